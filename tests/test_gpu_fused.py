"""The fused step on the GPU: next-step densities summed by the collide as it
pushes (flbm_set_density_mode 1) instead of a density pass re-reading every
population (mode 0).

The densities it carries from step to step must be the densities of
Eq. (density) of the state it produced, which the oracle computes directly.
Stepping must agree with the two-pass step to float32 rounding and with the
oracle to the parity tolerance. This must hold whatever the tile
raggedness, walls, planes per block (chunk seams on every plane or none),
and whether the particle crosses tiles, chunks and periodic faces."""
import numpy as np
import pytest

from paper_1909_01092_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def flbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_01092_gb300 import binding

    binding.load(build_if_missing=True)
    return binding


def _max_rel_mean(g, o, mask):
    g = g[:, :, mask].astype(np.float64)
    o = o[:, :, mask]
    return float(np.max(np.abs(g - o) / np.mean(np.abs(o), axis=2, keepdims=True)))


CASES = [
    # name, params, planes per block, particle start (X, V)
    ("periodic_3x3_tiles_particle_K3",
     W.params(lx=96, ly=24, lz=12, wall=(0, 0, 0), G=1.2, kT=1e-5, radius=3.3, delta_rho=0.2),
     3, ((31.6, 7.4, 9.3), (0.04, 0.03, 0.05))),
    ("periodic_3x3_tiles_particle_K1",
     W.params(lx=96, ly=24, lz=12, wall=(0, 0, 0), G=1.2, radius=3.3, delta_rho=-0.2),
     1, ((64.2, 15.6, 0.4), (-0.04, 0.03, -0.05))),
    ("ragged_all_walls_K2", W.params(lx=40, ly=17, lz=9, wall=(1, 1, 1), G=1.5, tau_s=0.8, tau_g=1.3), 2, None),
    ("ragged_all_walls_one_chunk",
     W.params(lx=40, ly=17, lz=9, wall=(1, 1, 1), G=1.2, kT=1e-4, radius=2.7, delta_rho=0.4), 9,
     ((31.2, 8.3, 4.1), (0.05, -0.02, 0.03))),
    ("channel_walls_xy_K4_forced",
     W.params(lx=48, ly=20, lz=23, wall=(1, 1, 0), G=1.2, fluid_force=(0.0, 0.0, 1e-5)), 4, None),
]


def _start(flbm, p, K, part, seed):
    sim = flbm.Sim(p)
    sim.set_density_mode(1, K)
    assert sim.density_mode() == (1, K)
    f0 = W.random_populations(p, seed).astype(np.float32)
    sim.write_f(f0)
    if part is not None:
        sim.set_particle(*part)
    return sim, f0


@pytest.mark.parametrize("name,p,K,part", CASES, ids=[c[0] for c in CASES])
def test_carried_densities_are_those_of_the_state(flbm, oracle_mod, name, p, K, part):
    """After each of 12 fused steps the carried densities (flbm_read_fields'
    rho: what the next step's Shan-Chen force reads) equal, on every fluid
    node, the densities the oracle computes from its own state after the same
    steps, within 1e-5 of the mean component density. The populations agree
    within the parity tolerance."""
    sim, f0 = _start(flbm, p, K, part, 11)
    orc = oracle_mod.Oracle(p)
    orc.set_f(f0.astype(np.float64))
    if part is not None:
        orc.set_particle(*part)
    for k in range(12):
        sim.step(1)
        orc.step(1)
        fo = orc.fields()
        fluid = ~fo["solid"]
        rg = sim.read_rho().astype(np.float64)
        for l in range(2):
            scale = np.mean(fo["rho"][l][fluid])
            err = np.max(np.abs(rg[l][fluid] - fo["rho"][l][fluid])) / scale
            assert err < 1e-5, f"{name} step {k + 1} component {l}: {err:.3e}"
    err = _max_rel_mean(sim.read_f(), orc.get_f(), ~orc.fields()["solid"])
    print(f"{name}: populations max rel err {err:.3e}")
    assert err < 1e-5


@pytest.mark.parametrize("name,p,K,part", CASES, ids=[c[0] for c in CASES])
def test_fused_and_two_pass_steps_agree(flbm, name, p, K, part):
    """The same 20 steps in both density modes: the sums differ only in their
    order, so populations and particle agree to float32 rounding growth
    (1e-6 of each population's mean magnitude), and each mode is
    reproducible bit for bit."""
    a, f0 = _start(flbm, p, K, part, 12)
    b, _ = _start(flbm, p, K, part, 12)
    c = flbm.Sim(p)
    c.set_density_mode(0)
    c.write_f(f0)
    if part is not None:
        c.set_particle(*part)
    a.step(20)
    b.step(20)
    c.step(20)
    fa, fb, fc = a.read_f(), b.read_f(), c.read_f()
    pa, pc = a.particle(), c.particle()
    assert np.array_equal(fa, fb)
    fluid = np.ones(fa.shape[2:], bool)
    if part is not None:
        z, y, x = np.meshgrid(np.arange(p["lz"]), np.arange(p["ly"]), np.arange(p["lx"]), indexing="ij")
        r2 = np.zeros(x.shape)
        for cc, ax, L, w in ((x, 0, p["lx"], p["wall"][0]), (y, 1, p["ly"], p["wall"][1]),
                             (z, 2, p["lz"], p["wall"][2])):
            d = cc - pa["X"][ax]
            if not w:
                d = (d + 0.5 * L) % L - 0.5 * L
            r2 = r2 + d * d
        fluid = r2 >= p["radius"] ** 2
        assert pa["nfluid"] == pc["nfluid"]
        assert np.max(np.abs(pa["V"] - pc["V"])) <= 1e-6 * max(np.max(np.abs(pc["V"])), 1e-3)
    err = _max_rel_mean(fa, fc.astype(np.float64), fluid)
    print(f"{name}: fused vs two-pass max rel err {err:.3e}")
    assert err < 1e-6


def test_density_mode_choice(flbm):
    """Two-pass by default; fused where the lattice allows it and it is asked
    for; lattices with tiles narrower than 8 nodes or fewer than 3 tiles
    along a periodic axis refuse it; the TMA-staged collide runs two-pass."""
    s = flbm.Sim(W.channel_small())
    assert s.density_mode() == (0, 0)
    s.set_density_mode(1)
    assert s.density_mode()[0] == 1
    s.set_density_mode(1, 5)
    assert s.density_mode() == (1, 5)
    narrow = flbm.Sim(W.params(lx=4, ly=8, lz=8, wall=(1, 1, 0)))
    assert narrow.density_mode() == (0, 0)
    with pytest.raises(flbm.FLBMError, match="UNSUPPORTED"):
        narrow.set_density_mode(1)
    few = flbm.Sim(W.params(lx=64, ly=16, lz=8, wall=(0, 1, 0)))  # 2 tiles along periodic x
    with pytest.raises(flbm.FLBMError, match="UNSUPPORTED"):
        few.set_density_mode(1)
    t = flbm.Sim(W.params(lx=64, ly=32, lz=8))
    t.set_density_mode(1)
    t.use_tma(True)
    assert t.density_mode() == (0, 0)
    t.use_tma(False)
    assert t.density_mode()[0] == 1
    with pytest.raises(flbm.FLBMError, match="INVAL"):
        t.set_density_mode(1, 9)


def test_benchmarked_channel_carries_the_densities_of_its_state(flbm):
    """The 128x128x512 fluctuating channel with the R = 12 sphere in fused
    mode with the default planes per block: after 6
    fused steps the densities the step carries equal, on every fluid node,
    a fresh density pass over the same populations (a second handle given
    those populations) within 1e-6 relative. The two sum the same values in
    different orders. The same holds after a graph replay of 8 more
    steps."""
    import torch

    p = W.channel_large()
    sim = flbm.Sim(p, stream=torch.cuda.Stream())
    sim.set_density_mode(1)
    assert sim.density_mode()[0] == 1
    for steps, graphs in ((6, False), (8, True)):
        sim.use_graphs(graphs)
        sim.step(steps)
        torch.cuda.synchronize()
        rho = sim.read_rho().astype(np.float64)
        ref = flbm.Sim(p)
        ref.set_density_mode(0)
        ref.write_f(sim.read_f())
        pg = sim.particle()
        ref.set_particle(pg["X"], pg["V"], pg["Omega"])
        want = ref.read_rho().astype(np.float64)
        fluid = want[0] > 0
        for l in range(2):
            err = float(np.max(np.abs(rho[l][fluid] - want[l][fluid]) / want[l][fluid]))
            print(f"128x128x512 after {steps} steps: component {l} max rel err {err:.2e}")
            assert err < 1e-6
        ref.close()
