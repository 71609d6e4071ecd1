"""Configurations beyond the benchmarked ones, each against the FP64 oracle:
a phase-separated mixture at the paper's G = 1.5 with the particle sitting on
the A/B interface, and the closed channel (walls on all three axes) of the
paper's production runs (Section 3)."""
import numpy as np
import pytest

from paper_1909_01092_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL_F = 1e-5


@pytest.fixture(scope="module")
def flbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_01092_gb300 import binding

    binding.load(build_if_missing=True)
    return binding


def _run(flbm, oracle_mod, p, f0, X, V, steps):
    sim = flbm.Sim(p)
    orc = oracle_mod.Oracle(p)
    f32 = f0.astype(np.float32)
    sim.write_f(f32)
    orc.set_f(f32.astype(np.float64))
    sim.set_particle(X, V)
    orc.set_particle(X, V)
    sim.step(steps)
    orc.step(steps)
    fluid = ~orc.fields()["solid"]
    g, o = sim.read_f()[:, :, fluid].astype(np.float64), orc.get_f()[:, :, fluid]
    err = float(np.max(np.abs(g - o) / np.mean(np.abs(o), axis=2, keepdims=True)))
    return sim, orc, err


@pytest.mark.parametrize("kT,drho", [(0.0, 0.3), (1e-5, -0.3)])
def test_particle_on_the_interface_of_a_separated_mixture(flbm, oracle_mod, kT, drho):
    p = W.channel_small(G=1.5, rho_a0=2.21, rho_b0=0.09, kT=kT, delta_rho=drho, g=1e-4, radius=3.0)
    f0 = W.layered_populations(p)  # A-rich slab 8 <= z < 24, interfaces at z = 8 and 24
    X = (p["pos0"][0], p["pos0"][1], 8.0)
    sim, orc, err = _run(flbm, oracle_mod, p, f0, X, (0.0, 0.0, 0.0), 60)
    assert err < RTOL_F, f"max rel err {err:.3e}"
    pg, po = sim.particle(), orc.particle()
    scale = max(np.max(np.abs(po["V"])), 1e-9)
    assert np.max(np.abs(pg["V"] - po["V"])) <= 1e-4 * scale
    assert pg["nfluid"] == po["nfluid"]
    # the slab stays separated: A-rich in the middle, B-rich outside
    rho = orc.fields()["rho"]
    assert rho[0, 16].mean() > 1.5 and rho[0, 0].mean() < 0.5


def test_closed_channel(flbm, oracle_mod):
    """Walls on x, y and z, a moving particle, noise."""
    p = W.params(lx=12, ly=12, lz=24, wall=(1, 1, 1), radius=3.0, rho_p_ratio=1.5, g=1e-4, kT=1e-5,
                 fluid_counterforce=1)
    f0 = W.random_populations(p, 11)
    X = (5.5, 5.5, 11.5)
    sim, orc, err = _run(flbm, oracle_mod, p, f0, X, (0.002, -0.001, 0.01), 80)
    assert err < RTOL_F, f"max rel err {err:.3e}"
    pg, po = sim.particle(), orc.particle()
    assert np.max(np.abs(pg["V"] - po["V"])) <= 1e-4 * np.max(np.abs(po["V"]))
    assert pg["nfluid"] == po["nfluid"]


def test_production_cross_section_closed_slab(flbm, oracle_mod):
    """The closed channel of the paper's production runs (Section 3: 60 x 60
    cross-section, walls on every axis, the paper's fluid G = 1.5 with
    rho_A = 2.21, rho_B = 0.09, rho_p = 2 rho_tot) on a 60 x 60 x 32 slab.
    Its 60-wide rows are not a multiple of the 32-node tile, so the last tile
    of each row is ragged. An R = 8 sphere (d/L = 0.27) moves through the
    slab with noise, kT = 1e-5, and is covered and uncovered. After 10 steps
    the populations agree with the oracle within 1e-5 (mean-normalised,
    noisy run), with the particle velocity within 1e-4 of its scale and the
    fluid count exact."""
    p = W.params(lx=60, ly=60, lz=32, wall=(1, 1, 1), G=1.5, rho_a0=2.21, rho_b0=0.09, radius=8.0,
                 rho_p_ratio=2.0, g=5e-6, kT=1e-5)
    sim = flbm.Sim(p)
    orc = oracle_mod.Oracle(p)
    orc.set_f(sim.read_f().astype(np.float64))
    X, V = (29.3, 30.1, 15.7), (0.01, -0.02, 0.03)
    sim.set_particle(X, V)
    orc.set_particle(X, V)
    n0, flips = orc.particle()["nfluid"], 0
    for _ in range(10):
        sim.step(1)
        orc.step(1)
        po = orc.particle()
        flips += po["nfluid"] != n0
        n0 = po["nfluid"]
    fluid = ~orc.fields()["solid"]
    g, o = sim.read_f()[:, :, fluid].astype(np.float64), orc.get_f()[:, :, fluid]
    err = float(np.max(np.abs(g - o) / np.mean(np.abs(o), axis=2, keepdims=True)))
    print(f"60x60x32 closed slab, R=8: max rel err {err:.3e}, {flips} steps with cover/uncover")
    assert err < RTOL_F, f"max rel err {err:.3e}"
    pg = sim.particle()
    assert np.max(np.abs(pg["V"] - po["V"])) <= 1e-4 * np.max(np.abs(po["V"]))
    assert pg["nfluid"] == po["nfluid"] and flips > 0


def test_normalised_fluctuations_grow_with_confinement(flbm):
    """The paper's Section 3 result in the Langevin picture, on the ensemble
    engine through paper_1909_01092_gb300.sweep: a fluctuating sphere (R = 3,
    kT = 1e-4, same body force) settles more slowly in narrower channels (c_m
    falls with d/L), while its velocity fluctuation stays at equipartition,
    sqrt(kT / m_p) (Eq. (FLUCTUATIONSSCALING)); so the normalised fluctuation
    Delta U / U grows with confinement (Eq. (normalizedconf)). Channels
    L = 16, 24, 32, 48 (length 2L, walls on x and y, counterforce on the
    fluid), two noise realisations each, in one ensemble; five-interval error
    bars as in the paper's figures."""
    from paper_1909_01092_gb300 import sweep

    Ls = (16, 24, 32, 48)
    plist = [W.params(lx=L, ly=L, lz=2 * L, radius=3.0, rho_p_ratio=5.0, g=2e-4, kT=1e-4, init_pert=0.0,
                      fluid_counterforce=1, replica=2 * k + s) for k, L in enumerate(Ls) for s in range(2)]
    rows = sweep.settling_sweep(plist, burn=10000, samples=1500, every=10)
    U = np.array([r["U"] for r in rows]).reshape(len(Ls), 2).mean(axis=1)
    Uerr = np.array([r["U_err"] for r in rows]).reshape(len(Ls), 2).mean(axis=1)
    cm = np.array([r["cm"] for r in rows]).reshape(len(Ls), 2).mean(axis=1)
    dU = np.array([r["dU"] / r["dU_pred"] for r in rows]).reshape(len(Ls), 2).mean(axis=1)
    ratio = np.array([r["dU_over_U"] for r in rows]).reshape(len(Ls), 2).mean(axis=1)
    assert np.all((cm > 0) & (cm < 1)), cm
    assert np.all(np.diff(U) > 3 * Uerr[1:]), (U, Uerr)  # c_m rises as d/L falls, beyond the error bars
    assert np.all(np.abs(dU - 1.0) < 0.15), dU           # equipartition in every channel
    assert np.all(np.diff(ratio) < 0), ratio              # Delta U / U falls as d/L falls


def test_hydrophilic_wetting_leaves_the_confined_drag_unchanged(flbm):
    """Section 3 finds almost no dependency of c_m on the wettability. With
    the particle wetted by the majority component (delta_rho = +0.5) the
    noise-free settling velocity in 16- and 32-wide channels (R = 4) equals
    the neutral one within 1 %."""
    from paper_1909_01092_gb300 import sweep

    plist = [W.params(lx=L, ly=L, lz=2 * L, radius=4.0, rho_p_ratio=1.5, g=1e-4, kT=0.0, init_pert=0.0,
                      delta_rho=dr, fluid_counterforce=1, replica=k)
             for k, (L, dr) in enumerate([(16, 0.0), (16, 0.5), (32, 0.0), (32, 0.5)])]
    cm = [r["cm"] for r in sweep.settling_sweep(plist, burn=8000, samples=100, every=10)]
    assert 0.0 < cm[0] < cm[2] < 1.0, cm
    assert abs(cm[1] / cm[0] - 1.0) < 0.01, cm
    assert abs(cm[3] / cm[2] - 1.0) < 0.01, cm
