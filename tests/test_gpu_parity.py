"""GPU parity: the sm_103a CUDA path (through the C-ABI) against the FP64 oracle.

Both sides start from the same seeded input (the method's own Philox-seeded
initial state, or a seeded random population field from
paper_1909_01092_gb300.workloads) and are compared element by element on the
fluid nodes. Tolerances:
* noise-free runs: every population within 1e-5 of its own value
  (element-wise relative error);
* noisy runs: every population within 1e-5 of the mean magnitude of its
  (component, direction) field. Both sides draw the same Philox normals, but a
  few populations of the minority component pass close to zero, where an
  element-wise ratio says nothing about the arithmetic;
* the particle velocity within 1e-4 of its velocity scale.
"""
import math

import numpy as np
import pytest

from paper_1909_01092_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL_F = 1e-5
RTOL_TRAJ = 1e-4


@pytest.fixture(scope="module")
def flbm():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need CUDA")
    from paper_1909_01092_gb300 import binding
    binding.load()
    return binding


def _launches_per_step(p):
    """Kernels of one step: densities, density shell with the virtual layer,
    the collide-stream pass of the tiles away from the particle, then either
    the near-particle collide (ending with the particle update), the
    next-position masks and cover/uncover (ending with the bookkeeping), or
    the finish kernel."""
    return 6 if p["radius"] > 0 else 4


def _fluid_mask(orc):
    return ~orc.fields()["solid"]


def _max_rel(g, o, mask):
    """max |g - o| / mean|o| per (component, direction), over fluid nodes
    (noisy runs)."""
    g = g[:, :, mask].astype(np.float64)
    o = o[:, :, mask]
    scale = np.mean(np.abs(o), axis=2, keepdims=True)
    return float(np.max(np.abs(g - o) / scale))


def _max_rel_elem(g, o, mask):
    """max |g - o| / |o| over every population of every fluid node
    (noise-free runs)."""
    g = g[:, :, mask].astype(np.float64)
    o = o[:, :, mask]
    return float(np.max(np.abs(g - o) / np.abs(o)))


def _rel_err(g, o, mask, p):
    """Element-wise relative error without noise, mean-normalised with it."""
    return (_max_rel_elem if p["kT"] == 0 else _max_rel)(g, o, mask)


def _pair(flbm, oracle_mod, p, init_seed=None, X=None, V=(0, 0, 0), Om=(0, 0, 0)):
    sim = flbm.Sim(p)
    orc = oracle_mod.Oracle(p)
    if init_seed is not None:
        f0 = W.random_populations(p, init_seed)
        f32 = f0.astype(np.float32)
        sim.write_f(f32)
        orc.set_f(f32.astype(np.float64))
    else:
        orc.set_f(sim.read_f().astype(np.float64))  # same Philox initial state, rounded to float32
    if X is not None:
        sim.set_particle(X, V, Om)
        orc.set_particle(X, V, Om)
    return sim, orc


def _compare_particle(pg, po, vscale, nsteps, tol=RTOL_TRAJ):
    """Velocity within tol of its largest magnitude so far; position within the
    displacement that velocity error can accumulate over nsteps."""
    assert np.max(np.abs(pg["V"] - po["V"])) <= tol * vscale + 1e-12
    assert np.max(np.abs(pg["X"] - po["X"])) <= tol * vscale * nsteps + 1e-9
    assert pg["nfluid"] == po["nfluid"]
    assert pg["step"] == po["step"]


def test_initial_state_matches_oracle(flbm, oracle_mod):
    p = W.channel_small(init_pert=1e-2)
    sim = flbm.Sim(p)
    orc = oracle_mod.Oracle(p)
    g, o = sim.read_f(), orc.get_f()
    assert np.max(np.abs(g - o) / o) < 3e-7  # three float32 roundings of the same formula


CASES = [
    # name, params, steps, random init seed
    ("periodic_sc", W.params(lx=8, ly=6, lz=10, wall=(0, 0, 0), G=1.5), 100, 1),
    ("walls_ragged_mrt", W.params(lx=37, ly=11, lz=9, wall=(1, 1, 1), G=1.2, tau_s=0.8, tau_d=1.3, tau_g=0.9),
     50, 2),
    ("noise_periodic", W.params(lx=12, ly=10, lz=8, wall=(0, 0, 0), G=1.2, kT=1e-4), 50, 3),
    ("noise_walls_forced", W.params(lx=9, ly=20, lz=7, wall=(1, 0, 1), G=1.5, kT=1e-5,
                                    fluid_force=(1e-5, -2e-5, 3e-5), tau_s=0.7), 40, 4),
    ("single_node", W.params(lx=1, ly=1, lz=1, wall=(0, 0, 0), kT=1e-4), 30, 5),
    ("thin_channel", W.params(lx=1, ly=33, lz=2, wall=(0, 1, 0), G=1.2, kT=1e-5), 30, 6),
    # noise amplitudes of all three relaxation classes, each at its own rate
    ("noise_three_rates", W.params(lx=10, ly=9, lz=11, wall=(0, 1, 0), G=1.2, kT=1e-4, tau_s=0.8, tau_d=0.7,
                                   tau_g=1.3), 40, 7),
    # a line of nodes between halfway walls, forced along z (one row per tile)
    ("line_walls_forced", W.params(lx=48, ly=1, lz=1, wall=(1, 0, 0), G=1.5, tau_s=0.875, tau_g=1.0,
                                   fluid_force=(0.0, 0.0, 1e-6)), 200, 8),
]


@pytest.mark.parametrize("name,p,steps,seed", CASES, ids=[c[0] for c in CASES])
def test_fluid_parity(flbm, oracle_mod, name, p, steps, seed):
    sim, orc = _pair(flbm, oracle_mod, p, init_seed=seed)
    sim.step(steps)
    orc.step(steps)
    assert sim.launches() == _launches_per_step(p) * steps
    err = _rel_err(sim.read_f(), orc.get_f(), _fluid_mask(orc), p)
    print(f"{name}: max rel err {err:.3e}")
    assert err < RTOL_F, f"{name}: max rel err {err:.3e}"


def test_channel_small_100_noise_free_steps(flbm, oracle_mod):
    """The 16x16x32 noise-free channel with the R=3 sphere: populations after
    100 steps within 1e-5. The settling velocity is a small difference between
    the driving impulse F_p t / m_p and the drag, so its tolerance is 1e-4 of
    that impulse velocity (float32 rounding of the exchanged momentum)."""
    p = W.channel_small()
    sim, orc = _pair(flbm, oracle_mod, p)
    for _ in range(100):
        sim.step(1)
        orc.step(1)
    po = orc.particle()
    assert sim.launches() == _launches_per_step(p)
    pg = sim.particle()
    vimp = po["Fp"] / po["mp"] * 100
    _compare_particle(pg, po, vimp, 100)
    # F is a near-cancelling sum of a few hundred link terms of size ~0.06 each:
    # float32 populations bound its error by ~1e-6 of that sum, i.e. well under
    # 1e-3 of the driving force F_p.
    assert np.max(np.abs(pg["F"] - po["F"])) <= 1e-3 * abs(po["Fp"])
    err = _max_rel_elem(sim.read_f(), orc.get_f(), _fluid_mask(orc))
    print(f"channel 16x16x32, 100 noise-free steps: element-wise max rel err {err:.3e}")
    assert err < RTOL_F, f"max rel err {err:.3e}"


PARTICLE_CASES = [
    ("moving_periodic_wetting_noise",
     W.params(lx=14, ly=14, lz=14, wall=(0, 0, 0), G=1.2, kT=1e-5, radius=2.6, delta_rho=0.3),
     (6.3, 6.8, 7.1), (0.03, -0.02, 0.05), (0.01, 0.0, -0.01), 60),
    ("wraps_periodic_z",
     W.params(lx=14, ly=14, lz=16, wall=(1, 1, 0), G=1.2, radius=3.2, delta_rho=-0.2),
     (6.5, 6.4, 1.0), (0.0, 0.01, -0.06), (0.0, 0.02, 0.0), 50),
    ("counterforce_clamped_wetting",
     W.params(lx=16, ly=16, lz=32, wall=(1, 1, 0), G=1.2, radius=3.0, g=1e-3, delta_rho=1.5,
              fluid_counterforce=1, fluid_force=(0.0, 1e-5, 0.0)),
     None, (0, 0, 0), (0, 0, 0), 40),
    ("near_wall_all_walls",
     W.params(lx=18, ly=15, lz=17, wall=(1, 1, 1), G=1.0, kT=1e-5, radius=3.4, delta_rho=0.5),
     (3.1, 7.2, 8.3), (-0.01, 0.02, 0.03), (0.0, 0.0, 0.05), 40),
]


@pytest.mark.parametrize("name,p,X,V,Om,steps", PARTICLE_CASES, ids=[c[0] for c in PARTICLE_CASES])
def test_particle_parity(flbm, oracle_mod, name, p, X, V, Om, steps):
    sim, orc = _pair(flbm, oracle_mod, p, init_seed=7, X=X, V=V, Om=Om)
    flips = 0
    n0 = orc.particle()["nfluid"]
    vmax = max(1e-6, float(np.max(np.abs(V))))
    for k in range(steps):
        sim.step(1)
        orc.step(1)
        po, pg = orc.particle(), sim.particle()
        vmax = max(vmax, float(np.max(np.abs(po["V"]))))
        _compare_particle(pg, po, vmax, k + 1)
        flips += po["nfluid"] != n0
        n0 = po["nfluid"]
    err = _rel_err(sim.read_f(), orc.get_f(), _fluid_mask(orc), p)
    print(f"{name}: max rel err {err:.3e}")
    assert err < RTOL_F, f"{name}: max rel err {err:.3e}"
    if X is not None:
        assert flips > 0, "expected cover/uncover events"


def test_trajectory_1000_fluctuating_steps(flbm, oracle_mod):
    """The 16x16x32 channel with thermal noise (kT = 1e-5) and the R=3 sphere
    started at V_z = 0.01, so that it crosses lattice nodes: 1000 steps with
    identical Philox noise on both sides.

    The kick decays within a few tens of steps. After that the velocity is
    thermal, sqrt(kT/m_p) = 2.4e-4, plus a settling drift of order 1e-5. The
    velocity error of every step must stay within 1e-4 of the velocity
    scale of the late part (steps 200 to 999): the largest |V| the oracle
    reaches there. That scale is at least sqrt(kT/m_p), not the kick, so
    the tolerance holds the fluctuating motion itself to 1e-4. The
    position error after k steps must stay within the velocity tolerance
    times k (the sum of the per-step velocity errors)."""
    p = W.channel_small(kT=1e-5)
    X0 = np.array(p["pos0"])
    sim, orc = _pair(flbm, oracle_mod, p, X=X0, V=(0.0, 0.0, 0.01))
    f0 = sim.read_f()
    traj = sim.run_host(f0, 1000, traj=True)
    Vg = np.array([t["V"] for t in traj])
    Xg = np.array([t["X"] for t in traj])
    Vo = np.empty_like(Vg)
    Xo = np.empty_like(Xg)
    for k in range(1000):
        orc.step(1)
        po = orc.particle()
        Vo[k], Xo[k] = po["V"], po["X"]
    v_th = math.sqrt(p["kT"] / po["mp"])
    scale = max(float(np.max(np.abs(Vo[200:]))), v_th)
    dv = np.max(np.abs(Vg - Vo), axis=1)
    dx = np.max(np.abs(Xg - Xo), axis=1)
    steps = np.arange(1, 1001)
    print(f"trajectory: velocity scale {scale:.3e} (thermal {v_th:.3e}); max velocity error "
          f"{dv.max():.3e} = {dv.max() / scale:.2e} of scale (steps 200-999: {dv[200:].max() / scale:.2e}); "
          f"max position error / (scale k) {np.max(dx / (scale * steps)):.2e}")
    assert dv.max() <= RTOL_TRAJ * scale
    assert np.all(dx <= RTOL_TRAJ * scale * steps)
    assert traj[-1]["step"] == 1000


def test_run_host_equals_step(flbm, oracle_mod):
    p = W.channel_small(kT=1e-5)
    a = flbm.Sim(p)
    b = flbm.Sim(p)
    f0 = a.read_f()
    out = np.empty_like(f0)
    traj = b.run_host(f0, 25, f_out=out, traj=True)
    a.step(25)
    assert np.array_equal(a.read_f(), out)  # both copies are initialised, so particle nodes match too
    pa = a.particle()
    assert np.array_equal(pa["X"], traj[-1]["X"]) and np.array_equal(pa["V"], traj[-1]["V"])


def test_full_size_translation_invariance(flbm, oracle_mod):
    """128x128x512 channel in the benchmark's launch configuration, noise-free,
    no particle: a state periodic in z with period 32 must give, after two
    steps, the oracle's result on the 128x128x32 channel tiled 16 times."""
    small = W.params(lx=128, ly=128, lz=32, wall=(1, 1, 0), G=1.2)
    big = W.params(lx=128, ly=128, lz=512, wall=(1, 1, 0), G=1.2)
    f0 = W.random_populations(small, 21).astype(np.float32)
    orc = oracle_mod.Oracle(small)
    orc.set_f(f0.astype(np.float64))
    orc.step(2)
    sim = flbm.Sim(big)
    sim.write_f(np.tile(f0, (1, 1, 16, 1, 1)))
    sim.step(2)
    g = sim.read_f()
    o = orc.get_f()
    for k in range(16):
        blk = g[:, :, 32 * k:32 * (k + 1)].astype(np.float64)
        err = float(np.max(np.abs(blk - o) / o))
        assert err < RTOL_F, f"z block {k}: max rel err {err:.3e}"


def test_full_size_workload_conserves_mass(flbm):
    """The 128x128x512 fluctuating channel with the R=12 sphere, exactly as
    benchmarked: after 20 steps every population is finite, the mass of each
    component plus the pending correction is conserved to float32 rounding,
    and the particle starts moving along the driving force."""
    p = W.channel_large()
    sim = flbm.Sim(p)
    a = sim.observables()
    sim.step(20)
    b = sim.observables()
    assert b["nonfinite"] == 0
    for l in range(2):
        m0 = a["mass"][l] + a["pending_mass"][l]
        m1 = b["mass"][l] + b["pending_mass"][l]
        assert abs(m1 - m0) < 1e-6 * m0
    pg = sim.particle()
    assert pg["V"][2] > 0 and pg["step"] == 20
    assert math.isclose(pg["Fp"], 4 / 3 * math.pi * 12 ** 3 * 0.5 * 1.05 * 1e-5, rel_tol=1e-12)


@pytest.mark.parametrize("drho", [-0.5, 0.0, 0.5])
def test_fluctuating_channel_with_each_wetting(flbm, oracle_mod, drho):
    """The 32x32x64 fluctuating channel (kT = 1e-5, R = 4) at each wetting
    parameter of that workload, the particle given a velocity that makes it
    cross nodes: 30 steps with identical Philox noise, populations within
    1e-5 and the particle velocity within 1e-4 of its scale."""
    p = W.channel_fluct(delta_rho=drho)
    V = (0.01, -0.02, 0.04)
    sim, orc = _pair(flbm, oracle_mod, p, X=p["pos0"], V=V, Om=(0.0, 0.01, 0.0))
    sim.step(30)
    orc.step(30)
    pg, po = sim.particle(), orc.particle()
    _compare_particle(pg, po, max(0.04, float(np.max(np.abs(po["V"])))), 30)
    err = _max_rel(sim.read_f(), orc.get_f(), _fluid_mask(orc))
    assert err < RTOL_F, f"max rel err {err:.3e}"


def test_benchmarked_channel_slab_with_moving_sphere(flbm, oracle_mod):
    """The benchmarked configuration against the oracle: 128-wide rows, walls
    on x and y, kT = 1e-5 and the R = 12 sphere, so the same bulk and
    near-particle launches (tile shapes, candidate grid around the particle
    box) as the 128x128x512 throughput run. It runs on a 128x128x32 slab,
    which the oracle steps in seconds. The sphere is given V_z = 0.02 so that
    nodes are covered and uncovered. After 12 steps with identical Philox
    noise, the populations must agree within 1e-5 (mean-normalised, noisy
    run) and the particle velocity within 1e-4 of its scale at every step,
    with the fluid node count exact."""
    p = W.channel_large(lz=32)
    V = (0.0, 0.0, 0.02)
    sim, orc = _pair(flbm, oracle_mod, p, X=p["pos0"], V=V)
    n0 = orc.particle()["nfluid"]
    flips = 0
    vmax = 0.02
    for k in range(12):
        sim.step(1)
        orc.step(1)
        po, pg = orc.particle(), sim.particle()
        vmax = max(vmax, float(np.max(np.abs(po["V"]))))
        _compare_particle(pg, po, vmax, k + 1)
        flips += po["nfluid"] != n0
        n0 = po["nfluid"]
    assert sim.launches() == _launches_per_step(p)
    err = _max_rel(sim.read_f(), orc.get_f(), _fluid_mask(orc))
    print(f"128x128x32 slab, R=12, kT=1e-5, 12 steps: max rel err {err:.3e}, {flips} steps with cover/uncover")
    assert err < RTOL_F, f"max rel err {err:.3e}"
    assert flips > 0, "expected cover/uncover events"


def test_mode_temperatures_match_the_oracle(flbm, oracle_mod):
    """The fluctuation temperatures of flbm_observables (modes 4..18 of each
    component, interdiffusion current, total momentum; Section 2's
    fluctuation-dissipation requirement) against the oracle's own reduction of
    its state. The run has 40 noisy steps with a moving, wetted sphere. The
    populations agree to about 1e-6, and the non-equilibrium modes are
    differences of them about a tenth of their size, so the temperatures
    must agree to 1e-3 relative. The bulk node count (fluid nodes with no
    particle neighbour) must be exact."""
    p = W.params(lx=14, ly=14, lz=14, wall=(0, 0, 0), G=1.2, kT=1e-4, radius=2.6, delta_rho=0.3)
    sim, orc = _pair(flbm, oracle_mod, p, init_seed=9, X=(6.3, 6.8, 7.1), V=(0.03, -0.02, 0.05))
    sim.step(40)
    orc.step(40)
    go = sim.observables()
    oo = orc.mode_temps()
    assert go["n_bulk"] == oo["n_bulk"] > 0
    for key in ("mode_temp", "diff_temp", "mom_temp"):
        err = float(np.max(np.abs(go[key] - oo[key]) / np.maximum(np.abs(oo[key]), 1e-300)))
        print(f"{key}: max rel err {err:.2e}")
        np.testing.assert_allclose(go[key], oo[key], rtol=1e-3, atol=0)
