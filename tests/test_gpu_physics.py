"""Physics of the settling particle on the GPU path, against the paper's
hydrodynamic-Langevin picture (Section 3): the velocity variance of a
thermalised sphere is kT / m_p per axis, and confinement in the square
channel lowers the settling velocity below Stokes' prediction, the more so
the larger d/L (the ratio c_m of Eq. (cm) decreases from 1)."""
import math

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


def _trajectory(flbm, p, burn, steps):
    """Half-step leap-frog velocity V and step average Vavg over `steps`
    steps after `burn`, and kT / m_p."""
    sim = flbm.Sim(p)
    sim.step(burn)
    tr = sim.run_host(sim.read_f(), steps, traj=True)
    V = np.array([t["V"] for t in tr])
    Va = np.array([t["Vavg"] for t in tr])
    s = p["kT"] / tr[-1]["mp"]
    sim.close()
    return V, Va, s


def _variances(flbm, p, burn, steps):
    """Velocity variances per axis in units of kT / m_p: V and Vavg."""
    V, Va, s = _trajectory(flbm, p, burn, steps)
    return V.var(axis=0) / s, Va.var(axis=0) / s


def test_heavy_sphere_velocity_equipartition(flbm):
    """rho_p = 5 rho, R = 3, fluctuating mixture in a 24x24x48 channel,
    200000 samples (a few thousand velocity relaxation times): both velocity
    estimates give kT / m_p to within their few-percent time-stepping bias,
    the half-step velocity above the step average, and the velocity is
    Gaussian."""
    p = W.params(lx=24, ly=24, lz=48, wall=(1, 1, 0), radius=3.0, rho_p_ratio=5.0, g=0.0, kT=1e-4, init_pert=0.0)
    V, Va, s = _trajectory(flbm, p, 2000, 200000)
    rv, ra = V.var(axis=0) / s, Va.var(axis=0) / s
    assert 0.95 <= rv.mean() <= 1.15, rv
    assert 0.88 <= ra.mean() <= 1.06, ra
    assert rv.mean() > ra.mean()
    # Gaussian velocity distribution (Section 3): kurtosis 3, no skew, 4.55 %
    # of the samples beyond two standard deviations (pooled over the axes).
    Z = (Va - Va.mean(axis=0)) / Va.std(axis=0)
    assert 2.8 <= (Z ** 4).mean() <= 3.2, (Z ** 4).mean(axis=0)
    assert abs((Z ** 3).mean()) <= 0.1, (Z ** 3).mean(axis=0)
    assert 0.038 <= (np.abs(Z) > 2).mean() <= 0.053


def test_light_sphere_leapfrog_estimates_bracket_equipartition(flbm):
    """rho_p = 1.5 rho (the benchmarked density ratio), R = 3: the explicit
    time stepping of the coupling makes the half-step velocity run hot and
    the step average run cold; they bracket kT / m_p."""
    p = W.params(lx=24, ly=24, lz=48, wall=(1, 1, 0), radius=3.0, rho_p_ratio=1.5, g=0.0, kT=1e-4, init_pert=0.0)
    rv, ra = _variances(flbm, p, 2000, 100000)
    assert 1.05 < rv.mean() < 1.6, rv
    assert 0.7 < ra.mean() < 1.0, ra


def test_confinement_lowers_the_settling_velocity(flbm):
    """Noise-free settling in a 32x32x64 channel (walls on x and y, the
    counterforce keeping the total momentum steady): c_m = U / U_0 with
    U_0 = F_p / (3 pi eta d) falls below 1 and decreases as d/L grows."""
    eta = 1.05 / 6
    cm = []
    for R in (2.0, 4.0, 6.0):
        p = W.params(lx=32, ly=32, lz=64, wall=(1, 1, 0), radius=R, rho_p_ratio=1.5, g=2e-4 * (4.0 / R) ** 2,
                     kT=0.0, init_pert=0.0, fluid_counterforce=1)
        sim = flbm.Sim(p)
        sim.step(8000)
        us = []
        for _ in range(50):
            sim.step(10)
            us.append(sim.particle()["V"][2])
        ob = sim.observables()
        U = np.mean(us) - ob["momentum"][2] / ob["mass"].sum()
        Fp = sim.particle()["Fp"]
        cm.append(U / (Fp / (3 * math.pi * eta * 2 * R)))
        sim.close()
    assert all(0.0 < c < 1.0 for c in cm), cm
    assert cm[0] > cm[1] > cm[2], cm


def test_fluctuating_modes_are_at_equipartition_on_the_benchmark_channel(flbm):
    """Fluctuation-dissipation (Section 2) on the GPU at the benchmarked size:
    the 128x128x512 channel (walls on x and y) at kT = 1e-5 as an ideal
    mixture (G = 0) without the sphere. There the populations are independent
    Gaussians of variance 3 kT rho_l w_i, walls included, so every mode
    temperature of flbm_observables (modes 4..18 of A and B), the
    interdiffusion temperature and the momentum temperature equal kT. After
    300 steps, the mean over 4 snapshots 5 steps apart must lie within
    6 sigma, sigma = sqrt(2 / (4 n)) = 2.4e-4 for the n = 8.4 M nodes
    (momentum: 8 sigma, its long waves decorrelate more slowly)."""
    p = W.channel_large(radius=0.0, G=0.0)
    kT = p["kT"]
    sim = flbm.Sim(p)
    sim.step(300)
    acc = []
    for _ in range(4):
        sim.step(5)
        acc.append(sim.observables())
    n = acc[0]["n_bulk"]
    assert n == 128 * 128 * 512
    sigma = math.sqrt(2.0 / (4 * n))
    mt = np.mean([a["mode_temp"] for a in acc], axis=0) / kT
    dt = np.mean([a["diff_temp"] for a in acc], axis=0) / kT
    jt = np.mean([a["mom_temp"] for a in acc], axis=0) / kT
    print("mode temperatures / kT, A:", np.round(mt[0, 4:], 5), "B:", np.round(mt[1, 4:], 5))
    print("interdiffusion / kT:", np.round(dt, 5), "momentum / kT:", np.round(jt, 5), f"sigma {sigma:.1e}")
    assert np.all(mt[:, :4] == 0.0)
    assert np.max(np.abs(mt[:, 4:] - 1.0)) < 6 * sigma
    assert np.max(np.abs(dt - 1.0)) < 6 * sigma
    assert np.max(np.abs(jt - 1.0)) < 8 * sigma
