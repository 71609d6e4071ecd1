"""The bulk collide kernel with TMA-staged inputs (flbm_use_tma) on the GPU.

It computes the same node update as the kernel that reads global memory
directly, so the two must agree bit for bit, whatever the tile raggedness,
walls, noise, relaxation times or particle. One case is also checked against
the FP64 oracle, and graph replay with it against plain launches."""
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


CASES = [
    dict(lx=64, ly=32, lz=24, radius=5.0, kT=1e-5, g=1e-4),
    dict(lx=36, ly=20, lz=9, wall=(1, 0, 1), radius=0.0, kT=1e-4),          # ragged tiles in x and y
    dict(lx=32, ly=40, lz=40, radius=4.0, kT=0.0, g=2e-4, tau_s=0.8),        # MRT with tau != 1
    dict(lx=44, ly=24, lz=30, wall=(0, 1, 0), radius=3.5, kT=1e-5, delta_rho=0.2, pos0=(1.0, 11.5, 0.5)),
    dict(lx=32, ly=32, lz=64, radius=4.0, kT=1e-5, g=5e-6, fluid_counterforce=1),
]


def _fluid(p, X):
    z, y, x = np.meshgrid(np.arange(p["lz"]), np.arange(p["ly"]), np.arange(p["lx"]), indexing="ij")
    r2 = np.zeros(x.shape)
    for c, a, L, w in ((x, 0, p["lx"], p["wall"][0]), (y, 1, p["ly"], p["wall"][1]), (z, 2, p["lz"], p["wall"][2])):
        d = c - X[a]
        if not w:
            d = (d + 0.5 * L) % L - 0.5 * L
        r2 = r2 + d * d
    return r2 >= p["radius"] ** 2 if p["radius"] > 0 else np.ones(x.shape, bool)


@pytest.mark.parametrize("case", range(len(CASES)))
def test_tma_equals_direct_kernel_bit_for_bit(flbm, case):
    p = W.params(**CASES[case])
    a, b = flbm.Sim(p), flbm.Sim(p)
    a.use_tma(True)
    b.use_tma(False)
    b.set_density_mode(0)  # the TMA-staged kernel runs with a density pass
    a.step(17)
    b.step(17)
    pa, pb = a.particle(), b.particle()
    for k in ("X", "V", "Omega", "F", "T", "delta"):
        assert np.array_equal(pa[k], pb[k]), k
    fl = _fluid(p, pa["X"])
    assert np.array_equal(a.read_f()[:, :, fl], b.read_f()[:, :, fl])
    assert a.observables()["nonfinite"] == 0


def test_tma_against_the_oracle(flbm, oracle_mod):
    p = W.params(lx=32, ly=32, lz=40, radius=4.0, kT=1e-5, g=1e-4)
    sim = flbm.Sim(p)
    sim.use_tma(True)
    orc = oracle_mod.Oracle(p)
    orc.set_f(sim.read_f().astype(np.float64))
    sim.step(10)
    orc.step(10)
    fl = ~orc.fields()["solid"]
    g, o = sim.read_f()[:, :, fl].astype(np.float64), orc.get_f()[:, :, fl]
    scale = np.mean(np.abs(o), axis=-1, keepdims=True)
    assert np.max(np.abs(g - o) / scale) < 1e-5
    pg, po = sim.particle(), orc.particle()
    assert np.max(np.abs(pg["V"] - po["V"])) <= 1e-4 * np.max(np.abs(po["V"])) + 1e-12


def test_graph_replay_with_tma(flbm):
    import torch

    p = W.params(lx=32, ly=32, lz=48, radius=4.0, kT=1e-5, g=1e-4)
    plain = flbm.Sim(p)
    plain.use_tma(True)
    plain.step(9)
    g = flbm.Sim(p, stream=torch.cuda.Stream())
    g.use_tma(True)
    g.use_graphs(True)
    g.step(9)
    torch.cuda.synchronize()
    pa, pb = plain.particle(), g.particle()
    assert np.array_equal(pa["V"], pb["V"]) and np.array_equal(pa["X"], pb["X"])
    fl = _fluid(p, pa["X"])
    assert np.array_equal(plain.read_f()[:, :, fl], g.read_f()[:, :, fl])


def test_tma_refused_where_rows_do_not_allow_it(flbm):
    for over in (dict(lx=16, ly=16, lz=32), dict(lx=34, ly=16, lz=8)):
        s = flbm.Sim(W.params(**over))
        with pytest.raises(flbm.FLBMError):
            s.use_tma(True)
        s.use_tma(False)
        s.step(2)
        assert s.observables()["nonfinite"] == 0


def test_a_wait_that_runs_out_reports_a_timeout_and_the_context_stays_usable(flbm):
    """Failure detection of the bounded waits, without a fault. The TMA-staged
    collide's waits for its tensor copies are given a limit of one SM cycle,
    so they give up before the copies land. Each block that gives up flags
    the error, waits (with the default limit) for its own copies still in
    flight, and returns. The host must then report FLBM_E_TIMEOUT from
    flbm_particle_state and flbm_observables. The lattice has no particle,
    so no kernel of the step indexes memory by values the skipped tiles
    left behind. Afterwards the context is still usable: a new handle with
    the default limit steps bit for bit as the direct kernel does."""
    p = W.params(lx=32, ly=32, lz=32, radius=0.0, kT=1e-5)
    broken = flbm.Sim(p)
    broken.use_tma(True)
    broken.set_tma_wait(1)
    broken.step(2)
    with pytest.raises(flbm.FLBMError, match="FLBM_E_TIMEOUT"):
        broken.particle()
    with pytest.raises(flbm.FLBMError, match="FLBM_E_TIMEOUT"):
        broken.observables(allow_nonfinite=True)
    broken.close()
    a, b = flbm.Sim(p), flbm.Sim(p)
    a.use_tma(True)
    b.set_density_mode(0)
    a.step(6)
    b.step(6)
    a.particle()  # no error flagged
    assert np.array_equal(a.read_f(), b.read_f())
