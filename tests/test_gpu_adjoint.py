"""Adjoint of the noise-free step (flbm_adjoint_run) on the GPU.

J = (1/T) sum_n Vavg_z(n), the time-averaged settling velocity; gradient with
respect to the body force g (Eq. (fp)), the wetting shift delta_rho (virtual
layer, Section 2) and the Shan-Chen coupling G (Eq. (sc-force)).

The reference gradient is the plain definition of the derivative: central
finite differences of J computed by the FP64 oracle, on a 16x16x32 channel,
starting from the GPU's own initial populations, with the particle given an
initial velocity so that cover/uncover events happen inside the horizon.
"""
import numpy as np
import pytest

from paper_1909_01092_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NAMES = ("g", "delta_rho", "G")
KEYS = ("dJ_dg", "dJ_ddelta_rho", "dJ_dG")


@pytest.fixture(scope="module")
def flbm():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1909_01092_gb300 import binding

    binding.load(build_if_missing=True)
    return binding


def _small(**over):
    base = dict(G=1.2, delta_rho=0.3, g=1e-4, kT=0.0)
    base.update(over)
    return W.channel_small(**base)


V0 = (0.01, -0.008, 0.05)


def _oracle_J(oracle_mod, p, f0, steps, v0):
    """J by the oracle, and whether the particle-node set changed on the way."""
    orc = oracle_mod.Oracle(p)
    orc.set_f(f0)
    orc.set_particle(p["pos0"], v0)
    solid0 = orc.fields()["solid"].copy()
    s = 0.0
    for _ in range(steps):
        orc.step(1)
        s += orc.particle()["Vavg"][2]
    return s / steps, bool(np.any(orc.fields()["solid"] != solid0))


def _gpu_start(flbm, p, v0):
    sim = flbm.Sim(p)
    sim.set_particle(p["pos0"], v0)
    return sim


@pytest.fixture(scope="module")
def small_case(flbm, oracle_mod):
    p = _small()
    T = 48
    sim = _gpu_start(flbm, p, V0)
    f0 = sim.read_f().astype(np.float64)
    res = sim.adjoint(T, checkpoint_every=16)
    J0, moved = _oracle_J(oracle_mod, p, f0, T, V0)
    fd = {}
    for name in NAMES:
        h = 1e-4 * abs(p[name])
        jp, _ = _oracle_J(oracle_mod, dict(p, **{name: p[name] + h}), f0, T, V0)
        jm, _ = _oracle_J(oracle_mod, dict(p, **{name: p[name] - h}), f0, T, V0)
        fd[name] = (jp - jm) / (2 * h)
    return dict(p=p, T=T, res=res, J0=J0, fd=fd, moved=moved, sim=sim)


def test_J_matches_the_oracle(small_case):
    c = small_case
    assert abs(c["res"]["J"] - c["J0"]) <= 1e-5 * abs(c["J0"])
    assert c["moved"], "no cover/uncover inside the horizon"


@pytest.mark.parametrize("k", range(3))
def test_gradient_matches_oracle_finite_differences(small_case, k):
    """Within 1e-4 of the FP64 difference quotient (the adjoint runs in FP64
    on a float32 forward trajectory; the difference quotient's own error is
    below 1e-7)."""
    c = small_case
    name = NAMES[k]
    adj, fd = c["res"][KEYS[k]], c["fd"][name]
    tol = 1e-4 * abs(fd) + 1e-8 * abs(c["J0"]) / abs(c["p"][name])
    assert abs(adj - fd) <= tol, f"{name}: adjoint {adj:.6e} vs oracle FD {fd:.6e}"


def test_strongly_coupled_mixture(flbm, oracle_mod):
    """A 50/50 mixture with 5 % density fluctuations and wetting, where J
    depends on G through the Shan-Chen forces everywhere."""
    p = _small(rho_a0=0.6, rho_b0=0.6, init_pert=0.05, delta_rho=0.1)
    T = 48
    sim = _gpu_start(flbm, p, V0)
    f0 = sim.read_f().astype(np.float64)
    res = sim.adjoint(T, 16)
    for name, key in zip(NAMES, KEYS):
        h = 1e-4 * abs(p[name])
        jp, _ = _oracle_J(oracle_mod, dict(p, **{name: p[name] + h}), f0, T, V0)
        jm, _ = _oracle_J(oracle_mod, dict(p, **{name: p[name] - h}), f0, T, V0)
        fd = (jp - jm) / (2 * h)
        assert abs(res[key] - fd) <= 1e-4 * abs(fd), f"{name}: adjoint {res[key]:.6e} vs oracle FD {fd:.6e}"


def test_gradient_of_g_after_one_step_is_exact(flbm):
    """T = 1 from rest: F of the first step does not depend on g, so
    dJ/dg = (1/2) dF_p/dg / m_p = (1 - rho_tot/rho_p) / 2 (Eq. (fp))."""
    p = _small()
    r = flbm.Sim(p).adjoint(1, 1)
    assert abs(r["dJ_dg"] - (1.0 - 1.0 / p["rho_p_ratio"]) / 2.0) < 1e-12


def test_checkpoint_interval_changes_nothing(flbm, small_case):
    p, T = small_case["p"], small_case["T"]
    ref = small_case["res"]
    for K in (1, 7, T):
        r = _gpu_start(flbm, p, V0).adjoint(T, K)
        for key in ("J",) + KEYS:
            assert r[key] == ref[key], (K, key)


def test_whole_tape_equals_checkpoint_recompute(flbm, small_case):
    """The small case fits the default tape limit, so its forward run keeps
    the tape of every step and nothing is recomputed. With the limit at 0
    (or below the store's size) the run checkpoints and recomputes each
    segment instead. Both must give the same J and gradient, and leave the
    same state, bit for bit, for full and ragged segments."""
    p, T = small_case["p"], small_case["T"]
    ref = small_case["res"]
    assert ref["whole_tape"]
    for K, limit in ((16, 0), (7, 0), (16, 1)):
        a = _gpu_start(flbm, p, V0)
        ra = a.adjoint(T, K, tape_limit=-1)
        c = _gpu_start(flbm, p, V0)
        rc = c.adjoint(T, K, tape_limit=limit)
        assert ra["whole_tape"] and not rc["whole_tape"], (K, limit)
        for key in ("J",) + KEYS:
            assert ra[key] == rc[key] == ref[key], (K, limit, key)
        assert np.array_equal(a.read_f(), c.read_f())
        pa, pc = a.particle(), c.particle()
        for k in ("X", "V", "Omega", "delta"):
            assert np.array_equal(pa[k], pc[k])
        assert pa["step"] == pc["step"] == T


def test_leaves_the_state_of_plain_steps(flbm, small_case):
    p, T = small_case["p"], small_case["T"]
    plain = _gpu_start(flbm, p, V0)
    plain.step(T)
    a, b = small_case["sim"].particle(), plain.particle()
    for k in ("X", "V", "Omega", "delta"):
        assert np.array_equal(a[k], b[k])
    assert a["step"] == b["step"] == T
    assert np.array_equal(small_case["sim"].read_f(), plain.read_f())


def test_autograd_function(flbm, small_case):
    import torch

    p, T = small_case["p"], small_case["T"]
    fn = flbm.settling_velocity(p, T, 16, v0=V0)
    th = [torch.tensor(p[n], dtype=torch.float64, requires_grad=True) for n in NAMES]
    J = fn(*th)
    J.backward()
    assert float(J.detach()) == small_case["res"]["J"]
    for t, key in zip(th, KEYS):
        assert float(t.grad) == small_case["res"][key]


def test_unsupported_configurations(flbm):
    for over in (dict(kT=1e-5), dict(radius=0.0), dict(tau_s=0.8), dict(fluid_counterforce=1)):
        with pytest.raises(flbm.FLBMError):
            flbm.Sim(_small(**over)).adjoint(2, 1)


@pytest.mark.slow
def test_full_size_against_gpu_finite_differences(flbm):
    """64x64x128 channel, R=8, delta_rho=0.3, G=1.2, 2000 steps, checkpoint
    every 100: the adjoint gradient against central differences of the GPU
    forward run (1e-2 relative step; J is smooth and the float32 forward
    sets the noise floor of the difference quotient)."""
    p = W.channel_adjoint()
    T = 2000
    r = flbm.Sim(p).adjoint(T, 100)
    assert r["checkpoint_every"] == 100 and r["steps"] == T

    def J(q):
        s = flbm.Sim(q)
        out = s.adjoint(T, 100)["J"]
        s.close()
        return out

    for name, key in zip(NAMES, KEYS):
        h = 1e-2 * abs(p[name])
        fd = (J(dict(p, **{name: p[name] + h})) - J(dict(p, **{name: p[name] - h}))) / (2 * h)
        assert abs(r[key] - fd) <= 2e-2 * abs(fd) + 1e-5 * abs(r["J"]) / abs(p[name]), (name, r[key], fd)
