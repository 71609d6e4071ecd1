"""Batched ensemble on the GPU.

Every replica of an ensemble must be the simulation a single handle makes
from the same parameters: bit for bit under tile policy 0 (whatever the
packing and persistence), to FP64 summation order of the particle force under
tile policy 1. One member is also checked against the FP64 oracle directly.
"""
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


def _members():
    """Uneven replicas covering every collide variant and particle/no particle."""
    return [
        W.params(lx=16, ly=16, lz=32, radius=3.0, kT=1e-5, g=1e-4, replica=0),
        W.params(lx=24, ly=24, lz=48, radius=4.0, kT=1e-4, g=5e-6, replica=1, delta_rho=0.3),
        W.params(lx=12, ly=10, lz=9, radius=0.0, kT=0.0, replica=2),
        W.params(lx=20, ly=12, lz=24, radius=2.5, kT=0.0, g=2e-5, replica=3, tau_s=0.8),
        W.params(lx=9, ly=20, lz=7, wall=(1, 0, 1), radius=0.0, kT=1e-5, tau_d=1.3, replica=4),
        W.params(lx=48, ly=48, lz=96, radius=6.0, kT=1e-6, g=1e-5, replica=5),
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


def _singles(flbm, plist, steps):
    """Single simulations in the ensemble's density mode (a density pass each
    step), so that members and singles do the same arithmetic."""
    out = []
    for p in plist:
        s = flbm.Sim(p)
        s.set_density_mode(0)
        s.step(steps)
        out.append((s.read_f(), s.particle()))
        s.close()
    return out


@pytest.fixture(scope="module")
def reference_runs(flbm):
    return _singles(flbm, _members(), 12)


@pytest.mark.parametrize("packing,ctas", [(0, 4), (1, 2), (2, 0), (1, 0)])
def test_members_equal_single_runs_bit_for_bit(flbm, reference_runs, packing, ctas):
    plist = _members()
    ens = flbm.Ensemble(plist, config=dict(packing=packing, ctas_per_sm=ctas, tile_policy=0))
    ens.step(5)
    ens.step(7)  # odd split: graph replays plus single steps
    parts = ens.particles()
    for r, p in enumerate(plist):
        f_ref, p_ref = reference_runs[r]
        fl = _fluid(p, p_ref["X"])
        assert np.array_equal(ens.read_f(r)[:, :, fl], f_ref[:, :, fl]), f"replica {r}"
        for k in ("X", "V", "Omega", "F", "T", "delta"):
            assert np.array_equal(parts[r][k], p_ref[k]), (r, k)
        assert parts[r]["step"] == 12
    ens.close()


def test_tile_policy_1_changes_only_rounding(flbm, reference_runs):
    plist = _members()
    ens = flbm.Ensemble(plist, config=dict(packing=0, ctas_per_sm=4, tile_policy=1))
    ens.step(12)
    parts = ens.particles()
    for r, p in enumerate(plist):
        f_ref, p_ref = reference_runs[r]
        fl = _fluid(p, p_ref["X"])
        g = ens.read_f(r)[:, :, fl].astype(np.float64)
        o = f_ref[:, :, fl].astype(np.float64)
        assert np.max(np.abs(g - o) / np.maximum(np.abs(o), 1e-6)) < 1e-5, f"replica {r}"
        if p["radius"] > 0:
            vs = max(np.max(np.abs(p_ref["V"])), 1e-12)
            assert np.max(np.abs(parts[r]["V"] - p_ref["V"])) <= 1e-6 * vs + 1e-14
    ens.close()


def test_member_matches_oracle(flbm, oracle_mod):
    """Replica 1 of a mixed ensemble against the FP64 oracle, 10 fluctuating steps."""
    plist = [W.channel_small(kT=0.0, replica=0), W.channel_small(kT=1e-5, g=1e-4, replica=7),
             W.params(lx=24, ly=24, lz=48, radius=4.0, kT=1e-5, replica=2)]
    ens = flbm.Ensemble(plist)
    orc = oracle_mod.Oracle(plist[1])
    ens.step(10)
    orc.step(10)
    fl = ~orc.fields()["solid"]
    g, o = ens.read_f(1)[:, :, fl].astype(np.float64), orc.get_f()[:, :, fl]
    scale = np.mean(np.abs(o), axis=-1, keepdims=True)
    assert np.max(np.abs(g - o) / scale) < 1e-5
    pg, po = ens.particles()[1], orc.particle()
    assert np.max(np.abs(pg["V"] - po["V"])) <= 1e-4 * np.max(np.abs(po["V"])) + 1e-12
    assert pg["nfluid"] == po["nfluid"]
    ens.close()


def test_launches_do_not_grow_with_replicas(flbm):
    small = flbm.Ensemble(_members()[:2])
    big = flbm.Ensemble(_members())
    small.step(4)
    big.step(4)
    assert big.launches() <= 4 * 15
    assert small.launches() <= big.launches()
    small.close()
    big.close()


def test_tuner_picks_a_config_and_resets_state(flbm, reference_runs):
    plist = _members()
    ens = flbm.Ensemble(plist)
    ens.step(3)
    cfg, ms = ens.tune(steps=2)
    assert ms > 0.0 and cfg == ens.config()
    assert all(p["step"] == 0 for p in ens.particles())
    ens.step(12)
    for r, p in enumerate(plist):
        f_ref, p_ref = reference_runs[r]
        fl = _fluid(p, p_ref["X"])
        g = ens.read_f(r)[:, :, fl]
        if cfg["tile_policy"] == 0:
            assert np.array_equal(g, f_ref[:, :, fl])
        else:
            assert np.max(np.abs(g - f_ref[:, :, fl]) / np.maximum(np.abs(f_ref[:, :, fl]), 1e-6)) < 1e-5
    ens.close()


@pytest.mark.slow
def test_full_ensemble_of_128_replicas(flbm):
    """The 128-replica workload: tuned, stepped, sampled members against their
    single runs, every member finite and at the same step."""
    plist = W.ensemble_members(128)
    ens = flbm.Ensemble(plist)
    cfg, _ = ens.tune(steps=2)
    ens.step(20)
    parts = ens.particles()
    assert all(p["step"] == 20 for p in parts)
    for r in (0, 37, 127):
        assert ens.observables(r)["nonfinite"] == 0
        s = flbm.Sim(plist[r])
        s.set_density_mode(0)  # the ensemble's density pass, so only the tile policy differs
        s.step(20)
        ps = s.particle()
        fl = _fluid(plist[r], ps["X"])
        f_ref = s.read_f()[:, :, fl].astype(np.float64)
        g = ens.read_f(r)[:, :, fl].astype(np.float64)
        assert np.max(np.abs(g - f_ref) / np.maximum(np.abs(f_ref), 1e-6)) < 1e-5
        assert np.max(np.abs(parts[r]["V"] - ps["V"])) <= 1e-6 * np.max(np.abs(ps["V"])) + 1e-14
        s.close()
    ens.close()
