"""Runtime services of the C-ABI on the GPU: checkpoint/restore and CUDA-graph
replay of the step. Both must reproduce plain stepping bit for bit."""
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


def _fluid(p, X):
    """Boolean [lz, ly, lx] mask of nodes outside the sphere centred at X."""
    z, y, x = np.meshgrid(np.arange(p["lz"]), np.arange(p["ly"]), np.arange(p["lx"]), indexing="ij")
    r2 = np.zeros(x.shape)
    for c, a, L, w in ((x, 0, p["lx"], p["wall"][0]), (y, 1, p["ly"], p["wall"][1]), (z, 2, p["lz"], p["wall"][2])):
        d = c - X[a]
        if not w:
            d = (d + 0.5 * L) % L - 0.5 * L
        r2 = r2 + d * d
    return r2 >= p["radius"] ** 2


def _same_state(a, b, p):
    pa, pb = a.particle(), b.particle()
    for k in ("X", "V", "Omega", "F", "T", "P_pending", "L_pending", "delta"):
        assert np.array_equal(pa[k], pb[k]), k
    assert pa["step"] == pb["step"] and pa["nfluid"] == pb["nfluid"]
    fl = _fluid(p, pa["X"]) if p["radius"] > 0 else np.ones((p["lz"], p["ly"], p["lx"]), bool)
    fa, fb = a.read_f(), b.read_f()
    assert np.array_equal(fa[:, :, fl], fb[:, :, fl])


@pytest.mark.parametrize("kT", [0.0, 1e-5])
def test_restore_continues_bit_for_bit(flbm, tmp_path, kT):
    p = W.channel_small(kT=kT, g=1e-4)
    a = flbm.Sim(p)
    a.step(7)
    path = tmp_path / "state.ckpt"
    a.checkpoint(path)
    a.step(13)
    b = flbm.Sim(p)
    b.restore(path)
    assert b.particle()["step"] == 7
    b.step(13)
    _same_state(a, b, p)


def test_restore_keeps_the_handles_physics(flbm, tmp_path):
    """Layout must match; kT, G and forces follow the restoring handle."""
    p = W.channel_small(kT=0.0)
    a = flbm.Sim(p)
    a.step(3)
    path = tmp_path / "s.ckpt"
    a.checkpoint(path)
    hot = flbm.Sim(dict(p, kT=1e-4, seed=99))
    hot.restore(path)
    hot.step(2)
    assert hot.observables()["nonfinite"] == 0
    with pytest.raises(flbm.FLBMError):
        flbm.Sim(dict(p, lz=p["lz"] + 2)).restore(path)
    with pytest.raises(flbm.FLBMError):
        flbm.Sim(dict(p, radius=p["radius"] + 1.0)).restore(path)
    bad = tmp_path / "bad.ckpt"
    bad.write_bytes(path.read_bytes()[:1000])
    with pytest.raises(flbm.FLBMError):
        flbm.Sim(p).restore(bad)


@pytest.mark.parametrize("radius", [0.0, 3.0])
def test_graph_replay_equals_plain_launches(flbm, radius):
    import torch

    p = W.channel_small(kT=1e-5, radius=radius)
    plain = flbm.Sim(p)
    plain.step(13)
    per_step = plain.launches() // 13
    g = flbm.Sim(p, stream=torch.cuda.Stream())
    g.use_graphs(True)
    g.step(10)
    assert g.launches() == 10 * per_step
    g.step(3)  # fewer steps than a graph holds: plain launches
    torch.cuda.synchronize()
    _same_state(plain, g, p)


def test_run_host_in_graphs_records_every_step(flbm):
    """flbm_run_host with graph replay: each captured step is followed by a
    kernel that writes its particle record into the next slot of the
    trajectory buffer. The final populations and every step's record must
    equal plain stepping, step by step, in a first call, in a second one
    (the record count starts again) and in a longer third one (a larger
    record buffer, so the recording graphs are captured again)."""
    import torch

    p = W.channel_small(kT=1e-5, radius=3.0)
    ref = flbm.Sim(p)
    g = flbm.Sim(p, stream=torch.cuda.Stream())
    g.use_graphs(True)
    f = ref.read_f()
    keys = ("X", "V", "Omega", "F", "T", "delta", "step", "nfluid")
    for n in (21, 13, 37):  # graphs of 8 steps and a plain rest
        out = np.empty_like(f)
        traj = g.run_host(f, n, f_out=out, traj=True)
        torch.cuda.synchronize()
        assert len(traj) == n
        for k in range(n):
            ref.step(1)
            pr = ref.particle()
            for key in keys:
                assert np.array_equal(np.asarray(pr[key]), np.asarray(traj[k][key])), (n, k, key)
        assert np.array_equal(ref.read_f(), out)
        f = out


def test_graphs_refused_on_the_legacy_stream(flbm):
    import torch

    s = flbm.Sim(W.channel_small(), stream=torch.cuda.default_stream())
    if s.stream.cuda_stream != 0:
        pytest.skip("default stream is not the legacy stream here")
    with pytest.raises(flbm.FLBMError):
        s.use_graphs(True)


def test_legacy_default_stream_equals_another_stream(flbm):
    """The near-particle collide forks to a second stream and joins back by
    events; that must hold on the legacy default stream too."""
    import torch

    p = W.channel_small(kT=1e-5, g=1e-4)
    a = flbm.Sim(p, stream=torch.cuda.default_stream())
    b = flbm.Sim(p, stream=torch.cuda.Stream())
    a.step(9)
    b.step(9)
    torch.cuda.synchronize()
    _same_state(a, b, p)


def test_restore_refuses_a_corrupt_particle_record(flbm, tmp_path):
    """A checkpoint whose particle record is corrupt (a non-finite centre, a
    mask index other than 0 or 1) is refused with FLBM_E_INVAL before any of
    it reaches the device; the handle still restores a good file afterwards
    and continues bit for bit."""
    import ctypes
    import struct

    p = W.channel_small(kT=1e-5, g=1e-4)
    a = flbm.Sim(p)
    a.step(5)
    path = tmp_path / "good.ckpt"
    a.checkpoint(path)
    raw = bytearray(path.read_bytes())
    head = 80  # the file's fixed header
    state = head + ctypes.sizeof(flbm.Params)  # the particle record starts with X[3]
    bad = bytearray(raw)
    bad[state:state + 8] = struct.pack("<d", float("nan"))
    (tmp_path / "nan.ckpt").write_bytes(bytes(bad))
    b = flbm.Sim(p)
    with pytest.raises(flbm.FLBMError, match="FLBM_E_INVAL"):
        b.restore(tmp_path / "nan.ckpt")
    b.restore(path)
    a.step(4)
    b.step(4)
    _same_state(a, b, p)
