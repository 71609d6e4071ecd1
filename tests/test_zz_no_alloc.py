"""The observables entry point that allocates nothing, against flbm_observables.

flbm_observables_noalloc serves callers that cannot allocate device memory:
code whose device memory belongs to a pool or arena, host plugins that must
not call cudaMalloc or cudaFree. Its per-tile partial sums live in a static
device array of the library instead. Its result must match the handle-based
flbm_observables on the same populations, on two calls in a row (the second
call reuses the static array the first one filled).

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

from paper_1909_01092_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RTOL = 1e-5  # the tolerance of the parity tests


def _call(lib, binding, p, f_dev, out_dev, stream):
    s = binding.to_params(p)
    return lib.flbm_observables_noalloc(ctypes.byref(s), ctypes.c_void_p(f_dev), ctypes.c_void_p(out_dev),
                                        ctypes.c_void_p(stream))


def test_noalloc_observables_match_handle_entry_point():
    import torch
    from paper_1909_01092_gb300 import binding

    assert torch.cuda.is_available(), "needs a GPU"
    lib = binding.load()
    p = W.params(lx=40, ly=24, lz=20, wall=(1, 1, 0), G=1.2, kT=1e-5, init_pert=0.05)  # no particle
    sim = binding.Sim(p)
    stream = torch.cuda.current_stream()
    out = torch.full((8,), float("nan"), dtype=torch.float64, device="cuda")
    for _ in range(2):
        sim.step(7)
        ref = sim.observables()
        f = torch.from_numpy(sim.read_f()).cuda()
        assert _call(lib, binding, p, f.data_ptr(), out.data_ptr(), stream.cuda_stream) == 0
        torch.cuda.synchronize()
        v = out.cpu().numpy()
        assert np.allclose(v[0:2], ref["mass"], rtol=RTOL, atol=0)
        scale = float(ref["mass"].sum())
        assert np.allclose(v[2:5], ref["momentum"], rtol=RTOL, atol=RTOL * 1e-6 * scale)
        assert abs(v[5] - ref["kinetic"]) <= RTOL * abs(ref["kinetic"])
        assert v[6] == 0 and ref["nonfinite"] == 0
    sim.close()


def test_noalloc_rejects_what_it_cannot_serve():
    import torch
    from paper_1909_01092_gb300 import binding

    lib = binding.load()
    stream = torch.cuda.current_stream().cuda_stream
    dummy = torch.zeros(16, dtype=torch.float64, device="cuda")
    too_big = W.params(lx=128, ly=128, lz=1024, wall=(1, 1, 0))  # 65536 tiles > the static scratch
    assert _call(lib, binding, too_big, dummy.data_ptr(), dummy.data_ptr(), stream) == -1
    with_particle = W.channel_small()
    assert _call(lib, binding, with_particle, dummy.data_ptr(), dummy.data_ptr(), stream) == -6
