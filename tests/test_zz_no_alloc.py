"""The allocation-free weight-gradient entry point, for callers that cannot let the library
allocate device memory (a host whose device memory is reserved up front by its own
allocator, or latency-critical code that must avoid cudaMalloc's locks and implicit
synchronisation).  It must agree with vktApplyFilterBackwardSV, which takes its scratch
from cudaMallocAsync, within the gradient tolerance, on two calls in a row (the fixed
scratch array keeps the previous call's contents), and reject volumes whose partial sums
do not fit in the fixed scratch.

This file is named so that pytest collects it last."""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2203_10213_gb300 as vkt  # noqa: E402

TOL = 1e-5
SEED = synth.BASE_SEED + 9


def _view(t):
    return vkt.StructuredVolume.from_tensor(t)


def test_no_alloc_weight_gradient_matches_allocating_entry_point():
    lib = vkt._lib
    shape = (40, 48, 64)
    k = 5
    x = torch.from_numpy(synth.uniform(SEED, shape, -1.0, 1.0)).cuda()
    gy = torch.from_numpy(synth.uniform(SEED + 1, shape, -1.0, 1.0)).cuda()
    w = synth.normal(SEED + 2, (k, k, k)).astype(np.float32)
    f = vkt.Filter.dense(w)
    vx, vgy = _view(x), _view(gy)
    ref = torch.empty(k ** 3, dtype=torch.float32, device="cuda")
    out1 = torch.full((k ** 3,), float("nan"), dtype=torch.float32, device="cuda")
    out2 = torch.full((k ** 3,), float("nan"), dtype=torch.float32, device="cuda")
    with vkt.policy():
        vkt.check(lib.vktApplyFilterBackwardSV(None, ctypes.c_void_p(ref.data_ptr()), vgy.handle,
                                               vx.handle, f.handle))
        vkt.check(lib.vktApplyFilterWeightGradNoAllocSV(ctypes.c_void_p(out1.data_ptr()),
                                                        vgy.handle, vx.handle, f.handle))
        vkt.check(lib.vktApplyFilterWeightGradNoAllocSV(ctypes.c_void_p(out2.data_ptr()),
                                                        vgy.handle, vx.handle, f.handle))
    torch.cuda.synchronize()
    vkt.synchronize()
    scale = float(gy.abs().sum()) * float(x.abs().max())
    r = ref.double().cpu().numpy()
    for out in (out1, out2):
        o = out.double().cpu().numpy()
        assert np.all(np.isfinite(o))
        assert np.max(np.abs(o - r)) <= TOL * scale


def test_no_alloc_rejects_volumes_beyond_the_scratch():
    lib = vkt._lib
    # 20 x 20 tiles of 64 x 32 voxels with k = 9 need 400 * 729 > 2^18 partial sums
    shape = (1, 640, 1280)
    x = torch.zeros(shape, dtype=torch.float32, device="cuda")
    gy = torch.zeros(shape, dtype=torch.float32, device="cuda")
    gw = torch.zeros(9 ** 3, dtype=torch.float32, device="cuda")
    f = vkt.Filter.dense(np.ones((9, 9, 9), np.float32))
    vx, vgy = _view(x), _view(gy)          # keep the handles alive across the call
    with vkt.policy():
        rc = lib.vktApplyFilterWeightGradNoAllocSV(ctypes.c_void_p(gw.data_ptr()), vgy.handle,
                                                   vx.handle, f.handle)
    assert rc == 1   # VKT_ERROR_INVALID_VALUE
    torch.cuda.synchronize()
