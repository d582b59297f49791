"""Helpers of the GPU parity tests: run the CUDA path through the C ABI, compare with the
oracle under the tolerances of the method.

Tolerances:
  float32 destination: max |gpu - oracle| <= 1e-5 * sum|w| * max|x| (x the mapped source);
  integer destination: codes equal the oracle's, except where the oracle's pre-rounding
  code lies within 1e-3 LSB of a .5 tie (there either neighbouring code is accepted).
"""
import numpy as np

import oracle

FLOAT_TOL = 1e-5


def mapped_absmax(src: np.ndarray, lo: float, hi: float) -> float:
    if src.dtype == np.float32:
        return float(np.max(np.abs(src))) if src.size else 0.0
    qmax = 255.0 if src.dtype == np.uint8 else 65535.0
    q = src.astype(np.float64)
    return float(np.max(np.abs(lo + (hi - lo) * q / qmax))) if src.size else 0.0


def run_gpu(vkt, src: np.ndarray, filt, dst_dtype, src_range=(0.0, 1.0), dst_range=(0.0, 1.0),
            path="auto"):
    import torch
    s = torch.from_numpy(np.ascontiguousarray(src)).cuda()
    out = torch.empty(src.shape, dtype=dst_dtype, device="cuda")
    vkt.filter_tensor(s, filt, src_range=src_range, dst_range=dst_range, path=path, out=out)
    torch.cuda.synchronize()
    vkt.synchronize()
    return out.cpu().numpy()


def compare(gpu: np.ndarray, ref: np.ndarray, w, src: np.ndarray, src_range, dst_range,
            what: str = ""):
    """Asserts parity of gpu results (float or integer codes) with oracle values ref."""
    if gpu.dtype == np.float32:
        scale = oracle.error_scale(w, mapped_absmax(src, *src_range))
        scale = scale if scale > 0 else 1.0
        err = float(np.max(np.abs(gpu.astype(np.float64) - ref))) / scale if ref.size else 0.0
        assert err <= FLOAT_TOL, f"{what}: normalised error {err:.3e} > {FLOAT_TOL}"
        return err
    fmt = oracle.U8 if gpu.dtype == np.uint8 else oracle.U16
    t, q, tie = oracle.quantize(ref, fmt, *dst_range)
    g = gpu.astype(np.int64).ravel()
    q = q.astype(np.int64).ravel()
    tie = tie.ravel()
    bad = (g != q) & ~tie
    assert not bad.any(), (f"{what}: {int(bad.sum())} integer codes differ outside tie windows; "
                           f"first at {np.flatnonzero(bad)[:5]}, gpu {g[bad][:5]}, "
                           f"oracle {q[bad][:5]}, t {t.ravel()[bad][:5]}")
    tg = g[tie]
    qmax = 255 if fmt == oracle.U8 else 65535
    lo_ok = np.floor(t.ravel()[tie]).astype(np.int64)
    ok = (tg == np.clip(lo_ok, 0, qmax)) | (tg == np.clip(lo_ok + 1, 0, qmax))
    assert ok.all(), f"{what}: tie voxels outside the two neighbouring codes"
    return 0.0
