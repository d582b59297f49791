"""GB300 ApplyFilter: Python binding of the C ABI in include/vkt.h.

This module only marshals arguments: every step of the filter runs in the CUDA kernels of
libvkt.so.  PyTorch supplies device memory and streams.  Importing it loads (and if
needed builds) the library and raises if that fails; there is no CPU fallback.

Volumes are (nz, ny, nx) tensors, x fastest, of dtype uint8, uint16 or float32.
"""
from __future__ import annotations

import contextlib
import ctypes

import numpy as np

from . import _build
from ._lib import ExecutionPolicy, load

U8, U16, F32 = 0, 1, 2
PATH_AUTO, PATH_DIRECT, PATH_SEPARABLE, PATH_TENSOR = 0, 1, 2, 3
PATHS = {"auto": PATH_AUTO, "direct": PATH_DIRECT, "separable": PATH_SEPARABLE,
         "tensor": PATH_TENSOR}
MAX_FILTER_SIZE = 9

ERRORS = {0: "VKT_NO_ERROR", 1: "VKT_ERROR_INVALID_VALUE", 2: "VKT_ERROR_INVALID_HANDLE",
          3: "VKT_ERROR_DIMS_MISMATCH", 4: "VKT_ERROR_UNSUPPORTED",
          5: "VKT_ERROR_OUT_OF_MEMORY", 6: "VKT_ERROR_NO_DEVICE", 7: "VKT_ERROR_CUDA",
          8: "VKT_ERROR_DEVICE_TIMEOUT"}

_lib = load()


class VktError(RuntimeError):
    def __init__(self, code: int, what: str = ""):
        self.code = code
        msg = _lib.vktGetErrorString(code).decode()
        super().__init__(f"{ERRORS.get(code, code)}: {msg}" + (f" ({what})" if what else ""))


def check(code: int, what: str = "") -> None:
    if code != 0:
        raise VktError(code, what)


def build(force: bool = False) -> str:
    return _build.build(force=force)


def _torch():
    import torch
    return torch


def _fmt_of_dtype(dtype) -> int:
    torch = _torch()
    table = {torch.uint8: U8, torch.float32: F32}
    if hasattr(torch, "uint16"):
        table[torch.uint16] = U16
    if dtype not in table:
        raise TypeError(f"unsupported voxel dtype {dtype}")
    return table[dtype]


def torch_dtype(fmt: int):
    torch = _torch()
    return {U8: torch.uint8, U16: torch.uint16, F32: torch.float32}[fmt]


# ------------------------------------------------------------------ execution policy

def get_policy() -> ExecutionPolicy:
    pol = ExecutionPolicy()
    check(_lib.vktGetThreadExecutionPolicy(ctypes.byref(pol)))
    return pol


DEBUG_LOG = 1
DEBUG_INJECT_WAIT_TIMEOUT = 2


def set_policy(stream=None, path=None, debug=None, print_times=None) -> None:
    """Sets the calling thread's policy.  stream None: torch's current stream; path, debug,
    print_times None: keep the current setting.  debug: True for DEBUG_LOG, or an int of
    DEBUG_* bits."""
    pol = get_policy()
    pol.stream = ctypes.c_void_p(_stream_handle(stream))
    if path is not None:
        pol.path = PATHS[path] if isinstance(path, str) else int(path)
    if debug is not None:
        pol.debug = int(debug)
    if print_times is not None:
        pol.printTimes = int(bool(print_times))
    check(_lib.vktSetThreadExecutionPolicy(pol))


@contextlib.contextmanager
def policy(stream=None, path=None, debug=None, print_times=None):
    """Temporarily sets the calling thread's execution policy (None: keep the setting)."""
    old = get_policy()
    set_policy(stream, path, debug, print_times)
    try:
        yield
    finally:
        check(_lib.vktSetThreadExecutionPolicy(old))


def _stream_handle(stream) -> int:
    if stream is None:
        torch = _torch()
        return int(torch.cuda.current_stream().cuda_stream) if torch.cuda.is_available() else 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)


def synchronize() -> None:
    """Waits for the policy stream; raises on a device-side timeout or CUDA error."""
    check(_lib.vktSynchronize(), "vktSynchronize")


def launch_count() -> int:
    n = ctypes.c_uint64()
    check(_lib.vktGetLaunchCount(ctypes.byref(n)))
    return int(n.value)


# ------------------------------------------------------------------ volumes

class StructuredVolume:
    """A structured volume handle (owning, or a view of a torch tensor)."""

    def __init__(self, handle: ctypes.c_void_p, tensor=None):
        self._h = handle
        self.tensor = tensor          # keeps a viewed tensor alive

    @classmethod
    def create(cls, dims, fmt: int, cell=(1.0, 1.0, 1.0), lo: float = 0.0, hi: float = 1.0):
        h = ctypes.c_void_p()
        nx, ny, nz = dims
        check(_lib.vktStructuredVolumeCreate(ctypes.byref(h), nx, ny, nz, fmt, *cell, lo, hi),
              "vktStructuredVolumeCreate")
        return cls(h)

    @classmethod
    def from_tensor(cls, t, lo: float = 0.0, hi: float = 1.0, cell=(1.0, 1.0, 1.0)):
        if t.dim() != 3 or not t.is_contiguous() or not t.is_cuda:
            raise ValueError("volume tensors are contiguous CUDA tensors of shape (nz, ny, nx)")
        nz, ny, nx = t.shape
        h = ctypes.c_void_p()
        check(_lib.vktStructuredVolumeCreateView(ctypes.byref(h), ctypes.c_void_p(t.data_ptr()),
                                                 nx, ny, nz, _fmt_of_dtype(t.dtype), *cell, lo,
                                                 hi), "vktStructuredVolumeCreateView")
        return cls(h, t)

    @property
    def handle(self):
        return self._h

    @property
    def dims(self):
        a, b, c = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        check(_lib.vktStructuredVolumeGetDims(self._h, ctypes.byref(a), ctypes.byref(b),
                                              ctypes.byref(c)))
        return (a.value, b.value, c.value)

    @property
    def format(self) -> int:
        f = ctypes.c_int()
        check(_lib.vktStructuredVolumeGetDataFormat(self._h, ctypes.byref(f)))
        return f.value

    @property
    def cell_size(self):
        a, b, c = ctypes.c_float(), ctypes.c_float(), ctypes.c_float()
        check(_lib.vktStructuredVolumeGetCellSize(self._h, ctypes.byref(a), ctypes.byref(b),
                                                  ctypes.byref(c)))
        return (a.value, b.value, c.value)

    @property
    def mapping(self):
        lo, hi = ctypes.c_float(), ctypes.c_float()
        check(_lib.vktStructuredVolumeGetVoxelMapping(self._h, ctypes.byref(lo), ctypes.byref(hi)))
        return (lo.value, hi.value)

    def set_mapping(self, lo: float, hi: float) -> None:
        check(_lib.vktStructuredVolumeSetVoxelMapping(self._h, lo, hi))

    @property
    def data_ptr(self) -> int:
        d = ctypes.c_void_p()
        check(_lib.vktStructuredVolumeGetData(self._h, ctypes.byref(d)))
        return int(d.value or 0)

    @property
    def nbytes(self) -> int:
        n = ctypes.c_uint64()
        check(_lib.vktStructuredVolumeGetSizeInBytes(self._h, ctypes.byref(n)))
        return int(n.value)

    def set_data(self, host: np.ndarray) -> None:
        """Asynchronous host-to-device copy of all voxels (keep `host` alive until synced)."""
        host = np.ascontiguousarray(host)
        if host.nbytes != self.nbytes:
            raise ValueError("host array size does not match the volume")
        check(_lib.vktStructuredVolumeSetData(self._h, ctypes.c_void_p(host.ctypes.data)))

    def copy_to_host(self, out: np.ndarray) -> None:
        if not out.flags["C_CONTIGUOUS"] or out.nbytes != self.nbytes:
            raise ValueError("output array must be contiguous and match the volume size")
        check(_lib.vktStructuredVolumeCopyToHost(self._h, ctypes.c_void_p(out.ctypes.data)))

    def destroy(self) -> None:
        if self._h is not None and self._h.value:
            check(_lib.vktStructuredVolumeDestroy(self._h))
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ------------------------------------------------------------------ filters

def _fptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


class Filter:
    """A k x k x k filter (dense, separable or Gaussian)."""

    def __init__(self, handle):
        self._h = handle

    @classmethod
    def dense(cls, w):
        w = np.ascontiguousarray(w, dtype=np.float32)
        k = round(w.size ** (1 / 3))
        if k ** 3 != w.size:
            raise ValueError("dense weights hold k^3 values")
        h = ctypes.c_void_p()
        check(_lib.vktFilterCreate(ctypes.byref(h), k, _fptr(w)), "vktFilterCreate")
        return cls(h)

    @classmethod
    def separable(cls, gx, gy, gz):
        gx, gy, gz = (np.ascontiguousarray(g, dtype=np.float32) for g in (gx, gy, gz))
        h = ctypes.c_void_p()
        check(_lib.vktFilterCreateSeparable(ctypes.byref(h), gx.size, _fptr(gx), _fptr(gy),
                                            _fptr(gz)), "vktFilterCreateSeparable")
        return cls(h)

    @classmethod
    def gaussian(cls, k: int, sigma: float):
        h = ctypes.c_void_p()
        check(_lib.vktFilterCreateGaussian(ctypes.byref(h), k, sigma), "vktFilterCreateGaussian")
        return cls(h)

    @property
    def handle(self):
        return self._h

    @property
    def k(self) -> int:
        k = ctypes.c_int32()
        check(_lib.vktFilterGetSize(self._h, ctypes.byref(k)))
        return k.value

    @property
    def is_separable(self) -> bool:
        s = ctypes.c_int32()
        check(_lib.vktFilterIsSeparable(self._h, ctypes.byref(s)))
        return bool(s.value)

    def weights(self) -> np.ndarray:
        k = self.k
        w = np.empty((k, k, k), np.float32)
        check(_lib.vktFilterGetWeights(self._h, _fptr(w)))
        return w

    def separable_weights(self):
        k = self.k
        g = [np.empty(k, np.float32) for _ in range(3)]
        check(_lib.vktFilterGetSeparableWeights(self._h, *(_fptr(x) for x in g)))
        return tuple(g)

    def set_weights(self, w) -> None:
        w = np.ascontiguousarray(w, dtype=np.float32)
        if w.size != self.k ** 3:
            raise ValueError("dense weights hold k^3 values")
        check(_lib.vktFilterSetWeights(self._h, _fptr(w)))

    def normalize(self) -> None:
        check(_lib.vktFilterNormalize(self._h), "vktFilterNormalize")

    def destroy(self) -> None:
        if self._h is not None and self._h.value:
            check(_lib.vktFilterDestroy(self._h))
        self._h = None

    def __del__(self):
        try:
            self.destroy()
        except Exception:
            pass


# ------------------------------------------------------------------ ApplyFilter

def apply_filter(dst: StructuredVolume, src: StructuredVolume, filt: Filter, path=None,
                 stream=None, roi=None) -> None:
    """Enqueues dst = filter(src) on `stream` (default: torch's current stream); path None
    keeps the thread policy's path.  roi ((x0, y0, z0), (x1, y1, z1)): only the voxels of
    that half-open box are written (vktApplyFilterRangeSV)."""
    with policy(stream=stream, path=path):
        if roi is None:
            check(_lib.vktApplyFilterSV(dst.handle, src.handle, filt.handle), "vktApplyFilterSV")
        else:
            (x0, y0, z0), (x1, y1, z1) = roi
            check(_lib.vktApplyFilterRangeSV(dst.handle, src.handle, filt.handle, int(x0), int(y0),
                                             int(z0), int(x1), int(y1), int(z1)),
                  "vktApplyFilterRangeSV")


def apply_filter_batch(dsts, srcs, filters, stream=None) -> None:
    n = len(dsts)
    if not (len(srcs) == n == len(filters)):
        raise ValueError("dsts, srcs and filters must have the same length")
    arr = ctypes.c_void_p * n
    d = arr(*(v.handle.value for v in dsts))
    s = arr(*(v.handle.value for v in srcs))
    f = arr(*(x.handle.value for x in filters))
    with policy(stream=stream):
        check(_lib.vktApplyFilterBatchSV(n, d, s, f), "vktApplyFilterBatchSV")


def apply_filter_backward(grad_src, grad_weights, grad_dst: StructuredVolume,
                          src: StructuredVolume, filt: Filter, stream=None) -> None:
    """grad_src: StructuredVolume or None; grad_weights: float32 CUDA tensor (k^3) or None."""
    gs = grad_src.handle if grad_src is not None else None
    gw = ctypes.c_void_p(grad_weights.data_ptr()) if grad_weights is not None else None
    with policy(stream=stream):
        check(_lib.vktApplyFilterBackwardSV(gs, gw, grad_dst.handle, src.handle, filt.handle),
              "vktApplyFilterBackwardSV")


def apply_filter_backward_batch(grad_srcs, grad_weights, grad_dsts, srcs, filt: Filter,
                                stream=None) -> None:
    """vktApplyFilterBackwardBatchSV: grad_srcs a list of StructuredVolume or None;
    grad_weights a float32 CUDA tensor of k^3 entries (dL/dw summed over the batch) or None."""
    n = len(srcs)
    if len(grad_dsts) != n or (grad_srcs is not None and len(grad_srcs) != n):
        raise ValueError("grad_srcs, grad_dsts and srcs must have the same length")
    arr = ctypes.c_void_p * n
    gs = arr(*(v.handle.value for v in grad_srcs)) if grad_srcs is not None else None
    gd = arr(*(v.handle.value for v in grad_dsts))
    sv = arr(*(v.handle.value for v in srcs))
    gw = ctypes.c_void_p(grad_weights.data_ptr()) if grad_weights is not None else None
    with policy(stream=stream):
        check(_lib.vktApplyFilterBackwardBatchSV(n, gs, gw, gd, sv, filt.handle),
              "vktApplyFilterBackwardBatchSV")


def brick_counts(src: StructuredVolume, brick) -> tuple:
    """(countX, countY, countZ) of vktBrickDecomposeCountSV for brick = (bx, by, bz)."""
    c = [ctypes.c_int32() for _ in range(3)]
    check(_lib.vktBrickDecomposeCountSV(*(ctypes.byref(x) for x in c), src.handle, *map(int, brick)),
          "vktBrickDecomposeCountSV")
    return tuple(x.value for x in c)


def brick_decompose(src_t, brick, ghost: int = 0, src_range=(0.0, 1.0), stream=None):
    """BrickDecompose of a (nz, ny, nx) CUDA tensor: allocates the bricks as tensors of the
    source dtype and fills them with vktBrickDecomposeSV.  Returns them in the order
    (kz, ky, kx), kx fastest."""
    torch = _torch()
    src = StructuredVolume.from_tensor(src_t, *src_range)
    cx, cy, cz = brick_counts(src, brick)
    nz, ny, nx = src_t.shape
    bx, by, bz = map(int, brick)
    tensors, views = [], []
    for kz in range(cz):
        for ky in range(cy):
            for kx in range(cx):
                shape = (min(bz, nz - kz * bz) + 2 * ghost, min(by, ny - ky * by) + 2 * ghost,
                         min(bx, nx - kx * bx) + 2 * ghost)
                t = torch.empty(shape, dtype=src_t.dtype, device=src_t.device)
                tensors.append(t)
                views.append(StructuredVolume.from_tensor(t, *src_range))
    arr = (ctypes.c_void_p * len(views))(*(v.handle.value for v in views))
    with policy(stream=stream):
        check(_lib.vktBrickDecomposeSV(arr, len(views), src.handle, bx, by, bz, int(ghost)),
              "vktBrickDecomposeSV")
    return tensors


class RenderParams(ctypes.Structure):
    _fields_ = [("eye", ctypes.c_float * 3), ("center", ctypes.c_float * 3), ("up", ctypes.c_float * 3),
                ("fovy", ctypes.c_float), ("step", ctypes.c_float), ("termination", ctypes.c_float),
                ("background", ctypes.c_float * 4), ("lutSize", ctypes.c_int32),
                ("lut", ctypes.POINTER(ctypes.c_float))]


def render(src_t, width: int, height: int, eye, center, up, fovy: float, step: float, lut,
           termination: float = 2.0, background=(0.0, 0.0, 0.0, 0.0), src_range=(0.0, 1.0),
           out=None, stream=None):
    """Headless ray marching of a (nz, ny, nx) CUDA volume tensor (vktRenderSV): returns an
    (height, width, 4) float32 CUDA tensor.  lut: (n, 4) straight RGBA transfer function."""
    import numpy as _np
    torch = _torch()
    table = _np.ascontiguousarray(_np.asarray(lut, dtype=_np.float32).reshape(-1, 4))
    if out is None:
        out = torch.empty((height, width, 4), dtype=torch.float32, device=src_t.device)
    vol = StructuredVolume.from_tensor(src_t, *src_range)
    prm = RenderParams()
    prm.eye[:] = [float(x) for x in eye]
    prm.center[:] = [float(x) for x in center]
    prm.up[:] = [float(x) for x in up]
    prm.fovy, prm.step, prm.termination = float(fovy), float(step), float(termination)
    prm.background[:] = [float(x) for x in background]
    prm.lutSize = table.shape[0]
    prm.lut = table.ctypes.data_as(ctypes.POINTER(ctypes.c_float))
    with policy(stream=stream):
        check(_lib.vktRenderSV(ctypes.c_void_p(out.data_ptr()), int(width), int(height), vol.handle,
                               ctypes.cast(ctypes.pointer(prm), ctypes.c_void_p)), "vktRenderSV")
    return out


def clahe3d(src_t, bricks, clip_limit: float, out=None, stream=None):
    """CLAHE-3D of a (nz, ny, nx) uint8 CUDA tensor (vktClahe3DSV); bricks = (bx, by, bz)
    bricks per axis dividing the dims.  Returns the uint8 result tensor."""
    torch = _torch()
    if out is None:
        out = torch.empty_like(src_t)
    src = StructuredVolume.from_tensor(src_t)
    dst = StructuredVolume.from_tensor(out)
    with policy(stream=stream):
        check(_lib.vktClahe3DSV(dst.handle, src.handle, *map(int, bricks), float(clip_limit)),
              "vktClahe3DSV")
    return out


def filter_tensor(src_t, filt: Filter, dst_dtype=None, src_range=(0.0, 1.0),
                  dst_range=(0.0, 1.0), path=None, out=None, roi=None):
    """Convenience: filters a (nz, ny, nx) CUDA tensor and returns the result tensor (roi:
    see apply_filter; voxels outside it keep the contents of `out`)."""
    torch = _torch()
    if out is None:
        out = torch.empty(src_t.shape, dtype=dst_dtype or torch.float32, device=src_t.device)
    src = StructuredVolume.from_tensor(src_t, *src_range)
    dst = StructuredVolume.from_tensor(out, *dst_range)
    apply_filter(dst, src, filt, path=path, roi=roi)
    return out


# ------------------------------------------------------------------ autograd

def _autograd_function():
    import torch

    class ApplyFilterFunction(torch.autograd.Function):
        """y = ApplyFilter(x, w) for float32 volumes x of shape (nz, ny, nx) or (B, nz, ny, nx)
        and a dense k^3 float32 kernel w.  Forward: vktApplyFilterBatchSV with one filter over
        the batch (one launch on the direct path).  Backward: vktApplyFilterBackwardBatchSV
        (exact adjoint for dL/dx, dL/dw summed over the batch and reduced in FP64 inside the
        library).  The kernel reads the weights as launch constants, so the forward copies w
        to the host once per step; the backward reuses that copy."""

        @staticmethod
        def forward(ctx, x, w, path="auto"):
            if x.dtype != torch.float32 or w.dtype != torch.float32:
                raise TypeError("ApplyFilterFunction takes float32 volumes and weights")
            xb = x.contiguous().reshape((-1,) + tuple(x.shape[-3:]))
            w_host = w.detach().float().cpu().numpy()
            filt = Filter.dense(w_host)
            y = torch.empty_like(xb)
            vx = [StructuredVolume.from_tensor(xb[b]) for b in range(xb.shape[0])]
            vy = [StructuredVolume.from_tensor(y[b]) for b in range(xb.shape[0])]
            with policy(path=path):
                apply_filter_batch(vy, vx, [filt] * len(vx))
            ctx.save_for_backward(xb)
            ctx.filt = filt
            ctx.w_shape = w.shape
            ctx.shape = x.shape
            return y.reshape(x.shape)

        @staticmethod
        def backward(ctx, gy):
            (xb,) = ctx.saved_tensors
            gyb = gy.contiguous().reshape(xb.shape)
            need_x, need_w = ctx.needs_input_grad[0], ctx.needs_input_grad[1]
            gx = torch.empty_like(xb) if need_x else None
            k3 = 1
            for d in ctx.w_shape:
                k3 *= d
            gw = torch.empty(k3, dtype=torch.float32, device=xb.device) if need_w else None
            n = xb.shape[0]
            apply_filter_backward_batch(
                [StructuredVolume.from_tensor(gx[b]) for b in range(n)] if need_x else None, gw,
                [StructuredVolume.from_tensor(gyb[b]) for b in range(n)],
                [StructuredVolume.from_tensor(xb[b]) for b in range(n)], ctx.filt)
            return ((gx.reshape(ctx.shape) if need_x else None),
                    (gw.reshape(ctx.w_shape) if need_w else None), None)

    return ApplyFilterFunction


_APPLY_FN = None


def apply_filter_autograd(x, w, path="auto"):
    """Differentiable ApplyFilter on float32 CUDA tensors (see ApplyFilterFunction)."""
    global _APPLY_FN
    if _APPLY_FN is None:
        _APPLY_FN = _autograd_function()
    return _APPLY_FN.apply(x, w, path)
