"""FP64 CPU oracle for ApplyFilter -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py``
may import this package.  The CUDA library never calls it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C loops, double precision, the definition
of the filtered value written out voxel by voxel; see the header there for the readings
of the paper it takes).  This module compiles it with gcc and wraps it for numpy.

Pins (tests/test_oracle.py): identity kernel, constant volume, linearity in input and
kernel, separable kernel = three 1-D clamped passes, hand-derived closed forms on small
volumes (tests/golden), scipy.ndimage.correlate(mode="nearest") and torch float64
replicate-padded conv3d, the adjoint dot-product identity, and central finite
differences of a quadratic loss.  ``brick_decompose`` (index arithmetic only, in numpy) is
pinned by exact reassembly, neighbour agreement and face replication.  ``clahe3d`` is
pinned by plain histogram equalisation (one brick, no clip), count conservation under the
clip limit, brick centres taking their own mapping, scipy's linear interpolation of the
mappings, and a constant volume.  ``render`` / ``render_pixels`` are pinned by the
background through a transparent volume, Beer-Lambert attenuation through a uniform slab,
early termination, linear blending of the lookup table, camera orientation and rays that
miss the volume.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

U8, U16, F32 = 0, 1, 2
BITS = {U8: 8, U16: 16}
TIE_WINDOW = 1e-3   # LSB; integer results this close to a .5 tie accept either code


def build(force: bool = False) -> str:
    src = os.path.join(_HERE, "oracle.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fno-fast-math", "-ffp-contract=off", "-shared", "-fPIC",
           "-std=c11", src, "-o", tmp, "-lm"]
    try:
        subprocess.run(cmd[:1] + ["-fopenmp"] + cmd[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(cmd, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            p, i64, d, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
            lib.oracle_correlate.restype = i32
            lib.oracle_correlate.argtypes = [p, i32, d, d, i64, i64, i64, p, i32, p]
            lib.oracle_correlate_points.restype = i32
            lib.oracle_correlate_points.argtypes = [p, i32, d, d, i64, i64, i64, p, i32, p, i64, p]
            lib.oracle_quantize.restype = i32
            lib.oracle_quantize.argtypes = [p, i64, i32, d, d, d, p, p, p]
            lib.oracle_gaussian_1d.restype = i32
            lib.oracle_gaussian_1d.argtypes = [i32, d, p]
            lib.oracle_separable_weights.restype = None
            lib.oracle_separable_weights.argtypes = [i32, p, p, p, p]
            lib.oracle_correlate_backward.restype = i32
            lib.oracle_correlate_backward.argtypes = [p, p, i64, i64, i64, p, i32, p, p]
            lib.oracle_backward_input_points.restype = i32
            lib.oracle_backward_input_points.argtypes = [p, i64, i64, i64, p, i32, p, i64, p]
            lib.oracle_num_threads.restype = i32
            lib.oracle_set_num_threads.restype = None
            lib.oracle_set_num_threads.argtypes = [i32]
            lib.oracle_render.restype = i32
            lib.oracle_render.argtypes = [p, i32, d, d, i64, i64, i64, i32, i32, p, p, p, d, d, d,
                                          p, i32, p, p]
            lib.oracle_render_pixels.restype = i32
            lib.oracle_render_pixels.argtypes = [p, i32, d, d, i64, i64, i64, i32, i32, p, p, p, d, d,
                                                 d, p, i32, p, p, i64, p]
            lib.oracle_clahe3d.restype = i32
            lib.oracle_clahe3d.argtypes = [p, i64, i64, i64, i32, i32, i32, d, p, p, p]
            _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _fmt_of(vol: np.ndarray) -> int:
    if vol.dtype == np.uint8:
        return U8
    if vol.dtype == np.uint16:
        return U16
    if vol.dtype == np.float32:
        return F32
    raise TypeError(f"unsupported voxel type {vol.dtype}")


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the oracle's parallel loops (timing only; results do not depend on it)."""
    _load().oracle_set_num_threads(int(n))


def dense_weights(w) -> np.ndarray:
    """k^3 weights as float64 (k, k, k) array, index [c][b][a] (a = x offset)."""
    w = np.asarray(w)
    k = round(w.size ** (1.0 / 3.0))
    if k ** 3 != w.size:
        raise ValueError("weights must hold k^3 values")
    return _c(w, np.float64).reshape(k, k, k)


def correlate(src: np.ndarray, w, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    """Filtered values (float64, same shape as src (nz, ny, nx)) of the clamp-to-edge
    correlation of the mapped source with the k^3 weights ``w``."""
    src = np.ascontiguousarray(src)
    fmt = _fmt_of(src)
    wd = dense_weights(w)
    k = wd.shape[0]
    nz, ny, nx = src.shape
    out = np.empty(src.shape, dtype=np.float64)
    rc = _load().oracle_correlate(_ptr(src), fmt, lo, hi, nx, ny, nz, _ptr(wd), k, _ptr(out))
    if rc:
        raise ValueError(f"oracle_correlate rejected its arguments ({rc})")
    return out


def correlate_points(src: np.ndarray, w, idx, lo: float = 0.0, hi: float = 1.0) -> np.ndarray:
    src = np.ascontiguousarray(src)
    fmt = _fmt_of(src)
    wd = dense_weights(w)
    k = wd.shape[0]
    nz, ny, nx = src.shape
    idx = _c(idx, np.int64)
    out = np.empty(idx.shape, dtype=np.float64)
    rc = _load().oracle_correlate_points(_ptr(src), fmt, lo, hi, nx, ny, nz, _ptr(wd), k,
                                         _ptr(idx), idx.size, _ptr(out))
    if rc:
        raise ValueError(f"oracle_correlate_points rejected its arguments ({rc})")
    return out


def quantize(v, fmt: int, lo: float, hi: float, window: float = TIE_WINDOW):
    """(t, q, tie): pre-rounding code values, expected codes, tie mask."""
    v = _c(v, np.float64)
    t = np.empty(v.shape, np.float64)
    q = np.empty(v.shape, np.uint32)
    tie = np.empty(v.shape, np.uint8)
    rc = _load().oracle_quantize(_ptr(v), v.size, BITS[fmt], lo, hi, window, _ptr(t), _ptr(q),
                                 _ptr(tie))
    if rc:
        raise ValueError("oracle_quantize rejected its arguments")
    return t, q, tie.astype(bool)


def gaussian_1d(k: int, sigma: float) -> np.ndarray:
    g = np.empty(k, np.float32)
    if _load().oracle_gaussian_1d(k, sigma, _ptr(g)):
        raise ValueError("bad Gaussian parameters")
    return g


def separable_weights(gx, gy, gz) -> np.ndarray:
    gx, gy, gz = (_c(g, np.float32) for g in (gx, gy, gz))
    k = gx.size
    w = np.empty((k, k, k), np.float64)
    _load().oracle_separable_weights(k, _ptr(gx), _ptr(gy), _ptr(gz), _ptr(w))
    return w


def gaussian_weights(k: int, sigma: float) -> np.ndarray:
    g = gaussian_1d(k, sigma)
    return separable_weights(g, g, g)


def laplacian_3() -> np.ndarray:
    """7-point Laplacian embedded in a 3^3 kernel: centre -6, the six face taps +1."""
    w = np.zeros((3, 3, 3), np.float64)
    w[1, 1, 1] = -6.0
    for c, b, a in ((0, 1, 1), (2, 1, 1), (1, 0, 1), (1, 2, 1), (1, 1, 0), (1, 1, 2)):
        w[c, b, a] = 1.0
    return w


def correlate_backward(x: np.ndarray, gy: np.ndarray, w, need_gx: bool = True,
                       need_gw: bool = True):
    """(gx, gw) of the float filter y = C_w x for upstream gradient gy."""
    x = _c(x, np.float64)
    gy = _c(gy, np.float64)
    wd = dense_weights(w)
    k = wd.shape[0]
    nz, ny, nx = x.shape
    gx = np.empty(x.shape, np.float64) if need_gx else None
    gw = np.empty((k, k, k), np.float64) if need_gw else None
    rc = _load().oracle_correlate_backward(_ptr(x), _ptr(gy), nx, ny, nz, _ptr(wd), k,
                                           _ptr(gx) if need_gx else None,
                                           _ptr(gw) if need_gw else None)
    if rc:
        raise ValueError("oracle_correlate_backward rejected its arguments")
    return gx, gw


def backward_input_points(gy: np.ndarray, w, idx) -> np.ndarray:
    gy = _c(gy, np.float64)
    wd = dense_weights(w)
    k = wd.shape[0]
    nz, ny, nx = gy.shape
    idx = _c(idx, np.int64)
    out = np.empty(idx.shape, np.float64)
    rc = _load().oracle_backward_input_points(_ptr(gy), nx, ny, nz, _ptr(wd), k, _ptr(idx),
                                              idx.size, _ptr(out))
    if rc:
        raise ValueError("oracle_backward_input_points rejected its arguments")
    return out


def error_scale(w, vmax_abs: float) -> float:
    """Normaliser of float errors: sum|w| * max|x| (the bound on any filtered value)."""
    return float(np.abs(dense_weights(w)).sum()) * float(vmax_abs)


def brick_decompose(src: np.ndarray, brick, ghost: int = 0):
    """BrickDecompose (Sec. 3.2, domain decomposition into subgrids with optional ghost
    cells): the bricks of ``src`` (shape (nz, ny, nx)) for a brick size ``brick`` = (bx, by,
    bz), in order (kz, ky, kx) with kx fastest.  Brick (kx, ky, kz) covers voxels [o, o + s),
    o = k * b, s = min(b, n - o), and holds s + 2 ghost voxels per axis: voxel (i, j, k) is
    src at clamp(o - ghost + (i, j, k)) per axis (clamp-to-edge beyond the faces)."""
    nz, ny, nx = src.shape
    bx, by, bz = brick
    out = []
    for oz in range(0, nz, bz):
        for oy in range(0, ny, by):
            for ox in range(0, nx, bx):
                zi = np.clip(np.arange(oz - ghost, min(oz + bz, nz) + ghost), 0, nz - 1)
                yi = np.clip(np.arange(oy - ghost, min(oy + by, ny) + ghost), 0, ny - 1)
                xi = np.clip(np.arange(ox - ghost, min(ox + bx, nx) + ghost), 0, nx - 1)
                out.append(src[np.ix_(zi, yi, xi)])
    return out


def clahe3d(src: np.ndarray, bricks, clip: float):
    """CLAHE-3D of a uint8 volume (Sec. 4.1 case study; the readings are listed in
    oracle.c): returns (codes uint8, blended values float64 before rounding, per-brick
    mappings uint8 of shape (nbz, nby, nbx, 256)).  bricks = (nbx, nby, nbz) bricks per axis,
    dividing the dims."""
    src = _c(src, np.uint8)
    nz, ny, nx = src.shape
    nbx, nby, nbz = (int(b) for b in bricks)
    out = np.empty_like(src)
    t = np.empty(src.shape, dtype=np.float64)
    luts = np.empty((nbz, nby, nbx, 256), dtype=np.uint8)
    rc = _load().oracle_clahe3d(_ptr(src), nx, ny, nz, nbx, nby, nbz, float(clip), _ptr(out),
                                _ptr(t), _ptr(luts))
    if rc != 0:
        raise ValueError("oracle_clahe3d: bricks must divide the dims")
    return out, t, luts


def render(src: np.ndarray, lo: float, hi: float, width: int, height: int, eye, center, up,
           fovy: float, step: float, termination: float, background, lut):
    """Headless ray marching with absorption and emission (Sec. 3.2 Render; readings in
    oracle.c): an (height, width, 4) float64 RGBA image.  lut: (n, 4) straight RGBA."""
    src = np.ascontiguousarray(src)
    fmt = _fmt_of(src)
    nz, ny, nx = src.shape
    lut = _c(lut, np.float64).reshape(-1, 4)
    out = np.empty((height, width, 4), dtype=np.float64)
    vec = lambda v: _c(v, np.float64).reshape(-1)
    e, c, u, bg = vec(eye), vec(center), vec(up), vec(background)
    rc = _load().oracle_render(_ptr(src), fmt, float(lo), float(hi), nx, ny, nz, int(width),
                               int(height), _ptr(e), _ptr(c), _ptr(u), float(fovy), float(step),
                               float(termination), _ptr(bg), lut.shape[0], _ptr(lut), _ptr(out))
    if rc != 0:
        raise ValueError("oracle_render: bad arguments")
    return out


def render_pixels(src: np.ndarray, lo: float, hi: float, width: int, height: int, eye, center,
                  up, fovy: float, step: float, termination: float, background, lut, pixels):
    """``render`` for the listed pixels only: pixels is an (n, 2) array of (px, py); returns
    (n, 4) float64 RGBA."""
    src = np.ascontiguousarray(src)
    fmt = _fmt_of(src)
    nz, ny, nx = src.shape
    lut = _c(lut, np.float64).reshape(-1, 4)
    pix = _c(pixels, np.int32).reshape(-1, 2)
    out = np.empty((pix.shape[0], 4), dtype=np.float64)
    vec = lambda v: _c(v, np.float64).reshape(-1)
    e, c, u, bg = vec(eye), vec(center), vec(up), vec(background)
    rc = _load().oracle_render_pixels(_ptr(src), fmt, float(lo), float(hi), nx, ny, nz, int(width),
                                      int(height), _ptr(e), _ptr(c), _ptr(u), float(fovy),
                                      float(step), float(termination), _ptr(bg), lut.shape[0],
                                      _ptr(lut), _ptr(pix), pix.shape[0], _ptr(out))
    if rc != 0:
        raise ValueError("oracle_render_pixels: bad arguments")
    return out
