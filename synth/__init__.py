"""Seeded synthetic inputs (volumes, weights) shared by the GPU tests, the benchmark and
the oracle checks.

This module draws inputs only: it holds none of the filter arithmetic, and neither the
oracle nor the CUDA path is imported here.  All draws are counter based (SplitMix64
hash of a counter, Box-Muller normals), implemented in ``synth.c``.

The paper times Gaussian blur on CT-like uint8 volumes (Heptane 302^3, RM
2048x2048x1920) and on DNS float32 fields (Table 1, Sec. 4.3).  Those datasets are not
available, so the recipes below stand in for them: ``blobs`` is a CT-like field, and
``fourier`` is a turbulence-like field with a k^(-5/3) spectrum.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "libsynth.so")
_lock = threading.Lock()
_lib = None

BASE_SEED = 220310213

U8, U16, F32 = 0, 1, 2
FORMAT_BITS = {U8: 8, U16: 16}
NP_DTYPE = {U8: np.uint8, U16: np.uint16, F32: np.float32}


def build(force: bool = False) -> str:
    """Compile ``synth.c`` into ``libsynth.so`` next to it (gcc, OpenMP if available)."""
    src = os.path.join(_HERE, "synth.c")
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(src):
        return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-shared", "-fPIC", "-std=c11", src, "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            u64, i64, d, i32 = ctypes.c_uint64, ctypes.c_int64, ctypes.c_double, ctypes.c_int
            p = ctypes.c_void_p
            lib.synth_u64.restype = u64
            lib.synth_u64.argtypes = [u64, u64, u64]
            lib.synth_u01.restype = d
            lib.synth_u01.argtypes = [u64, u64, u64]
            lib.synth_normal.restype = d
            lib.synth_normal.argtypes = [u64, u64, u64]
            lib.synth_uniform_f32.argtypes = [u64, u64, i64, ctypes.c_float, ctypes.c_float, p]
            lib.synth_normal_f32.argtypes = [u64, u64, i64, d, d, p]
            lib.synth_blobs_f32.restype = i32
            lib.synth_blobs_f32.argtypes = [u64, i64, i64, i64, i32, d, d, d, d, d, p]
            lib.synth_quantize.argtypes = [p, i64, i32, p]
            lib.synth_fourier_f32.restype = i32
            lib.synth_fourier_f32.argtypes = [u64, i64, i64, i64, i32, d, d, p]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def u01(seed: int, stream: int, i: int) -> float:
    return _load().synth_u01(seed, stream, i)


def uniform(seed: int, shape, lo: float = 0.0, hi: float = 1.0, stream: int = 0) -> np.ndarray:
    """float32 array, i.i.d. uniform[lo, hi); shape is (nz, ny, nx) for volumes."""
    out = np.empty(shape, dtype=np.float32)
    _load().synth_uniform_f32(seed, stream, out.size, lo, hi, _ptr(out))
    return out


def normal(seed: int, shape, mean: float = 0.0, sd: float = 1.0, stream: int = 0) -> np.ndarray:
    out = np.empty(shape, dtype=np.float32)
    _load().synth_normal_f32(seed, stream, out.size, mean, sd, _ptr(out))
    return out


def blobs(seed: int, dims, nblobs: int = 32, sigma=(8.0, 64.0), amp=(0.2, 1.0),
          noise: float = 0.02) -> np.ndarray:
    """CT-like float32 field in [0,1]; dims = (nx, ny, nz), returned as (nz, ny, nx)."""
    nx, ny, nz = dims
    out = np.empty((nz, ny, nx), dtype=np.float32)
    rc = _load().synth_blobs_f32(seed, nx, ny, nz, nblobs, sigma[0], sigma[1], amp[0], amp[1],
                                 noise, _ptr(out))
    if rc != 0:
        raise ValueError(f"synth_blobs_f32 failed ({rc})")
    return out


def quantize(v: np.ndarray, fmt: int) -> np.ndarray:
    """Codes q = floor(v*(2^N-1) + 1/2), clamped, for values v in [0,1]."""
    v = np.ascontiguousarray(v, dtype=np.float32)
    out = np.empty(v.shape, dtype=NP_DTYPE[fmt])
    _load().synth_quantize(_ptr(v), v.size, FORMAT_BITS[fmt], _ptr(out))
    return out


def fourier(seed: int, dims, nmodes: int = 64, kmin: float = 1.0, kmax: float = 32.0) -> np.ndarray:
    """Turbulence-like float32 field (k^-5/3 amplitudes); dims = (nx, ny, nz)."""
    nx, ny, nz = dims
    out = np.empty((nz, ny, nx), dtype=np.float32)
    rc = _load().synth_fourier_f32(seed, nx, ny, nz, nmodes, kmin, kmax, _ptr(out))
    if rc != 0:
        raise ValueError(f"synth_fourier_f32 failed ({rc})")
    return out


def random_kernel(seed: int, k: int, sd: float = 1.0, normalise_sum: bool = False,
                  stream: int = 7):
    """k^3 float32 weights, i.i.d. N(0, sd^2), x fastest.

    With ``normalise_sum`` the draw is divided by its (float64) sum; a draw whose |sum| < 1
    is redrawn with seed+1, seed+2, ... so the scale stays bounded.  Returns
    (weights, seed actually used).
    """
    s = seed
    while True:
        w = normal(s, (k, k, k), 0.0, sd, stream=stream).astype(np.float64)
        if not normalise_sum:
            return w.astype(np.float32), s
        tot = float(w.sum())
        if abs(tot) >= 1.0:
            return (w / tot).astype(np.float32), s
        s += 1


def laplacian_3() -> np.ndarray:
    """The 3x3x3 kernel of the Laplacian workload as float32 input weights, x fastest: the
    7-point stencil (centre -6, the six face neighbours +1, the other 20 taps 0).  A
    literal table: the filter that the GPU arm is given, written independently of the
    oracle's own copy."""
    w = np.zeros((3, 3, 3), np.float32)
    w[1, 1, 1] = -6.0
    w[0, 1, 1] = w[2, 1, 1] = 1.0
    w[1, 0, 1] = w[1, 2, 1] = 1.0
    w[1, 1, 0] = w[1, 1, 2] = 1.0
    return w


# ---------------------------------------------------------------------------------------
# Workload recipes.  Each returns host numpy arrays; shapes are (nz, ny, nx), x fastest.
# ---------------------------------------------------------------------------------------

def volume(kind: str, fmt: int, dims, seed: int):
    """A source volume of the given value model and storage format.

    kind: "uniform" (U[0,1) float), "blobs" (CT-like), "fourier" (turbulence-like).
    Integer formats store quantised codes of a [0,1] field (mapping range [0,1]).
    """
    if kind == "uniform":
        v = uniform(seed, tuple(reversed(dims)))
    elif kind == "blobs":
        v = blobs(seed, dims)
    elif kind == "fourier":
        v = fourier(seed, dims)
    else:
        raise ValueError(kind)
    if fmt == F32:
        return v
    if kind == "fourier":
        lo, hi = float(v.min()), float(v.max())
        v = (v - lo) / max(hi - lo, 1e-30)
    return quantize(v, fmt)


def batch_recipe(seed: int, n: int = 256, dmin: int = 16, dmax: int = 256, ks=(3, 5, 7)):
    """Mixed batch: per volume, dims log-uniform in [dmin, dmax] per axis, format uniform
    over {u8, u16, f32}, Gaussian filter size uniform over ``ks`` with sigma = k/3.

    Returns a list of dicts {dims, fmt, kind, k, sigma, seed}; values are drawn lazily by
    ``volume``.
    """
    items = []
    for i in range(n):
        d = []
        for a in range(3):
            u = u01(seed, 11, 8 * i + a)
            d.append(int(round(math.exp(math.log(dmin) + u * (math.log(dmax) - math.log(dmin))))))
        fmt = int(u01(seed, 11, 8 * i + 3) * 3) % 3
        k = ks[int(u01(seed, 11, 8 * i + 4) * len(ks)) % len(ks)]
        kind = "fourier" if fmt == F32 else "blobs"
        items.append(dict(dims=tuple(d), fmt=fmt, kind=kind, k=k, sigma=k / 3.0,
                          seed=seed * 1000 + i))
    return items
