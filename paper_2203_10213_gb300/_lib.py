"""ctypes declarations of every entry point of include/vkt.h (argument marshalling only).

Loading fails loudly when libvkt.so is missing or cannot be built: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

_lock = threading.Lock()
_lib = None

c_err = ctypes.c_int
p = ctypes.c_void_p
i32 = ctypes.c_int32
f32 = ctypes.c_float
pf = ctypes.POINTER(ctypes.c_float)
pi32 = ctypes.POINTER(ctypes.c_int32)


class ExecutionPolicy(ctypes.Structure):
    _fields_ = [("stream", ctypes.c_void_p), ("printTimes", ctypes.c_int32),
                ("debug", ctypes.c_int32), ("path", ctypes.c_int32)]


# name -> (argtypes); every function returns vktError (int) except vktGetErrorString
SIGNATURES = {
    "vktSetThreadExecutionPolicy": [ExecutionPolicy],
    "vktGetThreadExecutionPolicy": [ctypes.POINTER(ExecutionPolicy)],
    "vktGetErrorString": [c_err],
    "vktSynchronize": [],
    "vktGetLaunchCount": [ctypes.POINTER(ctypes.c_uint64)],
    "vktStructuredVolumeCreate": [ctypes.POINTER(p), i32, i32, i32, c_err, f32, f32, f32, f32, f32],
    "vktStructuredVolumeCreateView": [ctypes.POINTER(p), p, i32, i32, i32, c_err, f32, f32, f32,
                                      f32, f32],
    "vktStructuredVolumeDestroy": [p],
    "vktStructuredVolumeGetDims": [p, pi32, pi32, pi32],
    "vktStructuredVolumeGetDataFormat": [p, ctypes.POINTER(c_err)],
    "vktStructuredVolumeGetCellSize": [p, pf, pf, pf],
    "vktStructuredVolumeGetVoxelMapping": [p, pf, pf],
    "vktStructuredVolumeSetVoxelMapping": [p, f32, f32],
    "vktStructuredVolumeGetData": [p, ctypes.POINTER(p)],
    "vktStructuredVolumeGetSizeInBytes": [p, ctypes.POINTER(ctypes.c_uint64)],
    "vktStructuredVolumeSetData": [p, p],
    "vktStructuredVolumeCopyToHost": [p, p],
    "vktFilterCreate": [ctypes.POINTER(p), i32, pf],
    "vktFilterCreateSeparable": [ctypes.POINTER(p), i32, pf, pf, pf],
    "vktFilterCreateGaussian": [ctypes.POINTER(p), i32, f32],
    "vktFilterSetWeights": [p, pf],
    "vktFilterNormalize": [p],
    "vktFilterGetSize": [p, pi32],
    "vktFilterIsSeparable": [p, pi32],
    "vktFilterGetWeights": [p, pf],
    "vktFilterGetSeparableWeights": [p, pf, pf, pf],
    "vktFilterDestroy": [p],
    "vktApplyFilterSV": [p, p, p],
    "vktApplyFilterRangeSV": [p, p, p, i32, i32, i32, i32, i32, i32],
    "vktBrickDecomposeCountSV": [pi32, pi32, pi32, p, i32, i32, i32],
    "vktBrickDecomposeSV": [ctypes.POINTER(ctypes.c_void_p), i32, p, i32, i32, i32, i32],
    "vktClahe3DSV": [p, p, i32, i32, i32, ctypes.c_float],
    "vktRenderSV": [p, i32, i32, p, p],
    "vktApplyFilterBatchSV": [i32, ctypes.POINTER(p), ctypes.POINTER(p), ctypes.POINTER(p)],
    "vktApplyFilterBackwardSV": [p, p, p, p, p],
    "vktApplyFilterBackwardBatchSV": [i32, ctypes.POINTER(p), p, ctypes.POINTER(p), ctypes.POINTER(p), p],
    "vktApplyFilterWeightGradNoAllocSV": [p, p, p, p],
    "vktAutotuneSetEnabled": [i32],
    "vktAutotuneGetEnabled": [pi32],
    "vktAutotuneClear": [],
    "vktAutotuneGetCount": [pi32],
    "vktAutotuneSave": [ctypes.c_char_p],
    "vktAutotuneLoad": [ctypes.c_char_p],
}


def lib_path() -> str:
    return _build.LIB


def load(build: bool = True):
    """The loaded library (built first when sources changed and nvcc is available)."""
    global _lib
    with _lock:
        if _lib is None:
            if build:
                _build.build()
            if not os.path.exists(_build.LIB):
                raise ImportError(f"libvkt.so not found at {_build.LIB}; run build()")
            lib = ctypes.CDLL(_build.LIB)
            for name, args in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.argtypes = args
                fn.restype = ctypes.c_char_p if name == "vktGetErrorString" else c_err
            _lib = lib
    return _lib


def declared_symbols(header: str) -> list[str]:
    """Names of the functions declared in a C header (for the export check)."""
    import re
    with open(header) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(vkt[A-Za-z0-9_]+)\s*\(", text)))
