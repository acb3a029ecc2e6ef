"""The paper's CPU-parallel segmentation scheme (Sec. 4.2) with OpenMP: the
CPU-parallel baseline that ``bench.py`` reports beside the single-threaded
oracle.  ``msseg_omp.c`` holds the method; this module builds it with gcc and
drives it through ctypes.  It is measurement infrastructure: the GPU library
never calls it, and it shares no code with the GPU path or the oracle.

``python -m cpu_parallel FIELD.npy REPEATS`` times one warm-up and REPEATS
runs on all host cores and prints one JSON line.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "msseg_omp.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libmsseg_omp.so")
_lock = threading.Lock()
_lib = None

_ERR = {1: "NaN in the input field", 2: "invalid argument", 3: "out of memory"}


def build(force: bool = False) -> str:
    """Compile msseg_omp.c with gcc (C11, -O3, OpenMP, no arch flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O3", "-fopenmp", "-fPIC", "-shared", "-o", tmp,
                               _SRC])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            L.msseg_omp_segment.argtypes = [ctypes.c_void_p, ctypes.c_int64, ctypes.c_int64,
                                            ctypes.c_int64, i32p, i32p, i32p,
                                            ctypes.POINTER(ctypes.c_int64), ctypes.c_int]
            L.msseg_omp_segment.restype = ctypes.c_int
            L.msseg_omp_max_threads.restype = ctypes.c_int
            _lib = L
    return _lib


def max_threads() -> int:
    return int(lib().msseg_omp_max_threads())


def segment(field: np.ndarray, threads: int = 0):
    """asc, desc, ms (dense pair rank) and K of a float32 field of shape
    (nz, ny, nx) or (ny, nx)."""
    f = np.ascontiguousarray(field, dtype=np.float32)
    if f.ndim == 2:
        dims = (f.shape[1], f.shape[0], 1)
    elif f.ndim == 3:
        dims = (f.shape[2], f.shape[1], f.shape[0])
    else:
        raise ValueError("field must be 2D (ny, nx) or 3D (nz, ny, nx)")
    n = f.size
    out = [np.empty(n, np.int32) for _ in range(3)]
    k = ctypes.c_int64(0)
    i32p = ctypes.POINTER(ctypes.c_int32)
    st = lib().msseg_omp_segment(f.ctypes.data, dims[0], dims[1], dims[2],
                                 *(o.ctypes.data_as(i32p) for o in out), ctypes.byref(k), int(threads))
    if st != 0:
        raise RuntimeError(_ERR.get(st, f"error {st}"))
    return {"asc": out[0], "desc": out[1], "ms": out[2], "K": int(k.value)}
