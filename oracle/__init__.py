"""CPU oracle of the PL Morse-Smale segmentation (ctypes driver over
``ms_oracle.c``).

TEST INFRASTRUCTURE: only the test suite, the smoke check and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library, and the CUDA library never calls it.

The C file states which passage of the paper each function follows; this
driver only converts numpy arrays and builds the shared object with gcc.
Fields are numpy arrays of shape (nz, ny, nx) (x fastest) in float32,
float16 or float64; ``dims`` is always (nx, ny, nz).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ms_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "libmsoracle.so")
_lock = threading.Lock()
_lib = None

_DT = {np.dtype(np.float32): 0, np.dtype(np.float16): 1, np.dtype(np.float64): 2}
_ERR = {1: "NaN in the input field", 2: "invalid argument", 3: "out of memory",
        4: "pointer cycle (not a forest)", 5: "simplification regions neither nested nor disjoint"}

i32p = ctypes.POINTER(ctypes.c_int32)
i64p = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile ms_oracle.c with gcc (plain C11, -O2, no arch flags)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            L.ms_oracle_persistence.argtypes = [ctypes.c_void_p, ctypes.c_int, i64p, ctypes.c_int,
                                                i32p, i32p, ctypes.POINTER(ctypes.c_int64)]
            L.ms_oracle_persistence.restype = ctypes.c_int
            L.ms_oracle_simplify.argtypes = [ctypes.c_void_p, ctypes.c_int, i64p, ctypes.c_double, ctypes.c_int,
                                             i64p, ctypes.POINTER(ctypes.c_double), i64p]
            L.ms_oracle_simplify.restype = ctypes.c_int
            L.ms_oracle_neighbors.argtypes = [i64p, ctypes.c_int64, i64p]
            L.ms_oracle_neighbors.restype = ctypes.c_int
            L.ms_oracle_steepest.argtypes = [ctypes.c_void_p, ctypes.c_int, i64p, i32p, i32p]
            L.ms_oracle_steepest.restype = ctypes.c_int
            L.ms_oracle_follow.argtypes = [i32p, ctypes.c_int64, i32p]
            L.ms_oracle_follow.restype = ctypes.c_int
            L.ms_oracle_follow_brute.argtypes = [i32p, ctypes.c_int64, i32p]
            L.ms_oracle_follow_brute.restype = ctypes.c_int
            L.ms_oracle_walk.argtypes = [ctypes.c_void_p, ctypes.c_int, i64p, ctypes.c_int64,
                                         ctypes.c_int, ctypes.c_int64, i64p]
            L.ms_oracle_walk.restype = ctypes.c_int64
            L.ms_oracle_steepest_at.argtypes = [ctypes.c_void_p, ctypes.c_int, i64p, i64p,
                                                ctypes.c_int64, i32p, i32p]
            L.ms_oracle_steepest_at.restype = ctypes.c_int
            L.ms_oracle_ms_rank.argtypes = [i32p, i32p, ctypes.c_int64, i32p]
            L.ms_oracle_ms_rank.restype = ctypes.c_int64
            L.ms_oracle_segment.argtypes = [ctypes.c_void_p, ctypes.c_int, i64p, i32p, i32p, i32p,
                                            i64p, i32p, i32p]
            L.ms_oracle_segment.restype = ctypes.c_int
            L.ms_oracle_link_stats.argtypes = [ctypes.c_void_p, ctypes.c_int, i64p, i32p, i64p]
            L.ms_oracle_simplex_code.argtypes = [ctypes.c_int, i32p, ctypes.POINTER(ctypes.c_int)]
            L.ms_oracle_simplex_index.argtypes = [i32p, i64p, ctypes.c_void_p, i64p, i64p]
            L.ms_oracle_simplex_index_mode.argtypes = [i32p, i64p, ctypes.c_int, ctypes.c_void_p,
                                                       i64p, i64p]
            L.ms_oracle_simplex_geometry.argtypes = [i32p, i64p, ctypes.c_int, ctypes.c_void_p,
                                                     ctypes.c_void_p, i64p]
            L.ms_oracle_link_stats.restype = ctypes.c_int
            L.ms_oracle_coord_mean.argtypes = [ctypes.c_int64, ctypes.c_int]
            L.ms_oracle_coord_mean.restype = ctypes.c_float
            _lib = L
    return _lib


def _dims_of(field: np.ndarray):
    if field.ndim == 2:
        ny, nx = field.shape
        return (nx, ny, 1)
    if field.ndim != 3:
        raise ValueError("field must be (ny, nx) or (nz, ny, nx)")
    nz, ny, nx = field.shape
    return (nx, ny, nz)


def _prep(field: np.ndarray):
    f = np.ascontiguousarray(field)
    if f.dtype not in _DT:
        raise TypeError(f"unsupported dtype {f.dtype}")
    dims = (ctypes.c_int64 * 3)(*_dims_of(f))
    return f, _DT[f.dtype], dims


def _ptr32(a):
    return a.ctypes.data_as(i32p)


def _check(st):
    if st != 0:
        raise ValueError(_ERR.get(st, f"oracle error {st}"))


def neighbors(dims, v: int):
    out = (ctypes.c_int64 * 14)()
    d = (ctypes.c_int64 * 3)(*dims)
    c = lib().ms_oracle_neighbors(d, int(v), out)
    if c < 0:
        raise ValueError("bad vertex")
    return sorted(out[i] for i in range(c))


def steepest(field: np.ndarray):
    """(up, dn) int32 arrays of length N: the highest / lowest vertex of
    N(v) u {v} under the (value, index) order."""
    f, dt, dims = _prep(field)
    n = f.size
    up = np.empty(n, np.int32)
    dn = np.empty(n, np.int32)
    _check(lib().ms_oracle_steepest(f.ctypes.data, dt, dims, _ptr32(up), _ptr32(dn)))
    return up, dn


def steepest_at(field: np.ndarray, vertices):
    f, dt, dims = _prep(field)
    vs = np.ascontiguousarray(np.asarray(vertices, dtype=np.int64))
    up = np.empty(vs.size, np.int32)
    dn = np.empty(vs.size, np.int32)
    _check(lib().ms_oracle_steepest_at(f.ctypes.data, dt, dims, vs.ctypes.data_as(i64p), vs.size,
                                       _ptr32(up), _ptr32(dn)))
    return up, dn


def follow(ptr: np.ndarray, brute: bool = False) -> np.ndarray:
    p = np.ascontiguousarray(ptr, dtype=np.int32)
    out = np.empty_like(p)
    fn = lib().ms_oracle_follow_brute if brute else lib().ms_oracle_follow
    _check(fn(_ptr32(p), p.size, _ptr32(out)))
    return out


def ms_rank(asc: np.ndarray, desc: np.ndarray):
    a = np.ascontiguousarray(asc, dtype=np.int32)
    d = np.ascontiguousarray(desc, dtype=np.int32)
    ms = np.empty_like(a)
    k = lib().ms_oracle_ms_rank(_ptr32(a), _ptr32(d), a.size, _ptr32(ms))
    if k < 0:
        raise MemoryError("oracle ms_rank")
    return ms, int(k)


def walk(field: np.ndarray, v: int, direction: int, max_steps: int = 1 << 40):
    """Extremum reached from v (direction > 0: maximum, < 0: minimum) and
    the number of steps, by walking straight from the field."""
    f, dt, dims = _prep(field)
    steps = ctypes.c_int64(0)
    r = lib().ms_oracle_walk(f.ctypes.data, dt, dims, int(v), int(direction), int(max_steps),
                             ctypes.byref(steps))
    if r < 0:
        raise ValueError("walk exceeded max_steps")
    return int(r), int(steps.value)


def segment(field: np.ndarray):
    """The full segmentation: dict with asc (minimum reached), desc (maximum
    reached), ms (dense pair rank), K, up and dn."""
    f, dt, dims = _prep(field)
    n = f.size
    asc = np.empty(n, np.int32)
    desc = np.empty(n, np.int32)
    ms = np.empty(n, np.int32)
    up = np.empty(n, np.int32)
    dn = np.empty(n, np.int32)
    k = ctypes.c_int64(0)
    _check(lib().ms_oracle_segment(f.ctypes.data, dt, dims, _ptr32(asc), _ptr32(desc), _ptr32(ms),
                                   ctypes.byref(k), _ptr32(up), _ptr32(dn)))
    return {"asc": asc, "desc": desc, "ms": ms, "K": int(k.value), "up": up, "dn": dn}


def link_stats(field: np.ndarray, with_links: bool = False):
    """Per vertex: chi(Lk-), chi(Lk+), #components(Lk-), #components(Lk+),
    interior flag -- as an (N, 5) int32 array; optionally the link vertex
    sets as an (N, 14) int64 array padded with -1."""
    f, dt, dims = _prep(field)
    n = f.size
    out = np.empty((n, 5), np.int32)
    links = np.empty((n, 14), np.int64) if with_links else None
    _check(lib().ms_oracle_link_stats(f.ctypes.data, dt, dims, _ptr32(out),
                                      links.ctypes.data_as(i64p) if with_links else None))
    return (out, links) if with_links else out


def simplex_code(labels):
    """(code, element count) of one triangle (3 labels) or tetrahedron (4),
    the vertices in chain order (Sec. 4.3, Fig. 4, Tab. 1, Figs. 5-6)."""
    lab = np.ascontiguousarray(labels, dtype=np.int32)
    cnt = ctypes.c_int(0)
    code = lib().ms_oracle_simplex_code(int(lab.size), _ptr32(lab), ctypes.byref(cnt))
    if code < 0:
        raise ValueError("a simplex has 3 or 4 vertices")
    return int(code), int(cnt.value)


def simplex_cells(dims):
    nx, ny, nz = (int(d) for d in dims)
    if nz == 1:
        return max(nx - 1, 0) * max(ny - 1, 0), 2
    return max(nx - 1, 0) * max(ny - 1, 0) * max(nz - 1, 0), 6


def simplex_index(labels: np.ndarray, dims, mode: int = 0):
    """Index pass of the marching triangles / tetrahedra over a label grid:
    {'codes': uint8 per simplex, 'cell_offsets': int64 per cell, 'total'};
    mode 0 counts region separators, mode 1 region boundaries."""
    lab = np.ascontiguousarray(labels, dtype=np.int32).reshape(-1)
    nx, ny, nz = (int(d) for d in dims)
    if lab.size != nx * ny * nz:
        raise ValueError("labels do not match dims")
    cells, per = simplex_cells(dims)
    codes = np.zeros(cells * per, dtype=np.uint8)
    offs = np.zeros(max(cells, 1), dtype=np.int64)
    total = ctypes.c_int64(0)
    d = (ctypes.c_int64 * 3)(nx, ny, nz)
    _check(lib().ms_oracle_simplex_index_mode(_ptr32(lab), d, int(mode), codes.ctypes.data,
                                              offs.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                              ctypes.byref(total)))
    return {"codes": codes, "cell_offsets": offs[:cells], "total": int(total.value)}


def coord_mean(total: int, n: int) -> float:
    """The geometry pass's point coordinate: the mean of n corner coordinates
    whose exact sum is total, as a float32."""
    return float(np.float32(lib().ms_oracle_coord_mean(int(total), int(n))))


def simplex_geometry(labels: np.ndarray, dims, mode: int = 0):
    """Geometry pass (Sec. 4.3): mode 0 region separators, mode 1 region
    boundaries.  {'pos': float32 (total, points, dim), 'pairs': int32
    (total, 2), 'total'}."""
    lab = np.ascontiguousarray(labels, dtype=np.int32).reshape(-1)
    nx, ny, nz = (int(d) for d in dims)
    d = (ctypes.c_int64 * 3)(nx, ny, nz)
    total = ctypes.c_int64(0)
    _check(lib().ms_oracle_simplex_geometry(_ptr32(lab), d, int(mode), None, None,
                                            ctypes.byref(total)))
    dim = 2 if nz == 1 else 3
    npts = 2 if nz == 1 else 3
    n = int(total.value)
    pos = np.zeros((max(n, 1), npts, dim), dtype=np.float32)
    pairs = np.zeros((max(n, 1), 2), dtype=np.int32)
    _check(lib().ms_oracle_simplex_geometry(_ptr32(lab), d, int(mode), pos.ctypes.data,
                                            pairs.ctypes.data, ctypes.byref(total)))
    assert int(total.value) == n
    return {"pos": pos[:n], "pairs": pairs[:n], "total": n}


def persistence(field: np.ndarray, direction: int = -1):
    """0-dimensional persistence pairs of the extrema (direction -1: minima of
    the sublevel sets, +1: maxima of the superlevel sets): a dict with
    ``extremum`` and ``death`` (int32, in increasing extremum index; death
    -1 for the extremum that never dies)."""
    f, dt, dims = _prep(field)
    n = f.size
    ext = np.empty(n, np.int32)
    dth = np.empty(n, np.int32)
    k = ctypes.c_int64(0)
    _check(lib().ms_oracle_persistence(f.ctypes.data, dt, dims, int(direction), _ptr32(ext),
                                       _ptr32(dth), ctypes.byref(k)))
    return {"extremum": ext[:k.value].copy(), "death": dth[:k.value].copy()}


def simplify(field: np.ndarray, threshold: float, which: int = 3):
    """The field's order after removing the extrema whose persistence is below
    ``threshold`` (which: 1 minima, 2 maxima, 3 both, minima first): a dict
    with ``rank`` (int64, each vertex's position in the simplified order,
    ascending, shaped like the field), ``value`` (float64, the value each
    vertex carries), ``removed_minima`` and ``removed_maxima``.  ``rank`` as a
    float64 field is the simplified field to segment (its values are distinct,
    so the (value, index) order is the rank order)."""
    f, dt, dims = _prep(field)
    n = f.size
    rank = np.empty(n, np.int64)
    value = np.empty(n, np.float64)
    removed = np.zeros(3, np.int64)
    _check(lib().ms_oracle_simplify(f.ctypes.data, dt, dims, float(threshold), int(which),
                                    rank.ctypes.data_as(i64p),
                                    value.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    removed.ctypes.data_as(i64p)))
    return {"rank": rank.reshape(f.shape), "value": value.reshape(f.shape),
            "removed_minima": int(removed[0]), "removed_maxima": int(removed[1]), "rounds": int(removed[2])}
