"""Python binding of libmsseg -- the GB300 (sm_103a) piecewise-linear
Morse-Smale segmentation library declared in ``include/ms.h``.

The functions carry the C names and only marshal arguments: device tensors
become raw pointers, ``dims`` tuples become ``int64_t[3]``, and a non-OK
status becomes an ``MSError``.  Every step of the computation runs in the
library's CUDA kernels; there is no Python or CPU fallback -- if the library
cannot be built or loaded, importing the binding's functions raises.

PyTorch supplies device memory and streams only.  Fields are torch tensors
of shape (nz, ny, nx) or (ny, nx), x fastest, dtype float32 or float16, on a
CUDA device; label outputs are int32 tensors of the same number of elements.
"""
from __future__ import annotations

import ctypes
import os
import threading

from . import _build

__all__ = [
    "MSError", "MS_F32", "MS_F16", "load", "ms_status_string", "ms_create", "ms_destroy",
    "ms_segment", "ms_segment_host", "ms_last_region_count", "ms_order_keys", "ms_steepest",
    "ms_compress", "ms_pair_rank", "segment", "EXPORTED_SYMBOLS", "ms_profile_enable",
    "ms_profile_read", "ms_profile_stage_name", "STAGES", "ms_segment_staged",
    "ms_pair_rank_noalloc", "MS_NOALLOC_MAX_N", "ms_segment_batch", "ms_server_create",
    "ms_server_submit", "ms_server_wait", "ms_server_stats", "ms_server_destroy",
    "ms_batch_autotune", "ms_batch_graphs", "ms_simplex_index", "ms_simplex_geometry",
    "simplex_cells", "ms_segment_host_many", "ms_persistence", "persistence", "ms_slab_local",
    "ms_slab_resolve", "ms_slab_pairs", "ms_slab_rank", "ms_set_tuning", "ms_get_tuning",
    "TILE_SHAPES",
]

MS_F32, MS_F16 = 0, 1
STATUS = ["MS_OK", "MS_ERR_INVALID_ARG", "MS_ERR_UNSUPPORTED_DTYPE", "MS_ERR_TOO_LARGE",
          "MS_ERR_NAN_INPUT", "MS_ERR_OUT_OF_MEMORY", "MS_ERR_CUDA", "MS_ERR_NOT_CONVERGED",
          "MS_ERR_TIMEOUT", "MS_ERR_BUSY"]

EXPORTED_SYMBOLS = [
    "ms_status_string", "ms_create", "ms_destroy", "ms_segment", "ms_segment_host",
    "ms_last_region_count", "ms_order_keys", "ms_steepest", "ms_compress", "ms_pair_rank",
    "ms_profile_enable", "ms_profile_read", "ms_profile_stage_name", "ms_segment_staged",
    "ms_pair_rank_noalloc", "ms_segment_batch", "ms_server_create", "ms_server_submit",
    "ms_server_wait", "ms_server_stats", "ms_server_destroy", "ms_batch_autotune",
    "ms_batch_graphs", "ms_simplex_index", "ms_simplex_geometry", "ms_segment_host_many",
    "ms_persistence", "ms_slab_local", "ms_slab_resolve", "ms_slab_pairs", "ms_slab_rank",
    "ms_set_tuning", "ms_get_tuning",
]
MS_NOALLOC_MAX_N = 262144
# 3D tile shapes by ms_tuning.shape3 id: (x, y, z) vertices
TILE_SHAPES = {0: (32, 16, 16), 1: (64, 8, 16), 2: (16, 32, 16), 3: (16, 16, 16)}


class _Tuning(ctypes.Structure):
    _fields_ = [("tile_ctas", ctypes.c_int), ("write_ctas", ctypes.c_int),
                ("chase_blocks", ctypes.c_int), ("pair_blocks", ctypes.c_int),
                ("dynamic", ctypes.c_int), ("resolve_mode", ctypes.c_int), ("shape3", ctypes.c_int),
                ("default_ms", ctypes.c_double), ("best_ms", ctypes.c_double)]


class _PersistenceInfo(ctypes.Structure):
    _fields_ = [("n_extrema", ctypes.c_int64), ("basin_edges", ctypes.c_int64),
                ("rounds", ctypes.c_int32), ("pad", ctypes.c_int32), ("finish_edges", ctypes.c_int64)]


class _ServerInfo(ctypes.Structure):
    _fields_ = [("admitted", ctypes.c_uint64), ("completed", ctypes.c_uint64),
                ("queued", ctypes.c_uint64), ("bytes_in_use", ctypes.c_size_t),
                ("peak_bytes", ctypes.c_size_t), ("budget_bytes", ctypes.c_size_t),
                ("launches", ctypes.c_uint64), ("resident_bytes", ctypes.c_size_t)]


STAGES = ["tile_local", "resolve", "write", "h2d", "d2h", "graph"]


class _Profile(ctypes.Structure):
    _fields_ = [("calls", ctypes.c_int64), ("launches", ctypes.c_int64),
                ("stage_launches", ctypes.c_int64 * 8), ("stage_ms", ctypes.c_double * 8)]

_lock = threading.Lock()
_lib = None

c_i64p = ctypes.POINTER(ctypes.c_int64)
c_vp = ctypes.c_void_p


class MSError(RuntimeError):
    def __init__(self, status: int, where: str = ""):
        self.status = int(status)
        self.name = STATUS[status] if 0 <= status < len(STATUS) else f"status {status}"
        super().__init__(f"{where}: {self.name}" if where else self.name)


def load(build: bool = True) -> ctypes.CDLL:
    """Load libmsseg.so from the package's build folder (compiling it first
    if it is missing or stale and ``build`` is true)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build() if build else _build.LIB
            if not os.path.exists(path):
                raise OSError(f"libmsseg.so not built at {path}")
            L = ctypes.CDLL(path)
            L.ms_status_string.argtypes = [ctypes.c_int]
            L.ms_status_string.restype = ctypes.c_char_p
            L.ms_create.argtypes = [ctypes.POINTER(c_vp), ctypes.c_int, c_vp]
            L.ms_destroy.argtypes = [c_vp]
            L.ms_segment.argtypes = [c_vp, c_vp, c_i64p, ctypes.c_int, c_vp, c_vp, c_vp]
            L.ms_segment_batch.argtypes = [c_vp, ctypes.c_int, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp,
                                           c_i64p]
            L.ms_batch_autotune.argtypes = [c_vp, ctypes.c_int, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp,
                                            ctypes.POINTER(_Tuning)]
            L.ms_batch_graphs.argtypes = [c_vp, ctypes.c_int]
            L.ms_set_tuning.argtypes = [c_vp, ctypes.POINTER(_Tuning)]
            L.ms_get_tuning.argtypes = [c_vp, ctypes.POINTER(_Tuning)]
            L.ms_simplex_index.argtypes = [c_vp, c_vp, c_i64p, ctypes.c_int, c_vp, c_vp, c_i64p]
            L.ms_simplex_geometry.argtypes = [c_vp, c_vp, c_i64p, ctypes.c_int, c_vp, ctypes.c_int64,
                                              c_vp, c_vp]
            L.ms_persistence.argtypes = [c_vp, c_vp, c_i64p, ctypes.c_int, c_vp, ctypes.c_int, c_vp,
                                         c_vp, ctypes.c_int64, ctypes.POINTER(_PersistenceInfo)]
            L.ms_slab_local.argtypes = [c_vp, c_vp, c_i64p, ctypes.c_int, ctypes.c_int64,
                                        ctypes.c_int64, c_vp, c_vp]
            L.ms_slab_resolve.argtypes = [c_vp, c_i64p, c_vp, c_i64p, ctypes.c_int, c_vp, c_vp,
                                          ctypes.c_int64]
            L.ms_slab_pairs.argtypes = [c_vp, c_vp, c_vp, ctypes.c_int64, ctypes.c_int64, c_vp,
                                        ctypes.c_int64, c_i64p]
            L.ms_slab_rank.argtypes = [c_vp, c_vp, c_vp, ctypes.c_int64, ctypes.c_int64, c_vp,
                                       ctypes.c_int64, c_vp, c_i64p]
            L.ms_server_create.argtypes = [ctypes.POINTER(c_vp), ctypes.c_int, ctypes.c_size_t,
                                           ctypes.c_int]
            L.ms_server_submit.argtypes = [c_vp, c_vp, c_i64p, ctypes.c_int, c_vp, c_vp, c_vp,
                                           ctypes.POINTER(ctypes.c_uint64)]
            L.ms_server_wait.argtypes = [c_vp, ctypes.c_uint64, ctypes.c_int64,
                                         ctypes.POINTER(ctypes.c_int), c_i64p,
                                         ctypes.POINTER(ctypes.c_double)]
            L.ms_server_stats.argtypes = [c_vp, ctypes.POINTER(_ServerInfo)]
            L.ms_server_destroy.argtypes = [c_vp]
            L.ms_segment_staged.argtypes = [c_vp, c_vp, c_i64p, ctypes.c_int, c_vp, c_vp, c_vp]
            L.ms_segment_host.argtypes = [c_vp, c_vp, c_i64p, ctypes.c_int, c_vp, c_vp, c_vp]
            L.ms_segment_host_many.argtypes = [c_vp, ctypes.c_int, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp,
                                               c_i64p]
            L.ms_last_region_count.argtypes = [c_vp, c_i64p]
            L.ms_order_keys.argtypes = [c_vp, c_vp, ctypes.c_int64, ctypes.c_int, c_vp]
            L.ms_steepest.argtypes = [c_vp, c_vp, c_i64p, ctypes.c_int, c_vp, c_vp]
            L.ms_compress.argtypes = [c_vp, c_vp, ctypes.c_int64]
            L.ms_pair_rank.argtypes = [c_vp, c_vp, c_vp, ctypes.c_int64, c_vp, c_i64p]
            L.ms_pair_rank_noalloc.argtypes = [c_vp, c_vp, ctypes.c_int64, c_vp, c_i64p, c_vp]
            L.ms_profile_enable.argtypes = [c_vp, ctypes.c_int]
            L.ms_profile_read.argtypes = [c_vp, ctypes.POINTER(_Profile)]
            L.ms_profile_stage_name.argtypes = [ctypes.c_int]
            L.ms_profile_stage_name.restype = ctypes.c_char_p
            for name in EXPORTED_SYMBOLS[1:]:
                if name == "ms_profile_stage_name":
                    continue
                getattr(L, name).restype = ctypes.c_int
            _lib = L
    return _lib


def _check(st: int, where: str):
    if st != 0:
        raise MSError(st, where)


def _ptr(t) -> int:
    if t is None:
        return 0
    if isinstance(t, int):
        return t
    if hasattr(t, "data_ptr"):
        return t.data_ptr()
    if hasattr(t, "ctypes"):  # numpy
        return t.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(t)}")


def _dims(dims):
    d = tuple(int(v) for v in dims)
    if len(d) != 3:
        raise ValueError("dims must be (nx, ny, nz)")
    return (ctypes.c_int64 * 3)(*d)


def dims_of(field):
    """(nx, ny, nz) of a (nz, ny, nx) or (ny, nx) array / tensor."""
    shp = tuple(field.shape)
    if len(shp) == 2:
        return (shp[1], shp[0], 1)
    if len(shp) == 3:
        return (shp[2], shp[1], shp[0])
    raise ValueError("field must be 2D (ny, nx) or 3D (nz, ny, nx)")


def dtype_code(field) -> int:
    name = str(field.dtype)
    if name.endswith("float32"):
        return MS_F32
    if name.endswith("float16"):
        return MS_F16
    return 99  # rejected by the library as MS_ERR_UNSUPPORTED_DTYPE


def ms_status_string(status: int) -> str:
    return load().ms_status_string(int(status)).decode()


def ms_create(device: int = 0, stream=None) -> int:
    """Returns the context handle (an int).  ``stream``: a torch.cuda.Stream,
    a raw cudaStream_t int, or None for a context-owned stream."""
    h = c_vp()
    s = getattr(stream, "cuda_stream", stream)
    _check(load().ms_create(ctypes.byref(h), int(device), s if s else None), "ms_create")
    return h.value


def ms_destroy(ctx: int) -> None:
    _check(load().ms_destroy(ctx), "ms_destroy")


def ms_segment(ctx, field, dims, dtype, out_asc, out_desc, out_ms) -> None:
    _check(load().ms_segment(ctx, _ptr(field), _dims(dims), int(dtype), _ptr(out_asc),
                             _ptr(out_desc), _ptr(out_ms)), "ms_segment")


def ms_segment_batch(ctx, fields, dims_list, dtypes, ascs, descs, mss) -> list:
    """Segment many fields in one call; returns the list of per-field K.
    fields / ascs / descs / mss: device tensors (or pointers); dims_list:
    (nx, ny, nz) per field; dtypes: MS_F32 / MS_F16 per field."""
    n = len(fields)
    ptrs = lambda xs: (c_vp * n)(*[_ptr(x) for x in xs])
    dims = (ctypes.c_int64 * (3 * n))(*[int(v) for d in dims_list for v in d])
    dts = (ctypes.c_int * n)(*[int(t) for t in dtypes])
    ks = (ctypes.c_int64 * n)()
    _check(load().ms_segment_batch(ctx, n, ptrs(fields), ctypes.cast(dims, c_vp), ctypes.cast(dts, c_vp),
                                   ptrs(ascs), ptrs(descs), ptrs(mss), ks), "ms_segment_batch")
    return [int(k) for k in ks]




def ms_batch_autotune(ctx, fields, dims_list, dtypes, ascs, descs, mss) -> dict:
    """Pick the batched path's launch choices for these fields (see ms.h);
    returns them with the default and best times."""
    n = len(fields)
    ptrs = lambda xs: (c_vp * n)(*[_ptr(x) for x in xs])
    dims = (ctypes.c_int64 * (3 * n))(*[int(v) for d in dims_list for v in d])
    dts = (ctypes.c_int * n)(*[int(t) for t in dtypes])
    t = _Tuning()
    _check(load().ms_batch_autotune(ctx, n, ptrs(fields), ctypes.cast(dims, c_vp),
                                    ctypes.cast(dts, c_vp), ptrs(ascs), ptrs(descs), ptrs(mss),
                                    ctypes.byref(t)), "ms_batch_autotune")
    return {f: getattr(t, f) for f, _ in _Tuning._fields_}


def ms_simplex_index(ctx, labels, dims, codes, cell_offsets, mode: int = 0) -> int:
    """Index pass of the marching triangles / tetrahedra (see ms.h); returns
    the total number of elements (mode 0 separators, 1 boundaries)."""
    t = ctypes.c_int64(0)
    _check(load().ms_simplex_index(ctx, _ptr(labels), _dims(dims), int(mode), _ptr(codes),
                                   _ptr(cell_offsets), ctypes.byref(t)), "ms_simplex_index")
    return int(t.value)


def ms_simplex_geometry(ctx, labels, dims, cell_offsets, total, points, pairs=None,
                        mode: int = 0) -> None:
    """Geometry pass (see ms.h) into points (and pairs, optional)."""
    _check(load().ms_simplex_geometry(ctx, _ptr(labels), _dims(dims), int(mode), _ptr(cell_offsets),
                                      int(total), _ptr(points), _ptr(pairs)), "ms_simplex_geometry")


def simplex_cells(dims):
    """(cells, simplices per cell) of a grid."""
    nx, ny, nz = (int(d) for d in dims)
    if nz == 1:
        return max(nx - 1, 0) * max(ny - 1, 0), 2
    return max(nx - 1, 0) * max(ny - 1, 0) * max(nz - 1, 0), 6


def ms_persistence(ctx, field, dims, dtype, labels, direction, extremum, death, capacity) -> dict:
    """Persistence pairs of the minima (direction -1, labels = asc) or maxima
    (+1, labels = desc) into ``extremum`` / ``death`` (int32 device buffers of
    ``capacity`` entries).  Returns the info counts; raises MSError
    (MS_ERR_TOO_LARGE with ``.info`` set) when capacity is too small."""
    info = _PersistenceInfo()
    st = load().ms_persistence(ctx, _ptr(field), _dims(dims), int(dtype), _ptr(labels), int(direction),
                               _ptr(extremum), _ptr(death), int(capacity), ctypes.byref(info))
    out = {k: int(getattr(info, k)) for k in ("n_extrema", "basin_edges", "rounds", "finish_edges")}
    if st != 0:
        err = MSError(st, "ms_persistence")
        err.info = out
        raise err
    return out


def persistence(ctx, field, labels, direction: int = -1):
    """(extremum, death, info) of a device field and its asc (minima) or desc
    (maxima) labels; extremum and death are int32 device tensors."""
    import torch
    dims, dt = dims_of(field), dtype_code(field)
    cap = min(field.numel(), 1 << 20)
    for _ in range(2):
        ext = torch.empty(max(cap, 1), dtype=torch.int32, device=field.device)
        dth = torch.empty_like(ext)
        try:
            info = ms_persistence(ctx, field, dims, dt, labels, direction, ext, dth, cap)
        except MSError as e:
            if e.status != 3 or not getattr(e, "info", None) or e.info["n_extrema"] <= cap:
                raise
            cap = e.info["n_extrema"]
            continue
        return ext[:info["n_extrema"]], dth[:info["n_extrema"]], info
    raise RuntimeError("ms_persistence: extremum count changed between calls")


def ms_slab_local(ctx, field, dims, dtype, z0, z1, out_asc, out_desc) -> None:
    _check(load().ms_slab_local(ctx, _ptr(field), _dims(dims), int(dtype), int(z0), int(z1),
                                _ptr(out_asc), _ptr(out_desc)), "ms_slab_local")


def ms_slab_resolve(ctx, dims, rows, plane_z, asc, desc, n_owned) -> None:
    zs = (ctypes.c_int64 * max(1, len(plane_z)))(*[int(z) for z in plane_z])
    _check(load().ms_slab_resolve(ctx, _dims(dims), _ptr(rows), zs, len(plane_z), _ptr(asc),
                                  _ptr(desc), int(n_owned)), "ms_slab_resolve")


def ms_slab_pairs(ctx, asc, desc, n, n_labels, keys, capacity) -> int:
    """Count of distinct pairs; raises MSError (with ``.count``) when it
    exceeds capacity."""
    m = ctypes.c_int64(0)
    st = load().ms_slab_pairs(ctx, _ptr(asc), _ptr(desc), int(n), int(n_labels), _ptr(keys),
                              int(capacity), ctypes.byref(m))
    if st != 0:
        err = MSError(st, "ms_slab_pairs")
        err.count = m.value
        raise err
    return m.value


def ms_slab_rank(ctx, asc, desc, n, n_labels, keys, n_keys, ms) -> int:
    k = ctypes.c_int64(0)
    _check(load().ms_slab_rank(ctx, _ptr(asc), _ptr(desc), int(n), int(n_labels), _ptr(keys),
                               int(n_keys), _ptr(ms), ctypes.byref(k)), "ms_slab_rank")
    return k.value


def ms_get_tuning(ctx) -> dict:
    t = _Tuning()
    _check(load().ms_get_tuning(ctx, ctypes.byref(t)), "ms_get_tuning")
    return {f: getattr(t, f) for f, _ in _Tuning._fields_ if not f.endswith("_ms")}


def ms_set_tuning(ctx, **choices) -> dict:
    """Set some of the context's default launch choices (see ms.h); returns
    the previous ones."""
    prev = ms_get_tuning(ctx)
    t = _Tuning(**{**prev, **choices})
    _check(load().ms_set_tuning(ctx, ctypes.byref(t)), "ms_set_tuning")
    return prev


def ms_batch_graphs(ctx, on: bool = True) -> None:
    _check(load().ms_batch_graphs(ctx, 1 if on else 0), "ms_batch_graphs")

def ms_server_create(device: int = 0, budget_bytes: int = 120 << 30, n_slots: int = 4) -> int:
    h = c_vp()
    _check(load().ms_server_create(ctypes.byref(h), int(device), int(budget_bytes), int(n_slots)),
           "ms_server_create")
    return h.value


def ms_server_submit(srv, field, dims, dtype, out_asc, out_desc, out_ms) -> int:
    t = ctypes.c_uint64(0)
    _check(load().ms_server_submit(srv, _ptr(field), _dims(dims), int(dtype), _ptr(out_asc),
                                   _ptr(out_desc), _ptr(out_ms), ctypes.byref(t)), "ms_server_submit")
    return int(t.value)


def ms_server_wait(srv, ticket: int, timeout_ms: int = -1):
    """(status, K, latency_ms) of a finished request; raises MSError with
    MS_ERR_TIMEOUT if it is still running after timeout_ms."""
    st, k, lat = ctypes.c_int(0), ctypes.c_int64(0), ctypes.c_double(0.0)
    _check(load().ms_server_wait(srv, int(ticket), int(timeout_ms), ctypes.byref(st), ctypes.byref(k),
                                 ctypes.byref(lat)), "ms_server_wait")
    return int(st.value), int(k.value), float(lat.value)


def ms_server_stats(srv) -> dict:
    i = _ServerInfo()
    _check(load().ms_server_stats(srv, ctypes.byref(i)), "ms_server_stats")
    return {f: int(getattr(i, f)) for f, _ in _ServerInfo._fields_}


def ms_server_destroy(srv) -> None:
    _check(load().ms_server_destroy(srv), "ms_server_destroy")


def ms_segment_staged(ctx, field, dims, dtype, out_asc, out_desc, out_ms) -> None:
    _check(load().ms_segment_staged(ctx, _ptr(field), _dims(dims), int(dtype), _ptr(out_asc),
                                    _ptr(out_desc), _ptr(out_ms)), "ms_segment_staged")


def ms_segment_host_many(ctx, host_fields, dims, dtypes, host_asc, host_desc, host_ms) -> list:
    """Many host fields through the pipelined host path; returns the region
    counts."""
    n = len(host_fields)
    ptrs = lambda xs: (c_vp * n)(*[_ptr(x) for x in xs])
    d = (ctypes.c_int64 * (3 * n))(*[int(v) for dd in dims for v in dd])
    t = (ctypes.c_int * n)(*[int(x) for x in dtypes])
    k = (ctypes.c_int64 * n)()
    _check(load().ms_segment_host_many(ctx, n, ptrs(host_fields), ctypes.cast(d, c_vp),
                                       ctypes.cast(t, c_vp), ptrs(host_asc), ptrs(host_desc),
                                       ptrs(host_ms), k), "ms_segment_host_many")
    return [int(x) for x in k]


def ms_segment_host(ctx, host_field, dims, dtype, host_asc, host_desc, host_ms) -> None:
    _check(load().ms_segment_host(ctx, _ptr(host_field), _dims(dims), int(dtype), _ptr(host_asc),
                                  _ptr(host_desc), _ptr(host_ms)), "ms_segment_host")


def ms_last_region_count(ctx) -> int:
    k = ctypes.c_int64(0)
    _check(load().ms_last_region_count(ctx, ctypes.byref(k)), "ms_last_region_count")
    return int(k.value)


def ms_order_keys(ctx, field, n, dtype, keys) -> None:
    _check(load().ms_order_keys(ctx, _ptr(field), int(n), int(dtype), _ptr(keys)), "ms_order_keys")


def ms_steepest(ctx, field, dims, dtype, up, dn) -> None:
    _check(load().ms_steepest(ctx, _ptr(field), _dims(dims), int(dtype), _ptr(up), _ptr(dn)),
           "ms_steepest")


def ms_compress(ctx, ptr, n) -> None:
    _check(load().ms_compress(ctx, _ptr(ptr), int(n)), "ms_compress")


def ms_pair_rank(ctx, asc, desc, n, ms) -> int:
    k = ctypes.c_int64(0)
    _check(load().ms_pair_rank(ctx, _ptr(asc), _ptr(desc), int(n), _ptr(ms), ctypes.byref(k)),
           "ms_pair_rank")
    return int(k.value)


def ms_pair_rank_noalloc(asc, desc, n, ms, stream=None) -> int:
    """MS ids of (asc, desc) without allocating device memory (n <=
    MS_NOALLOC_MAX_N); returns K.  ``stream``: torch.cuda.Stream, raw
    cudaStream_t int, or None for the default stream."""
    k = ctypes.c_int64(0)
    s = getattr(stream, "cuda_stream", stream)
    _check(load().ms_pair_rank_noalloc(_ptr(asc), _ptr(desc), int(n), _ptr(ms), ctypes.byref(k),
                                       s if s else None), "ms_pair_rank_noalloc")
    return int(k.value)


def ms_profile_enable(ctx, on: bool = True) -> None:
    _check(load().ms_profile_enable(ctx, 1 if on else 0), "ms_profile_enable")


def ms_profile_read(ctx) -> dict:
    """{'calls', 'launches', 'stages': {name: {'ms': total, 'launches': n}}}"""
    p = _Profile()
    _check(load().ms_profile_read(ctx, ctypes.byref(p)), "ms_profile_read")
    return {"calls": int(p.calls), "launches": int(p.launches),
            "stages": {STAGES[i]: {"ms": float(p.stage_ms[i]), "launches": int(p.stage_launches[i])}
                       for i in range(len(STAGES))}}


def ms_profile_stage_name(stage: int) -> str:
    return load().ms_profile_stage_name(int(stage)).decode()


def segment(ctx, field):
    """Convenience over ms_segment for a CUDA tensor: allocates the three
    int32 outputs with torch and returns (asc, desc, ms, K)."""
    import torch

    n = field.numel()
    asc = torch.empty(n, dtype=torch.int32, device=field.device)
    desc = torch.empty_like(asc)
    ms = torch.empty_like(asc)
    ms_segment(ctx, field, dims_of(field), dtype_code(field), asc, desc, ms)
    return asc, desc, ms, ms_last_region_count(ctx)
