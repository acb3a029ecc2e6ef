// Sharding one field over several processes by z-slabs: the distributed
// computation the paper names as future work (Sec. 8), built from the same
// definitions (Sec. 4.2.1: steepest steps, then pointer jumping to the
// extremum each line reaches).
//
// A slab owns planes [z0, z1) and holds one halo plane on each side that
// exists.  The steepest step of an owned vertex needs only its stencil, which
// the halo completes, so it equals the whole field's step; jumping inside the
// slab then ends either at an owned extremum or at a halo vertex, where the
// line leaves the slab (an exit, stored as -(global index + 1)).  A line
// enters another slab only through that slab's first or last owned plane, so
// the slabs publish the labels of those planes; jumping over the published
// rows (each exit replaced by the row entry it points at) resolves every
// exit, and each slab then replaces its own exits.  The kernels here are that
// jumping and the encoding; the steepest step and the in-slab jumping are the
// step-by-step path's kernels.
#include "ms_internal.cuh"

namespace msseg {
namespace {

__global__ void k_slab_halo_self(int32_t *up, int32_t *dn, int64_t nxy, int64_t lo_planes,
                                 int64_t owned_planes, int64_t hi_planes) {
  const int64_t lo = lo_planes * nxy, hi = hi_planes * nxy;
  const int64_t hi_base = (lo_planes + owned_planes) * nxy;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < lo + hi; i += stride) {
    const int64_t v = i < lo ? i : hi_base + (i - lo);
    up[v] = (int32_t)v;
    dn[v] = (int32_t)v;
  }
}

__device__ __forceinline__ int32_t encode_root(int32_t r, int64_t owned_lo, int64_t owned_hi,
                                               int64_t base) {
  const int64_t g = (int64_t)r + base;
  return (r < owned_lo || r >= owned_hi) ? (int32_t)(-g - 1) : (int32_t)g;
}

__global__ void k_slab_encode(const int32_t *__restrict__ up, const int32_t *__restrict__ dn,
                              int64_t nxy, int64_t lo_planes, int64_t owned_planes, int64_t base,
                              int32_t *__restrict__ out_asc, int32_t *__restrict__ out_desc) {
  const int64_t owned_lo = lo_planes * nxy, owned_hi = (lo_planes + owned_planes) * nxy;
  const int64_t n = owned_planes * nxy;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    out_asc[i] = encode_root(dn[owned_lo + i], owned_lo, owned_hi, base);
    out_desc[i] = encode_root(up[owned_lo + i], owned_lo, owned_hi, base);
  }
}

// Row of the published plane holding global vertex h (binary search over the
// planes' z, sorted), or -1.
__device__ __forceinline__ int plane_slot(const long long *__restrict__ zs, const int *__restrict__ slot,
                                          int n_planes, long long z) {
  int lo = 0, hi = n_planes;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (zs[mid] < z)
      lo = mid + 1;
    else
      hi = mid;
  }
  return (lo < n_planes && zs[lo] == z) ? slot[lo] : -1;
}

// The row entry an exit code points at, or 0 with *bad set.
__device__ __forceinline__ int32_t follow_exit(const int32_t *rows, int32_t code, int kind,
                                               int64_t nxy, int64_t n_global,
                                               const long long *zs, const int *slot, int n_planes,
                                               bool *bad) {
  const int64_t h = -(int64_t)code - 1;
  if (h >= n_global) {
    *bad = true;
    return 0;
  }
  const int s = plane_slot(zs, slot, n_planes, h / nxy);
  if (s < 0) {
    *bad = true;
    return 0;
  }
  return __ldcg(rows + ((int64_t)s * 2 + kind) * nxy + h % nxy);
}

// One jumping round over the published rows ([plane][asc, desc][x + nx y]);
// rounds after one that left nothing open return at once.
__global__ void k_slab_rows_round(int32_t *rows, int n_planes, int64_t nxy, int64_t n_global,
                                  const long long *zs, const int *slot, DevStatus *st, int round) {
  if (round > 0 && *(volatile unsigned int *)&st->round_open[round - 1] == 0u) return;
  bool open = false, bad = false;
  const int64_t n = (int64_t)n_planes * 2 * nxy;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    const int32_t code = __ldcg(rows + i);
    if (code >= 0) continue;
    const int kind = (int)((i / nxy) & 1);
    const int32_t next = follow_exit(rows, code, kind, nxy, n_global, zs, slot, n_planes, &bad);
    if (bad) break;
    __stcg(rows + i, next);
    open |= next < 0;
  }
  if (__any_sync(0xffffffffu, open) && (threadIdx.x & 31) == 0)
    atomicOr(&st->round_open[round], 1u);
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->bad_index, 1u);
}

// The slab's own exits replaced by the resolved rows.
__global__ void k_slab_apply(int32_t *asc, int32_t *desc, int64_t n, const int32_t *rows,
                             int64_t nxy, int64_t n_global, const long long *zs, const int *slot,
                             int n_planes, DevStatus *st) {
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    int32_t a = asc[i], d = desc[i];
    if (a < 0) a = follow_exit(rows, a, 0, nxy, n_global, zs, slot, n_planes, &bad);
    if (d < 0) d = follow_exit(rows, d, 1, nxy, n_global, zs, slot, n_planes, &bad);
    if (a < 0 || d < 0) bad = true;  // an exit the rows left unresolved
    asc[i] = a;
    desc[i] = d;
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->bad_index, 1u);
}

__global__ void k_check_nonneg(const int32_t *p, int64_t n, DevStatus *st) {
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    bad |= p[i] < 0;
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->bad_index, 1u);
}

unsigned int blocks_for(int64_t n) {
  static int sms = 0;
  if (!sms) {
    int dev = 0, v = 152;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) v = 152;
    sms = v;
  }
  int64_t b = (n + 255) / 256;
  const int64_t cap = (int64_t)sms * 8;
  if (b > cap) b = cap;
  return (unsigned int)(b > 0 ? b : 1);
}

}  // namespace

cudaError_t launch_slab_halo_self(int32_t *up, int32_t *dn, int64_t nxy, int64_t lo_planes,
                                  int64_t owned_planes, int64_t hi_planes, cudaStream_t s) {
  const int64_t n = (lo_planes + hi_planes) * nxy;
  if (n <= 0) return cudaSuccess;
  ++tl_launches;
  k_slab_halo_self<<<blocks_for(n), 256, 0, s>>>(up, dn, nxy, lo_planes, owned_planes, hi_planes);
  return cudaGetLastError();
}

cudaError_t launch_slab_encode(const int32_t *up, const int32_t *dn, int64_t nxy, int64_t lo_planes,
                               int64_t owned_planes, int64_t base, int32_t *out_asc,
                               int32_t *out_desc, cudaStream_t s) {
  ++tl_launches;
  k_slab_encode<<<blocks_for(owned_planes * nxy), 256, 0, s>>>(up, dn, nxy, lo_planes, owned_planes,
                                                               base, out_asc, out_desc);
  return cudaGetLastError();
}

cudaError_t launch_slab_rows_round(int32_t *rows, int n_planes, int64_t nxy, int64_t n_global,
                                   const long long *zs, const int *slot, DevStatus *st, int round,
                                   cudaStream_t s) {
  ++tl_launches;
  k_slab_rows_round<<<blocks_for((int64_t)n_planes * 2 * nxy), 256, 0, s>>>(
      rows, n_planes, nxy, n_global, zs, slot, st, round);
  return cudaGetLastError();
}

cudaError_t launch_slab_apply(int32_t *asc, int32_t *desc, int64_t n, const int32_t *rows,
                              int64_t nxy, int64_t n_global, const long long *zs, const int *slot,
                              int n_planes, DevStatus *st, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ++tl_launches;
  k_slab_apply<<<blocks_for(n), 256, 0, s>>>(asc, desc, n, rows, nxy, n_global, zs, slot, n_planes,
                                             st);
  return cudaGetLastError();
}

cudaError_t launch_check_nonneg(const int32_t *p, int64_t n, DevStatus *st, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ++tl_launches;
  k_check_nonneg<<<blocks_for(n), 256, 0, s>>>(p, n, st);
  return cudaGetLastError();
}

}  // namespace msseg
