// Step 3 of the segmentation: path compression by pointer jumping
// (Sec. 4.2.1, Fig. 3) -- ptr[v] <- ptr[ptr[v]] until every pointer sits on a
// self-pointer (a maximum for up, a minimum for dn).
//
// Rounds are kernel launches.  Within a round each thread jumps its own
// vertex up to `iters` times, in place; a read may see another vertex's
// pointer before or after that vertex's own update in this round, and both
// lie on the same integral line, so the fixed point is the paper's (the order
// of evaluation changes the number of iterations, not the result -- Fig. 3's
// caption).  The first jump of round r reads pointers that already span at
// least 2^r steps, so round r leaves every pointer at least 2^(r+1) steps
// along its line or at the root: ceil(log2 n) + 1 rounds always suffice for a
// forest.  A round that finds nothing left to do clears its flag and all
// later rounds return at once, so the host can queue a fixed schedule
// without reading anything back.
#include "ms_internal.cuh"

namespace msseg {
namespace {

__device__ __forceinline__ bool jump_vertex(int32_t *__restrict__ p, int64_t v, int iters) {
  const int32_t p0 = __ldcg(p + v);
  int32_t cur = p0;
  bool done = false;
  for (int it = 0; it < iters; ++it) {
    const int32_t nxt = __ldcg(p + cur);
    if (nxt == cur) {
      done = true;
      break;
    }
    cur = nxt;
  }
  if (cur != p0) __stcg(p + v, cur);
  return done;
}

__global__ void k_compress_round(int32_t *a, int32_t *b, int64_t n, int iters, int round,
                                 DevStatus *st) {
  if (round > 0 && *(volatile unsigned int *)&st->round_open[round - 1] == 0u) return;
  bool open = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    open |= !jump_vertex(a, v, iters);
    if (b) open |= !jump_vertex(b, v, iters);
  }
  if (__any_sync(0xffffffffu, open) && (threadIdx.x & 31) == 0)
    atomicOr(&st->round_open[round], 1u);
}

__global__ void k_check_range(const int32_t *__restrict__ p, int64_t n, DevStatus *st) {
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
    const int32_t q = p[v];
    bad |= (q < 0) || ((int64_t)q >= n);
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(&st->bad_index, 1u);
}

int grid_for(int64_t n, int per_sm) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = (n + 255) / 256;
  const int64_t cap = (int64_t)sms * per_sm;
  return (int)(blocks < cap ? (blocks > 0 ? blocks : 1) : cap);
}

}  // namespace

cudaError_t launch_compress_round(int32_t *a, int32_t *b, int64_t n, int iters, int round,
                                  DevStatus *st, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ++tl_launches;
  k_compress_round<<<grid_for(n, 8), 256, 0, s>>>(a, b, n, iters, round, st);
  return cudaGetLastError();
}

cudaError_t launch_check_range(const int32_t *p, int64_t n, DevStatus *st, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ++tl_launches;
  k_check_range<<<grid_for(n, 8), 256, 0, s>>>(p, n, st);
  return cudaGetLastError();
}

}  // namespace msseg
