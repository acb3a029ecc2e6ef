// Steps 1 and 2 of the segmentation: order keys (Sec. 4.1) and steepest
// neighbours (Sec. 4.2.1, first step) -- the one-thread-per-vertex form.
#include "ms_internal.cuh"

namespace msseg {
namespace {

__device__ __forceinline__ void flag_warp(unsigned int *word, bool pred) {
  if (__any_sync(0xffffffffu, pred) && (threadIdx.x & 31) == 0) atomicOr(word, 1u);
}

__device__ __forceinline__ void count_warp(unsigned int *counter, bool pred) {
  const unsigned int m = __ballot_sync(0xffffffffu, pred);
  if (m && (threadIdx.x & 31) == 0) atomicAdd(counter, (unsigned int)__popc(m));
}

__global__ void k_order_keys(const void *__restrict__ field, int64_t n, int dtype,
                             uint32_t *__restrict__ keys, DevStatus *st) {
  bool nan = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    if (i < n) {
      const uint32_t b = load_bits(field, dtype, i);
      nan |= is_nan_bits(b);
      keys[i] = order_key_bits(b);
    }
  }
  flag_warp(&st->nan_flag, nan);
}

// The 14 Freudenthal neighbours: every non-zero offset whose components are
// all >= 0 or all <= 0.
__constant__ int8_t kNbr[14][3] = {
    {-1, -1, -1}, {0, -1, -1}, {-1, 0, -1}, {0, 0, -1}, {-1, -1, 0}, {0, -1, 0}, {-1, 0, 0},
    {1, 0, 0},    {0, 1, 0},   {1, 1, 0},   {0, 0, 1},  {1, 0, 1},   {0, 1, 1},  {1, 1, 1}};

// One thread per vertex: the candidates are packed as (key << 32 | index), so
// that a plain 64-bit max / min is the (value, index) order of Sec. 4.1.
__global__ void k_steepest_simple(const void *__restrict__ field, int dtype, int64_t nx,
                                  int64_t ny, int64_t nz, int32_t *__restrict__ up,
                                  int32_t *__restrict__ dn, DevStatus *st) {
  const int64_t n = nx * ny * nz;
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool nan = false, is_max = false, is_min = false;
  if (v < n) {
    const int64_t x = v % nx, r = v / nx, y = r % ny, z = r / ny;
    const uint32_t b = load_bits(field, dtype, v);
    nan = is_nan_bits(b);
    const unsigned long long self = ((unsigned long long)order_key_bits(b) << 32) | (uint32_t)v;
    unsigned long long hi = self, lo = self;
#pragma unroll
    for (int k = 0; k < 14; ++k) {
      const int64_t X = x + kNbr[k][0], Y = y + kNbr[k][1], Z = z + kNbr[k][2];
      if (X < 0 || Y < 0 || Z < 0 || X >= nx || Y >= ny || Z >= nz) continue;
      const int64_t u = X + nx * (Y + ny * Z);
      const unsigned long long pk =
          ((unsigned long long)order_key_bits(load_bits(field, dtype, u)) << 32) | (uint32_t)u;
      hi = pk > hi ? pk : hi;
      lo = pk < lo ? pk : lo;
    }
    up[v] = (int32_t)(uint32_t)hi;
    dn[v] = (int32_t)(uint32_t)lo;
    is_max = hi == self;
    is_min = lo == self;
  }
  flag_warp(&st->nan_flag, nan);
  count_warp(&st->n_max, is_max);
  count_warp(&st->n_min, is_min);
}

}  // namespace

cudaError_t launch_order_keys(const void *field, int64_t n, int dtype, uint32_t *keys,
                              DevStatus *st, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int64_t blocks = (n + 255) / 256;
  if (blocks > (int64_t)sms * 16) blocks = (int64_t)sms * 16;
  ++tl_launches;
  k_order_keys<<<(unsigned)blocks, 256, 0, s>>>(field, n, dtype, keys, st);
  return cudaGetLastError();
}

cudaError_t launch_steepest_simple(const void *field, const int64_t dims[3], int dtype,
                                   int32_t *up, int32_t *dn, DevStatus *st, cudaStream_t s) {
  const int64_t n = dims[0] * dims[1] * dims[2];
  if (n <= 0) return cudaSuccess;
  ++tl_launches;
  k_steepest_simple<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(field, dtype, dims[0], dims[1],
                                                                 dims[2], up, dn, st);
  return cudaGetLastError();
}

}  // namespace msseg
