// ms_pair_rank_noalloc: the pair-ranking step (MS ids from asc / desc
// labels) for callers that cannot allocate device memory.  Its working
// memory is one file-scope device array, so the call itself never allocates:
// the array is part of the library's device image and every GPU that loads
// the library holds it until the process exits.
#include <mutex>

#include "ms_internal.cuh"

namespace msseg {
namespace {

// Largest n accepted: the hash set then needs at most 2 * n slots.
constexpr int64_t kNoAllocMaxN = MS_NOALLOC_MAX_N;
constexpr unsigned int kNoAllocCapacity = 1u << 19;  // power of two >= 2 * kNoAllocMaxN
static_assert((int64_t)kNoAllocCapacity >= 2 * kNoAllocMaxN, "hash set too small");

constexpr size_t kStatusBytes = (sizeof(DevStatus) + 255) & ~(size_t)255;
constexpr size_t kRankBytes = (size_t)kNoAllocCapacity * 8 + (size_t)kNoAllocCapacity * 4 +
                              (size_t)(kNoAllocCapacity / 2) * 8 * 2 + 256 * (size_t)kSortBlocks * 4 +
                              4 * 256;
constexpr size_t kScratchBytes = kStatusBytes + kRankBytes;

// The shared working memory: a status block, then the rank scratch.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void *g_scratch_ptr[kMaxDevices] = {};

// Device address of the array on the current device (set up once per device;
// the first call on a device does this, so it must come before any stream
// capture on that device).
cudaError_t scratch_address(int device, void **out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[device] = p;
  }
  *out = g_scratch_ptr[device];
  return cudaSuccess;
}

int bits_for(int64_t x) {
  int b = 0;
  while (x > 0) {
    ++b;
    x >>= 1;
  }
  return b;
}

}  // namespace
}  // namespace msseg

using namespace msseg;

extern "C" ms_status ms_pair_rank_noalloc(const int32_t *asc, const int32_t *desc, int64_t n,
                                          int32_t *ms, int64_t *k_out, void *cuda_stream) {
  if (n < 0 || (n > 0 && (!asc || !desc || !ms))) return MS_ERR_INVALID_ARG;
  if (n > kNoAllocMaxN) return MS_ERR_TOO_LARGE;
  if (n == 0) {
    if (k_out) *k_out = 0;
    return MS_OK;
  }
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess || device < 0 || device >= kMaxDevices) {
    cudaGetLastError();
    return MS_ERR_CUDA;
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  void *base = nullptr;
  if (scratch_address(device, &base) != cudaSuccess) {
    cudaGetLastError();
    return MS_ERR_CUDA;
  }
  if (rank_scratch_bytes(kNoAllocCapacity) > kRankBytes) return MS_ERR_CUDA;  // layouts agree
  DevStatus *st = static_cast<DevStatus *>(base);
  RankScratch rs;
  rank_scratch_carve(static_cast<char *>(base) + kStatusBytes, kNoAllocCapacity, &rs);
  // the array keeps the previous call's contents: clear what must start at
  // zero (the status block; the hash set is reset by the insert launcher)
  if (cudaMemsetAsync(st, 0, sizeof(DevStatus), s) != cudaSuccess) return MS_ERR_CUDA;
  if (launch_pairs_insert(asc, desc, n, rs, st, s) != cudaSuccess) return MS_ERR_CUDA;
  DevStatus h;
  if (cudaMemcpyAsync(&h, st, sizeof(DevStatus), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MS_ERR_CUDA;
  if (h.bad_index) return MS_ERR_INVALID_ARG;
  if (h.hash_overflow) return MS_ERR_CUDA;  // cannot happen: capacity >= 2 * n
  const unsigned int m = h.n_unique;
  if (launch_pairs_sort(rs, m, bits_for(n - 1), s) != cudaSuccess) return MS_ERR_CUDA;
  if (launch_pairs_assign(rs, m, s) != cudaSuccess) return MS_ERR_CUDA;
  if (launch_pairs_lookup(asc, desc, n, rs, ms, s) != cudaSuccess) return MS_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return MS_ERR_CUDA;
  if (k_out) *k_out = m;
  return MS_OK;
}
