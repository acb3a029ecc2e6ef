// ms_pair_rank_noalloc: the pair-ranking step (MS ids from asc / desc
// labels) for callers that cannot allocate device memory.  Its working
// memory is one file-scope device array, so the call itself never allocates:
// the array is part of the library's device image and every GPU that loads
// the library holds it until the process exits.
#include <cuda.h>

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
// Per device: the array's address and the id of the context it was looked up
// in.  A module's device variables live in one context; after
// cudaDeviceReset (or any other end of the primary context) the next context
// loads the module again and the variable may sit elsewhere, so the address
// is looked up again whenever the current context's id differs.
struct ScratchAddr {
  unsigned long long ctx_id = 0;
  void *ptr = nullptr;
};
ScratchAddr g_scratch[kMaxDevices];

typedef CUresult (*CtxGetCurrentFn)(CUcontext *);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long *);

// Id of the calling thread's current context (0 if none or unavailable).
unsigned long long current_ctx_id() {
  static CtxGetCurrentFn get_current = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_current = reinterpret_cast<CtxGetCurrentFn>(p);
    p = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      get_id = reinterpret_cast<CtxGetIdFn>(p);
    cudaGetLastError();
  });
  CUcontext c = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&c) != CUDA_SUCCESS || !c ||
      get_id(c, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of the array on the current device, for the current
// context.  The first call on a device (and the first after its context
// changed) looks it up, so it must come before any stream capture.
cudaError_t scratch_address(int device, void **out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  ScratchAddr &a = g_scratch[device];
  const unsigned long long id = current_ctx_id();
  if (!a.ptr || id == 0 || id != a.ctx_id) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);  // makes the context current
    if (e != cudaSuccess) return e;
    a.ptr = p;
    a.ctx_id = current_ctx_id();
  }
  *out = a.ptr;
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
