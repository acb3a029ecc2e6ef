// Step 4 of the segmentation: MS ids (Sec. 3.4, Sec. 4.2.2).  Vertices with
// the same (asc, desc) pair share a region; the id is the rank of the pair
// among the distinct pairs, lexicographic with asc first.
//
//   insert : every vertex's pair goes into an open-addressing hash set
//            (lanes of a warp holding the same pair insert it once); each new
//            pair is also appended to a compact list.
//   sort   : LSD radix sort of the list on the compacted key (asc << b) | desc,
//            b = bit width of n - 1, 8 bits per pass, stable scatter.
//   assign : the sorted position of each pair is stored in its table slot.
//   lookup : every vertex reads its pair's rank from the table.
#include <algorithm>

#include "ms_internal.cuh"

namespace msseg {
namespace {

constexpr unsigned long long kEmpty = ~0ull;

__device__ __forceinline__ unsigned long long pack_pair(int32_t a, int32_t d) {
  return ((unsigned long long)(uint32_t)a << 32) | (uint32_t)d;
}

__device__ __forceinline__ unsigned int lane_id() { return threadIdx.x & 31u; }

__device__ void table_insert(const RankScratch &rs, unsigned long long key, DevStatus *st) {
  if (*(volatile unsigned int *)&st->hash_overflow) return;  // the caller retries larger
  const unsigned int mask = rs.capacity - 1u;
  unsigned int slot = (unsigned int)hash_mix64(key) & mask;
  for (unsigned int probe = 0; probe < rs.probe_limit; ++probe) {
    unsigned long long cur = *(volatile unsigned long long *)&rs.table_keys[slot];
    if (cur == key) return;
    if (cur == kEmpty) {
      cur = atomicCAS(&rs.table_keys[slot], kEmpty, key);
      if (cur == kEmpty) {
        const unsigned int at = atomicAdd(&st->n_unique, 1u);
        if (at < rs.max_unique)
          rs.list[at] = key;
        else
          atomicOr(&st->hash_overflow, 1u);
        return;
      }
      if (cur == key) return;
    }
    slot = (slot + 1u) & mask;
  }
  atomicOr(&st->hash_overflow, 1u);
}

__device__ __forceinline__ int table_find(const RankScratch &rs, unsigned long long key) {
  const unsigned int mask = rs.capacity - 1u;
  unsigned int slot = (unsigned int)hash_mix64(key) & mask;
  for (unsigned int probe = 0; probe < rs.capacity; ++probe) {
    const unsigned long long cur = __ldg(&rs.table_keys[slot]);
    if (cur == key) return (int)slot;
    if (cur == kEmpty) return -1;
    slot = (slot + 1u) & mask;
  }
  return -1;
}

// Labels must lie in [0, bound).
__global__ void k_pairs_insert(const int32_t *__restrict__ asc, const int32_t *__restrict__ desc,
                               int64_t n, int64_t bound, RankScratch rs, DevStatus *st) {
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  // the loop bound keeps whole warps together for __match_any_sync
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t v = base + threadIdx.x;
    unsigned long long key = kEmpty;
    if (v < n) {
      const int32_t a = asc[v], d = desc[v];
      if (a < 0 || d < 0 || (int64_t)a >= bound || (int64_t)d >= bound)
        bad = true;
      else
        key = pack_pair(a, d);
    }
    const unsigned int peers = __match_any_sync(0xffffffffu, key);
    if (key != kEmpty && (__ffs(peers) - 1) == (int)lane_id()) table_insert(rs, key, st);
  }
  if (__any_sync(0xffffffffu, bad) && lane_id() == 0) atomicOr(&st->bad_index, 1u);
}

// Packed (asc << 32) | desc keys, labels in [0, bound); keys may repeat.
__global__ void k_keys_insert(const unsigned long long *__restrict__ keys, int64_t n, int64_t bound,
                              RankScratch rs, DevStatus *st) {
  bool bad = false;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t i = base + threadIdx.x;
    unsigned long long key = kEmpty;
    if (i < n) {
      key = keys[i];
      const int64_t a = (int64_t)(key >> 32), d = (int64_t)(key & 0xffffffffull);
      if (a >= bound || d >= bound) {
        bad = true;
        key = kEmpty;
      }
    }
    const unsigned int peers = __match_any_sync(0xffffffffu, key);
    if (key != kEmpty && (__ffs(peers) - 1) == (int)lane_id()) table_insert(rs, key, st);
  }
  if (__any_sync(0xffffffffu, bad) && lane_id() == 0) atomicOr(&st->bad_index, 1u);
}

// b >= 0: the key is (asc << 32) | desc with labels below 2^b, sorted on the
// compacted (asc << b) | desc; b < 0: the key is sorted as it is.
__device__ __forceinline__ unsigned int sort_digit(unsigned long long key, int b, int shift) {
  const unsigned long long compact = b >= 0 ? (((key >> 32) << b) | (key & 0xffffffffull)) : key;
  return (unsigned int)(compact >> shift) & 255u;
}

// m_dev (optional): the key count on the device, at most m (graph replays
// size their launches from the capacity m and read the count here).
__device__ __forceinline__ unsigned int count_of(unsigned int m, const unsigned int *m_dev) {
  return m_dev ? min(*m_dev, m) : m;
}

__global__ void k_radix_hist(const unsigned long long *__restrict__ in, unsigned int m,
                             const unsigned int *m_dev, int b, int shift,
                             unsigned int *__restrict__ hist) {
  m = count_of(m, m_dev);
  __shared__ unsigned int h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const unsigned int chunk = (m + gridDim.x - 1) / gridDim.x;
  const unsigned int lo = blockIdx.x * chunk;
  const unsigned int hi = min(m, lo + chunk);
  for (unsigned int i = lo + threadIdx.x; i < hi; i += blockDim.x)
    atomicAdd(&h[sort_digit(in[i], b, shift)], 1u);
  __syncthreads();
  hist[threadIdx.x * gridDim.x + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan, in place, of the digit-major histogram hist[d * B + j]:
// afterwards entry (d, j) is where block j's keys of digit d start.  Two
// launches over chunks of kScanChunk entries (n is a multiple of 256, so
// every chunk starts 16-byte aligned): the chunk sums, then each chunk's
// scan from the sum of the chunks before it.  Every thread reads and writes
// 8 consecutive entries as two 16-byte vectors.
constexpr int kScanThreads = 1024;
constexpr int kScanChunk = kScanThreads * 8;
constexpr int kScanMaxChunks = 256;  // rank scratch keeps this many chunk sums
// Sorts of more keys than this use 2048-key blocks and the scan launches.
constexpr unsigned int kSortScanFrom = 1u << 16;

__device__ __forceinline__ void load8(const unsigned int *p, unsigned int i0, unsigned int n,
                                      unsigned int (&v)[8]) {
  if (i0 + 8 <= n) {
    const uint4 a = *reinterpret_cast<const uint4 *>(p + i0), b = *reinterpret_cast<const uint4 *>(p + i0 + 4);
    v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w, v[4] = b.x, v[5] = b.y, v[6] = b.z, v[7] = b.w;
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = i0 + k < n ? p[i0 + k] : 0u;
  }
}

// Block-wide exclusive sum of one value per thread (kScanThreads threads);
// also the total.
__device__ __forceinline__ unsigned int scan_block_excl(unsigned int v, unsigned int *total,
                                                        unsigned int *sh) {
  const unsigned int lane = lane_id(), warp = threadIdx.x >> 5;
  unsigned int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= (unsigned)o) incl += t;
  }
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    const unsigned int w = sh[lane];
    unsigned int wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= (unsigned)o) wi += t;
    }
    sh[lane] = wi - w;  // exclusive
    if (lane == 31) sh[32] = wi;
  }
  __syncthreads();
  *total = sh[32];
  return sh[warp] + incl - v;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_sums(const unsigned int *__restrict__ hist,
                                                            unsigned int n,
                                                            unsigned int *__restrict__ sums) {
  __shared__ unsigned int sh[33];
  unsigned int v[8];
  load8(hist, blockIdx.x * kScanChunk + threadIdx.x * 8, n, v);
  unsigned int t = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) t += v[k];
  unsigned int tot = 0;
  scan_block_excl(t, &tot, sh);
  if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) k_scan_chunks(unsigned int *__restrict__ hist,
                                                              unsigned int n,
                                                              const unsigned int *__restrict__ sums) {
  __shared__ unsigned int sh[33];
  __shared__ unsigned int s_before;
  if (threadIdx.x < 32) {  // the chunks before this one (at most kScanMaxChunks)
    unsigned int b = 0;
    for (unsigned int j = threadIdx.x; j < blockIdx.x; j += 32) b += sums[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) b += __shfl_xor_sync(0xffffffffu, b, o);
    if (threadIdx.x == 0) s_before = b;
  }
  const unsigned int i0 = blockIdx.x * kScanChunk + threadIdx.x * 8;
  unsigned int v[8];
  load8(hist, i0, n, v);
  unsigned int t = 0;
#pragma unroll
  for (int k = 0; k < 8; ++k) t += v[k];
  unsigned int tot = 0;
  unsigned int run = scan_block_excl(t, &tot, sh) + s_before;  // the scan's barriers order s_before
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    const unsigned int x = v[k];
    v[k] = run;
    run += x;
  }
  if (i0 + 8 <= n) {
    *reinterpret_cast<uint4 *>(hist + i0) = make_uint4(v[0], v[1], v[2], v[3]);
    *reinterpret_cast<uint4 *>(hist + i0 + 4) = make_uint4(v[4], v[5], v[6], v[7]);
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k)
      if (i0 + k < n) hist[i0 + k] = v[k];
  }
}

// Stable scatter: block j re-reads the chunk it histogrammed, 256 keys at a
// time; a key's destination is its digit's start (all keys of lower digits)
// plus the keys of the same digit in earlier blocks, in earlier warps of the
// tile and in earlier lanes of its own warp.  The per-block digit offsets are
// computed here from the raw histogram (no separate scan launch).
__global__ void __launch_bounds__(256) k_radix_scatter(const unsigned long long *__restrict__ in,
                                                       unsigned long long *__restrict__ out,
                                                       unsigned int m, const unsigned int *m_dev,
                                                       int b, int shift,
                                                       const unsigned int *__restrict__ hist,
                                                       int scanned) {
  m = count_of(m, m_dev);
  __shared__ unsigned int run[256];
  __shared__ unsigned int wcnt[8][256];
  const unsigned int warp = threadIdx.x >> 5, lane = lane_id();
  if (scanned) {
    // the histogram scan left each (digit, block) its first output position
    run[threadIdx.x] = hist[threadIdx.x * gridDim.x + blockIdx.x];
    __syncthreads();
  } else {
    // digit d = threadIdx.x: total over all blocks, and over blocks before this one
    const unsigned int *row = hist + threadIdx.x * gridDim.x;
    unsigned int tot = 0, before = 0;
#pragma unroll 8
    for (unsigned int j = 0; j < gridDim.x; ++j) {
      const unsigned int v = row[j];
      tot += v;
      if (j < blockIdx.x) before += v;
    }
    // exclusive scan of the 256 digit totals
    unsigned int incl = tot;
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
      if ((int)lane >= o) incl += t;
    }
    if (lane == 31) wcnt[0][warp] = incl;
    __syncthreads();
    unsigned int wbase = 0;
    for (unsigned int k = 0; k < warp; ++k) wbase += wcnt[0][k];
    run[threadIdx.x] = wbase + incl - tot + before;
    __syncthreads();
  }
  const unsigned int chunk = (m + gridDim.x - 1) / gridDim.x;
  const unsigned int lo = blockIdx.x * chunk;
  const unsigned int hi = min(m, lo + chunk);
  for (unsigned int t0 = lo; t0 < hi; t0 += 256) {
    for (int w = 0; w < 8; ++w) wcnt[w][threadIdx.x] = 0;
    __syncthreads();
    const unsigned int i = t0 + threadIdx.x;
    const bool valid = i < hi;
    unsigned long long key = 0;
    unsigned int d = 0x100u + lane;  // invalid lanes get distinct private digits
    if (valid) {
      key = in[i];
      d = sort_digit(key, b, shift);
    }
    const unsigned int peers = __match_any_sync(0xffffffffu, d);
    const unsigned int below = __popc(peers & ((1u << lane) - 1u));
    if (valid && below == 0) wcnt[warp][d] = __popc(peers);
    __syncthreads();
    if (valid) {
      unsigned int pre = 0;
      for (unsigned int w = 0; w < warp; ++w) pre += wcnt[w][d];
      out[run[d] + pre + below] = key;
    }
    __syncthreads();
    unsigned int tot = 0;
    for (int w = 0; w < 8; ++w) tot += wcnt[w][threadIdx.x];
    run[threadIdx.x] += tot;
    __syncthreads();
  }
}

__global__ void k_pairs_assign(const unsigned long long *__restrict__ sorted, unsigned int m,
                               const unsigned int *m_dev, RankScratch rs) {
  m = count_of(m, m_dev);
  const unsigned int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int slot = table_find(rs, sorted[i]);
  if (slot >= 0) rs.table_vals[slot] = (int32_t)i;
}

__global__ void k_pairs_lookup(const int32_t *__restrict__ asc, const int32_t *__restrict__ desc,
                               int64_t n, RankScratch rs, int32_t *__restrict__ ms) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < n; base += stride) {
    const int64_t v = base + threadIdx.x;
    unsigned long long key = kEmpty;
    if (v < n) key = pack_pair(asc[v], desc[v]);
    const unsigned int peers = __match_any_sync(0xffffffffu, key);
    const int leader = __ffs(peers) - 1;
    int32_t r = -1;
    if (key != kEmpty && leader == (int)lane_id()) {
      const int slot = table_find(rs, key);
      r = slot >= 0 ? rs.table_vals[slot] : -1;
    }
    r = __shfl_sync(0xffffffffu, r, leader);
    if (v < n) ms[v] = r;
  }
}

int sm_count() {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms;
}

unsigned int grid_n(int64_t n, int per_sm) {
  int64_t blocks = (n + 255) / 256;
  const int64_t cap = (int64_t)sm_count() * per_sm;
  if (blocks > cap) blocks = cap;
  return (unsigned int)(blocks > 0 ? blocks : 1);
}

}  // namespace

unsigned int sort_blocks_cap_of(unsigned int capacity) {
  return std::max<unsigned int>(kSortBlocks, capacity / 2 / 4096);
}

size_t rank_scratch_bytes(unsigned int capacity) {
  const size_t maxu = capacity / 2;
  return (size_t)capacity * 8 + (size_t)capacity * 4 + maxu * 8 * 2 +
         256 * (size_t)sort_blocks_cap_of(capacity) * 4 + 4 * 256;
}

void rank_scratch_carve(void *base, unsigned int capacity, RankScratch *rs) {
  char *p = static_cast<char *>(base);
  rs->capacity = capacity;
  rs->max_unique = capacity / 2;
  rs->probe_limit = capacity;
  rs->table_keys = reinterpret_cast<unsigned long long *>(p);
  p += (size_t)capacity * 8;
  rs->list = reinterpret_cast<unsigned long long *>(p);
  p += (size_t)rs->max_unique * 8;
  rs->tmp = reinterpret_cast<unsigned long long *>(p);
  p += (size_t)rs->max_unique * 8;
  rs->table_vals = reinterpret_cast<int32_t *>(p);
  p += (size_t)capacity * 4;
  rs->hist = reinterpret_cast<unsigned int *>(p);
  p += 256 * (size_t)sort_blocks_cap_of(capacity) * 4;
  rs->scan_sums = reinterpret_cast<unsigned int *>(p);  // the last 4 * 256 bytes
  rs->sort_blocks_cap = sort_blocks_cap_of(capacity);
}

cudaError_t launch_pairs_insert(const int32_t *asc, const int32_t *desc, int64_t n,
                                const RankScratch &rs, DevStatus *st, cudaStream_t s,
                                int64_t label_bound) {
  cudaError_t e = cudaMemsetAsync(rs.table_keys, 0xff, (size_t)rs.capacity * 8, s);
  if (e != cudaSuccess || n <= 0) return e;
  ++tl_launches;
  k_pairs_insert<<<grid_n(n, 8), 256, 0, s>>>(asc, desc, n, label_bound > 0 ? label_bound : n, rs,
                                              st);
  return cudaGetLastError();
}

cudaError_t launch_keys_insert(const unsigned long long *keys, int64_t n, int64_t label_bound,
                               const RankScratch &rs, DevStatus *st, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(rs.table_keys, 0xff, (size_t)rs.capacity * 8, s);
  if (e != cudaSuccess || n <= 0) return e;
  ++tl_launches;
  k_keys_insert<<<grid_n(n, 8), 256, 0, s>>>(keys, n, label_bound, rs, st);
  return cudaGetLastError();
}

// Sorts rs.list[0, m) in place (the result always ends in rs.list).
cudaError_t launch_pairs_sort(const RankScratch &rs, unsigned int m, int key_bits,
                              cudaStream_t s, int raw_bits, const unsigned int *m_dev) {
  if (m <= 1) return cudaSuccess;
  unsigned long long *src = rs.list, *dst = rs.tmp;
  const int b = raw_bits > 0 ? -1 : key_bits;  // bit width of one label, or raw keys
  const int total = raw_bits > 0 ? raw_bits : 2 * key_bits;
  // small sorts: 1024 keys a block (at most 64 blocks up to 2^16 keys, so each
  // block's offset computation, a pass over its digit's row, stays short;
  // 4096-key blocks made 13.5K keys a 4-block pass of 26 us);
  // larger ones: 2048 keys a block (up to 8 blocks an SM) and the histogram
  // scanned by two launches (a block with 4096 or more keys walks them 256 at
  // a time, three barriers each: at 350K keys, 85 blocks took 33 us a pass)
  unsigned int blocks = std::max(1u, std::min((unsigned)kSortBlocks, (m + 1023) / 1024));
  const bool large = m > kSortScanFrom;
  if (large)
    blocks = std::max(1u, std::min({rs.sort_blocks_cap, (m + 2047) / 2048,
                                    (unsigned)sm_count() * 8}));
  for (int shift = 0; shift < total; shift += 8) {
    ++tl_launches;
    k_radix_hist<<<blocks, 256, 0, s>>>(src, m, m_dev, b, shift, rs.hist);
    if (large) {
      const unsigned int n = 256 * blocks, chunks = (n + kScanChunk - 1) / kScanChunk;
      if (chunks > (unsigned)kScanMaxChunks) return cudaErrorInvalidValue;  // blocks <= 8 an SM
      tl_launches += 2;
      k_scan_sums<<<chunks, kScanThreads, 0, s>>>(rs.hist, n, rs.scan_sums);
      k_scan_chunks<<<chunks, kScanThreads, 0, s>>>(rs.hist, n, rs.scan_sums);
    }
    ++tl_launches;
    k_radix_scatter<<<blocks, 256, 0, s>>>(src, dst, m, m_dev, b, shift, rs.hist, large ? 1 : 0);
    unsigned long long *t = src;
    src = dst;
    dst = t;
  }
  if (src != rs.list)
    return cudaMemcpyAsync(rs.list, src, (size_t)m * 8, cudaMemcpyDeviceToDevice, s);
  return cudaGetLastError();
}

cudaError_t launch_pairs_assign(const RankScratch &rs, unsigned int m, cudaStream_t s,
                                const unsigned int *m_dev) {
  if (m == 0) return cudaSuccess;
  ++tl_launches;
  k_pairs_assign<<<(m + 255) / 256, 256, 0, s>>>(rs.list, m, m_dev, rs);
  return cudaGetLastError();
}

cudaError_t launch_pairs_lookup(const int32_t *asc, const int32_t *desc, int64_t n,
                                const RankScratch &rs, int32_t *ms, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  ++tl_launches;
  k_pairs_lookup<<<grid_n(n, 8), 256, 0, s>>>(asc, desc, n, rs, ms);
  return cudaGetLastError();
}

cudaError_t launch_fill_u64(unsigned long long *p, size_t count, unsigned long long v,
                            cudaStream_t s) {
  (void)v;
  return cudaMemsetAsync(p, 0xff, count * 8, s);
}

}  // namespace msseg
