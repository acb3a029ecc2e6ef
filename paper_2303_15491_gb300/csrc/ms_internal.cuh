// Internal declarations shared by the CUDA translation units of libmsseg.
#pragma once

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/ms.h"

namespace msseg {

// Device-side status words, zeroed at the start of every call.
struct DevStatus {
  unsigned int nan_flag;       // a NaN was seen in the field
  unsigned int bad_index;      // an index outside [0, n) was seen
  unsigned int not_converged;  // set by the last compression round that did not finish
  unsigned int hash_overflow;  // the pair table ran out of room
  unsigned int n_unique;       // distinct (asc, desc) pairs inserted
  unsigned int n_max;          // maxima found by the steepest step
  unsigned int n_min;          // minima found by the steepest step
  unsigned int pool_overflow;  // the tiled path's pair pool ran out of room
  unsigned int timeout;        // a bounded wait in a kernel gave up
  unsigned int pending;         // probe: sampled tile roots whose chase needs more hops
  unsigned int sampled;         // probe: tile roots sampled
  unsigned int pad;
  unsigned int round_open[64];  // round_open[r] != 0: round r left work for round r+1
};

// Order key of an IEEE binary32 bit pattern (Sec. 4.1): -0 is folded onto +0
// so that equal reals tie and fall through to the index comparison; then
// positives get the sign bit set and negatives are complemented, which makes
// unsigned integer order equal real order.  NaN patterns are the caller's to
// reject; no real value maps to 0 or to 0xFFFFFFFF.
__host__ __device__ __forceinline__ uint32_t order_key_bits(uint32_t b) {
  if ((b << 1) == 0u) b = 0u;
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

// 64-bit finaliser of MurmurHash3 (Appleby): spreads a packed key over an
// open-addressing table.
__device__ __forceinline__ unsigned long long hash_mix64(unsigned long long k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

__host__ __device__ __forceinline__ bool is_nan_bits(uint32_t b) {
  return (b & 0x7fffffffu) > 0x7f800000u;
}

__device__ __forceinline__ uint32_t load_bits(const void *field, int dtype, int64_t i) {
  if (dtype == MS_F16) {
    const __half h = reinterpret_cast<const __half *>(field)[i];
    return __float_as_uint(__half2float(h));  // exact widening
  }
  return __ldg(reinterpret_cast<const uint32_t *>(field) + i);
}

// Kernels launched by this host thread (read by the profiler).
extern thread_local long long tl_launches;

// Device bytes a context holds between calls (its scratch, staging and status
// buffers), and the release of everything but its status block (the next call
// allocates again).  Used by the request loop to keep its slots within budget.
size_t ctx_resident_bytes(const ms_ctx *c);
void ctx_release_scratch(ms_ctx *c);

// ---- launchers (stream-ordered, no synchronisation) ----------------------
cudaError_t launch_order_keys(const void *field, int64_t n, int dtype, uint32_t *keys,
                              DevStatus *st, cudaStream_t s);
cudaError_t launch_steepest_simple(const void *field, const int64_t dims[3], int dtype,
                                   int32_t *up, int32_t *dn, DevStatus *st, cudaStream_t s);
cudaError_t launch_check_range(const int32_t *p, int64_t n, DevStatus *st, cudaStream_t s);
cudaError_t launch_compress_round(int32_t *a, int32_t *b, int64_t n, int iters, int round,
                                  DevStatus *st, cudaStream_t s);

// Pair ranking (Sec. 4.2.2) working memory.
struct RankScratch {
  unsigned long long *table_keys;  // capacity entries, empty = ~0ull
  int32_t *table_vals;             // capacity entries
  unsigned long long *list;        // unique keys, up to max_unique
  unsigned long long *tmp;         // sort ping-pong, up to max_unique
  unsigned int *hist;              // 256 * sort_blocks_cap
  unsigned int *scan_sums;         // 256 chunk sums of the histogram scan
  unsigned int capacity;           // power of two
  unsigned int max_unique;         // capacity / 2
  unsigned int probe_limit;        // longest insert probe before the set counts as full
  unsigned int sort_blocks_cap;    // most blocks a sort pass may use
};
// Sort passes over up to 2^16 keys use at most kSortBlocks blocks, each
// computing its digit offsets from the raw histogram; larger sorts use
// 2048-key blocks and a separate scan of the histogram.
constexpr int kSortBlocks = 240;
// Insert probes allowed when the set was sized from an estimate: at a load
// factor of at most one half such a run essentially never happens, and a
// full-capacity probe on an over-full set would take time quadratic in its
// size.  Sets sized from an exact bound probe up to their capacity.
constexpr unsigned int kEstimateProbeLimit = 256;
size_t rank_scratch_bytes(unsigned int capacity);
// Most blocks a sort pass over up to capacity / 2 keys uses.
unsigned int sort_blocks_cap_of(unsigned int capacity);

void rank_scratch_carve(void *base, unsigned int capacity, RankScratch *rs);
// Labels must lie in [0, label_bound) (label_bound <= 0: [0, n)).
cudaError_t launch_pairs_insert(const int32_t *asc, const int32_t *desc, int64_t n,
                                const RankScratch &rs, DevStatus *st, cudaStream_t s,
                                int64_t label_bound = 0);
// Inserts packed (asc << 32) | desc keys (repeats allowed), labels in
// [0, label_bound).
cudaError_t launch_keys_insert(const unsigned long long *keys, int64_t n, int64_t label_bound,
                               const RankScratch &rs, DevStatus *st, cudaStream_t s);
// Sorts the pair list: (asc << 32) | desc keys with labels below 2^key_bits,
// or (raw_bits > 0) keys compared on their low raw_bits bits as they are.
// With m_dev, n_unique is a capacity that sizes the launches and the kernels
// read the actual count from m_dev (no host round trip; graph-capturable).
cudaError_t launch_pairs_sort(const RankScratch &rs, unsigned int n_unique, int key_bits,
                              cudaStream_t s, int raw_bits = 0,
                              const unsigned int *m_dev = nullptr);
cudaError_t launch_pairs_assign(const RankScratch &rs, unsigned int n_unique, cudaStream_t s,
                                const unsigned int *m_dev = nullptr);
cudaError_t launch_pairs_lookup(const int32_t *asc, const int32_t *desc, int64_t n,
                                const RankScratch &rs, int32_t *ms, cudaStream_t s);
cudaError_t launch_fill_u64(unsigned long long *p, size_t count, unsigned long long v,
                            cudaStream_t s);

// Index pass of the marching triangles / tetrahedra (ms_simplex.cu).
size_t simplex_scratch_bytes(int64_t ncells);
cudaError_t launch_simplex_index(const int32_t *labels, const int64_t dims[3], int mode,
                                 uint8_t *codes, int64_t *offsets, void *scratch,
                                 unsigned long long **total_dev, int64_t *ncells_out, DevStatus *st,
                                 cudaStream_t s);
cudaError_t launch_simplex_geometry(const int32_t *labels, const int64_t dims[3], int mode,
                                    const int64_t *offsets, int64_t total, float *points,
                                    int32_t *pairs, DevStatus *st, cudaStream_t s);

// z-slab sharding (ms_slab.cu).
cudaError_t launch_slab_halo_self(int32_t *up, int32_t *dn, int64_t nxy, int64_t lo_planes,
                                  int64_t owned_planes, int64_t hi_planes, cudaStream_t s);
cudaError_t launch_slab_encode(const int32_t *up, const int32_t *dn, int64_t nxy, int64_t lo_planes,
                               int64_t owned_planes, int64_t base, int32_t *out_asc,
                               int32_t *out_desc, cudaStream_t s);
cudaError_t launch_slab_rows_round(int32_t *rows, int n_planes, int64_t nxy, int64_t n_global,
                                   const long long *zs, const int *slot, DevStatus *st, int round,
                                   cudaStream_t s);
cudaError_t launch_slab_apply(int32_t *asc, int32_t *desc, int64_t n, const int32_t *rows,
                              int64_t nxy, int64_t n_global, const long long *zs, const int *slot,
                              int n_planes, DevStatus *st, cudaStream_t s);
cudaError_t launch_check_nonneg(const int32_t *p, int64_t n, DevStatus *st, cudaStream_t s);

// 0-dimensional persistence pairing from the basin graph (ms_persist.cu).
struct PersistCall {
  const void *field;
  int dtype;
  const int32_t *labels;
  int64_t dims[3];
  int64_t n;
  int direction;          // -1 minima, +1 maxima
  int32_t *extremum;      // capacity entries, device
  int32_t *death;         // capacity entries, device
  int64_t capacity;
  uint64_t max_pairs;     // basin pairs the scratch holds
  uint64_t max_minima;    // extrema the scratch holds
  int min_rounds;         // parallel rounds before a stalled call finishes in order
};
struct PersistOutcome {
  enum Kind { kDone, kGrow, kTooSmall, kBadLabels, kNan };
  Kind kind = kDone;
  uint64_t n_minima = 0;  // extrema found (a lower bound after kGrow)
  uint64_t n_pairs = 0;   // basin pairs found (a lower bound after kGrow)
  bool pairs_full = false;
  int rounds = 0;
  uint64_t finish_edges = 0;  // edges left to the in-order finish (0: none)
};
size_t persist_scratch_bytes(uint64_t max_pairs, uint64_t max_minima);
size_t persist_counters_bytes();
// Runs the pairing on stream s (synchronising it between steps);
// host_counters: pinned, persist_counters_bytes() long.
cudaError_t persist_run(const PersistCall &P, void *scratch, void *host_counters, cudaStream_t s,
                        PersistOutcome *out);

}  // namespace msseg
