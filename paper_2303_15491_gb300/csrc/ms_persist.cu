// 0-dimensional persistence pairing of the extrema (Sec. 4.1: the
// topological simplification the paper runs before segmenting removes the
// extrema whose persistence is below a threshold, Sec. 6), computed from the
// basins that the segmentation already produced.
//
// Why the basins suffice.  The pairing is the elder rule on sublevel-set
// components (minima; superlevel sets for maxima) of the vertex-edge graph:
// vertices enter in (value, index) order, and when an entering vertex joins
// several components, all but the one whose extremum entered first end there.
// A vertex's steepest-descent step goes to a vertex that entered earlier, so
// a vertex is connected to its basin's minimum the moment it enters, and the
// component of a minimum at any time is a union of whole entered basin parts.
// Two basins' parts become connected exactly when the later endpoint of a
// grid edge between them enters.  Hence:
//   1. basin edges: every grid edge whose endpoints lie in different basins
//      joins the two basins from the entry of its later endpoint on; for each
//      pair of basins only the earliest such entry matters;
//   2. the elder rule over the basin graph with those entry times.
//
// Step 2 runs as rounds of one parallel rule instead of one pass in entry
// order.  Components are kept as forests over the basins, each rooted at its
// oldest extremum.  In a round, every component looks at its earliest live
// outgoing edge (ties broken by edge position); if the component at the other
// end holds an older extremum, this component's extremum ends at that edge's
// entering vertex and the component is hung below the other one.  That is the
// elder rule's answer: the component has had no outgoing edge before that
// entry (so it was alone), and the component it meets then holds an older
// extremum.  Hanging it there keeps every later answer, because every edge
// leaving it enters no earlier than the edge it was hung along.  Each round
// hangs at least the youngest component touching the earliest live edge, so
// the rounds end.  Where few components move in a round (long chains whose
// earliest edges lead to younger extrema), the remaining edges are sorted by
// entry and finished by one thread in entry order; edges that enter together
// (one entering vertex) may be taken in any order, as each merge ends the
// younger side at that same vertex.
#include <algorithm>

#include "fastdiv.h"
#include "ms_internal.cuh"

namespace msseg {
namespace {

constexpr unsigned long long kEmptyKey = ~0ull;
constexpr uint32_t kNoEdge = ~0u;
constexpr uint32_t kFull = 0xffffffffu;
constexpr uint32_t kProbeLimit = 512;  // longest insert probe before the table counts as full

// Device counters of one call.
struct Counters {
  unsigned int n_minima;
  unsigned int n_pairs;
  unsigned int minima_overflow;
  unsigned int pairs_overflow;
  unsigned int bad_label;
  unsigned int nan_flag;
  unsigned int live[2];  // live edges kept by a round (alternating)
  unsigned int hooks;    // components hung in a round
  unsigned int roots;    // components with a live edge in a round
  unsigned int pad[6];
};
static_assert(sizeof(Counters) == 64, "one 64-byte block");

struct BasinEdge {
  uint32_t a, b;            // basins (or roots of components that held them)
  unsigned long long when;  // entry key of the later endpoint
};

struct Scratch {
  Counters *cnt;
  unsigned long long *keys, *vals;  // basin-pair table: (lo << 32 | hi) -> earliest entry
  uint32_t *slots;                  // table slots in insertion order (later: tie counters)
  BasinEdge *e0, *e1;               // edge lists, alternating between rounds
  unsigned long long *minima, *mtmp;  // extremum vertices (sorted) and sort ping-pong
  unsigned int *hist, *scan_sums;
  uint32_t *comp;                  // parent of a component in the forest
  unsigned long long *age;         // entry key of the basin's extremum
  unsigned long long *best;        // earliest live edge entry of a root
  uint32_t *best_e;                // its position in the live list
  int32_t *death;                  // entering vertex where the extremum ends, or -1
  uint32_t table_cap, max_pairs, max_minima, sort_blocks_cap;
};

size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

unsigned int table_cap_of(uint64_t max_pairs) {
  uint64_t t = 1024;
  while (t < 2 * max_pairs) t <<= 1;
  return (unsigned int)t;
}

// Carves the scratch; with base == nullptr only the size is computed.
size_t carve(void *base, uint64_t max_pairs, uint64_t max_minima, Scratch *S) {
  Scratch s{};
  s.table_cap = table_cap_of(max_pairs);
  s.max_pairs = (uint32_t)max_pairs;
  s.max_minima = (uint32_t)max_minima;
  s.sort_blocks_cap = sort_blocks_cap_of(2 * (unsigned int)std::max(max_pairs, max_minima));
  char *p = static_cast<char *>(base);
  size_t at = 0;
  auto take = [&](size_t bytes) {
    void *r = p ? p + at : nullptr;
    at += align256(bytes);
    return r;
  };
  s.cnt = static_cast<Counters *>(take(sizeof(Counters)));
  s.keys = static_cast<unsigned long long *>(take((size_t)s.table_cap * 8));
  s.vals = static_cast<unsigned long long *>(take((size_t)s.table_cap * 8));
  s.slots = static_cast<uint32_t *>(take((size_t)max_pairs * 4));
  s.e0 = static_cast<BasinEdge *>(take((size_t)max_pairs * sizeof(BasinEdge)));
  s.e1 = static_cast<BasinEdge *>(take((size_t)max_pairs * sizeof(BasinEdge)));
  s.minima = static_cast<unsigned long long *>(take((size_t)max_minima * 8));
  s.mtmp = static_cast<unsigned long long *>(take((size_t)max_minima * 8));
  s.hist = static_cast<unsigned int *>(take((size_t)256 * s.sort_blocks_cap * 4));
  s.scan_sums = static_cast<unsigned int *>(take(256 * 4));
  s.comp = static_cast<uint32_t *>(take((size_t)max_minima * 4));
  s.age = static_cast<unsigned long long *>(take((size_t)max_minima * 8));
  s.best = static_cast<unsigned long long *>(take((size_t)max_minima * 8));
  s.best_e = static_cast<uint32_t *>(take((size_t)max_minima * 4));
  s.death = static_cast<int32_t *>(take((size_t)max_minima * 4));
  if (S) *S = s;
  return at;
}

// A RankScratch view that sorts `list` with `tmp` as its ping-pong buffer.
RankScratch sort_view(const Scratch &S, unsigned long long *list, unsigned long long *tmp) {
  RankScratch rs{};
  rs.list = list;
  rs.tmp = tmp;
  rs.hist = S.hist;
  rs.scan_sums = S.scan_sums;
  rs.sort_blocks_cap = S.sort_blocks_cap;
  return rs;
}

// Entry key of vertex v: it increases with entry -- (order key, index) for
// minima (increasing order), its complement for maxima (decreasing order).
__device__ __forceinline__ unsigned long long entry_key(uint32_t bits, uint32_t v, bool maxima) {
  const unsigned long long k = ((unsigned long long)order_key_bits(bits) << 32) | v;
  return maxima ? ~k : k;
}

__device__ __forceinline__ int32_t entering_vertex(unsigned long long when, bool maxima) {
  return (int32_t)(uint32_t)(maxima ? ~when : when);
}

struct ScanArgs {
  const void *field;
  int dtype;
  const int32_t *labels;
  uint32_t nx, ny, nz, n, nxy;
  FastDivU32 div_x, div_y;
  bool maxima;
  Scratch S;
};

__device__ void pair_insert(const ScanArgs &A, unsigned long long key, unsigned long long when) {
  Counters *cnt = A.S.cnt;
  if (*(volatile unsigned int *)&cnt->pairs_overflow) return;  // the call retries larger
  const uint32_t mask = A.S.table_cap - 1u;
  uint32_t slot = (uint32_t)hash_mix64(key) & mask;
  for (uint32_t probe = 0; probe < kProbeLimit; ++probe) {
    unsigned long long cur = *(volatile unsigned long long *)&A.S.keys[slot];
    if (cur == kEmptyKey) {
      cur = atomicCAS(&A.S.keys[slot], kEmptyKey, key);
      if (cur == kEmptyKey) {
        const uint32_t at = atomicAdd(&cnt->n_pairs, 1u);
        if (at < A.S.max_pairs)
          A.S.slots[at] = slot;
        else
          atomicOr(&cnt->pairs_overflow, 1u);
        cur = key;
      }
    }
    if (cur == key) {
      // most edges of a basin pair enter after the earliest one: read first,
      // so that only an earlier entry pays for the atomic
      if (when < *(volatile unsigned long long *)&A.S.vals[slot]) atomicMin(&A.S.vals[slot], when);
      return;
    }
    slot = (slot + 1u) & mask;
  }
  atomicOr(&cnt->pairs_overflow, 1u);
}

// A block's own table of basin pairs.  A block scans kChunk consecutive
// vertices at a time (a sheet of rows of one or two planes), which meet a
// few hundred basin pairs but cross basin boundaries tens of thousands of
// times: the crossings meet in shared memory, and only each pair's earliest
// entry goes to the global table when the chunk ends.
constexpr uint32_t kChunk = 8192;
constexpr uint32_t kBlockSlots = 1024;  // about four times the pairs of a chunk of a 3D field

struct BlockTable {
  unsigned long long keys[kBlockSlots], vals[kBlockSlots];
};

// Slot of basin pair (lo, hi) in the block's table: multiplicative hashing
// (Knuth, TAOCP vol. 3, Sec. 6.4) of both halves, the top bits kept.
__device__ __forceinline__ uint32_t block_slot(uint32_t lo, uint32_t hi) {
  static_assert((kBlockSlots & (kBlockSlots - 1u)) == 0 && kBlockSlots >= 2, "a power of two");
  return (lo * 0x9e3779b1u ^ hi * 0x85ebca77u) >> (32 - __builtin_ctz(kBlockSlots));
}

__device__ __forceinline__ void block_insert(BlockTable &T, const ScanArgs &A, uint32_t lo, uint32_t hi,
                                             unsigned long long when) {
  const unsigned long long key = ((unsigned long long)lo << 32) | hi;  // lo != hi: never the empty key
  uint32_t slot = block_slot(lo, hi);
  for (uint32_t probe = 0; probe < kBlockSlots; ++probe) {
    unsigned long long cur = *(volatile unsigned long long *)&T.keys[slot];
    if (cur == kEmptyKey) cur = atomicCAS(&T.keys[slot], kEmptyKey, key);
    if (cur == kEmptyKey || cur == key) {
      if (when < *(volatile unsigned long long *)&T.vals[slot]) atomicMin(&T.vals[slot], when);
      return;
    }
    slot = (slot + 1u) & (kBlockSlots - 1u);
  }
  pair_insert(A, key, when);  // the block's table is full: straight to the global one
}

// Step 1 over every vertex v: checks its label (in range and an extremum's
// own label), lists v if it is an extremum, and for each of its forward
// stencil neighbours w in another basin records the basin pair with the
// entry key of the later of v, w, in the block's table.  (Merging a lane's
// or a warp's crossings of one pair first costs more instructions than the
// shared-memory inserts it saves.)
template <bool kFlat, bool kHalf>
__global__ void __launch_bounds__(256) k_basin_edges(ScanArgs A) {
  __shared__ BlockTable T;
  // forward half of the Freudenthal stencil (the other half is its negation)
  constexpr int kNb = kFlat ? 3 : 7;
  constexpr int8_t kOx[7] = {1, 0, 1, 0, 1, 0, 1};
  constexpr int8_t kOy[7] = {0, 1, 1, 0, 0, 1, 1};
  constexpr int8_t kOz[7] = {0, 0, 0, 1, 1, 1, 1};
  const uint32_t lane = threadIdx.x & 31u;
  bool bad = false, nan = false;
  for (uint32_t i = threadIdx.x; i < kBlockSlots; i += blockDim.x) {
    T.keys[i] = kEmptyKey;
    T.vals[i] = kEmptyKey;
  }
  __syncthreads();
  const uint32_t chunks = (uint32_t)(((uint64_t)A.n + kChunk - 1) / kChunk);
  for (uint32_t c = blockIdx.x; c < chunks; c += gridDim.x) {
    const uint32_t end = (uint32_t)min((uint64_t)A.n, (uint64_t)(c + 1) * kChunk);
    // the loop bound is the same for the whole block (ballots, matches, barriers)
    for (uint32_t base = c * kChunk; base < end; base += blockDim.x) {
      const uint32_t v = base + threadIdx.x;
      int32_t lv = -1;
      unsigned long long kv = 0;
      uint32_t x = 0, y = 0, z = 0;
      if (v < end) {
        lv = __ldg(&A.labels[v]);
        if (lv < 0 || (uint32_t)lv >= A.n) {
          bad = true;
          lv = -1;
        } else if (__ldg(&A.labels[lv]) != lv) {
          bad = true;
        }
        const uint32_t bits = load_bits(A.field, kHalf ? MS_F16 : MS_F32, v);
        nan |= is_nan_bits(bits);
        kv = entry_key(bits, v, A.maxima);
        uint32_t q;
        A.div_x.divmod(v, &q, &x);
        if (kFlat)
          y = q;
        else
          A.div_y.divmod(q, &z, &y);
      }
      const bool own = lv == (int32_t)v;
      const uint32_t mine = __ballot_sync(kFull, own);
      if (mine) {
        const int leader = __ffs(mine) - 1;
        uint32_t at = 0;
        if ((int)lane == leader) at = atomicAdd(&A.S.cnt->n_minima, (unsigned)__popc(mine));
        at = __shfl_sync(kFull, at, leader) + __popc(mine & ((1u << lane) - 1u));
        if (own) {
          if (at < A.S.max_minima)
            A.S.minima[at] = v;
          else
            atomicOr(&A.S.cnt->minima_overflow, 1u);
        }
      }
      // every neighbour's label first, then the values of those across a
      // boundary: the loads of a vertex are in flight together
      const bool hx = x + 1u < A.nx, hy = y + 1u < A.ny, hz = !kFlat && z + 1u < A.nz;
      int32_t lw[kNb];
      uint32_t bw[kNb];
#pragma unroll
      for (int j = 0; j < kNb; ++j) {
        lw[j] = lv;
        if (lv >= 0 && (!kOx[j] || hx) && (!kOy[j] || hy) && (!kOz[j] || hz))
          lw[j] = __ldg(&A.labels[v + kOx[j] + kOy[j] * A.nx + (kFlat ? 0u : kOz[j] * A.nxy)]);
      }
#pragma unroll
      for (int j = 0; j < kNb; ++j) {
        bw[j] = 0;
        if (lw[j] != lv)
          bw[j] = load_bits(A.field, kHalf ? MS_F16 : MS_F32,
                            v + kOx[j] + kOy[j] * A.nx + (kFlat ? 0u : kOz[j] * A.nxy));
      }
#pragma unroll
      for (int j = 0; j < kNb; ++j) {
        if (lw[j] != lv) {
          const unsigned long long k =
              entry_key(bw[j], v + kOx[j] + kOy[j] * A.nx + (kFlat ? 0u : kOz[j] * A.nxy), A.maxima);
          const uint32_t a = (uint32_t)lv, b = (uint32_t)lw[j];
          block_insert(T, A, min(a, b), max(a, b), kv > k ? kv : k);
        }
      }
    }
    // the chunk's pairs to the global table; the block's table empties
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kBlockSlots; i += blockDim.x) {
      const unsigned long long key = T.keys[i];
      if (key != kEmptyKey) {
        pair_insert(A, key, T.vals[i]);
        T.keys[i] = kEmptyKey;
        T.vals[i] = kEmptyKey;
      }
    }
    __syncthreads();
  }
  if (__any_sync(kFull, bad) && lane == 0) atomicOr(&A.S.cnt->bad_label, 1u);
  if (__any_sync(kFull, nan) && lane == 0) atomicOr(&A.S.cnt->nan_flag, 1u);
}

__device__ __forceinline__ uint32_t lower_bound(const unsigned long long *a, uint32_t n,
                                                unsigned long long x) {
  uint32_t lo = 0, hi = n;
  while (lo < hi) {
    const uint32_t mid = lo + ((hi - lo) >> 1);
    if (a[mid] < x)
      lo = mid + 1;
    else
      hi = mid;
  }
  return lo;
}

// The recorded basin pairs as edges between extremum numbers (the positions
// of the extrema in increasing vertex order).
__global__ void k_edges_collect(Scratch S, uint32_t m, uint32_t nmin) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const uint32_t slot = S.slots[i];
    const unsigned long long key = S.keys[slot];
    const uint32_t a = (uint32_t)(key >> 32), b = (uint32_t)key;
    const uint32_t ca = lower_bound(S.minima, nmin, a), cb = lower_bound(S.minima, nmin, b);
    BasinEdge e{0u, 0u, S.vals[slot]};
    if (ca < nmin && cb < nmin && S.minima[ca] == a && S.minima[cb] == b) {
      e.a = ca;
      e.b = cb;
    } else {
      atomicOr(&S.cnt->bad_label, 1u);  // a label that is no extremum's own
    }
    S.e0[i] = e;
  }
}

__global__ void k_nodes_init(Scratch S, uint32_t nmin, const void *field, int dtype, bool maxima) {
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nmin; c += gridDim.x * blockDim.x) {
    const uint32_t v = (uint32_t)S.minima[c];
    S.comp[c] = c;
    S.age[c] = entry_key(load_bits(field, dtype, v), v, maxima);
    S.best[c] = kEmptyKey;
    S.best_e[c] = kNoEdge;
    S.death[c] = -1;
  }
}

// Round, part 1: each live edge is moved onto its endpoints' current roots;
// edges inside one component are dropped, the rest are kept (in any order)
// and give each root its earliest live outgoing entry.
__global__ void k_round_filter(const BasinEdge *__restrict__ in, const unsigned int *m_in,
                               BasinEdge *__restrict__ out, unsigned int *m_out, Scratch S) {
  const uint32_t m = *m_in;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x; base < m; base += stride) {
    const uint32_t i = base + threadIdx.x;
    BasinEdge e{0u, 0u, 0ull};
    bool live = false;
    if (i < m) {
      e = in[i];
      e.a = S.comp[e.a];
      e.b = S.comp[e.b];
      live = e.a != e.b;
    }
    const uint32_t keep = __ballot_sync(kFull, live);
    if (!keep) continue;
    const int leader = __ffs(keep) - 1;
    uint32_t at = 0;
    if ((int)lane == leader) at = atomicAdd(m_out, (unsigned)__popc(keep));
    at = __shfl_sync(kFull, at, leader) + __popc(keep & ((1u << lane) - 1u));
    if (live) {
      out[at] = e;
      atomicMin(&S.best[e.a], e.when);
      atomicMin(&S.best[e.b], e.when);
    }
  }
}

// Round, part 2: among a root's edges with its earliest entry, the first in
// the list.
__global__ void k_round_pick(const BasinEdge *__restrict__ e, const unsigned int *m_dev, Scratch S) {
  const uint32_t m = *m_dev;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const BasinEdge ed = e[i];
    if (ed.when == S.best[ed.a]) atomicMin(&S.best_e[ed.a], i);
    if (ed.when == S.best[ed.b]) atomicMin(&S.best_e[ed.b], i);
  }
}

// Round, part 3: a root whose earliest edge leads to an older root ends there
// and is hung below it.  Reads no parent entry, so the writes do not race.
__global__ void k_round_hook(const BasinEdge *__restrict__ e, uint32_t nmin, Scratch S, bool maxima) {
  uint32_t roots = 0, hooks = 0;
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nmin; c += gridDim.x * blockDim.x) {
    const uint32_t i = S.best_e[c];
    if (i == kNoEdge) continue;
    const BasinEdge ed = e[i];
    const uint32_t other = ed.a == c ? ed.b : ed.a;
    ++roots;
    if (S.age[other] < S.age[c]) {
      S.comp[c] = other;
      S.death[c] = entering_vertex(ed.when, maxima);
      ++hooks;
    }
    S.best[c] = kEmptyKey;
    S.best_e[c] = kNoEdge;
  }
  roots = __reduce_add_sync(kFull, roots);
  hooks = __reduce_add_sync(kFull, hooks);
  if ((threadIdx.x & 31u) == 0 && roots) {
    atomicAdd(&S.cnt->roots, roots);
    atomicAdd(&S.cnt->hooks, hooks);
  }
}

// Round, part 4: every entry points at its root.  Parents only ever move to
// ancestors (every hang goes to an older root), so concurrent shortcuts by
// other threads are ancestors too and each walk ends at the root.
__global__ void k_flatten(Scratch S, uint32_t nmin) {
  for (uint32_t x = blockIdx.x * blockDim.x + threadIdx.x; x < nmin; x += gridDim.x * blockDim.x) {
    uint32_t r = S.comp[x];
    uint32_t p = S.comp[r];
    if (p == r) continue;
    do {
      r = p;
      p = S.comp[r];
    } while (p != r);
    S.comp[x] = r;
  }
}

// Finish, part 1: the entry keys of the remaining edges, to be sorted.
__global__ void k_finish_keys(const BasinEdge *__restrict__ e, uint32_t m,
                              unsigned long long *__restrict__ keys) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x)
    keys[i] = e[i].when;
}

// Finish, part 2: each edge goes to the first free position of its entry key
// in the sorted keys (edges with equal keys in any order).
__global__ void k_finish_scatter(const BasinEdge *__restrict__ e, uint32_t m,
                                 const unsigned long long *__restrict__ sorted,
                                 uint32_t *__restrict__ ties, BasinEdge *__restrict__ out) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const BasinEdge ed = e[i];
    const uint32_t p = lower_bound(sorted, m, ed.when);
    const uint32_t at = p + atomicAdd(&ties[p], 1u);
    if (at < m) out[at] = ed;
  }
}

__device__ uint32_t find_root(uint32_t *comp, uint32_t x) {
  while (comp[x] != x) {
    const uint32_t g = comp[comp[x]];  // path halving
    comp[x] = g;
    x = g;
  }
  return x;
}

// Finish, part 3: the elder rule in entry order, by one thread.
__global__ void k_finish_union(const BasinEdge *__restrict__ e, uint32_t m, Scratch S, bool maxima) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  for (uint32_t i = 0; i < m; ++i) {
    const BasinEdge ed = e[i];
    const uint32_t ra = find_root(S.comp, ed.a), rb = find_root(S.comp, ed.b);
    if (ra == rb) continue;
    const bool a_younger = S.age[ra] > S.age[rb];
    const uint32_t young = a_younger ? ra : rb, old = a_younger ? rb : ra;
    S.comp[young] = old;
    S.death[young] = entering_vertex(ed.when, maxima);
  }
}

__global__ void k_write_pairs(Scratch S, uint32_t nmin, int32_t *extremum, int32_t *death) {
  for (uint32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < nmin; c += gridDim.x * blockDim.x) {
    extremum[c] = (int32_t)S.minima[c];
    death[c] = S.death[c];
  }
}

int sms() {
  static int n = 0;
  if (!n) {
    int dev = 0, v = 152;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) v = 152;
    n = v;
  }
  return n;
}

unsigned int grid_for(uint64_t n, int per_sm = 8) {
  uint64_t b = (n + 255) / 256;
  const uint64_t cap = (uint64_t)sms() * per_sm;
  if (b > cap) b = cap;
  return (unsigned int)(b ? b : 1);
}

// One resident wave of the basin-edge scan (a block takes chunks in turn).
template <bool kFlat, bool kHalf>
unsigned int edges_grid(uint64_t n) {
  static int per_sm = 0;
  if (!per_sm && (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_basin_edges<kFlat, kHalf>, 256, 0) !=
                      cudaSuccess ||
                  per_sm < 1))
    per_sm = 1;
  const uint64_t chunks = (n + kChunk - 1) / kChunk;
  return (unsigned int)std::max<uint64_t>(1, std::min<uint64_t>(chunks, (uint64_t)sms() * per_sm));
}

int bits_of(uint64_t x) {
  int b = 0;
  while (x) {
    ++b;
    x >>= 1;
  }
  return b;
}

cudaError_t read_counters(const Scratch &S, Counters *h, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(h, S.cnt, sizeof(Counters), cudaMemcpyDeviceToHost, s);
  if (e != cudaSuccess) return e;
  return cudaStreamSynchronize(s);
}

}  // namespace

size_t persist_scratch_bytes(uint64_t max_pairs, uint64_t max_minima) {
  return carve(nullptr, max_pairs, max_minima, nullptr);
}

size_t persist_counters_bytes() { return sizeof(Counters); }

cudaError_t persist_run(const PersistCall &P, void *scratch, void *host_counters, cudaStream_t s,
                        PersistOutcome *out) {
  *out = PersistOutcome{};
  Scratch S;
  carve(scratch, P.max_pairs, P.max_minima, &S);
  Counters *h = static_cast<Counters *>(host_counters);
  const bool maxima = P.direction > 0;
  const uint32_t n = (uint32_t)P.n;
  cudaError_t e;

  // step 1: basin edges and the extremum list
  if ((e = cudaMemsetAsync(S.cnt, 0, sizeof(Counters), s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(S.keys, 0xff, (size_t)S.table_cap * 8, s)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(S.vals, 0xff, (size_t)S.table_cap * 8, s)) != cudaSuccess) return e;
  ScanArgs A;
  A.field = P.field;
  A.dtype = P.dtype;
  A.labels = P.labels;
  A.nx = (uint32_t)P.dims[0];
  A.ny = (uint32_t)P.dims[1];
  A.nz = (uint32_t)P.dims[2];
  A.n = n;
  A.nxy = A.nx * A.ny;
  A.div_x = FastDivU32(A.nx);
  A.div_y = FastDivU32(A.ny);
  A.maxima = maxima;
  A.S = S;
  ++tl_launches;
  const bool half = A.dtype == MS_F16;
  if (A.nz == 1 && half)
    k_basin_edges<true, true><<<edges_grid<true, true>(n), 256, 0, s>>>(A);
  else if (A.nz == 1)
    k_basin_edges<true, false><<<edges_grid<true, false>(n), 256, 0, s>>>(A);
  else if (half)
    k_basin_edges<false, true><<<edges_grid<false, true>(n), 256, 0, s>>>(A);
  else
    k_basin_edges<false, false><<<edges_grid<false, false>(n), 256, 0, s>>>(A);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = read_counters(S, h, s)) != cudaSuccess) return e;
  if (h->nan_flag) {
    out->kind = PersistOutcome::kNan;
    return cudaSuccess;
  }
  if (h->bad_label) {
    out->kind = PersistOutcome::kBadLabels;
    return cudaSuccess;
  }
  out->n_minima = h->n_minima;
  out->n_pairs = h->n_pairs;
  if (h->minima_overflow || h->pairs_overflow) {
    out->kind = PersistOutcome::kGrow;
    out->pairs_full = h->pairs_overflow != 0;
    return cudaSuccess;
  }
  const uint32_t nmin = h->n_minima, npairs = h->n_pairs;
  if (nmin == 0) {  // labels without an extremum cannot come from a segmentation
    out->kind = PersistOutcome::kBadLabels;
    return cudaSuccess;
  }
  if ((int64_t)nmin > P.capacity) {
    out->kind = PersistOutcome::kTooSmall;
    return cudaSuccess;
  }

  // the extrema in increasing vertex order; edges between their numbers
  RankScratch rs = sort_view(S, S.minima, S.mtmp);
  if ((e = launch_pairs_sort(rs, nmin, 0, s, std::max(1, bits_of(n - 1)))) != cudaSuccess) return e;
  tl_launches += 2;
  k_nodes_init<<<grid_for(nmin), 256, 0, s>>>(S, nmin, P.field, P.dtype, maxima);
  if (npairs) k_edges_collect<<<grid_for(npairs), 256, 0, s>>>(S, npairs, nmin);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if (npairs) {
    if ((e = read_counters(S, h, s)) != cudaSuccess) return e;
    if (h->bad_label) {
      out->kind = PersistOutcome::kBadLabels;
      return cudaSuccess;
    }
  }

  // step 2: rounds of the parallel rule, then (if they stall) the finish
  BasinEdge *in = S.e0, *outl = S.e1;
  const unsigned int *m_in = &S.cnt->n_pairs;
  uint32_t m = npairs;
  int slot = 0;
  while (m > 0) {
    unsigned int *m_out = &S.cnt->live[slot];
    if ((e = cudaMemsetAsync(m_out, 0, 4, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(&S.cnt->hooks, 0, 8, s)) != cudaSuccess) return e;
    tl_launches += 4;
    k_round_filter<<<grid_for(m), 256, 0, s>>>(in, m_in, outl, m_out, S);
    k_round_pick<<<grid_for(m), 256, 0, s>>>(outl, m_out, S);
    k_round_hook<<<grid_for(nmin), 256, 0, s>>>(outl, nmin, S, maxima);
    k_flatten<<<grid_for(nmin), 256, 0, s>>>(S, nmin);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = read_counters(S, h, s)) != cudaSuccess) return e;
    const uint32_t live = h->live[slot];
    if (live == 0) break;
    ++out->rounds;
    if (out->rounds >= P.min_rounds && (uint64_t)h->hooks * 16 < h->roots) {
      // few components moved: sort the live edges by entry, finish in order
      unsigned long long *keys = S.keys, *tmp = S.vals;  // the table is no longer needed
      tl_launches += 1;
      k_finish_keys<<<grid_for(live), 256, 0, s>>>(outl, live, keys);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      RankScratch fs = sort_view(S, keys, tmp);
      if ((e = launch_pairs_sort(fs, live, 0, s, 64)) != cudaSuccess) return e;
      if ((e = cudaMemsetAsync(S.slots, 0, (size_t)live * 4, s)) != cudaSuccess) return e;
      tl_launches += 2;
      k_finish_scatter<<<grid_for(live), 256, 0, s>>>(outl, live, keys, S.slots, in);
      k_finish_union<<<1, 32, 0, s>>>(in, live, S, maxima);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      out->finish_edges = live;
      break;
    }
    BasinEdge *t = in;
    in = outl;
    outl = t;
    m_in = m_out;
    m = live;
    slot ^= 1;
  }
  ++tl_launches;
  k_write_pairs<<<grid_for(nmin), 256, 0, s>>>(S, nmin, P.extremum, P.death);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return e;
  out->kind = PersistOutcome::kDone;
  return cudaSuccess;
}

}  // namespace msseg
