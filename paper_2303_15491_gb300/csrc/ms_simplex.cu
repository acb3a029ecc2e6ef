// Index pass of the multi-label marching triangles / tetrahedra (Sec. 4.3):
// per simplex of the Freudenthal triangulation, the binary code of its label
// configuration (Fig. 4, Tab. 1); per cell, where its separating elements
// start in the output (exclusive prefix sum of the element counts drawn in
// Figs. 5 and 6).
//
// Simplices: cell (x, y[, z]) is cut along its (0,..,0)->(1,..,1) diagonal
// into one simplex per order in which the axes are stepped (2D: x-then-y,
// y-then-x; 3D: xyz, xzy, yxz, yzx, zxy, zyx), numbered 2c + p / 6c + p with
// c the cell's linear index (x fastest); a simplex's vertices in stepping
// order are a, b, c(, d).
//
// One launch computes the codes and the offsets (k_simplex_index); a second
// kernel writes the separating elements into those slots
// (k_simplex_geometry).
#include <stdint.h>

#include "fastdiv.h"
#include "ms_internal.cuh"

namespace msseg {
namespace {

constexpr int kCellThreads = 512;

struct SimplexGeom {
  int64_t nx, ny;        // vertices per row / per plane row count
  int64_t cx, cy;        // cells along x and y
  int64_t ncells;
  int per;               // simplices per cell: 2 (2D) or 6 (3D)
  int mode;              // 0: region separators, 1: region boundaries
  FastDivU32 div_cx, div_cy;
};

// Local label of position k given its equality to the earlier positions
// (Sec. 4.3: the first earlier vertex with the same label lends its local
// label, else the position itself).
__device__ __forceinline__ int tri_code(int32_t a, int32_t b, int32_t c) {
  const int lb = b != a;
  const int lc = c == a ? 0 : (c == b ? 1 : 2);
  return (lb << 2) | lc;
}

__device__ __forceinline__ int tet_code(int32_t a, int32_t b, int32_t c, int32_t d) {
  const int lb = b == a ? 0 : 1;
  const int lc = c == a ? 0 : (c == b ? lb : 2);
  const int ld = d == a ? 0 : (d == b ? lb : (d == c ? lc : 3));
  return (lb << 4) | (lc << 2) | ld;
}

// Separating elements of a configuration (Figs. 5, 6): by the sizes of its
// label classes -- triangles: {3} 0, {2,1} 1, {1,1,1} 3 segments;
// tetrahedra: {4} 0, {3,1} 1, {2,2} 2, {2,1,1} 5, {1,1,1,1} 12 triangles.
__device__ __forceinline__ int tri_elements(int code) {
  // codes: 0 = {3}; 2, 4, 5 = {2,1}; 6 = {1,1,1}
  return code == 0 ? 0 : (code == 6 ? 3 : 1);
}

__device__ __forceinline__ int tet_elements(int code) {
  const int b = code >> 4, c = (code >> 2) & 3, d = code & 3;
  // class sizes of the local labels 0..3
  const int n0 = 1 + (b == 0) + (c == 0) + (d == 0);
  const int n1 = (b == 1) + (c == 1) + (d == 1);
  const int n2 = (c == 2) + (d == 2);
  const int n3 = d == 3;
  const int classes = 1 + (n1 > 0) + (n2 > 0) + n3;
  if (classes == 1) return 0;
  if (classes == 2) return (n0 == 2 || n1 == 2 || n2 == 2) ? 2 : 1;
  return classes == 3 ? 5 : 12;
}

__device__ __forceinline__ void cell_xyz(const SimplexGeom &g, uint32_t c, uint32_t *x, uint32_t *y,
                                         uint32_t *z) {
  uint32_t q;
  g.div_cx.divmod(c, &q, x);
  g.div_cy.divmod(q, z, y);
}

// Region boundaries (Sec. 4.3): a tetrahedron with exactly three vertices of
// one label gives the triangle of those three, a triangle with exactly two
// the edge between them: one element for the splits 3+1 / 2+1.
__device__ __forceinline__ int tri_boundaries(int code) { return code == 2 || code == 4 || code == 5; }

__device__ __forceinline__ int tet_boundaries(int code) {
  // a class of three: local label 0 thrice, or b, c, d all joining b's class
  const int b = code >> 4, c = (code >> 2) & 3, d = code & 3;
  const int n0 = 1 + (b == 0) + (c == 0) + (d == 0);
  const int n1 = (b == 1) + (c == 1) + (d == 1);
  return n0 == 3 || (n0 == 1 && n1 == 3);
}

// Element counts of all 32 codes (valid or not), one word per code so that
// lookups of different codes hit different banks.  mode 0: separators,
// mode 1: boundaries.
__device__ __forceinline__ void fill_elements(unsigned int *lut, int per, int mode) {
  if (threadIdx.x < 32) {
    const int code = per == 2 ? (int)(threadIdx.x & 7) : (int)threadIdx.x;
    lut[threadIdx.x] = per == 2 ? (unsigned int)(mode ? tri_boundaries(code) : tri_elements(code))
                                : (unsigned int)(mode ? tet_boundaries(code) : tet_elements(code));
  }
}

// Codes of the six tetrahedra of a cell from its corner labels (corner
// bits x = 1, y = 2, z = 4; axis orders xyz, xzy, yxz, yzx, zxy, zyx give the
// b and c corners 1,3 / 1,5 / 2,3 / 2,6 / 4,5 / 4,6), packed into the byte
// lanes of w starting at byte `at` (a constant once the caller's loop is
// unrolled); returns the cell's element count.
__device__ __forceinline__ uint32_t cell_codes3(const int32_t (&l)[8], int at, uint32_t *w,
                                                const unsigned int *lut) {
  constexpr int kb[6] = {1, 1, 2, 2, 4, 4};
  constexpr int kc[6] = {3, 5, 3, 6, 5, 6};
  uint32_t n = 0;
#pragma unroll
  for (int p = 0; p < 6; ++p) {
    const uint32_t code = (uint32_t)tet_code(l[0], l[kb[p]], l[kc[p]], l[7]);
    w[(at + p) / 4] |= code << (8 * ((at + p) % 4));
    n += lut[code];
  }
  return n;
}

__device__ __forceinline__ uint32_t cell_codes2(int32_t l00, int32_t l10, int32_t l01, int32_t l11,
                                                int at, uint32_t *w, const unsigned int *lut) {
  const uint32_t k0 = (uint32_t)tri_code(l00, l10, l11), k1 = (uint32_t)tri_code(l00, l01, l11);
  w[at / 4] |= k0 << (8 * (at % 4));
  w[(at + 1) / 4] |= k1 << (8 * ((at + 1) % 4));
  return lut[k0] + lut[k1];
}

// One persistent launch.  A block's warps split into kComputeWarps that
// compute and one look-back warp.  The compute warps take tiles of
// kTileCells cells in turn (tile ids from an atomic counter), each thread
// kRunCells consecutive cells: along a row the thread slides a window of
// corner labels (4 new labels a cell in 3D, 2 in 2D, restarting at the next
// row's first column when the run reaches a row's end), codes go out as
// 16-byte vectors, and the tile's element total is published at once.  The
// look-back warp then finds the tile's base by decoupled look-back over the
// earlier tiles' published words (flag and value in one 64-bit word: the
// tile's own total, or its inclusive prefix), while the compute warps go on
// with their next tile; they write a tile's offsets one tile later, when its
// base is known.  So no warp computing codes waits for a look-back.
//
// Hand-offs within the block are named barriers with fixed counts: compute
// warps arrive on kBarTile + (i & 1) when tile i is counted, the look-back
// warp arrives on kBarBase + (i & 1) when its base is in s_base; alternating
// by parity keeps a fast side from arriving twice on one barrier before the
// other side has waited on it (each side's arrival for tile i + 2 comes after
// its wait for the other side's arrival for tile i + 1).
constexpr int kRunCells = 8;
constexpr int kComputeWarps = kCellThreads / 32 - 1;
constexpr int kComputeThreads = kComputeWarps * 32;
constexpr int kTileCells = kComputeThreads * kRunCells;
constexpr unsigned long long kFlagAgg = 1ull << 62, kFlagPrefix = 2ull << 62,
                             kValueMask = (1ull << 62) - 1;
// Look-back waits are bounded: past this many polls the call reports a
// timeout (and the waiting tile takes base 0, so nothing waits on it).
constexpr int kLookbackPolls = 1 << 22;
constexpr unsigned int kNoTile = 0xffffffffu;
constexpr int kBarCompute = 1, kBarTile = 2, kBarBase = 4;  // 2, 3 and 4, 5 by parity

template <int kId>
__device__ __forceinline__ void named_sync(int count) {
  asm volatile("bar.sync %0, %1;" ::"n"(kId), "r"(count) : "memory");
}
template <int kId>
__device__ __forceinline__ void named_arrive(int count) {
  asm volatile("bar.arrive %0, %1;" ::"n"(kId), "r"(count) : "memory");
}
// the barrier of parity b (ids fixed at compile time)
template <int kId>
__device__ __forceinline__ void named_sync_by(int b, int count) {
  if (b)
    named_sync<kId + 1>(count);
  else
    named_sync<kId>(count);
}
template <int kId>
__device__ __forceinline__ void named_arrive_by(int b, int count) {
  if (b)
    named_arrive<kId + 1>(count);
  else
    named_arrive<kId>(count);
}

// Codes and element counts of the run of kRunCells cells at c0 (c0 <
// ncells); the codes are stored.
template <int kPer>
__device__ __forceinline__ void run_codes(const int32_t *__restrict__ lab, const SimplexGeom &g,
                                          int64_t c0, uint8_t *__restrict__ codes,
                                          const unsigned int *lut, uint32_t (&n)[kRunCells]) {
  constexpr int kWords = kPer * kRunCells / 4;  // code bytes of a run, 4 a word
  const int64_t sy = g.nx, sz = g.nx * g.ny;
  uint32_t w[kWords];
#pragma unroll
  for (int i = 0; i < kWords; ++i) w[i] = 0;
#pragma unroll
  for (int j = 0; j < kRunCells; ++j) n[j] = 0;
  const bool full = c0 + kRunCells <= g.ncells;
  uint32_t x, y, z;
  cell_xyz(g, (uint32_t)c0, &x, &y, &z);
  // the window: the column at the cell's x (rows y, y+1 of planes z, z+1)
  // and the one at x + 1
  const int32_t *r = lab + ((int64_t)x + g.nx * ((int64_t)y + g.ny * z));
  const bool three = kPer == 6;
  int32_t a0 = __ldg(r), a1 = __ldg(r + sy), a2 = three ? __ldg(r + sz) : 0,
          a3 = three ? __ldg(r + sy + sz) : 0;
#pragma unroll
  for (int j = 0; j < kRunCells; ++j) {
    if (full || c0 + j < g.ncells) {
      const int32_t b0 = __ldg(r + 1), b1 = __ldg(r + sy + 1), b2 = three ? __ldg(r + sz + 1) : 0,
                    b3 = three ? __ldg(r + sy + sz + 1) : 0;
      if (three) {
        const int32_t l[8] = {a0, b0, a1, b1, a2, b2, a3, b3};
        n[j] = cell_codes3(l, 6 * j, w, lut);
      } else {
        n[j] = cell_codes2(a0, b0, a1, b1, 2 * j, w, lut);
      }
      a0 = b0;
      a1 = b1;
      a2 = b2;
      a3 = b3;
      ++r;
      if (++x == (uint32_t)g.cx && j + 1 < kRunCells && c0 + j + 1 < g.ncells) {
        // r is at vertex x = nx - 1: one more is the next row's first vertex,
        // and past the last row of cells skip the plane's last vertex row
        x = 0;
        ++r;
        if (++y == (uint32_t)g.cy) {
          y = 0;
          r += g.nx;
        }
        a0 = __ldg(r);
        a1 = __ldg(r + sy);
        a2 = three ? __ldg(r + sz) : 0;
        a3 = three ? __ldg(r + sy + sz) : 0;
      }
    }
  }
  if (full) {  // c0 * kPer is a multiple of 16 bytes
    uint4 *dst = reinterpret_cast<uint4 *>(codes + c0 * kPer);
#pragma unroll
    for (int i = 0; i < kWords / 4; ++i) dst[i] = make_uint4(w[4 * i], w[4 * i + 1], w[4 * i + 2], w[4 * i + 3]);
  } else {
#pragma unroll
    for (int i = 0; i < kPer * kRunCells; ++i)
      if (c0 + i / kPer < g.ncells) codes[c0 * kPer + i] = (uint8_t)(w[i / 4] >> (8 * (i % 4)));
  }
}

// Base of `tile` (whose own total is already published): the sum of the
// earlier tiles' totals, read back 32 words at a time until one holds an
// inclusive prefix.  Run by one whole warp; the result is in every lane.
__device__ unsigned long long look_back(unsigned long long *status, unsigned int tile,
                                        DevStatus *st) {
  const int lane = threadIdx.x & 31;
  unsigned long long base = 0;
  long long j = (long long)tile - 1;  // newest tile not yet summed
  int polls = 0;
  for (;;) {
    const long long idx = j - lane;
    unsigned long long word = kFlagPrefix;  // before tile 0: a prefix of 0
    if (idx >= 0) word = *(volatile unsigned long long *)&status[idx];
    unsigned int pm;
    for (;;) {  // until every lane before the nearest prefix has published
      pm = __ballot_sync(0xffffffffu, (word >> 62) == 2);
      const unsigned int em = __ballot_sync(0xffffffffu, (word >> 62) == 0);
      const unsigned int need = pm ? em & ((pm & (~pm + 1u)) - 1u) : em;
      if (!need) break;
      if (__any_sync(0xffffffffu, ++polls > kLookbackPolls ||
                                      *(volatile unsigned int *)&st->timeout != 0)) {
        if (lane == 0) atomicOr(&st->timeout, 1u);
        return 0;
      }
      __nanosleep(32);
      if (need >> lane & 1u) word = *(volatile unsigned long long *)&status[idx];
    }
    const int stop = pm ? __ffs(pm) - 1 : 31;  // lanes 0..stop are summed
    unsigned long long v = lane <= stop ? (word & kValueMask) : 0ull;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    base += v;
    if (pm) return base;
    j -= 32;
  }
}

template <int kPer>
__global__ void __launch_bounds__(kCellThreads, 2) k_simplex_index(
    const int32_t *__restrict__ lab, SimplexGeom g, uint8_t *__restrict__ codes,
    int64_t *__restrict__ offsets, int vec_offsets, unsigned long long *hdr,
    unsigned long long *status, unsigned int ntiles, DevStatus *st) {
  __shared__ unsigned int lut[32];
  __shared__ unsigned int s_fetch[2];                       // tile ids, by parity
  __shared__ unsigned int s_tile[2];
  __shared__ unsigned int s_wtot[2][kComputeWarps];         // each compute warp's total
  __shared__ unsigned long long s_wbase[2][kComputeWarps];  // each compute warp's base
  fill_elements(lut, kPer, g.mode);
  if (threadIdx.x == 0) s_fetch[0] = atomicAdd(reinterpret_cast<unsigned int *>(hdr + 1), 1u);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (warp == kComputeWarps) {
    // ---- the look-back warp: tile i of this block, in the order computed.
    // It sums the compute warps' totals, publishes the tile's total, looks
    // back for the tile's base and hands each compute warp its base.
    for (int i = 0;; ++i) {
      const int b = i & 1;
      named_sync_by<kBarTile>(b, kCellThreads);
      const unsigned int t = s_tile[b];
      if (t == kNoTile) return;  // the compute warps have finished
      const unsigned int wv = lane < kComputeWarps ? s_wtot[b][lane] : 0u;
      unsigned int wi = wv;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int u = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += u;
      }
      const unsigned int tot = __shfl_sync(0xffffffffu, wi, 31);
      if (lane == 0)  // the tile's total (tile 0: its prefix) for later tiles' look-back
        *(volatile unsigned long long *)&status[t] = (t == 0 ? kFlagPrefix : kFlagAgg) | tot;
      const unsigned long long base = t == 0 ? 0ull : look_back(status, t, st);
      if (lane < kComputeWarps) s_wbase[b][lane] = base + (wi - wv);
      if (lane == 0) {
        if (t != 0) *(volatile unsigned long long *)&status[t] = kFlagPrefix | ((base + tot) & kValueMask);
        if (t + 1 == ntiles) hdr[0] = base + tot;  // the element total
      }
      __threadfence_block();
      named_arrive_by<kBarBase>(b, kCellThreads);
    }
  }
  // ---- the compute warps
  uint32_t prev_n[kRunCells / 4];  // the previous tile's counts (a byte each), exclusive sum, run
  unsigned int prev_ex = 0;
  int64_t prev_c0 = -1;
  for (int i = 0;; ++i) {
    const int b = i & 1;
    // tile i's id is in s_fetch[b] (tile 0's from before the role split);
    // s_fetch[b] is written again for tile i + 2 only after every compute
    // thread has passed the base barrier of tile i + 1, so after this read
    if (i > 0) {
      if (threadIdx.x == 0) s_fetch[b] = atomicAdd(reinterpret_cast<unsigned int *>(hdr + 1), 1u);
      named_sync<kBarCompute>(kComputeThreads);
    }
    const unsigned int t = s_fetch[b] < ntiles ? s_fetch[b] : kNoTile;
    uint32_t n[kRunCells];
    unsigned int ex = 0;
    const int64_t c0 = t == kNoTile ? -1 : (int64_t)t * kTileCells + (int64_t)threadIdx.x * kRunCells;
    if (t != kNoTile) {
      if (c0 < g.ncells) {
        run_codes<kPer>(lab, g, c0, codes, lut, n);
      } else {
#pragma unroll
        for (int j = 0; j < kRunCells; ++j) n[j] = 0;
      }
      uint32_t mine = 0;
#pragma unroll
      for (int j = 0; j < kRunCells; ++j) mine += n[j];
      // the exclusive sum within the warp; the warp's total goes to the
      // look-back warp, which returns the warp's base
      unsigned int incl = mine;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned int u = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += u;
      }
      ex = incl - mine;
      if (lane == 31) s_wtot[b][warp] = incl;
    }
    if (threadIdx.x == 0) s_tile[b] = t;
    __threadfence_block();
    named_arrive_by<kBarTile>(b, kCellThreads);
    // the previous tile's offsets, now that its base is known
    if (i > 0) {  // tile i - 1 was a tile: the block stops at its first kNoTile
      named_sync_by<kBarBase>(b ^ 1, kCellThreads);
      if (prev_c0 >= 0 && prev_c0 < g.ncells) {
        long long o[kRunCells];
        unsigned long long run = s_wbase[b ^ 1][warp] + prev_ex;
#pragma unroll
        for (int j = 0; j < kRunCells; ++j) {
          o[j] = (long long)run;
          run += (prev_n[j / 4] >> (8 * (j % 4))) & 0xffu;
        }
        if (prev_c0 + kRunCells <= g.ncells && vec_offsets) {
          longlong2 *dst = reinterpret_cast<longlong2 *>(offsets + prev_c0);
#pragma unroll
          for (int j = 0; j < kRunCells / 2; ++j) dst[j] = make_longlong2(o[2 * j], o[2 * j + 1]);
        } else {
#pragma unroll
          for (int j = 0; j < kRunCells; ++j)
            if (prev_c0 + j < g.ncells) offsets[prev_c0 + j] = o[j];
        }
      }
    }
    if (t == kNoTile) return;
#pragma unroll
    for (int j = 0; j < kRunCells / 4; ++j)
      prev_n[j] = n[4 * j] | n[4 * j + 1] << 8 | n[4 * j + 2] << 16 | n[4 * j + 3] << 24;  // each <= 72
    prev_ex = ex;
    prev_c0 = c0;
  }
}

// ---- geometry pass ---------------------------------------------------------
//
// A simplex's elements depend on its code only.  Each block first tabulates,
// for all 32 codes, the elements as corner subsets: a point of an element is
// the mean of a subset of the simplex's corners (bit k = corner k in chain
// order: a midpoint has two bits, a face centre three, the tetrahedron centre
// four), and an element names the two corners whose labels it separates.
// A coordinate is the subset's mean rounded once to nearest even (see
// mean_wide and the narrow path's table of fractions below).
//
// The pass then takes chunks of 32 cells per warp.  A chunk's elements are one
// contiguous range of the output (the index pass's offsets); they are handed
// out 32 at a time, one per lane, so that the lanes do equal work whatever the
// cells' element counts.  A lane finds its element's cell by a binary search
// over the chunk's running counts and the simplex by the cell's per-simplex
// counts, writes the points to a shared-memory window, and the warp stores
// the window as consecutive words; the separated labels come from the owner
// cell's corner labels, which each lane leaves in shared memory.
constexpr int kMaxElems = 12;  // four labels in a tetrahedron
constexpr int kGeoThreads = 256;

// Element descriptor: point masks m0 | m1 << 4 | m2 << 8, separated corners
// i << 12 | j << 14 (m2 = 0 for a segment).
struct ElemRecorder {
  uint32_t *desc;  // kMaxElems per code
  int code;
  int n;
  __device__ void put(const unsigned (&m)[3], int i, int j) {
    if (n < kMaxElems)
      desc[code * kMaxElems + n] =
          m[0] | m[1] << 4 | m[2] << 8 | (unsigned)i << 12 | (unsigned)j << 14;
    ++n;
  }
};

// Separators of a triangle (Fig. 5) or tetrahedron (Fig. 6), n = 3 or 4
// corners with labels L in chain order.
__device__ void separators(ElemRecorder &o, const int32_t *L, int n) {
  // classes of equal labels: cls[k] = first corner with L[k]
  int cls[4], size[4] = {0, 0, 0, 0};
  for (int k = 0; k < n; ++k) {
    cls[k] = k;
    for (int j = 0; j < k; ++j)
      if (L[j] == L[k]) {
        cls[k] = cls[j];
        break;
      }
    size[cls[k]]++;
  }
  int classes = 0;
  for (int k = 0; k < n; ++k) classes += size[k] > 0;
  if (classes == 1) return;
  if (n == 3) {
    if (classes == 3) {  // from the centre to the edge midpoints ab, bc, ac
      const unsigned e[3] = {3u, 6u, 5u};
      for (int k = 0; k < 3; ++k) {
        const unsigned m[3] = {7u, e[k], 0u};
        o.put(m, __ffs(e[k]) - 1, 31 - __clz(e[k]));
      }
      return;
    }
    int lone = 0;
    for (int k = 0; k < 3; ++k)
      if (size[cls[k]] == 1) lone = k;
    const int o1 = lone == 0 ? 1 : 0, o2 = lone == 2 ? 1 : 2;
    const unsigned m[3] = {(1u << lone) | (1u << o1), (1u << lone) | (1u << o2), 0u};
    o.put(m, lone, o1);
    return;
  }
  if (classes == 2) {
    int lone = -1;
    for (int k = 0; k < 4; ++k)
      if (size[cls[k]] == 1) lone = k;
    if (lone >= 0) {  // 3 + 1: the midpoints of the lone corner's edges
      unsigned m[3];
      int t = 0, first = -1;
      for (int k = 0; k < 4; ++k)
        if (k != lone) {
          m[t++] = (1u << lone) | (1u << k);
          if (first < 0) first = k;
        }
      o.put(m, lone, first);
      return;
    }
    // 2 + 2: the quad between {p0, p1} (the class of corner 0) and {q0, q1}
    int p[2], q[2], np = 0, nq = 0;
    for (int k = 0; k < 4; ++k) {
      if (cls[k] == 0)
        p[np++] = k;
      else
        q[nq++] = k;
    }
    const unsigned p0q0 = (1u << p[0]) | (1u << q[0]), p0q1 = (1u << p[0]) | (1u << q[1]),
                   p1q0 = (1u << p[1]) | (1u << q[0]), p1q1 = (1u << p[1]) | (1u << q[1]);
    const unsigned m1[3] = {p0q0, p0q1, p1q0}, m2[3] = {p0q1, p1q0, p1q1};
    o.put(m1, p[0], q[0]);
    o.put(m2, p[0], q[1]);
    return;
  }
  if (classes == 3) {
    int P = -1, Q = -1, R = -1, S = -1;
    for (int k = 0; k < 4; ++k) {
      if (size[cls[k]] == 2) {
        if (P < 0)
          P = k;
        else
          Q = k;
      } else if (R < 0) {
        R = k;
      } else {
        S = k;
      }
    }
    const unsigned bP = 1u << P, bQ = 1u << Q, bR = 1u << R, bS = 1u << S;
    const unsigned T1 = bP | bR | bS, T2 = bQ | bR | bS;
    const unsigned e1[3] = {T1, T2, bP | bR}, e2[3] = {T2, bP | bR, bQ | bR},
                   e3[3] = {T1, T2, bR | bS}, e4[3] = {T1, T2, bP | bS},
                   e5[3] = {T2, bP | bS, bQ | bS};
    o.put(e1, P, R);
    o.put(e2, P, R);
    o.put(e3, R, S);
    o.put(e4, P, S);
    o.put(e5, P, S);
    return;
  }
  // four labels: centre, face centre, edge midpoint for each face's edges
  const unsigned faces[4] = {0x7u, 0xBu, 0xDu, 0xEu};  // abc, abd, acd, bcd
  for (int f = 0; f < 4; ++f) {
    int v[3], t = 0;
    for (int k = 0; k < 4; ++k)
      if (faces[f] >> k & 1u) v[t++] = k;
    const int ea[3] = {v[0], v[0], v[1]}, eb[3] = {v[1], v[2], v[2]};
    for (int k = 0; k < 3; ++k) {
      const unsigned m[3] = {0xFu, faces[f], (1u << ea[k]) | (1u << eb[k])};
      o.put(m, ea[k], eb[k]);
    }
  }
}

// Boundaries: the corners that share a label held by all but one of them.
__device__ void boundaries(ElemRecorder &o, const int32_t *L, int n) {
  for (int lone = 0; lone < n; ++lone) {
    const int ref = lone == 0 ? 1 : 0;
    bool same = L[lone] != L[ref];
    for (int k = 0; k < n && same; ++k)
      if (k != lone && L[k] != L[ref]) same = false;
    if (same) {
      unsigned m[3] = {0u, 0u, 0u};
      int t = 0;
      for (int k = 0; k < n; ++k)
        if (k != lone) m[t++] = 1u << k;
      o.put(m, ref, lone);
      return;
    }
  }
}

// Per-block tables: the elements of every code (mode 0: separators, mode 1:
// boundaries); per chain p the offset bits of its corners (x = 1, y = 2,
// z = 4; corner k in bits 3k..3k+2); and per chain p and corner subset m,
// |m| | k_x << 3 | k_y << 6 | k_z << 9 with k_a the corners of m past axis
// a's step (their coordinate along a is the cell's plus one).
struct GeoTables {
  float4 frac[6 * 16];  // per chain and subset: k_a / |m| rounded (x, y, z), w: the axes where it is 2/3
  uint32_t desc[32 * kMaxElems];
  uint32_t count[32];
  uint32_t corners[6];
  uint32_t subset[6 * 16];
};

__device__ void fill_geo_tables(GeoTables &t, int per, int mode) {
  const int tid = threadIdx.x;
  if (tid < 32) {
    // labels with the equality pattern the code describes (local labels)
    const int code = per == 2 ? (tid & 7) : tid;
    int32_t L[4];
    L[0] = 0;
    if (per == 2) {
      L[1] = (code >> 2) & 1;
      L[2] = code & 3;
      L[3] = 0;
    } else {
      L[1] = code >> 4;
      L[2] = (code >> 2) & 3;
      L[3] = code & 3;
    }
    ElemRecorder r{t.desc, tid, 0};
    if (mode)
      boundaries(r, L, per == 2 ? 3 : 4);
    else
      separators(r, L, per == 2 ? 3 : 4);
    t.count[tid] = (uint32_t)min(r.n, kMaxElems);
  } else if (tid < 32 + per) {
    const int p = tid - 32;
    // axis stepped before corner k: 2D x,y / y,x; 3D xyz, xzy, yxz, yzx, zxy, zyx
    // (axis a stepped k-th in bits 4(k-1)..4(k-1)+3)
    const uint32_t orders3[6] = {0x210u, 0x120u, 0x201u, 0x021u, 0x102u, 0x012u};
    const uint32_t order = per == 2 ? (p == 0 ? 0x10u : 0x01u) : orders3[p];
    const int steps = per == 2 ? 2 : 3;
    uint32_t bits = 0, corners = 0, above = 0;
    for (int k = 1; k <= steps; ++k) {
      const int a = (order >> (4 * (k - 1))) & 15;
      bits |= 1u << a;
      corners |= bits << (3 * k);
      for (int kk = k; kk <= steps; ++kk) above |= 1u << (4 * a + kk);
    }
    t.corners[p] = corners;
    for (unsigned m = 0; m < 16; ++m) {
      const uint32_t cnt = (uint32_t)__popc(m), kx = (uint32_t)__popc(m & above & 15u),
                     ky = (uint32_t)__popc(m & (above >> 4) & 15u),
                     kz = (uint32_t)__popc(m & (above >> 8) & 15u);
      t.subset[p * 16 + m] = cnt | kx << 3 | ky << 6 | kz << 9;
      const float c = (float)(cnt ? cnt : 1u);
      const uint32_t two_thirds = (cnt == 3 && kx == 2) | (cnt == 3 && ky == 2) << 1 |
                                  (cnt == 3 && kz == 2) << 2;
      t.frac[p * 16 + m] = make_float4(__fdiv_rn((float)kx, c), __fdiv_rn((float)ky, c),
                                       __fdiv_rn((float)kz, c), __uint_as_float(two_thirds));
    }
  }
}

// Largest vertex coordinate of the narrow path.
constexpr int64_t kNarrowCoord = (1 << 21) - 1;
// 5/3 rounded to float: the one narrow-path coordinate that o + fl(2/3) rounds
// the other way (o = 1)
constexpr uint32_t kFiveThirdsBits = 0x3FD55555u;

// A point coordinate is the mean of cnt corners (1..4) whose coordinate along
// the axis is o for cnt - k of them and o + 1 for k: (cnt o + k) / cnt rounded
// to nearest even.  Narrow path (o below 2^21): fl(o) + fl(k / cnt), which is
// exact for cnt = 1, 2, 4 and the correctly rounded value for thirds except
// k / cnt = 2/3 at o = 1 -- checked for every o below 2^21 against the exact
// quotient.  Wide path: the exact sum in 64 bits, divided in double and
// rounded to float -- one correct rounding of the exact quotient, as the
// double quotient is exact for cnt = 1, 2, 4 and for thirds never within a
// double rounding error of a float rounding midpoint.
__device__ __forceinline__ float mean_wide(uint32_t o, uint32_t k, uint32_t cnt) {
  return __double2float_rn(__ddiv_rn((double)((uint64_t)cnt * o + k), (double)cnt));
}

template <int kPer, bool kWide>
__global__ void __launch_bounds__(kGeoThreads, 6) k_simplex_geometry(
    const int32_t *__restrict__ lab, SimplexGeom g, const int64_t *__restrict__ offsets,
    int64_t total, float *__restrict__ pos, int32_t *__restrict__ pairs, int pairs8, DevStatus *st) {
  constexpr int kDim = kPer == 2 ? 2 : 3;  // coordinates per point = points per element
  constexpr int kF = kDim * kDim;          // floats per element
  constexpr int kS = kF | 1;               // window stride per element (odd: no bank conflicts)
  constexpr int kWarps = kGeoThreads / 32;
  constexpr unsigned kAll = 0xffffffffu;
  constexpr int kCorners = kPer == 2 ? 4 : 8;  // a cell's corner labels, kept for the pairs
  constexpr int kLS = kCorners + 1;             // their stride (odd: no bank conflicts)
  __shared__ GeoTables tab;
  __shared__ float window[kWarps][32 * kS];
  __shared__ int32_t corner_labels[kWarps][32 * kLS];
  fill_geo_tables(tab, kPer, g.mode);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  float *win = window[threadIdx.x >> 5];
  int32_t *cl = corner_labels[threadIdx.x >> 5];
  const int64_t sy = g.nx, sz = g.nx * g.ny;
  const int64_t nchunks = (g.ncells + 31) / 32;
  for (int64_t ch = (int64_t)blockIdx.x * kWarps + (threadIdx.x >> 5); ch < nchunks;
       ch += (int64_t)gridDim.x * kWarps) {
    const int64_t c = ch * 32 + lane;
    uint32_t x = 0, y = 0, z = 0, codes = 0, counts = 0, n = 0;
    int64_t off = 0;
    if (c < g.ncells) {
      cell_xyz(g, (uint32_t)c, &x, &y, &z);
      const int64_t v = (int64_t)x + g.nx * ((int64_t)y + g.ny * z);
      if (kPer == 2) {
        const int32_t l00 = __ldg(lab + v), l10 = __ldg(lab + v + 1), l01 = __ldg(lab + v + sy),
                      l11 = __ldg(lab + v + sy + 1);
        cl[lane * kLS] = l00;  // corner bits x = 1, y = 2
        cl[lane * kLS + 1] = l10;
        cl[lane * kLS + 2] = l01;
        cl[lane * kLS + 3] = l11;
        const int k0 = tri_code(l00, l10, l11), k1 = tri_code(l00, l01, l11);
        const uint32_t n0 = tab.count[k0], n1 = tab.count[k1];
        codes = (uint32_t)k0 | (uint32_t)k1 << 5;
        counts = n0 | n1 << 4;
        n = n0 + n1;
      } else {
        int32_t l[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          l[k] = __ldg(lab + v + ((k & 1) ? 1 : 0) + ((k & 2) ? sy : 0) + ((k & 4) ? sz : 0));
          cl[lane * kLS + k] = l[k];
        }
        const int kb[6] = {1, 1, 2, 2, 4, 4};
        const int kc[6] = {3, 5, 3, 6, 5, 6};
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          const int code = tet_code(l[0], l[kb[p]], l[kc[p]], l[7]);
          const uint32_t np = tab.count[code];
          codes |= (uint32_t)code << (5 * p);
          counts |= np << (4 * p);
          n += np;
        }
      }
      off = offsets[c];
    }
    __syncwarp();  // the corner labels are read by other lanes below
    // running element counts over the chunk's cells
    uint32_t incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(kAll, incl, o);
      if (lane >= o) incl += t;
    }
    const uint32_t nw = __shfl_sync(kAll, incl, 31);
    const int64_t base = __shfl_sync(kAll, off, 0);
    int64_t end = 0;
    if (lane == 0) end = ch * 32 + 32 < g.ncells ? offsets[ch * 32 + 32] : total;
    end = __shfl_sync(kAll, end, 0);
    // the offsets must be the running counts: then every write below stays
    // inside [offsets[first cell], end) and end <= total
    const bool bad = c < g.ncells && off != base + (int64_t)(incl - n);
    if (__any_sync(kAll, bad) || base < 0 || end != base + (int64_t)nw || end > total) {
      if (lane == 0) atomicOr(&st->bad_index, 1u);
      continue;
    }
    const uint32_t excl = incl - n;
    for (uint32_t e0 = 0; e0 < nw; e0 += 32) {
      const uint32_t e = e0 + lane;
      // the element's cell: the first lane whose running count exceeds e
      int owner = 0;
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) {
        const uint32_t t = __shfl_sync(kAll, incl, owner + s - 1);
        if (t <= e) owner += s;
      }
      const uint32_t oc = __shfl_sync(kAll, codes, owner), on = __shfl_sync(kAll, counts, owner);
      const uint32_t ox = __shfl_sync(kAll, x, owner), oy = __shfl_sync(kAll, y, owner),
                     oz = __shfl_sync(kAll, z, owner), oe = __shfl_sync(kAll, excl, owner);
      if (e < nw) {
        // the simplex within the cell, and the element within the simplex
        uint32_t r = e - oe;
        int p = 0;
#pragma unroll
        for (int q = 0; q < kPer - 1; ++q) {
          const uint32_t cq = (on >> (4 * q)) & 15u;
          if (p == q && r >= cq) {
            r -= cq;
            p = q + 1;
          }
        }
        const int code = (int)((oc >> (5 * p)) & 31u);
        const uint32_t d = tab.desc[code * kMaxElems + r];
        if (kWide) {
          const uint32_t *sub = tab.subset + p * 16;
#pragma unroll
          for (int k = 0; k < kDim; ++k) {
            const uint32_t q = sub[(d >> (4 * k)) & 15u];
            const uint32_t cnt = q & 7u;
            win[lane * kS + k * kDim] = mean_wide(ox, (q >> 3) & 7u, cnt);
            win[lane * kS + k * kDim + 1] = mean_wide(oy, (q >> 6) & 7u, cnt);
            if (kDim == 3) win[lane * kS + k * kDim + 2] = mean_wide(oz, (q >> 9) & 7u, cnt);
          }
        } else {
          const float fx = (float)ox, fy = (float)oy, fz = (float)oz;  // exact below 2^24
          const uint32_t one = (ox == 1u) | (oy == 1u) << 1 | (oz == 1u) << 2;
          const float five_thirds = __uint_as_float(kFiveThirdsBits);
          const float4 *fr = tab.frac + p * 16;
#pragma unroll
          for (int k = 0; k < kDim; ++k) {
            const float4 q = fr[(d >> (4 * k)) & 15u];
            const uint32_t fix = __float_as_uint(q.w) & one;
            win[lane * kS + k * kDim] = (fix & 1u) ? five_thirds : fx + q.x;
            win[lane * kS + k * kDim + 1] = (fix & 2u) ? five_thirds : fy + q.y;
            if (kDim == 3) win[lane * kS + k * kDim + 2] = (fix & 4u) ? five_thirds : fz + q.z;
          }
        }
        if (pairs) {
          const uint32_t cb = tab.corners[p];
          const uint32_t bi = (cb >> (3 * ((d >> 12) & 3u))) & 7u, bj = (cb >> (3 * ((d >> 14) & 3u))) & 7u;
          const int32_t li = cl[owner * kLS + bi], lj = cl[owner * kLS + bj];
          const int64_t at = base + e;
          if (pairs8) {
            *reinterpret_cast<int2 *>(pairs + 2 * at) = make_int2(min(li, lj), max(li, lj));
          } else {
            pairs[2 * at] = min(li, lj);
            pairs[2 * at + 1] = max(li, lj);
          }
        }
      }
      __syncwarp();
      const int nf = (int)min(32u, nw - e0) * kF;
      float *dst = pos + (base + e0) * kF;
      for (int i = lane; i < nf; i += 32) {
        const int el = i / kF;
        dst[i] = win[el * kS + (i - el * kF)];
      }
      __syncwarp();  // the window is refilled by the next round
    }
  }
}

int geometry_grid(int64_t nchunks, const void *kernel) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kGeoThreads, 0);
  const int64_t want = (nchunks + kGeoThreads / 32 - 1) / (kGeoThreads / 32);
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  return (int)(want < cap ? want : cap);
}

}  // namespace

size_t simplex_scratch_bytes(int64_t ncells) {
  const int64_t nb = (ncells + kTileCells - 1) / kTileCells;
  return 256 + (size_t)nb * 8;
}

namespace {
SimplexGeom simplex_geom(const int64_t dims[3], int mode) {
  SimplexGeom g;
  g.nx = dims[0];
  g.ny = dims[1];
  const bool flat = dims[2] == 1;
  g.cx = dims[0] - 1;
  g.cy = dims[1] - 1;
  const int64_t cz = flat ? 1 : dims[2] - 1;
  g.ncells = (g.cx > 0 && g.cy > 0 && cz > 0) ? g.cx * g.cy * cz : 0;
  g.per = flat ? 2 : 6;
  g.mode = mode;
  if (g.ncells) {
    g.div_cx = FastDivU32((uint32_t)g.cx);
    g.div_cy = FastDivU32((uint32_t)g.cy);
  }
  return g;
}
}  // namespace

cudaError_t launch_simplex_geometry(const int32_t *labels, const int64_t dims[3], int mode,
                                    const int64_t *offsets, int64_t total, float *points,
                                    int32_t *pairs, DevStatus *st, cudaStream_t s) {
  const SimplexGeom g = simplex_geom(dims, mode);
  if (g.ncells == 0) return cudaSuccess;
  const int64_t nchunks = (g.ncells + 31) / 32;
  const int pairs8 = (reinterpret_cast<uintptr_t>(pairs) & 7) == 0;
  const bool wide = dims[0] > kNarrowCoord || dims[1] > kNarrowCoord || dims[2] > kNarrowCoord;
  ++tl_launches;
#define MS_GEO_LAUNCH(per, w)                                                                   \
  k_simplex_geometry<per, w><<<geometry_grid(nchunks, (const void *)k_simplex_geometry<per, w>), \
                               kGeoThreads, 0, s>>>(labels, g, offsets, total, points, pairs, pairs8, st)
  if (g.per == 2) {
    if (wide)
      MS_GEO_LAUNCH(2, true);
    else
      MS_GEO_LAUNCH(2, false);
  } else {
    if (wide)
      MS_GEO_LAUNCH(6, true);
    else
      MS_GEO_LAUNCH(6, false);
  }
#undef MS_GEO_LAUNCH
  return cudaGetLastError();
}

// labels: int32[N]; codes: uint8[ncells * per] (16-byte aligned); offsets:
// int64[ncells]; scratch: simplex_scratch_bytes(ncells) bytes; *total_dev:
// the sum; a look-back that waited too long sets st->timeout.
cudaError_t launch_simplex_index(const int32_t *labels, const int64_t dims[3], int mode,
                                 uint8_t *codes, int64_t *offsets, void *scratch,
                                 unsigned long long **total_dev, int64_t *ncells_out, DevStatus *st,
                                 cudaStream_t s) {
  const SimplexGeom g = simplex_geom(dims, mode);
  *ncells_out = g.ncells;
  // scratch: the total (8 bytes) and the tile counter, then one word per tile
  unsigned long long *hdr = reinterpret_cast<unsigned long long *>(scratch);
  *total_dev = hdr;
  const int64_t nb = (g.ncells + kTileCells - 1) / kTileCells;
  cudaError_t e = cudaMemsetAsync(scratch, 0, 256 + (size_t)nb * 8, s);
  if (e != cudaSuccess || g.ncells == 0) return e;
  unsigned long long *status = reinterpret_cast<unsigned long long *>(static_cast<char *>(scratch) + 256);
  const int vec = (reinterpret_cast<uintptr_t>(offsets) & 15) == 0;
  // persistent: as many blocks as are resident at once, at most one a tile
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void *kern = g.per == 2 ? (const void *)k_simplex_index<2> : (const void *)k_simplex_index<6>;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kCellThreads, 0);
  const int64_t cap = (int64_t)(sms > 0 ? sms : 1) * (per_sm > 0 ? per_sm : 1);
  const unsigned int grid = (unsigned)(nb < cap ? nb : cap);
  ++tl_launches;
  if (g.per == 2)
    k_simplex_index<2><<<grid, kCellThreads, 0, s>>>(labels, g, codes, offsets, vec, hdr, status,
                                                     (unsigned)nb, st);
  else
    k_simplex_index<6><<<grid, kCellThreads, 0, s>>>(labels, g, codes, offsets, vec, hdr, status,
                                                     (unsigned)nb, st);
  return cudaGetLastError();
}

}  // namespace msseg
