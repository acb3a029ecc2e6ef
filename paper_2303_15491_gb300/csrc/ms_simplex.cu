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
// Three launches: codes, per-cell element counts (one byte) and per-block
// totals (one thread per cell of each of a block's kSub groups of 256 cells,
// a group's codes staged in shared memory and stored as 16-byte vectors), an
// exclusive scan of the block totals, and the per-cell offsets (block scans
// of the counts, plus the block's base).
#include <stdint.h>

#include "fastdiv.h"
#include "ms_internal.cuh"

namespace msseg {
namespace {

constexpr int kCellThreads = 256;
constexpr int kSub = 8;  // groups of kCellThreads cells per block

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

// Block-wide exclusive sum of one value per thread; also the block total.
__device__ __forceinline__ unsigned int block_excl(unsigned int v, unsigned int *total,
                                                   unsigned int *sh) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned int incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) sh[warp] = incl;
  __syncthreads();
  unsigned int base = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kCellThreads / 32; ++w) {
    const unsigned int s = sh[w];
    if (w < warp) base += s;
    tot += s;
  }
  *total = tot;
  return base + incl - v;
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

__global__ void __launch_bounds__(kCellThreads) k_simplex_codes(const int32_t *__restrict__ lab,
                                                                SimplexGeom g,
                                                                uint8_t *__restrict__ codes,
                                                                uint8_t *__restrict__ counts,
                                                                unsigned int *__restrict__ block_tot) {
  __shared__ __align__(16) uint8_t sc[kCellThreads * 6];
  __shared__ unsigned int sh[kCellThreads / 32];
  __shared__ unsigned int lut[32];
  fill_elements(lut, g.per, g.mode);
  __syncthreads();
  unsigned int block_sum = 0;
  // kSub consecutive groups of kCellThreads cells per block
  for (int sub = 0; sub < kSub; ++sub) {
    const int64_t c0 = ((int64_t)blockIdx.x * kSub + sub) * kCellThreads;
    if (c0 >= g.ncells) break;  // block-uniform
    const int64_t c = c0 + threadIdx.x;
    unsigned int count = 0;
    if (c < g.ncells) {
      uint32_t x, y, z;
      cell_xyz(g, (uint32_t)c, &x, &y, &z);
      const int64_t v = (int64_t)x + g.nx * ((int64_t)y + g.ny * z);
      const int64_t sy = g.nx, sz = g.nx * g.ny;
      if (g.per == 2) {
        const int32_t l00 = __ldg(lab + v), l10 = __ldg(lab + v + 1), l01 = __ldg(lab + v + sy),
                      l11 = __ldg(lab + v + sy + 1);
        const int k0 = tri_code(l00, l10, l11), k1 = tri_code(l00, l01, l11);
        sc[threadIdx.x * 2] = (uint8_t)k0;
        sc[threadIdx.x * 2 + 1] = (uint8_t)k1;
        count = lut[k0] + lut[k1];
      } else {
        // corners by offset bits (x = 1, y = 2, z = 4)
        int32_t l[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
          l[k] = __ldg(lab + v + ((k & 1) ? 1 : 0) + ((k & 2) ? sy : 0) + ((k & 4) ? sz : 0));
        // axis orders xyz, xzy, yxz, yzx, zxy, zyx: b and c corners of each chain
        const int kb[6] = {1, 1, 2, 2, 4, 4};
        const int kc[6] = {3, 5, 3, 6, 5, 6};
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          const int code = tet_code(l[0], l[kb[p]], l[kc[p]], l[7]);
          sc[threadIdx.x * 6 + p] = (uint8_t)code;
          count += lut[code];
        }
      }
    }
    if (c < g.ncells) counts[c] = (uint8_t)count;  // at most 6 x 12
    __syncthreads();
    // the group's codes are one contiguous byte range
    const int64_t nvalid = min((int64_t)kCellThreads, g.ncells - c0);
    const int64_t bytes = nvalid * g.per;
    uint8_t *dst = codes + c0 * g.per;  // 16-byte aligned: c0 * per is a multiple of 512
    const int vec = (int)(bytes / 16);
    for (int i = threadIdx.x; i < vec; i += kCellThreads)
      reinterpret_cast<uint4 *>(dst)[i] = reinterpret_cast<const uint4 *>(sc)[i];
    for (int64_t i = (int64_t)vec * 16 + threadIdx.x; i < bytes; i += kCellThreads) dst[i] = sc[i];
    unsigned int tot = 0;
    block_excl(count, &tot, sh);
    block_sum += tot;
    __syncthreads();  // sc and sh are reused by the next group
  }
  if (threadIdx.x == 0) block_tot[blockIdx.x] = block_sum;
}

// Exclusive scan of the per-block totals into 64-bit bases, by one block:
// thread t sums its contiguous chunk, the chunk sums are scanned, and the
// chunk is walked again writing bases.  *total receives the sum.
__global__ void __launch_bounds__(1024) k_scan_blocks(const unsigned int *__restrict__ tot,
                                                      int64_t nblocks,
                                                      unsigned long long *__restrict__ base,
                                                      unsigned long long *__restrict__ total) {
  __shared__ unsigned long long sh[1024];
  const int64_t chunk = (nblocks + 1023) / 1024;
  const int64_t lo = (int64_t)threadIdx.x * chunk, hi = min(nblocks, lo + chunk);
  unsigned long long s = 0;
  for (int64_t i = lo; i < hi; ++i) s += tot[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const unsigned long long t = threadIdx.x >= o ? sh[threadIdx.x - o] : 0ull;
    __syncthreads();
    sh[threadIdx.x] += t;
    __syncthreads();
  }
  unsigned long long run = sh[threadIdx.x] - s;
  for (int64_t i = lo; i < hi; ++i) {
    base[i] = run;
    run += tot[i];
  }
  if (threadIdx.x == 1023) *total = sh[1023];
}

__global__ void __launch_bounds__(kCellThreads) k_simplex_offsets(const uint8_t *__restrict__ counts,
                                                                  SimplexGeom g,
                                                                  const unsigned long long *__restrict__ base,
                                                                  int64_t *__restrict__ offsets) {
  __shared__ unsigned int sh[kCellThreads / 32];
  unsigned long long running = base[blockIdx.x];
  for (int sub = 0; sub < kSub; ++sub) {
    const int64_t c0 = ((int64_t)blockIdx.x * kSub + sub) * kCellThreads;
    if (c0 >= g.ncells) break;  // block-uniform
    const int64_t c = c0 + threadIdx.x;
    const unsigned int count = c < g.ncells ? __ldg(counts + c) : 0u;
    unsigned int tot = 0;
    const unsigned int ex = block_excl(count, &tot, sh);
    if (c < g.ncells) offsets[c] = (int64_t)(running + ex);
    running += tot;
    __syncthreads();  // sh is reused by the next group
  }
}

// ---- geometry pass ---------------------------------------------------------
//
// A simplex's elements depend on its code only.  Each block first tabulates,
// for all 32 codes, the elements as corner subsets: a point of an element is
// the mean of a subset of the simplex's corners (bit k = corner k in chain
// order: a midpoint has two bits, a face centre three, the tetrahedron centre
// four), and an element names the two corners whose labels it separates.
// Each coordinate's sum is formed exactly and divided once with IEEE rounding.
//
// The pass then takes chunks of 32 cells per warp.  A chunk's elements are one
// contiguous range of the output (the index pass's offsets); they are handed
// out 32 at a time, one per lane, so that the lanes do equal work whatever the
// cells' element counts.  A lane finds its element's cell by a binary search
// over the chunk's running counts and the simplex by the cell's per-simplex
// counts, writes the points to a shared-memory window, and the warp stores
// the window as consecutive words.
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
// boundaries), and per chain p the offset bits of its corners (x = 1, y = 2,
// z = 4; corner k in bits 3k..3k+2) and the corners past each axis's step
// (axis a: bit 4a + k set when corner k has +1 along a).
struct GeoTables {
  uint32_t desc[32 * kMaxElems];
  uint32_t count[32];
  uint32_t corners[6];
  uint32_t above[6];
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
    t.above[p] = above;
  }
}

// Mean of cnt corners whose coordinates sum to s (cnt * base + k, k <= cnt):
// halves and quarters are exact scalings, thirds take the rounded division.
__device__ __forceinline__ float mean_of(int64_t s, int cnt) {
  const float f = (float)s;
  return cnt == 3 ? __fdiv_rn(f, 3.0f) : (cnt == 1 ? f : (cnt == 2 ? f * 0.5f : f * 0.25f));
}

template <int kPer>
__global__ void __launch_bounds__(kGeoThreads) k_simplex_geometry(
    const int32_t *__restrict__ lab, SimplexGeom g, const int64_t *__restrict__ offsets,
    int64_t total, float *__restrict__ pos, int32_t *__restrict__ pairs, int pairs8, DevStatus *st) {
  constexpr int kDim = kPer == 2 ? 2 : 3;  // coordinates per point = points per element
  constexpr int kF = kDim * kDim;          // floats per element
  constexpr int kS = kF | 1;               // window stride per element (odd: no bank conflicts)
  constexpr int kWarps = kGeoThreads / 32;
  constexpr unsigned kAll = 0xffffffffu;
  __shared__ GeoTables tab;
  __shared__ float window[kWarps][32 * kS];
  fill_geo_tables(tab, kPer, g.mode);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  float *win = window[threadIdx.x >> 5];
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
        const int k0 = tri_code(l00, l10, l11), k1 = tri_code(l00, l01, l11);
        const uint32_t n0 = tab.count[k0], n1 = tab.count[k1];
        codes = (uint32_t)k0 | (uint32_t)k1 << 5;
        counts = n0 | n1 << 4;
        n = n0 + n1;
      } else {
        int32_t l[8];
#pragma unroll
        for (int k = 0; k < 8; ++k)
          l[k] = __ldg(lab + v + ((k & 1) ? 1 : 0) + ((k & 2) ? sy : 0) + ((k & 4) ? sz : 0));
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
        const uint32_t above = tab.above[p];
        const uint32_t o3[3] = {ox, oy, oz};
#pragma unroll
        for (int k = 0; k < kDim; ++k) {
          const uint32_t m = (d >> (4 * k)) & 15u;
          const int cnt = __popc(m);
#pragma unroll
          for (int a = 0; a < kDim; ++a) {
            const int64_t s = (int64_t)cnt * o3[a] + __popc(m & (above >> (4 * a)) & 15u);
            win[lane * kS + k * kDim + a] = mean_of(s, cnt);
          }
        }
        if (pairs) {
          const uint32_t cb = tab.corners[p];
          const uint32_t bi = (cb >> (3 * ((d >> 12) & 3u))) & 7u, bj = (cb >> (3 * ((d >> 14) & 3u))) & 7u;
          const int64_t v = (int64_t)ox + g.nx * ((int64_t)oy + g.ny * oz);
          const int32_t li = __ldg(lab + v + (bi & 1u) + ((bi & 2u) ? sy : 0) + ((bi & 4u) ? sz : 0));
          const int32_t lj = __ldg(lab + v + (bj & 1u) + ((bj & 2u) ? sy : 0) + ((bj & 4u) ? sz : 0));
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
  const int64_t nb = (ncells + kCellThreads * kSub - 1) / (kCellThreads * kSub);
  return 256 + (size_t)nb * 4 + (size_t)nb * 8 + 256 + 256 + (size_t)ncells;
}

// labels: int32[N]; codes: uint8[ncells * per]; offsets: int64[ncells];
// scratch: simplex_scratch_bytes(ncells) bytes; *total_dev: the sum.
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
  ++tl_launches;
  if (g.per == 2) {
    k_simplex_geometry<2><<<geometry_grid(nchunks, (const void *)k_simplex_geometry<2>), kGeoThreads, 0,
                            s>>>(labels, g, offsets, total, points, pairs, pairs8, st);
  } else {
    k_simplex_geometry<6><<<geometry_grid(nchunks, (const void *)k_simplex_geometry<6>), kGeoThreads, 0,
                            s>>>(labels, g, offsets, total, points, pairs, pairs8, st);
  }
  return cudaGetLastError();
}

cudaError_t launch_simplex_index(const int32_t *labels, const int64_t dims[3], int mode,
                                 uint8_t *codes, int64_t *offsets, void *scratch,
                                 unsigned long long **total_dev, int64_t *ncells_out,
                                 cudaStream_t s) {
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
  *ncells_out = g.ncells;
  unsigned long long *total = reinterpret_cast<unsigned long long *>(scratch);
  *total_dev = total;
  cudaError_t e = cudaMemsetAsync(total, 0, 8, s);
  if (e != cudaSuccess || g.ncells == 0) return e;
  g.div_cx = FastDivU32((uint32_t)g.cx);
  g.div_cy = FastDivU32((uint32_t)g.cy);
  const int64_t nb = (g.ncells + kCellThreads * kSub - 1) / (kCellThreads * kSub);
  unsigned int *btot = reinterpret_cast<unsigned int *>(static_cast<char *>(scratch) + 256);
  const size_t tot_bytes = ((size_t)nb * 4 + 255) & ~(size_t)255;
  unsigned long long *bbase =
      reinterpret_cast<unsigned long long *>(static_cast<char *>(scratch) + 256 + tot_bytes);
  uint8_t *counts = static_cast<uint8_t *>(scratch) + 256 + tot_bytes +
                    (((size_t)nb * 8 + 255) & ~(size_t)255);
  ++tl_launches;
  k_simplex_codes<<<(unsigned)nb, kCellThreads, 0, s>>>(labels, g, codes, counts, btot);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  ++tl_launches;
  k_scan_blocks<<<1, 1024, 0, s>>>(btot, nb, bbase, total);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  ++tl_launches;
  k_simplex_offsets<<<(unsigned)nb, kCellThreads, 0, s>>>(counts, g, bbase, offsets);
  return cudaGetLastError();
}

}  // namespace msseg
