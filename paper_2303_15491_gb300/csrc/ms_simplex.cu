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
// Points of an element are subsets of its simplex's corners, as bit masks
// (bit k = corner k in chain order): a midpoint has two bits, a face centre
// three, the tetrahedron centre four; the point is the subset's mean, each
// coordinate's sum formed exactly and divided once with IEEE rounding.
struct GeoOut {
  float *pos;
  int32_t *pairs;
  int64_t at, end;  // next element, end of this cell's range
  int npts, dim;
  bool overrun;
};

__device__ __forceinline__ void put(GeoOut &o, const int (*cc)[3], const unsigned (&m)[3],
                                    int32_t l1, int32_t l2) {
  if (o.at >= o.end) {
    o.overrun = true;
    return;
  }
  for (int k = 0; k < o.npts; ++k) {
    const int cnt = __popc(m[k]);
    for (int d = 0; d < o.dim; ++d) {
      int sum = 0;
      for (int j = 0; j < 4; ++j)
        if (m[k] >> j & 1u) sum += cc[j][d];
      o.pos[(o.at * o.npts + k) * o.dim + d] = __fdiv_rn((float)sum, (float)cnt);
    }
  }
  if (o.pairs) {
    o.pairs[2 * o.at] = min(l1, l2);
    o.pairs[2 * o.at + 1] = max(l1, l2);
  }
  ++o.at;
}

// Separators of a triangle (Fig. 5) or tetrahedron (Fig. 6), n = 3 or 4
// corners with labels L in chain order.
__device__ void separators(GeoOut &o, const int (*cc)[3], const int32_t *L, int n) {
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
        const int i = __ffs(e[k]) - 1, j = 31 - __clz(e[k]);
        put(o, cc, m, L[i], L[j]);
      }
      return;
    }
    int lone = 0;
    for (int k = 0; k < 3; ++k)
      if (size[cls[k]] == 1) lone = k;
    const int o1 = lone == 0 ? 1 : 0, o2 = lone == 2 ? 1 : 2;
    const unsigned m[3] = {(1u << lone) | (1u << o1), (1u << lone) | (1u << o2), 0u};
    put(o, cc, m, L[lone], L[o1]);
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
      put(o, cc, m, L[lone], L[first]);
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
    put(o, cc, m1, L[p[0]], L[q[0]]);
    put(o, cc, m2, L[p[0]], L[q[1]]);
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
    put(o, cc, e1, L[P], L[R]);
    put(o, cc, e2, L[P], L[R]);
    put(o, cc, e3, L[R], L[S]);
    put(o, cc, e4, L[P], L[S]);
    put(o, cc, e5, L[P], L[S]);
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
      put(o, cc, m, L[ea[k]], L[eb[k]]);
    }
  }
}

// Boundaries: the corners that share a label held by all but one of them.
__device__ __forceinline__ void boundaries(GeoOut &o, const int (*cc)[3], const int32_t *L, int n) {
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
      put(o, cc, m, L[ref], L[lone]);
      return;
    }
  }
}

// One thread per cell, writing its cell's elements where the index pass put
// them (a store-staged variant that regenerated the elements per window of
// shared memory measured twice as slow).
__global__ void __launch_bounds__(kCellThreads) k_simplex_geometry(const int32_t *__restrict__ lab,
                                                                   SimplexGeom g,
                                                                   const int64_t *__restrict__ offsets,
                                                                   int64_t total, float *pos,
                                                                   int32_t *pairs, DevStatus *st) {
  const int64_t c = (int64_t)blockIdx.x * kCellThreads + threadIdx.x;
  if (c >= g.ncells) return;
  uint32_t x, y, z;
  cell_xyz(g, (uint32_t)c, &x, &y, &z);
  GeoOut o;
  o.pos = pos;
  o.pairs = pairs;
  o.at = offsets[c];
  o.end = c + 1 < g.ncells ? offsets[c + 1] : total;
  o.dim = g.per == 2 ? 2 : 3;
  o.npts = o.dim;
  o.overrun = o.at > o.end || o.end > total;
  if (o.overrun) {
    atomicOr(&st->bad_index, 1u);
    return;
  }
  const int64_t v = (int64_t)x + g.nx * ((int64_t)y + g.ny * z);
  const int64_t sy = g.nx, sz = g.nx * g.ny;
  if (g.per == 2) {
    int cc[3][3];
    int32_t L[3];
    for (int p = 0; p < 2; ++p) {
      // chains (0,0) -> (1,0) -> (1,1) and (0,0) -> (0,1) -> (1,1)
      const int dx[3] = {0, p == 0 ? 1 : 0, 1}, dy[3] = {0, p == 0 ? 0 : 1, 1};
      for (int k = 0; k < 3; ++k) {
        cc[k][0] = (int)x + dx[k];
        cc[k][1] = (int)y + dy[k];
        cc[k][2] = 0;
        L[k] = __ldg(lab + v + dx[k] + sy * dy[k]);
      }
      if (g.mode)
        boundaries(o, cc, L, 3);
      else
        separators(o, cc, L, 3);
    }
  } else {
    const int ax[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int p = 0; p < 6; ++p) {
      int cc[4][3];
      int32_t L[4];
      int pt[3] = {(int)x, (int)y, (int)z};
      int64_t vv = v;
      for (int k = 0; k < 4; ++k) {
        if (k > 0) {
          const int a = ax[p][k - 1];
          pt[a] += 1;
          vv += a == 0 ? 1 : (a == 1 ? sy : sz);
        }
        cc[k][0] = pt[0];
        cc[k][1] = pt[1];
        cc[k][2] = pt[2];
        L[k] = __ldg(lab + vv);
      }
      if (g.mode)
        boundaries(o, cc, L, 4);
      else
        separators(o, cc, L, 4);
    }
  }
  if (o.overrun || o.at != o.end) atomicOr(&st->bad_index, 1u);
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
  ++tl_launches;
  k_simplex_geometry<<<(unsigned)((g.ncells + kCellThreads - 1) / kCellThreads), kCellThreads, 0, s>>>(
      labels, g, offsets, total, points, pairs, st);
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
