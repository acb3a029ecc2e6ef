// The fused, tiled form of the segmentation used by ms_segment.
//
// The grid is cut into tiles of TX x TY x TZ vertices.  Three phases:
//
//  1. k_tile_local (one CTA per tile, persistent): streams the tile's field
//     plus a one-vertex halo from HBM, computes up / dn of every tile vertex
//     (Sec. 4.2.1 first step), compresses the paths inside the tile in shared
//     memory (Sec. 4.2.1 second step, Fig. 3) until each pointer reaches a
//     local maximum/minimum or the first vertex outside the tile (an "exit"),
//     then numbers the distinct (dn-root, up-root) pairs of the tile.  Per
//     vertex it writes only the 16-bit number of its pair; per tile the pair
//     list (roots as global vertex indices, exits flagged) and, for the
//     vertices on the tile's faces, their local roots (other tiles' paths
//     enter through those vertices).
//  2. k_resolve_pairs: every tile pair's exits are followed from face to face
//     through the other tiles' face roots until they end at an extremum;
//     the resulting (asc, desc) pairs are deduplicated in a global hash set,
//     sorted (ms_rank.cu) and each tile pair gets its MS id (Sec. 4.2.2).
//  3. k_tile_write: per tile, the small pair table is staged in shared memory
//     and the three int32 labels of every vertex are streamed out.
//
// Steepest neighbours without 14 comparisons: the Freudenthal neighbourhood
// of v together with v is the union of the two unit cubes [v, v+(1,1,1)] and
// [v-(1,1,1), v] (their 2 x 8 corners minus the shared v are the 14 offsets
// whose components are all >= 0 or all <= 0).  The maximum over a unit cube
// is separable: pairs along x, then y, then z.  Every comparison is between
// two candidate sets one of which lies entirely at higher vertex indices (the
// +x / +y / +z half, or the upper cube), so the (value, index) order needs
// only the 32-bit order key: on equal keys the higher-index operand wins for
// the maximum and the lower-index one for the minimum.
#include <cuda.h>
#include <string.h>

#include "ms_internal.cuh"
#include "ms_tiled.cuh"

namespace msseg {
namespace {

constexpr uint32_t kEmpty32 = 0xffffffffu;

struct Cand {
  uint32_t k;  // order key (max side) or key - 1 (min side)
  uint32_t i;  // extended-box index of the candidate
};

template <class S>
__device__ __forceinline__ int ext_of(int lx, int ly, int lz) {
  return (lx + kXO) + S::EX * ((ly + 1) + S::EY * (lz + 1));
}

template <class S>
__device__ __forceinline__ void tile_origin(const TileGeom &g, int64_t t, int64_t *x0, int64_t *y0,
                                            int64_t *z0) {
  uint32_t r, tx, ty, tz;
  g.div_tx.divmod((uint32_t)t, &r, &tx);
  g.div_ty.divmod(r, &tz, &ty);
  *x0 = (int64_t)tx * S::TX;
  *y0 = (int64_t)ty * S::TY;
  *z0 = (int64_t)tz * S::TZ;
}

// Slot of a face vertex in its tile's face-root array (first face that
// contains it, in the order z-low, z-high, y-low, y-high, x-low, x-high), or
// -1 for an interior vertex.
template <class S>
__device__ __forceinline__ int face_slot(int lx, int ly, int lz) {
  constexpr int TX = S::TX, TY = S::TY, TZ = S::TZ;
  if (lz == 0) return lx + TX * ly;
  if (lz == TZ - 1) return TX * TY + lx + TX * ly;
  if (ly == 0) return 2 * TX * TY + lx + TX * lz;
  if (ly == TY - 1) return 2 * TX * TY + TX * TZ + lx + TX * lz;
  if (lx == 0) return 2 * TX * TY + 2 * TX * TZ + ly + TY * lz;
  if (lx == TX - 1) return 2 * TX * TY + 2 * TX * TZ + TY * TZ + ly + TY * lz;
  return -1;
}

// Reference to a tile root at box index e: its global vertex index, with
// kExitFlag set when e lies in the halo (the path continues in another tile).
template <class S>
__device__ __forceinline__ int32_t root_ref(const TileGeom &g, int64_t x0, int64_t y0, int64_t z0,
                                            int e) {
  constexpr int EX = S::EX, EY = S::EY, EZ = S::EZ;
  const uint32_t ue = (uint32_t)e;
  const uint32_t ez = ue / (EX * EY), r = ue - ez * (EX * EY);
  const uint32_t ey = r / EX, ex = r - ey * EX;
  const bool halo = ex == kXO - 1 || ex == kXO + S::TX || ey == 0 || ez == 0 || ey == EY - 1 ||
                    ez == EZ - 1;
  const int64_t v = (x0 + (int)ex - kXO) + g.nx * ((y0 + (int)ey - 1) + g.ny * (z0 + (int)ez - 1));
  return (int32_t)v | (halo ? kExitFlag : 0);
}

// Inverse of face_slot's layout: the vertex a face slot describes.
template <class S>
__device__ __forceinline__ void face_coords(int fs, int *lx, int *ly, int *lz) {
  constexpr int TX = S::TX, TY = S::TY, TZ = S::TZ;
  constexpr int kZ = TX * TY, kY = TX * TZ, kX = TY * TZ;
  if (fs < 2 * kZ) {
    *lz = fs < kZ ? 0 : TZ - 1;
    const int r = fs % kZ;
    *lx = r % TX;
    *ly = r / TX;
  } else if (fs < 2 * kZ + 2 * kY) {
    const int q = fs - 2 * kZ;
    *ly = q < kY ? 0 : TY - 1;
    const int r = q % kY;
    *lx = r % TX;
    *lz = r / TX;
  } else {
    const int q = fs - 2 * kZ - 2 * kY;
    *lx = q < kX ? 0 : TX - 1;
    const int r = q % kX;
    *ly = r % TY;
    *lz = r / TY;
  }
}

// ---- 2D tiles (k2TX x k2TY; see ms_tiled.cuh) -----------------------------
__device__ __forceinline__ int ext2_of(int lx, int ly) { return (lx + kXO) + k2EX * (ly + 1); }

__device__ __forceinline__ void tile_origin2(const TileGeom &g, int64_t t, int64_t *x0,
                                             int64_t *y0) {
  uint32_t tx, ty;
  g.div_tx.divmod((uint32_t)t, &ty, &tx);
  *x0 = (int64_t)tx * k2TX;
  *y0 = (int64_t)ty * k2TY;
}

// Face slots of a 2D tile: the y-low row, the y-high row, the x-low column,
// the x-high column (corners in the first that contains them).
__device__ __forceinline__ int face_slot2(int lx, int ly) {
  if (ly == 0) return lx;
  if (ly == k2TY - 1) return k2TX + lx;
  if (lx == 0) return 2 * k2TX + ly;
  if (lx == k2TX - 1) return 2 * k2TX + k2TY + ly;
  return -1;
}

__device__ __forceinline__ void face_coords2(int fs, int *lx, int *ly) {
  if (fs < 2 * k2TX) {
    *lx = fs % k2TX;
    *ly = fs < k2TX ? 0 : k2TY - 1;
  } else {
    const int q = fs - 2 * k2TX;
    *lx = q < k2TY ? 0 : k2TX - 1;
    *ly = q % k2TY;
  }
}

__device__ __forceinline__ int32_t root_ref2(const TileGeom &g, int64_t x0, int64_t y0, int e) {
  const uint32_t ue = (uint32_t)e;
  const uint32_t ey = ue / k2EX, ex = ue - ey * k2EX;
  const bool halo = ex == kXO - 1 || ex == kXO + k2TX || ey == 0 || ey == k2EY - 1;
  const int64_t v = (x0 + (int)ex - kXO) + g.nx * (y0 + (int)ey - 1);
  return (int32_t)v | (halo ? kExitFlag : 0);
}

// Exclusive block scan of two values per thread (kWarps warps); also returns
// both totals.  Uses scratch[2][kWarps]; ends with a barrier.
template <int kWarps>
__device__ __forceinline__ void block_scan2(int a, int b, int *ea, int *eb, int *ta, int *tb,
                                            int (*scratch)[kWarps]) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int ia = a, ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int xa = __shfl_up_sync(0xffffffffu, ia, o);
    const int xb = __shfl_up_sync(0xffffffffu, ib, o);
    if (lane >= o) {
      ia += xa;
      ib += xb;
    }
  }
  if (lane == 31) {
    scratch[0][warp] = ia;
    scratch[1][warp] = ib;
  }
  __syncthreads();
  int pa = 0, pb = 0, sa = 0, sb = 0;
#pragma unroll
  for (int k = 0; k < kWarps; ++k) {
    const int va = scratch[0][k], vb = scratch[1][k];
    if (k < warp) {
      pa += va;
      pb += vb;
    }
    sa += va;
    sb += vb;
  }
  *ea = pa + ia - a;
  *eb = pb + ib - b;
  *ta = sa;
  *tb = sb;
  __syncthreads();
}

template <int kBits>
__device__ __forceinline__ uint32_t hash32(uint32_t k) { return (k * 0x9E3779B1u) >> (32 - kBits); }

// Order key of one field value (Sec. 4.1): see order_key_bits; written
// branch-free.  Out-of-box positions get the sentinel 0, which no real value
// has.
__device__ __forceinline__ uint32_t key_of(uint32_t b) {
  b = (b == 0x80000000u) ? 0u : b;
  const uint32_t m = (uint32_t)((int32_t)b >> 31);
  return b ^ (m | 0x80000000u);
}

// float16 bits widened exactly to float32 bits.
__device__ __forceinline__ uint32_t half_bits_to_float(uint16_t h) {
  return __float_as_uint(__half2float(__ushort_as_half(h)));
}

__device__ __forceinline__ uint32_t raw_bits(const void *__restrict__ field, int dtype, int64_t i) {
  if (dtype == MS_F16)
    return __float_as_uint(__half2float(reinterpret_cast<const __half *>(field)[i]));
  return __ldg(reinterpret_cast<const uint32_t *>(field) + i);
}

// ---- TMA and mbarrier helpers (inline PTX, sm_90+ forms, single CTA) -----
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Box load of the tile + halo: x from x0 - kXO, y from y0 - 1, z from z0 - 1;
// the unit zero-fills whatever lies outside the field.
__device__ __forceinline__ void tma_load_box(void *dst, const CUtensorMap *map, uint64_t *bar,
                                             int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_addr(bar))
      : "memory");
}

// 2D box load of a 2D tile + halo: x from x0 - kXO, y from y0 - 1.
__device__ __forceinline__ void tma_load_box2(void *dst, const CUtensorMap *map, uint64_t *bar,
                                              int x, int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_addr(bar))
      : "memory");
}

constexpr long long kWaitPolls = 1ll << 26;  // about a second of polling: a TMA never takes that

// Bounded wait for the tile's box load (thread 0).  Past the bound the call
// is flagged MS_ERR_TIMEOUT and the block stops; before it leaves, it polls up
// to four times longer still, so that a copy still in flight does not land in
// shared memory that another block (of this or another call) owns next.
__device__ __forceinline__ void wait_box(uint64_t *bar, uint32_t parity, DevStatus *st, int *s_abort) {
  long long polls = 0;
  while (!mbar_try_wait(bar, parity)) {
    if (++polls > kWaitPolls) {
      atomicOr(&st->timeout, 1u);
      *s_abort = 1;
      for (long long q = 0; q < 4 * kWaitPolls && !mbar_try_wait(bar, parity); ++q) __nanosleep(64);
      break;
    }
    __nanosleep(64);
  }
}

// One pointer jump of a packed (up | dn << 16) entry through the pointer
// area: up of its up, dn of its dn (Sec. 4.2.1 second step).
__device__ __forceinline__ uint32_t jump1(const uint32_t *P, uint32_t x) {
  return __byte_perm(P[x & 0xffffu], P[x >> 16], 0x7610);
}

// Comparisons of staged values.  Interior tiles (tile and halo inside the
// field) compare the raw float32 values: IEEE ">=" is the real order, equal
// reals (including -0 and +0) tie and fall to the index rule, and nvcc does
// not flush subnormals in comparisons unless told to.  Boundary tiles hold
// integer order keys with the out-of-field sentinel 0, and the minimum side
// compares key - 1 so that the sentinel sorts last there too.
template <bool kRaw>
struct Ord;
template <>
struct Ord<true> {
  static __device__ __forceinline__ bool ge(uint32_t b, uint32_t a) {
    return __uint_as_float(b) >= __uint_as_float(a);
  }
  static __device__ __forceinline__ bool lt(uint32_t b, uint32_t a) {
    return __uint_as_float(b) < __uint_as_float(a);
  }
  static __device__ __forceinline__ uint32_t mk(uint32_t k) { return k; }
};
template <>
struct Ord<false> {
  static __device__ __forceinline__ bool ge(uint32_t b, uint32_t a) { return b >= a; }
  static __device__ __forceinline__ bool lt(uint32_t b, uint32_t a) { return b < a; }
  static __device__ __forceinline__ uint32_t mk(uint32_t k) { return k - 1u; }
};

// b lies at higher vertex indices than a.
template <bool kRaw>
__device__ __forceinline__ Cand omax(Cand a, Cand b) {
  const bool t = Ord<kRaw>::ge(b.k, a.k);
  return Cand{t ? b.k : a.k, t ? b.i : a.i};
}
template <bool kRaw>
__device__ __forceinline__ Cand omin(Cand a, Cand b) {
  const bool t = Ord<kRaw>::lt(b.k, a.k);
  return Cand{t ? b.k : a.k, t ? b.i : a.i};
}

// Cube extrema.  A unit cube with minimum corner c = (cx, cy, cz), cx in
// [-1, TX-1], cy in [-1, TY-1], cz in [-1, TZ-1] (tile coordinates), has its
// (max, min) winners' box indices at C[cube_of(c)] as max | min << 16.
template <class S>
__device__ __forceinline__ int cube_of(int cx, int cy, int cz) {
  return (cx + 1) + S::CX * ((cy + 1) + S::CY * (cz + 1));
}

// Max and min of two candidates in one step (b at higher indices); the
// min side compares Ord::mk-transformed keys.
template <bool kRaw>
__device__ __forceinline__ void mm2(Cand a_max, Cand a_min, Cand b_max, Cand b_min, Cand *o_max,
                                    Cand *o_min) {
  *o_max = omax<kRaw>(a_max, b_max);
  *o_min = omin<kRaw>(a_min, b_min);
}

// The extremum pair of one cube from 8 box loads, x pairs, then y, then z.
template <class S, bool kRaw>
__device__ __forceinline__ uint32_t cube_extrema(const uint32_t *__restrict__ K, int cx, int cy,
                                                 int cz) {
  typedef Ord<kRaw> O;
  Cand zmax[2], zmin[2];
#pragma unroll
  for (int dz = 0; dz < 2; ++dz) {
    Cand ymax[2], ymin[2];
#pragma unroll
    for (int dy = 0; dy < 2; ++dy) {
      const uint32_t e = (uint32_t)((cx + kXO) + S::EX * ((cy + dy + 1) + S::EY * (cz + dz + 1)));
      const uint32_t k0 = K[e], k1 = K[e + 1];
      ymax[dy] = omax<kRaw>(Cand{k0, e}, Cand{k1, e + 1});
      ymin[dy] = omin<kRaw>(Cand{O::mk(k0), e}, Cand{O::mk(k1), e + 1});
    }
    zmax[dz] = omax<kRaw>(ymax[0], ymax[1]);
    zmin[dz] = omin<kRaw>(ymin[0], ymin[1]);
  }
  const Cand m = omax<kRaw>(zmax[0], zmax[1]), n = omin<kRaw>(zmin[0], zmin[1]);
  return m.i | (n.i << 16);
}

// up / dn of the tile's vertices.  N(v) u {v} is the union of the unit cubes
// [v, v+(1,1,1)] and [v-(1,1,1), v]; a cube's extremum is taken along x, then
// y, then z, and each cube serves two vertices (as the upper cube of its
// minimum corner and the lower cube of its maximum corner), so it is
// computed once: the cubes with c = (lx, ly, .) by thread (lx, ly) streaming
// z, the remaining cubes (some coordinate -1) spread over the block.  The
// results go to w[] in registers; C lives in P's area until then.
template <class S, bool kRaw>
__device__ __forceinline__ void steepest_tile(const uint32_t *__restrict__ K, uint32_t *C, int lx,
                                              int ly, bool col_in, int nz_here, uint32_t *w,
                                              bool *nan) {
  typedef Ord<kRaw> O;
  constexpr int kEX = S::EX, kEY = S::EY, kTZ_ = S::TZ;
  {
    Cand h2max{}, h2min{};
#pragma unroll 2
    for (int p = 0; p <= kTZ_; ++p) {
      const uint32_t e = (uint32_t)((lx + kXO) + kEX * ((ly + 1) + kEY * (p + 1)));
      const uint32_t k00 = K[e], k10 = K[e + 1], k01 = K[e + kEX], k11 = K[e + kEX + 1];
      if (kRaw && p < nz_here && col_in) *nan |= is_nan_bits(k00);
      const Cand a_max = omax<kRaw>(Cand{k00, e}, Cand{k10, e + 1});
      const Cand b_max = omax<kRaw>(Cand{k01, e + kEX}, Cand{k11, e + kEX + 1});
      const Cand a_min = omin<kRaw>(Cand{O::mk(k00), e}, Cand{O::mk(k10), e + 1});
      const Cand b_min = omin<kRaw>(Cand{O::mk(k01), e + kEX}, Cand{O::mk(k11), e + kEX + 1});
      const Cand pmax = omax<kRaw>(a_max, b_max), pmin = omin<kRaw>(a_min, b_min);
      if (p >= 1) {
        const Cand m = omax<kRaw>(h2max, pmax), n = omin<kRaw>(h2min, pmin);
        C[cube_of<S>(lx, ly, p - 1)] = m.i | (n.i << 16);
      }
      h2max = pmax;
      h2min = pmin;
    }
  }
  // cubes with a coordinate at -1: cz = -1 (CX x CY), then cy = -1 with cz
  // >= 0 (CX x TZ), then cx = -1 with cy, cz >= 0 (TY x TZ)
  constexpr int kCX = S::CX, kCY = S::CY, kTY = S::TY;
  constexpr int kA = kCX * kCY, kB = kCX * kTZ_, kCn = kTY * kTZ_;
  for (int j = threadIdx.x; j < kA + kB + kCn; j += S::Threads) {
    int cx, cy, cz;
    if (j < kA) {
      cz = -1;
      cx = j % kCX - 1;
      cy = j / kCX - 1;
    } else if (j < kA + kB) {
      const int q = j - kA;
      cy = -1;
      cx = q % kCX - 1;
      cz = q / kCX;
    } else {
      const int q = j - kA - kB;
      cx = -1;
      cy = q % kTY;
      cz = q / kTY;
    }
    C[cube_of<S>(cx, cy, cz)] = cube_extrema<S, kRaw>(K, cx, cy, cz);
  }
  __syncthreads();
#pragma unroll
  for (int lz = 0; lz < kTZ_; ++lz) {
    const uint32_t ev = (uint32_t)ext_of<S>(lx, ly, lz);
    const uint32_t hi = C[cube_of<S>(lx, ly, lz)], lo = C[cube_of<S>(lx - 1, ly - 1, lz - 1)];
    const uint32_t ua = lo & 0xffffu, ub = hi & 0xffffu, da = lo >> 16, db = hi >> 16;
    const uint32_t up = O::ge(K[ub], K[ua]) ? ub : ua;  // the upper cube lies at higher indices
    const uint32_t dn = O::lt(O::mk(K[db]), O::mk(K[da])) ? db : da;
    w[lz] = (col_in && lz < nz_here) ? (up | (dn << 16)) : ev * 0x10001u;
  }
  __syncthreads();  // C is dead; P may be written
}

// First-fit insert of key into the open-addressing pair set H of kHashN
// slots, starting at slot s; returns the key's slot.
template <int kHashN>
__device__ __forceinline__ uint32_t pairset_insert(uint32_t *H, uint32_t key, uint32_t s) {
  for (int probe = 0; probe < kHashN; ++probe) {
    uint32_t cur = H[s];
    if (cur == kEmpty32) cur = atomicCAS(&H[s], kEmpty32, key);
    if (cur == kEmpty32 || cur == key) return s;
    s = (s + 1) & (kHashN - 1);
  }
  return 0;  // unreachable: the set holds one slot per vertex
}

// An empty tile record (a tile skipped for a NaN): no pairs, no roots.
__device__ __forceinline__ void empty_tile(const TiledScratch &ts, int64_t gt) {
  if (threadIdx.x == 0) {
    TileMeta m;
    m.pbase = 0;
    m.rbase = 0;
    m.npairs = 0;
    m.nd = 0;
    m.nu = 0;
    m.pad = 0;
    ts.meta[gt] = m;
  }
}

// The distinct (dn-root, up-root) pairs and the distinct roots of a tile whose
// final pointers are in w[] (one run of kRun per thread, both tile shapes).
//   (1) every run entry whose pair differs from the entry before it inserts
//       the pair into the open-addressing set H (first fit);
//   (2) the used slots of H get dense numbers by a block scan (thread t owns
//       slots 16t .. 16t + 15), in which order they form the pair list PL;
//       each listed pair marks its dn root and its up root in two bitmaps
//       over the extended box;
//   (3) a block scan of the bitmap words' popcounts ranks the roots: the
//       tile's root list holds its dn roots in box order, then its up roots;
//   (4) the pair pool gets each pair as (dn-root index, up-root index) in the
//       root list, the root list gets each root's box index, and every
//       vertex its pair's dense number.
// A (kHash + kHash / 2 words) and B (kTileV + 4 kBmW words) are free
// shared-memory areas; valid run entries are those of a column with col_in,
// below n_here.  A tile of kThreads threads holds kTileV = 16 kThreads
// vertices, and its set kHash = kTileV slots (thread t numbers slots
// 16t .. 16t + 15).
template <int kThreads, int kBmW>
__device__ __forceinline__ void number_tile_pairs(uint32_t *A, uint32_t *B, const uint32_t (&w)[kRun],
                                                  bool col_in, int n_here, int64_t gt,
                                                  const TiledScratch &ts, DevStatus *st,
                                                  int (*s_scan2)[kThreads / 32],
                                                  unsigned long long *s_base) {
  constexpr int kTileV = kThreads * kRun;
  constexpr int kHash = kTileV;
  constexpr int kHashBits = ilog2(kHash);
  static_assert(kBmW <= kThreads, "two bitmap words per thread cover both root bitmaps");
  const int t = threadIdx.x;
  uint32_t *H = A;
  uint16_t *D = reinterpret_cast<uint16_t *>(A + kHash);
  uint32_t *PL = B;
  uint32_t *BW = B + kTileV;
  uint32_t *PW = BW + 2 * kBmW;
  for (int i = t; i < kHash / 4; i += kThreads)
    reinterpret_cast<uint4 *>(H)[i] = make_uint4(kEmpty32, kEmpty32, kEmpty32, kEmpty32);
  for (int i = t; i < 2 * kBmW; i += kThreads) BW[i] = 0u;
  __syncthreads();
  // (1) inserts: one per change of pair along the run
  uint32_t slot2[kRun / 2];  // two 16-bit set slots per word
  {
    uint32_t prev = kEmpty32, ps = 0;
#pragma unroll
    for (int j = 0; j < kRun; ++j) {
      const uint32_t key = w[j];
      if (col_in && j < n_here && key != prev) {
        ps = pairset_insert<kHash>(H, key, hash32<kHashBits>(key));
        prev = key;
      }
      if (j & 1)
        slot2[j / 2] |= ps << 16;
      else
        slot2[j / 2] = ps;
    }
  }
  __syncthreads();
  // (2) dense numbers of the used slots; the pair list; roots marked
  int npairs;
  {
    uint32_t hk[16];
    const uint4 *h4 = reinterpret_cast<const uint4 *>(H + 16 * t);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const uint4 v = h4[q];
      hk[4 * q] = v.x, hk[4 * q + 1] = v.y, hk[4 * q + 2] = v.z, hk[4 * q + 3] = v.w;
    }
    int cnt = 0;
#pragma unroll
    for (int k = 0; k < 16; ++k) cnt += hk[k] != kEmpty32;
    int ex, e2, t2;
    block_scan2<kThreads / 32>(cnt, 0, &ex, &e2, &npairs, &t2, s_scan2);
    int id = ex;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const uint32_t key = hk[k];
      if (key != kEmpty32) {
        D[16 * t + k] = (uint16_t)id;
        PL[id] = key;
        const uint32_t dn = key >> 16, up = key & 0xffffu;
        atomicOr(&BW[dn >> 5], 1u << (dn & 31u));
        atomicOr(&BW[kBmW + (up >> 5)], 1u << (up & 31u));
        ++id;
      }
    }
  }
  __syncthreads();
  // (3) root ranks: exclusive prefix popcounts over the dn words, then the up words
  int nroots;
  {
    const int w0 = t, w1 = t + kThreads;
    const int a = w0 < 2 * kBmW ? __popc(BW[w0]) : 0;
    const int b = w1 < 2 * kBmW ? __popc(BW[w1]) : 0;
    int ea, eb, ta, tb;
    block_scan2<kThreads / 32>(a, b, &ea, &eb, &ta, &tb, s_scan2);  // ends with a barrier
    if (w0 < 2 * kBmW) PW[w0] = (uint32_t)ea;
    if (w1 < 2 * kBmW) PW[w1] = (uint32_t)(ta + eb);
    nroots = ta + tb;
    if (t == 0) s_base[0] = atomicAdd(&ts.counters[0], (unsigned long long)npairs);
    if (t == 32) s_base[1] = atomicAdd(&ts.counters[1], (unsigned long long)nroots);
  }
  __syncthreads();
  const unsigned long long pbase = s_base[0], rbase = s_base[1];
  const int nd = (int)PW[kBmW];
  if (t == 0) {
    TileMeta m;
    m.pbase = pbase;
    m.rbase = rbase;
    m.npairs = npairs;
    m.nd = nd;
    m.nu = nroots - nd;
    m.pad = 0;
    ts.meta[gt] = m;
    if (pbase + (unsigned long long)npairs > ts.pool_cap) atomicOr(&st->pool_overflow, 1u);
    if (rbase + (unsigned long long)nroots > ts.root_cap) atomicOr(&st->pool_overflow, 1u);
  }
  // (4) pool entries, root list, per-vertex numbers
  if (pbase + (unsigned long long)npairs <= ts.pool_cap) {
    for (int i = t; i < npairs; i += kThreads) {
      const uint32_t key = PL[i];
      const uint32_t dn = key >> 16, up = key & 0xffffu;
      const uint32_t wd = dn >> 5, wu = kBmW + (up >> 5);
      const uint32_t di = PW[wd] + __popc(BW[wd] & ((1u << (dn & 31u)) - 1u));
      const uint32_t ui = PW[wu] + __popc(BW[wu] & ((1u << (up & 31u)) - 1u));
      // the pair's two roots as indices into the global root list
      ts.pool_pair[pbase + i] = make_uint2((uint32_t)(rbase + di), (uint32_t)(rbase + ui));
    }
  }
  if (rbase + (unsigned long long)nroots <= ts.root_cap) {
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int wi = t + q * kThreads;
      if (wi < 2 * kBmW) {
        uint32_t bits = BW[wi];
        uint32_t r = PW[wi];
        const uint32_t box0 = 32u * (uint32_t)(wi < kBmW ? wi : wi - kBmW);
        while (bits) {
          const uint32_t b = (uint32_t)(__ffs(bits) - 1);
          bits &= bits - 1u;
          ts.root_box[rbase + r] = (uint16_t)(box0 + b) | (wi < kBmW ? (uint16_t)0 : kUpRoot);
          if (ts.root_tile) ts.root_tile[rbase + r] = (uint32_t)gt;
          ++r;
        }
      }
    }
  }
  if (col_in) {
    uint32_t packed[kRun / 2];
#pragma unroll
    for (int j = 0; j < kRun; j += 2)
      packed[j / 2] = (uint32_t)D[slot2[j / 2] & 0xffffu] | ((uint32_t)D[slot2[j / 2] >> 16] << 16);
    uint4 *pid4 = reinterpret_cast<uint4 *>(ts.pid + gt * (int64_t)kPidStride +
                                            (int64_t)threadIdx.x * kRun);
    pid4[0] = make_uint4(packed[0], packed[1], packed[2], packed[3]);
    pid4[1] = make_uint4(packed[4], packed[5], packed[6], packed[7]);
  }
  __syncthreads();  // A and B are reused by the next tile
}

// Tile scheduling of the persistent kernels: a static stride over the tile
// range, or a work queue -- an atomic counter that thread 0 reads one tile
// ahead into *s_next (all threads have read the current index when it does).
__device__ __forceinline__ long long queue_first(bool dyn, unsigned int *ctr, long long *s_next) {
  if (!dyn) return blockIdx.x;
  if (threadIdx.x == 0) *s_next = atomicAdd(ctr, 1u);
  __syncthreads();
  return *s_next;
}
__device__ __forceinline__ void queue_prefetch(bool dyn, unsigned int *ctr, long long *s_next) {
  if (!dyn) return;
  __syncthreads();
  if (threadIdx.x == 0) *s_next = atomicAdd(ctr, 1u);
}
__device__ __forceinline__ long long queue_next(bool dyn, long long k, const long long *s_next) {
  return dyn ? *s_next : k + gridDim.x;
}

// One CTA per tile (persistent).  Thread t owns the z-column of vertices
// (x0 + t % TX, y0 + t / TX, z0 .. z0 + TZ - 1).
//
// Shared memory (dynamic): K, the staged field values of the tile and its
// halo in box order (reused for the pair set once the steepest step is
// done), and P, the up / dn pointers in the same order.
// Field of global tile gt: the last field whose first tile is <= gt.
__device__ __forceinline__ int field_of(const Batch &b, int64_t gt) {
  int lo = 0, hi = b.n_fields - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (b.fields[mid].tile_base <= gt)
      lo = mid;
    else
      hi = mid - 1;
  }
  return lo;
}

template <bool kSingle, class S>
__global__ void __launch_bounds__(S::Threads, 1024 / S::Threads) k_tile_local(Batch bt, TiledScratch ts,
                                                                             DevStatus *st) {
  constexpr int kTX = S::TX, kTY = S::TY, kTZ_ = S::TZ, kEX = S::EX, kEY = S::EY, kEZ = S::EZ;
  constexpr int kExt = S::Ext, kThreads = S::Threads, kFace = S::Face;
  // float16 boxes start kXO16 values left of the tile (16 bytes) and are kE16X wide
  constexpr int kXO16 = 8, kE16X = S::TX + 2 * kXO16;
  static_assert(kE16X * S::EY * S::EZ * 2 <= kExt * 4, "a float16 box fits the pointer area");
  static_assert((kExt * 4) % 128 == 0, "the pointer area starts 128-byte aligned");
  extern __shared__ __align__(128) uint32_t dsmem[];
  uint32_t *K = dsmem;         // kExt words: values / keys, then pair-numbering scratch
  uint32_t *P = dsmem + kExt;  // kExt words: up | dn << 16, box indices
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ unsigned long long s_base[2];
  __shared__ int s_abort;
  __shared__ int s_scan2[2][kThreads / 32];
  const int lane = threadIdx.x & 31;
  const int lx = threadIdx.x % kTX, ly = threadIdx.x / kTX;
  bool nan = false;
  uint32_t parity = 0;
  if (threadIdx.x == 0) s_abort = 0;
  if (threadIdx.x == 0) mbar_init(&s_bar, 1);
  __syncthreads();

  __shared__ long long s_next;
  const bool dyn = bt.tune.dynamic != 0;
  for (long long k = queue_first(dyn, ts.queue + kQTile3, &s_next); k < bt.tiles3;
       k = queue_next(dyn, k, &s_next)) {
    queue_prefetch(dyn, ts.queue + kQTile3, &s_next);
    const int64_t gt = k;
    const int fi = kSingle ? 0 : field_of(bt, gt);
    const FieldDesc &fd = kSingle ? bt.f0 : bt.fields[fi];
    const TileGeom &g = fd.g;
    const void *__restrict__ field = fd.field;
    const int dtype = fd.dtype;
    const bool tma = fd.tma != 0;
    const bool f16 = dtype == MS_F16;
    const int64_t tile = gt - fd.tile_base;  // within the field
    int64_t x0, y0, z0;
    tile_origin<S>(g, tile, &x0, &y0, &z0);
    // float32 tile and halo entirely inside the field: raw float comparisons
    const bool raw = tma && !f16 && x0 >= 1 && y0 >= 1 && z0 >= 1 && x0 + kTX < g.nx &&
                     y0 + kTY < g.ny && z0 + kTZ_ < g.nz;

    // ---- field values of the tile + halo into K (float16: a 16-bit box from
    // x0 - 8, the nearest 16-byte boundary, into P's area, widened below)
    if (tma) {
      if (threadIdx.x == 0) {
        // K and P were last written by ordinary stores; order them before the copy
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (f16) {
          mbar_expect_tx(&s_bar, (uint32_t)(kE16X * kEY * kEZ * 2));
          tma_load_box(P, &bt.tmaps[fi], &s_bar, (int)(x0 - kXO16), (int)(y0 - 1), (int)(z0 - 1));
        } else {
          mbar_expect_tx(&s_bar, (uint32_t)(kExt * 4));
          tma_load_box(K, &bt.tmaps[fi], &s_bar, (int)(x0 - kXO), (int)(y0 - 1), (int)(z0 - 1));
        }
      }
      if (threadIdx.x == 0) wait_box(&s_bar, parity, st, &s_abort);
      __syncthreads();
      if (s_abort) return;  // block-uniform
      parity ^= 1u;
    }
    // ---- boundary tiles: order keys in place (sentinel 0 outside the
    // field).  All tiles: halo pointers are self-loops.  The kTX threads of
    // a row group (one y of the tile) take one box row at a time; the first
    // two also take the row's halo columns.
    if (!raw) {
      const int exe = lx == 0 ? kXO - 1 : kXO + kTX;  // threads lx = 0, 1: the halo columns
      const int64_t xl = x0 + lx, xe = x0 + exe - kXO;
      const bool x_in = xl < g.nx, xe_in = xe >= 0 && xe < g.nx;
#pragma unroll 4
      for (int r = ly; r < kEY * kEZ; r += kTY) {
        const int ey = r % kEY, ez = r / kEY;
        const bool interior = ey >= 1 && ey <= kTY && ez >= 1 && ez <= kTZ_;
        const int eb = kEX * r;
        {
          const int64_t y = y0 + ey - 1, z = z0 + ez - 1;
          const bool row_in = y >= 0 && y < g.ny && z >= 0 && z < g.nz;
          uint32_t b, be = 0;
          if (tma && f16) {  // the staged 16-bit row: box column c is staged column c + kXO16 - kXO
            const uint16_t *row16 = reinterpret_cast<const uint16_t *>(P) + kE16X * r + (kXO16 - kXO);
            b = half_bits_to_float(row16[kXO + lx]);
            if (lx < 2) be = half_bits_to_float(row16[exe]);
          } else if (tma) {
            b = K[eb + kXO + lx];
            if (lx < 2) be = K[eb + exe];
          } else {
            const int64_t row = y * g.nx + z * g.nx * g.ny;
            b = (row_in && x_in) ? raw_bits(field, dtype, row + xl) : 0u;
            if (lx < 2 && row_in && xe_in) be = raw_bits(field, dtype, row + xe);
          }
          if (row_in && x_in && interior) nan |= is_nan_bits(b);
          K[eb + kXO + lx] = (row_in && x_in) ? key_of(b) : 0u;
          if (lx < 2) K[eb + exe] = (row_in && xe_in) ? key_of(be) : 0u;
        }
      }
    }
    __syncthreads();

    // ---- steepest neighbours: the extremum of every unit cube the tile's
    // vertices need, once each, into C (in P's area); then per vertex the
    // better of its two cubes; then P = pointers, halo = self-loops
    const bool col_in = x0 + lx < g.nx && y0 + ly < g.ny;
    const int nz_here = (int)min((int64_t)kTZ_, g.nz - z0);
    uint32_t w[kRun];
    if (raw)
      steepest_tile<S, true>(K, P, lx, ly, col_in, nz_here, w, &nan);
    else
      steepest_tile<S, false>(K, P, lx, ly, col_in, nz_here, w, &nan);
    if (__syncthreads_or(nan)) {
      // the call fails with MS_ERR_NAN_INPUT; skip the rest of this tile
      empty_tile(ts, gt);
      __syncthreads();
      continue;
    }
#pragma unroll
    for (int lz = 0; lz < kTZ_; ++lz) P[ext_of<S>(lx, ly, lz)] = w[lz];
    // the halo points at itself: the 2 kEZ + 2 kTY box rows with ey or ez on
    // the halo (one row group per row), then the two halo columns of the
    // kTY x kTZ inner rows
    for (int j = ly; j < 2 * kEZ + 2 * kTY; j += kTY) {
      int ey, ez;
      if (j < 2 * kEZ) {
        ey = (j & 1) ? kEY - 1 : 0;
        ez = j >> 1;
      } else {
        const int q = j - 2 * kEZ;
        ez = (q & 1) ? kEZ - 1 : 0;
        ey = 1 + (q >> 1);
      }
      const int eb = kEX * (ey + kEY * ez);
      P[eb + kXO + lx] = (uint32_t)(eb + kXO + lx) * 0x10001u;
      if (lx < 2) {
        const int e = eb + (lx == 0 ? kXO - 1 : kXO + kTX);
        P[e] = (uint32_t)e * 0x10001u;
      }
    }
    for (int i = threadIdx.x; i < 2 * kTY * kTZ_; i += kThreads) {
      const int row = i >> 1;
      const int e = kEX * ((1 + (row % kTY)) + kEY * (1 + row / kTY)) +
                    ((i & 1) ? kXO + kTX : kXO - 1);
      P[e] = (uint32_t)e * 0x10001u;
    }
    __syncthreads();

    // ---- path compression inside the tile.  Halo entries and extrema are
    // self-pointers, so every pointer ends on a local extremum or an exit.
    // Each thread keeps its own 16 pointers in registers (it alone writes
    // them) and jumps them in place until a pass changes nothing in its
    // warp; reads of other vertices' pointers may see them before or after
    // their own jumps, and either lies on the same path.
    // An entry that a pass leaves unchanged points at two roots (only roots
    // point at themselves) and is final; a warp skips the entries that are
    // final in all its lanes.
    {
      uint32_t open = 0xffffu;
      for (int it = 0; it < kExt; ++it) {
        // the entries still open in some lane of the warp (one reduction a pass)
        const uint32_t rows = __reduce_or_sync(0xffffffffu, open);
        if (!rows) break;
        uint32_t still = 0;
#pragma unroll
        for (int lz = 0; lz < kTZ_; ++lz) {
          if ((rows >> lz) & 1u) {
            const uint32_t nw = jump1(P, w[lz]);
            if (nw != w[lz]) {
              w[lz] = nw;
              P[ext_of<S>(lx, ly, lz)] = nw;
              still |= 1u << lz;
            }
          }
        }
        open = still;
      }
    }
    __syncthreads();

    // ---- face roots (final pointers of the tile's face vertices), written
    // cooperatively from P: other tiles' paths enter through these vertices
    {
      uint32_t *face = ts.face + gt * (int64_t)bt.face_stride;
      for (int fs = threadIdx.x; fs < kFace; fs += kThreads) {
        int fx, fy, fz;
        face_coords<S>(fs, &fx, &fy, &fz);
        if (x0 + fx < g.nx && y0 + fy < g.ny && fz < nz_here) face[fs] = P[ext_of<S>(fx, fy, fz)];
      }
    }
    __syncthreads();

    number_tile_pairs<kThreads, S::BmW>(K, P, w, col_in, nz_here, gt, ts, st, s_scan2, s_base);
  }
  if (__any_sync(0xffffffffu, nan) && lane == 0) atomicOr(&st->nan_flag, 1u);
}

// up / dn of a thread's run of kRun vertices in a 2D tile.  N(v) u {v} is
// the union of the unit squares [v, v+(1,1)] and [v-(1,1), v]; with
// A(y) = extremum of {(x-1, y), (x, y)} and B(y) = extremum of {(x, y),
// (x+1, y)}, the lower square is A(y-1), A(y) and the upper one B(y), B(y+1).
// The thread streams the rows y0 - 1 .. y0 + kRun of its column, keeping two
// rows of A and B in registers (every operand pair again has its second
// operand at higher vertex indices).
template <bool kRaw>
__device__ __forceinline__ void steepest_run2(const uint32_t *__restrict__ K, int cx, int cy0,
                                              bool col_in, int n_here, uint32_t *w, bool *nan) {
  typedef Ord<kRaw> O;
  const uint32_t e0 = (uint32_t)((cx + kXO) + k2EX * cy0);  // box row of y = cy0 - 1
  Cand a0x, a0n, a1x, a1n, b1x, b1n;
  uint32_t kc1;
  {
    const uint32_t e = e0;
    const uint32_t kl = K[e - 1], kc = K[e];
    a0x = omax<kRaw>(Cand{kl, e - 1}, Cand{kc, e});
    a0n = omin<kRaw>(Cand{O::mk(kl), e - 1}, Cand{O::mk(kc), e});
  }
  {
    const uint32_t e = e0 + k2EX;
    const uint32_t kl = K[e - 1], kc = K[e], kr = K[e + 1];
    a1x = omax<kRaw>(Cand{kl, e - 1}, Cand{kc, e});
    a1n = omin<kRaw>(Cand{O::mk(kl), e - 1}, Cand{O::mk(kc), e});
    b1x = omax<kRaw>(Cand{kc, e}, Cand{kr, e + 1});
    b1n = omin<kRaw>(Cand{O::mk(kc), e}, Cand{O::mk(kr), e + 1});
    kc1 = kc;
  }
#pragma unroll
  for (int j = 0; j < kRun; ++j) {
    const uint32_t e = e0 + (uint32_t)(j + 2) * k2EX;  // the row below vertex j
    const uint32_t kl = K[e - 1], kc = K[e], kr = K[e + 1];
    const Cand a2x = omax<kRaw>(Cand{kl, e - 1}, Cand{kc, e});
    const Cand a2n = omin<kRaw>(Cand{O::mk(kl), e - 1}, Cand{O::mk(kc), e});
    const Cand b2x = omax<kRaw>(Cand{kc, e}, Cand{kr, e + 1});
    const Cand b2n = omin<kRaw>(Cand{O::mk(kc), e}, Cand{O::mk(kr), e + 1});
    const uint32_t up = omax<kRaw>(omax<kRaw>(a0x, a1x), omax<kRaw>(b1x, b2x)).i;
    const uint32_t dn = omin<kRaw>(omin<kRaw>(a0n, a1n), omin<kRaw>(b1n, b2n)).i;
    const bool valid = col_in && j < n_here;
    if (kRaw && valid) *nan |= is_nan_bits(kc1);
    const uint32_t ev = e0 + (uint32_t)(j + 1) * k2EX;
    w[j] = valid ? (up | (dn << 16)) : ev * 0x10001u;
    a0x = a1x;
    a0n = a1n;
    a1x = a2x;
    a1n = a2n;
    b1x = b2x;
    b1n = b2n;
    kc1 = kc;
  }
}

// The 2D form of k_tile_local, for fields with nz = 1 (the tiles after the
// 3D fields' in a batch).  Thread (lane, warp) owns the run of kRun vertices
// at x = lane + 32 (warp % 4), y = kRun (warp / 4) + 0 .. kRun - 1.
// float16 2D boxes: k2E16X values from x0 - k2XO16 (16-byte aligned), staged
// in P's area from its first 128-byte boundary (word k2StageOff).
constexpr int k2XO16 = 8, k2E16X = k2TX + 2 * k2XO16;
constexpr int k2StageOff = ((k2KArea * 4 + 127) / 128 * 128 - k2KArea * 4) / 4;
static_assert(k2StageOff * 4 + k2E16X * k2EY * 2 <= k2PArea * 4, "a float16 2D box fits P's area");

template <bool kSingle>
__global__ void __launch_bounds__(k2Threads, 2) k_tile_local2(Batch bt, TiledScratch ts, DevStatus *st) {
  extern __shared__ __align__(128) uint32_t dsmem[];
  uint32_t *K = dsmem;            // k2KArea words: values / keys, then the pair list and bitmaps
  uint32_t *P = dsmem + k2KArea;  // k2PArea words: up | dn << 16, then the pair set
  __shared__ __align__(8) uint64_t s_bar;
  __shared__ unsigned long long s_base[2];
  __shared__ int s_abort;
  __shared__ int s_scan2[2][k2Threads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int cx = lane + 32 * (warp & 3), cy0 = kRun * (warp >> 2);
  bool nan = false;
  uint32_t parity = 0;
  if (threadIdx.x == 0) s_abort = 0;
  if (threadIdx.x == 0) mbar_init(&s_bar, 1);
  __syncthreads();

  __shared__ long long s_next;
  const bool dyn = bt.tune.dynamic != 0;
  for (long long k = queue_first(dyn, ts.queue + kQTile2, &s_next); k < bt.total_tiles - bt.tiles3;
       k = queue_next(dyn, k, &s_next)) {
    queue_prefetch(dyn, ts.queue + kQTile2, &s_next);
    const int64_t gt = bt.tiles3 + k;
    const int fi = kSingle ? 0 : field_of(bt, gt);
    const FieldDesc &fd = kSingle ? bt.f0 : bt.fields[fi];
    const TileGeom &g = fd.g;
    const void *__restrict__ field = fd.field;
    const int dtype = fd.dtype;
    const bool tma = fd.tma != 0;
    const bool f16 = dtype == MS_F16;
    int64_t x0, y0;
    tile_origin2(g, gt - fd.tile_base, &x0, &y0);
    const bool raw = tma && !f16 && x0 >= 1 && y0 >= 1 && x0 + k2TX < g.nx && y0 + k2TY < g.ny;
    // float16: a 16-bit box from x0 - 8 staged at a 128-byte boundary in P's area
    const uint16_t *S16 = reinterpret_cast<const uint16_t *>(P + k2StageOff);

    if (tma) {
      if (threadIdx.x == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (f16) {
          mbar_expect_tx(&s_bar, (uint32_t)(k2E16X * k2EY * 2));
          tma_load_box2(P + k2StageOff, &bt.tmaps[fi], &s_bar, (int)(x0 - k2XO16), (int)(y0 - 1));
        } else {
          mbar_expect_tx(&s_bar, (uint32_t)(k2Ext * 4));
          tma_load_box2(K, &bt.tmaps[fi], &s_bar, (int)(x0 - kXO), (int)(y0 - 1));
        }
        wait_box(&s_bar, parity, st, &s_abort);
      }
      __syncthreads();
      if (s_abort) return;  // block-uniform
      parity ^= 1u;
    }
    // boundary tiles: order keys in place, sentinel 0 outside the field
    if (!raw) {
      constexpr int kCols = k2TX + 2;  // the tile's columns and the two halo columns
      for (int i = threadIdx.x; i < k2EY * kCols; i += k2Threads) {
        const int r = i / kCols, c = i - r * kCols + kXO - 1;
        const int e = r * k2EX + c;
        const int64_t x = x0 + c - kXO, y = y0 + r - 1;
        const bool in = x >= 0 && x < g.nx && y >= 0 && y < g.ny;
        uint32_t b = 0;
        if (tma && f16)
          b = half_bits_to_float(S16[r * k2E16X + c + (k2XO16 - kXO)]);
        else if (tma)
          b = K[e];
        else if (in)
          b = raw_bits(field, dtype, y * g.nx + x);
        if (in && r >= 1 && r <= k2TY && c >= kXO && c < kXO + k2TX) nan |= is_nan_bits(b);
        K[e] = in ? key_of(b) : 0u;
      }
    }
    __syncthreads();

    const bool col_in = x0 + cx < g.nx && y0 + cy0 < g.ny;
    const int n_here = (int)min((int64_t)kRun, g.ny - (y0 + cy0));
    uint32_t w[kRun];
    if (raw)
      steepest_run2<true>(K, cx, cy0, col_in, n_here, w, &nan);
    else
      steepest_run2<false>(K, cx, cy0, col_in, n_here, w, &nan);
    if (__syncthreads_or(nan)) {
      empty_tile(ts, gt);
      __syncthreads();
      continue;
    }
#pragma unroll
    for (int j = 0; j < kRun; ++j) P[ext2_of(cx, cy0 + j)] = w[j];
    // the halo ring points at itself
    for (int i = threadIdx.x; i < 2 * (k2TX + 2) + 2 * k2TY; i += k2Threads) {
      int e;
      if (i < k2TX + 2)
        e = kXO - 1 + i;
      else if (i < 2 * (k2TX + 2))
        e = (k2EY - 1) * k2EX + kXO - 1 + (i - (k2TX + 2));
      else {
        const int q = i - 2 * (k2TX + 2);
        e = (1 + (q >> 1)) * k2EX + ((q & 1) ? kXO + k2TX : kXO - 1);
      }
      P[e] = (uint32_t)e * 0x10001u;
    }
    __syncthreads();

    // in-place pointer jumping, as in the 3D tiles
    {
      uint32_t open = 0xffffu;
      for (int it = 0; it < k2Ext; ++it) {
        const uint32_t rows = __reduce_or_sync(0xffffffffu, open);
        if (!rows) break;
        uint32_t still = 0;
#pragma unroll
        for (int j = 0; j < kRun; ++j) {
          if ((rows >> j) & 1u) {
            const uint32_t nw = jump1(P, w[j]);
            if (nw != w[j]) {
              w[j] = nw;
              P[ext2_of(cx, cy0 + j)] = nw;
              still |= 1u << j;
            }
          }
        }
        open = still;
      }
    }
    __syncthreads();

    {
      uint32_t *face = ts.face + gt * (int64_t)bt.face_stride;
      for (int fs = threadIdx.x; fs < k2Face; fs += k2Threads) {
        int fx, fy;
        face_coords2(fs, &fx, &fy);
        if (x0 + fx < g.nx && y0 + fy < g.ny) face[fs] = P[ext2_of(fx, fy)];
      }
    }
    __syncthreads();

    number_tile_pairs<k2Threads, kBmW2>(P, K, w, col_in, n_here, gt, ts, st, s_scan2, s_base);
  }
  if (__any_sync(0xffffffffu, nan) && lane == 0) atomicOr(&st->nan_flag, 1u);
}

// Global face-graph slot of a face vertex v (a tile exit) of a field whose
// first tile is tile_base (fstride slots a tile).
template <class S>
__device__ __forceinline__ uint32_t slot_of_vertex(const TileGeom &g, long long tile_base,
                                                   uint32_t v, int fstride) {
  if (g.flat) {
    uint32_t x, y;
    g.div_nx.divmod(v, &y, &x);
    const uint32_t tx = x / k2TX, ty = y / k2TY;
    const int fs = face_slot2((int)(x - tx * k2TX), (int)(y - ty * k2TY));
    return (uint32_t)((tile_base + tx + (long long)g.tx * ty) * fstride + fs);
  }
  uint32_t q, x, y, z;
  g.div_nx.divmod(v, &q, &x);
  g.div_ny.divmod(q, &z, &y);
  const uint32_t tx = x / S::TX, ty = y / S::TY, tz = z / S::TZ;
  const int fs = face_slot<S>((int)(x - tx * S::TX), (int)(y - ty * S::TY), (int)(z - tz * S::TZ));
  return (uint32_t)((tile_base + tx + (long long)g.tx * (ty + (long long)g.ty * tz)) * fstride + fs);
}

// Face-graph slots are numbered face_stride per tile (the 3D shape's face
// count); 2D tiles use the first k2Face.  Valid slot i (of
// face_graph_valid(b)) -> (tile, face slot).
__device__ __forceinline__ void valid_slot(const Batch &b, long long i, long long *gt, int *fs) {
  const long long f3 = b.face_stride;
  const long long n3 = b.tiles3 * f3;
  if (i < n3) {
    *gt = i / f3;
    *fs = (int)(i - *gt * f3);
  } else {
    const long long j = i - n3;
    *gt = b.tiles3 + j / k2Face;
    *fs = (int)(j - (*gt - b.tiles3) * k2Face);
  }
}

__host__ __device__ __forceinline__ long long face_graph_valid(const Batch &b) {
  return b.tiles3 * (long long)b.face_stride + (b.total_tiles - b.tiles3) * (long long)k2Face;
}

// The face graph from the tiles' face roots (local box indices): exits
// become the global slot of the exit vertex, extrema their vertex index |
// kSlotFinal.  Slots of vertices outside their field get a final dummy.
template <class S>
__global__ void k_face_graph_build(Batch bt, TiledScratch ts, int2 *__restrict__ graph) {
  const long long nvalid = face_graph_valid(bt);
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nvalid;
       i += (long long)gridDim.x * blockDim.x) {
    long long gt;
    int fs;
    valid_slot(bt, i, &gt, &fs);
    const int fi = field_of(bt, gt);
    const FieldDesc &fd = bt.fields[fi];
    const TileGeom &g = fd.g;
    const long long tile = gt - fd.tile_base;
    const long long slot = gt * (long long)bt.face_stride + fs;
    int32_t ru, rd;
    bool in;
    const uint32_t w = ts.face[slot];
    if (g.flat) {
      int64_t x0, y0;
      tile_origin2(g, tile, &x0, &y0);
      int fx, fy;
      face_coords2(fs, &fx, &fy);
      in = x0 + fx < g.nx && y0 + fy < g.ny;
      ru = in ? root_ref2(g, x0, y0, (int)(w & 0xffffu)) : 0;
      rd = in ? root_ref2(g, x0, y0, (int)(w >> 16)) : 0;
    } else {
      int64_t x0, y0, z0;
      tile_origin<S>(g, tile, &x0, &y0, &z0);
      int fx, fy, fz;
      face_coords<S>(fs, &fx, &fy, &fz);
      in = x0 + fx < g.nx && y0 + fy < g.ny && z0 + fz < g.nz;
      ru = in ? root_ref<S>(g, x0, y0, z0, (int)(w & 0xffffu)) : 0;
      rd = in ? root_ref<S>(g, x0, y0, z0, (int)(w >> 16)) : 0;
    }
    auto enc = [&](int32_t r) -> int32_t {
      if (!(r & kExitFlag)) return (int32_t)((uint32_t)r | kSlotFinal);
      return (int32_t)slot_of_vertex<S>(g, fd.tile_base, (uint32_t)(r & ~kExitFlag), bt.face_stride);
    };
    graph[slot] = in ? make_int2(enc(ru), enc(rd)) : make_int2((int32_t)kSlotFinal, (int32_t)kSlotFinal);
  }
}

// One in-place pointer-jumping round over the face graph (each entry moves to
// its successor's entry; entries read mid-round are still on the same path).
// Sets st->round_open[round] if any entry is still not final.
__global__ void k_face_graph_round(Batch bt, int2 *__restrict__ graph, int round, DevStatus *st) {
  const long long nvalid = face_graph_valid(bt);
  const long long nslots = bt.total_tiles * (long long)bt.face_stride;
  bool open = false;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nvalid;
       i += (long long)gridDim.x * blockDim.x) {
    long long gt;
    int fs;
    valid_slot(bt, i, &gt, &fs);
    const long long slot = gt * (long long)bt.face_stride + fs;
    int2 a = graph[slot];
    bool ch = false;
    // two jumps per round: an entry then points (more than) three times as far
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      if (!((uint32_t)a.x & kSlotFinal)) {
        if ((long long)a.x >= nslots) {  // cannot happen for a well-formed graph
          atomicOr(&st->bad_index, 1u);
          a.x = (int32_t)kSlotFinal;
        } else {
          a.x = graph[a.x].x;
        }
        ch = true;
      }
      if (!((uint32_t)a.y & kSlotFinal)) {
        if ((long long)a.y >= nslots) {
          atomicOr(&st->bad_index, 1u);
          a.y = (int32_t)kSlotFinal;
        } else {
          a.y = graph[a.y].y;
        }
        ch = true;
      }
    }
    if (ch) {
      graph[slot] = a;
      open |= !((uint32_t)a.x & kSlotFinal) || !((uint32_t)a.y & kSlotFinal);
    }
  }
  if (__any_sync(0xffffffffu, open) && (threadIdx.x & 31) == 0) st->round_open[round] = 1u;
}



// Returns true (block-uniform) when an earlier stage of the call found its
// buffers too small or the input bad: the tile records are then not valid to
// read (a replayed graph runs every stage regardless; the host runs the call
// again step by step or reports the error).
__device__ __forceinline__ bool call_failed(const DevStatus *st) {
  return (st->pool_overflow | st->nan_flag | st->timeout | st->bad_index) != 0u;
}

// Decoding table of the root chase: for every extended-box index of a tile
// shape, either its tile coordinates (a vertex inside the tile: the chase
// ends there) or, for a halo vertex, the direction of the neighbouring tile
// that holds it and its slot in that tile's face array.  Built once per
// block; a hop is then one table read and one face read.
//   inside:  bits 0-6 lx, 7-12 ly, 13-17 lz
//   halo:    bit 31, bits 0-11 face slot, 12-13 dx + 1, 14-15 dy + 1, 16-17 dz + 1
constexpr uint32_t kHaloBit = 0x80000000u;

template <bool kFlat, class S>
__device__ __forceinline__ uint32_t chase_code(int e) {
  int lx, ly, lz = 0;
  if (kFlat) {
    const int ey = e / k2EX;
    lx = e - ey * k2EX - kXO, ly = ey - 1;
  } else {
    const int ez = e / (S::EX * S::EY), r = e - ez * (S::EX * S::EY), ey = r / S::EX;
    lx = r - ey * S::EX - kXO, ly = ey - 1, lz = ez - 1;
  }
  constexpr int TX = kFlat ? k2TX : S::TX, TY = kFlat ? k2TY : S::TY, TZ = kFlat ? 1 : S::TZ;
  const int dx = lx < 0 ? -1 : (lx >= TX ? 1 : 0);
  const int dy = ly < 0 ? -1 : (ly >= TY ? 1 : 0);
  const int dz = kFlat ? 0 : (lz < 0 ? -1 : (lz >= TZ ? 1 : 0));
  if ((dx | dy | dz) == 0) return (uint32_t)lx | ((uint32_t)ly << 7) | ((uint32_t)lz << 13);
  if (lx < -1 || lx > TX) return kHaloBit;  // a padding column: never a root
  const int fs = kFlat ? face_slot2(lx - dx * TX, ly - dy * TY)
                       : face_slot<S>(lx - dx * TX, ly - dy * TY, lz - dz * TZ);
  return kHaloBit | (uint32_t)fs | ((uint32_t)(dx + 1) << 12) | ((uint32_t)(dy + 1) << 14) |
         ((uint32_t)(dz + 1) << 16);
}

// Root chase, flat over the root list (see launch_chase_roots; calls with
// few tiles): a lane takes
// roots r, r + T, r + 2T, ... (T threads in all) and keeps kInFlight chases
// going at once, starting the next root in a chase's place as soon as it ends,
// so that neither a long chain nor a tile with many roots holds up others.
// A root knows its tile; its field is found from the tile.  kFlat: the 2D
// tiles' roots, which follow the 3D tiles' in the list.
constexpr int kChaseThreads = 512;
constexpr int kInFlight = 4;

template <bool kFlat, bool kSingle, class S>
__global__ void __launch_bounds__(kChaseThreads, 2) k_chase_flat(Batch bt, TiledScratch ts,
                                                                  const int2 *__restrict__ graph,
                                                                  long long probe_stride,
                                                                  DevStatus *st) {
  if (call_failed(st)) return;
  extern __shared__ uint32_t LUT[];
  constexpr int kE = kFlat ? k2Ext : S::Ext;
  constexpr int TX = kFlat ? k2TX : S::TX, TY = kFlat ? k2TY : S::TY, TZ = kFlat ? 1 : S::TZ;
  constexpr int kFaceN = kFlat ? k2Face : S::Face;
  const long long fstride = bt.face_stride;
  for (int e = threadIdx.x; e < kE; e += kChaseThreads) LUT[e] = chase_code<kFlat, S>(e);
  __syncthreads();
  const bool probe = probe_stride > 0;
  const unsigned long long cap = ts.root_cap;
  const unsigned long long r0 = kFlat ? min(ts.counters[2], cap) : 0ull;
  const unsigned long long r1 = min(kFlat ? ts.counters[1] : ts.counters[2], cap);
  const unsigned long long nroots = r1 > r0 ? r1 - r0 : 0ull;
  const unsigned long long nwork =
      probe ? (nroots + (unsigned long long)probe_stride - 1) / (unsigned long long)probe_stride : nroots;
  const unsigned long long T = (unsigned long long)gridDim.x * kChaseThreads;
  unsigned int sampled = 0, pending = 0, bad = 0;
  // per chase in flight: its work item, root, field, tile, box index, hops
  unsigned long long w[kInFlight];
  uint32_t e[kInFlight];
  int fi[kInFlight], tx[kInFlight], ty[kInFlight], tz[kInFlight], hops[kInFlight];
  bool up[kInFlight];
  unsigned long long next = (unsigned long long)blockIdx.x * kChaseThreads + threadIdx.x;
  auto start = [&](int q) {
    w[q] = next;
    next += T;
    if (w[q] >= nwork) return;
    const unsigned long long r = r0 + (probe ? w[q] * (unsigned long long)probe_stride : w[q]);
    const uint32_t b = ts.root_box[r];
    const int64_t gt = ts.root_tile[r];
    const int f = kSingle ? 0 : field_of(bt, gt);
    const FieldDesc &fd = kSingle ? bt.f0 : bt.fields[f];
    uint32_t rr, x, y, z = 0;
    if (kFlat) {
      fd.g.div_tx.divmod((uint32_t)(gt - fd.tile_base), &y, &x);
    } else {
      fd.g.div_tx.divmod((uint32_t)(gt - fd.tile_base), &rr, &x);
      fd.g.div_ty.divmod(rr, &z, &y);
    }
    fi[q] = f, tx[q] = (int)x, ty[q] = (int)y, tz[q] = (int)z;
    e[q] = b & (uint32_t)(kUpRoot - 1);
    up[q] = (b & kUpRoot) != 0;
    hops[q] = 0;
  };
#pragma unroll
  for (int q = 0; q < kInFlight; ++q) start(q);
  for (;;) {
    bool any = false;
#pragma unroll
    for (int q = 0; q < kInFlight; ++q) {
      if (w[q] >= nwork) continue;
      any = true;
      const FieldDesc &fd = kSingle ? bt.f0 : bt.fields[fi[q]];
      const uint32_t code = LUT[e[q]];
      int32_t label = 0;
      bool done = false;
      if (!(code & kHaloBit)) {  // inside its tile: the extremum
        const uint32_t lx = code & 127u, ly = (code >> 7) & 63u, lz = (code >> 13) & 31u;
        label = (int32_t)((uint32_t)(tx[q] * TX) + lx +
                          (uint32_t)fd.g.nx * ((uint32_t)(ty[q] * TY) + ly +
                                               (uint32_t)fd.g.ny * ((uint32_t)(tz[q] * TZ) + lz)));
        done = true;
      } else {
        const int gtx = (int)fd.g.tx, gty = (int)fd.g.ty, gtz = (int)fd.g.tz;
        const int ntx = tx[q] + (int)((code >> 12) & 3u) - 1;
        const int nty = ty[q] + (int)((code >> 14) & 3u) - 1;
        const int ntz = tz[q] + (int)((code >> 16) & 3u) - 1;
        if ((unsigned)ntx >= (unsigned)gtx || (unsigned)nty >= (unsigned)gty ||
            (unsigned)ntz >= (unsigned)gtz) {  // cannot happen: every root lies in the field
          ++bad;
          done = true;
        } else {
          const long long slot =
              (fd.tile_base + (long long)ntx + (long long)gtx * (nty + (long long)gty * ntz)) * fstride +
              (code & 0xfffu);
          if (graph) {  // the jumped face graph knows where the path ends
            const int2 gv = graph[slot];
            const uint32_t f = (uint32_t)(up[q] ? gv.x : gv.y);
            if (!(f & kSlotFinal)) atomicOr(&st->not_converged, 1u);
            label = (int32_t)(f & ~kSlotFinal);
            done = true;
          } else {
            const int64_t n = fd.g.nx * fd.g.ny * fd.g.nz;
            const int64_t slots = fd.g.ntiles * (int64_t)kFaceN;
            const int64_t max_hops = probe ? kProbeHops : (n < slots ? n : slots);
            if (++hops[q] > max_hops) {
              if (probe)
                ++pending;
              else
                atomicOr(&st->not_converged, 1u);
              done = true;
            } else {
              const uint32_t wv = __ldg(&ts.face[slot]);
              e[q] = up[q] ? (wv & 0xffffu) : (wv >> 16);
              tx[q] = ntx, ty[q] = nty, tz[q] = ntz;
            }
          }
        }
      }
      if (done) {
        if (probe)
          ++sampled;
        else
          ts.root_label[r0 + w[q]] = label;
        start(q);
      }
    }
    if (!__any_sync(0xffffffffu, any)) break;
  }
  if (bad) atomicOr(&st->bad_index, 1u);
  if (probe) {
    if (sampled) atomicAdd(&st->sampled, sampled);
    if (pending) atomicAdd(&st->pending, pending);
  }
}

// Root chase, a tile a warp (see launch_chase_roots; calls with many tiles).
// A warp takes one tile at a time from
// a work queue; its lanes take the tile's roots in turn (lane l roots l,
// l + 32, ...).  Each hop of a chase is one dependent load, so every lane
// keeps kInFlight chases going at once, and a lane whose chase ends starts
// its next root in that place: one long chain holds up no other chase.
// kFlat: the 2D tiles (which follow the 3D ones).

template <bool kFlat, bool kSingle, class S>
__global__ void __launch_bounds__(kChaseThreads) k_chase_tiles(Batch bt, TiledScratch ts,
                                                               const int2 *__restrict__ graph,
                                                               long long probe_stride,
                                                               DevStatus *st) {
  if (call_failed(st)) return;
  extern __shared__ uint32_t LUT[];
  constexpr int kE = kFlat ? k2Ext : S::Ext;
  constexpr int TX = kFlat ? k2TX : S::TX, TY = kFlat ? k2TY : S::TY, TZ = kFlat ? 1 : S::TZ;
  constexpr int kFaceN = kFlat ? k2Face : S::Face;
  const long long fstride = bt.face_stride;
  for (int e = threadIdx.x; e < kE; e += kChaseThreads) LUT[e] = chase_code<kFlat, S>(e);
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const bool probe = probe_stride > 0;
  const long long t0 = kFlat ? bt.tiles3 : 0;
  const long long ntiles = kFlat ? bt.total_tiles - bt.tiles3 : bt.tiles3;
  const long long nwork = probe ? (ntiles + probe_stride - 1) / probe_stride : ntiles;
  unsigned int *ctr = ts.queue + (kFlat ? kQChase2 : kQChase);
  unsigned int sampled = 0, pending = 0, bad = 0;
  for (;;) {
    long long k = 0;
    if (lane == 0) k = (long long)atomicAdd(ctr, 1u);
    k = __shfl_sync(0xffffffffu, k, 0);
    if (k >= nwork) break;
    const int64_t gt = t0 + (probe ? k * probe_stride : k);
    const TileMeta m = ts.meta[gt];
    const int fi = kSingle ? 0 : field_of(bt, gt);
    const FieldDesc &fd = kSingle ? bt.f0 : bt.fields[fi];
    const TileGeom &g = fd.g;
    const uint32_t *__restrict__ face = ts.face + fd.tile_base * fstride;
    const int gtx = (int)g.tx, gty = (int)g.ty, gtz = (int)g.tz;
    const uint32_t nx = (uint32_t)g.nx, ny = (uint32_t)g.ny;
    int tx0, ty0, tz0 = 0;
    {
      const int64_t tile = gt - fd.tile_base;
      uint32_t r, tx, ty, tz = 0;
      if (kFlat) {
        g.div_tx.divmod((uint32_t)tile, &ty, &tx);
      } else {
        g.div_tx.divmod((uint32_t)tile, &r, &tx);
        g.div_ty.divmod(r, &tz, &ty);
      }
      tx0 = (int)tx, ty0 = (int)ty, tz0 = (int)tz;
    }
    const int nr = m.nd + m.nu;
    const int64_t n = g.nx * g.ny * g.nz;
    const int64_t slots = g.ntiles * (int64_t)kFaceN;
    const int max_hops = probe ? kProbeHops : (int)(n < slots ? n : slots);
    const uint16_t *__restrict__ rb = ts.root_box + m.rbase;
    int32_t *__restrict__ rl = ts.root_label + m.rbase;
    uint32_t e[kInFlight];
    int tx[kInFlight], ty[kInFlight], tz[kInFlight], idx[kInFlight], hops[kInFlight];
    int next = lane + 32 * kInFlight;  // this lane's next root to start
    uint32_t nb = next < nr ? ((uint32_t)rb[next] & (uint32_t)(kUpRoot - 1)) : 0u;  // its box index, loaded ahead
#pragma unroll
    for (int q = 0; q < kInFlight; ++q) {
      idx[q] = lane + 32 * q;
      hops[q] = 0;
      tx[q] = tx0, ty[q] = ty0, tz[q] = tz0;
      e[q] = idx[q] < nr ? ((uint32_t)rb[idx[q]] & (uint32_t)(kUpRoot - 1)) : 0u;
    }
    for (;;) {
      bool any = false;
#pragma unroll
      for (int q = 0; q < kInFlight; ++q) {
        if (idx[q] >= nr) continue;
        any = true;
        const bool up = idx[q] >= m.nd;
        const uint32_t code = LUT[e[q]];
        int32_t label = 0;
        bool done = false;
        if (!(code & kHaloBit)) {  // inside its tile: the extremum
          const uint32_t lx = code & 127u, ly = (code >> 7) & 63u, lz = (code >> 13) & 31u;
          label = (int32_t)((uint32_t)(tx[q] * TX) + lx +
                            nx * ((uint32_t)(ty[q] * TY) + ly + ny * ((uint32_t)(tz[q] * TZ) + lz)));
          done = true;
        } else {
          const int ntx = tx[q] + (int)((code >> 12) & 3u) - 1;
          const int nty = ty[q] + (int)((code >> 14) & 3u) - 1;
          const int ntz = tz[q] + (int)((code >> 16) & 3u) - 1;
          if ((unsigned)ntx >= (unsigned)gtx || (unsigned)nty >= (unsigned)gty ||
              (unsigned)ntz >= (unsigned)gtz) {  // cannot happen: every root lies in the field
            ++bad;
            done = true;
          } else {
            const long long slot =
                ((long long)ntx + (long long)gtx * (nty + (long long)gty * ntz)) * fstride +
                (code & 0xfffu);
            if (graph) {  // the jumped face graph knows where the path ends
              const int2 gv = graph[fd.tile_base * fstride + slot];
              const uint32_t f = (uint32_t)(up ? gv.x : gv.y);
              if (!(f & kSlotFinal)) atomicOr(&st->not_converged, 1u);
              label = (int32_t)(f & ~kSlotFinal);
              done = true;
            } else if (++hops[q] > max_hops) {
              if (probe)
                ++pending;
              else
                atomicOr(&st->not_converged, 1u);
              done = true;
            } else {
              const uint32_t wv = __ldg(&face[slot]);
              e[q] = up ? (wv & 0xffffu) : (wv >> 16);
              tx[q] = ntx, ty[q] = nty, tz[q] = ntz;
            }
          }
        }
        if (done) {
          if (probe)
            ++sampled;
          else
            rl[idx[q]] = label;
          idx[q] = next;
          e[q] = nb;
          next += 32;
          nb = next < nr ? ((uint32_t)rb[next] & (uint32_t)(kUpRoot - 1)) : 0u;
          hops[q] = 0;
          tx[q] = tx0, ty[q] = ty0, tz[q] = tz0;
        }
      }
      if (!__any_sync(0xffffffffu, any)) break;
    }
  }
  if (bad) atomicOr(&st->bad_index, 1u);
  if (probe) {
    if (sampled) atomicAdd(&st->sampled, sampled);
    if (pending) atomicAdd(&st->pending, pending);
  }
}

// First-fit insert into the global pair set; returns the key's slot (and
// *fresh when this call placed it), or 0xffffffff when the probe limit ran
// out (the set is too small: the host retries with a larger one).
__device__ __forceinline__ uint32_t global_insert(const RankScratch &rs, unsigned long long key,
                                                  bool *fresh) {
  const unsigned int mask = rs.capacity - 1u;
  unsigned int slot = (unsigned int)hash_mix64(key) & mask;
  for (unsigned int probe = 0; probe < rs.probe_limit; ++probe) {
    unsigned long long cur = __ldcg(&rs.table_keys[slot]);
    if (cur == ~0ull) {
      cur = atomicCAS(&rs.table_keys[slot], ~0ull, key);
      if (cur == ~0ull) {
        *fresh = true;
        return slot;
      }
    }
    if (cur == key) return slot;
    slot = (slot + 1u) & mask;
  }
  return 0xffffffffu;
}

// New keys join the sorted-list input with one counter update per warp.
__device__ __forceinline__ void list_append(const RankScratch &rs, unsigned long long key, bool fresh,
                                            uint32_t slot, DevStatus *st) {
  const unsigned int am = __activemask();
  const unsigned int nm = __ballot_sync(am, fresh);
  if (nm) {
    const int lane = threadIdx.x & 31, leader = __ffs(nm) - 1;
    unsigned int base = 0;
    if (lane == leader) base = atomicAdd(&st->n_unique, (unsigned int)__popc(nm));
    base = __shfl_sync(am, base, leader);
    if (fresh) {
      const unsigned int at = base + __popc(nm & ((1u << lane) - 1u));
      if (at < rs.max_unique)
        rs.list[at] = key;
      else
        atomicOr(&st->hash_overflow, 1u);
    }
  }
  if (slot == 0xffffffffu) atomicOr(&st->hash_overflow, 1u);
}

// list_append for a converged warp: the lanes with inserted set true are
// the ones that inserted (fresh: placed a new key); a failed insert (slot
// 0xffffffff) flags the set as too small.
__device__ __forceinline__ void list_append_warp(const RankScratch &rs, unsigned long long key, bool fresh,
                                                 bool inserted, uint32_t slot, DevStatus *st) {
  const unsigned int nm = __ballot_sync(0xffffffffu, fresh);
  const int lane = threadIdx.x & 31;
  if (nm) {
    const int leader = __ffs(nm) - 1;
    unsigned int base = 0;
    if (lane == leader) base = atomicAdd(&st->n_unique, (unsigned int)__popc(nm));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (fresh) {
      const unsigned int at = base + __popc(nm & ((1u << lane) - 1u));
      if (at < rs.max_unique)
        rs.list[at] = key;
      else
        atomicOr(&st->hash_overflow, 1u);
    }
  }
  if (inserted && slot == 0xffffffffu) atomicOr(&st->hash_overflow, 1u);
}

// Tile pairs, flat over the pair pool (see launch_tile_pairs; calls with few
// tiles): every tile
// pair's (asc, desc) from its two roots' labels into the global set.  A lane
// handles kPairBatch pairs at once (their loads overlap); lanes of a warp
// holding the same pair -- mostly the same tile's pairs reaching the same
// extrema -- insert it once (__match_any_sync), and every lane stores the
// slot.  An overflowing set stops the pass early (the host retries larger).
constexpr int kPairThreads = 256;
constexpr int kPairBatch = 8;

__device__ __forceinline__ unsigned long long final_key(int key_mode, uint32_t fi, int32_t a, int32_t d) {
  return key_mode == kKeyBatch
             ? (((unsigned long long)fi << 48) | ((unsigned long long)(uint32_t)a << 24) | (uint32_t)d)
             : (((unsigned long long)(uint32_t)a << 32) | (uint32_t)d);
}

template <bool kSingle>
__global__ void __launch_bounds__(kPairThreads) k_pairs_flat(Batch bt, TiledScratch ts, RankScratch rs,
                                                             DevStatus *st) {
  if (call_failed(st) || st->not_converged) return;
  const int lane = threadIdx.x & 31;
  const bool keep_ad = rs.capacity > kSetInL2;
  const unsigned long long npairs = min(ts.counters[0], ts.pool_cap);
  const unsigned long long nroots = min(ts.counters[1], ts.root_cap);
  const unsigned long long step = (unsigned long long)gridDim.x * kPairThreads * kPairBatch;
  unsigned int it = 0;
  // the loop bound is the warp's first pair, so the whole warp iterates together
  for (unsigned long long wb = (unsigned long long)blockIdx.x * kPairThreads * kPairBatch +
                               (threadIdx.x & ~31u) * kPairBatch;
       wb < npairs; wb += step) {
    const unsigned long long p0 = wb + lane;
    // a set found too small ends the pass; the flag is one word every warp
    // would read, so it is read on every 8th iteration only
    if ((it++ & 7u) == 0 && __shfl_sync(0xffffffffu, __ldcg(&st->hash_overflow), 0)) break;
    uint2 pp[kPairBatch];
#pragma unroll
    for (int u = 0; u < kPairBatch; ++u)
      pp[u] = p0 + 32 * u < npairs ? __ldcs(&ts.pool_pair[p0 + 32 * u]) : make_uint2(0u, 0u);
    int32_t a[kPairBatch], d[kPairBatch];
#pragma unroll
    for (int u = 0; u < kPairBatch; ++u) {
      const bool ok = p0 + 32 * u < npairs && pp[u].x < nroots && pp[u].y < nroots;
      if (p0 + 32 * u < npairs && !ok) atomicOr(&st->bad_index, 1u);  // cannot happen
      a[u] = ok ? __ldg(&ts.root_label[pp[u].x]) : 0;
      d[u] = ok ? __ldg(&ts.root_label[pp[u].y]) : 0;
    }
#pragma unroll
    for (int u = 0; u < kPairBatch; ++u) {
      const unsigned long long p = p0 + 32 * u;
      const bool valid = p < npairs;
      const uint32_t fi = (kSingle || !valid) ? 0u : (uint32_t)field_of(bt, ts.root_tile[pp[u].x]);
      const unsigned long long key = valid ? final_key(bt.key_mode, fi, a[u], d[u]) : ~0ull;
      const unsigned int peers = __match_any_sync(0xffffffffu, key);
      const int leader = __ffs(peers) - 1;
      bool fresh = false;
      uint32_t gs = 0;
      if (valid && lane == leader) gs = global_insert(rs, key, &fresh);
      list_append_warp(rs, key, fresh, valid && lane == leader, gs, st);
      gs = __shfl_sync(0xffffffffu, gs, leader);
      if (valid) {
        ts.pool_slot[p] = gs;
        if (keep_ad) ts.pool_ad[p] = make_int2(a[u], d[u]);
      }
    }
  }
}

// Tile pairs, a tile a warp (see launch_tile_pairs; calls with many tiles),
// taken from a work queue: each tile pair's (asc, desc) from its two roots' labels; the tile's
// distinct pairs -- a few dozen where the tile has about a thousand root
// pairs -- are found in the warp's shared-memory set and only they are
// inserted into the global set.  Lanes work on kPairBatch pairs at once, so
// their loads overlap.  A tile with more distinct pairs than the warp's set
// holds inserts the rest directly.
constexpr int kWarpHash = 256;
constexpr int kWarpProbes = 8;
constexpr int kWarpFill = kWarpHash * 3 / 4;  // entries past which the set takes no new keys

__device__ __forceinline__ uint32_t warp_slot_of(unsigned long long key) {
  uint32_t h = ((uint32_t)key * 0x9E3779B1u) ^ ((uint32_t)(key >> 32) * 0x85EBCA77u);
  h ^= h >> 15;
  return h & (kWarpHash - 1);
}

template <bool kSingle>
__global__ void __launch_bounds__(kPairThreads) k_pairs_tiles(Batch bt, TiledScratch ts, RankScratch rs,
                                                             DevStatus *st) {
  if (call_failed(st) || st->not_converged) return;
  __shared__ unsigned long long HKs[kPairThreads / 32][kWarpHash];
  __shared__ uint32_t HSs[kPairThreads / 32][kWarpHash];
  __shared__ int s_fill[kPairThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long *HK = HKs[wid];
  uint32_t *HS = HSs[wid];
  const bool keep_ad = rs.capacity > kSetInL2;
  for (;;) {
    long long k = 0;
    if (lane == 0) k = (long long)atomicAdd(ts.queue + kQPairs, 1u);
    k = __shfl_sync(0xffffffffu, k, 0);
    if (k >= bt.total_tiles) break;
    // a set found too small ends the pass (the host retries larger)
    if (__shfl_sync(0xffffffffu, lane == 0 ? __ldcg(&st->hash_overflow) : 0u, 0)) break;
    const int64_t gt = k;
    const TileMeta m = ts.meta[gt];
    const uint32_t fi = kSingle ? 0u : (uint32_t)field_of(bt, gt);
    const uint32_t nr = (uint32_t)(m.nd + m.nu);
    const int np = m.npairs;
    const uint2 *__restrict__ pp_src = ts.pool_pair + m.pbase;
    for (int i = lane; i < kWarpHash; i += 32) HK[i] = ~0ull;
    if (lane == 0) s_fill[wid] = 0;
    __syncwarp();
    auto label_of = [&](uint32_t r) -> int32_t {
      if (r < m.rbase || r >= m.rbase + nr) {  // cannot happen for a pair the tile pass listed
        atomicOr(&st->bad_index, 1u);
        return 0;
      }
      return __ldg(&ts.root_label[r]);  // written by the previous launch
    };
    // pass 1: every pair into the warp's set (or, past it, the global set)
    for (int i0 = lane; i0 < np; i0 += 32 * kPairBatch) {
      uint2 pp[kPairBatch];
      int32_t a[kPairBatch], d[kPairBatch];
#pragma unroll
      for (int u = 0; u < kPairBatch; ++u) pp[u] = i0 + 32 * u < np ? __ldg(&pp_src[i0 + 32 * u]) : make_uint2(0u, 0u);
#pragma unroll
      for (int u = 0; u < kPairBatch; ++u) {
        a[u] = i0 + 32 * u < np ? label_of(pp[u].x) : 0;
        d[u] = i0 + 32 * u < np ? label_of(pp[u].y) : 0;
      }
#pragma unroll
      for (int u = 0; u < kPairBatch; ++u) {
        const int i = i0 + 32 * u;
        if (i >= np) continue;
        const unsigned long long key = final_key(bt.key_mode, fi, a[u], d[u]);
        uint32_t sl = warp_slot_of(key);
        bool placed = false;
        for (int probe = 0; probe < kWarpProbes; ++probe) {
          unsigned long long cur = HK[sl];
          if (cur == key) {
            placed = true;
            break;
          }
          if (cur == ~0ull) {
            // a full set takes no new keys: its probe chains stay short
            if (*(volatile int *)&s_fill[wid] >= kWarpFill) break;
            cur = atomicCAS(&HK[sl], ~0ull, key);
            if (cur == ~0ull) atomicAdd(&s_fill[wid], 1);
            if (cur == ~0ull || cur == key) {
              placed = true;
              break;
            }
          }
          sl = (sl + 1) & (kWarpHash - 1);
        }
        if (!placed) {  // the warp's set is full: straight into the global set
          bool fresh = false;
          const uint32_t gs = global_insert(rs, key, &fresh);
          list_append(rs, key, fresh, gs, st);
          ts.pool_slot[m.pbase + i] = gs;
          if (keep_ad) ts.pool_ad[m.pbase + i] = make_int2(a[u], d[u]);
        }
      }
    }
    __syncwarp();
    // the tile's distinct pairs into the global set
    for (int sl = lane; sl < kWarpHash; sl += 32) {
      const unsigned long long key = HK[sl];
      if (key != ~0ull) {
        bool fresh = false;
        const uint32_t gs = global_insert(rs, key, &fresh);
        list_append(rs, key, fresh, gs, st);
        HS[sl] = gs;
      }
    }
    __syncwarp();
    // pass 2: every pair's set slot
    for (int i0 = lane; i0 < np; i0 += 32 * kPairBatch) {
      uint2 pp[kPairBatch];
      int32_t a[kPairBatch], d[kPairBatch];
#pragma unroll
      for (int u = 0; u < kPairBatch; ++u) pp[u] = i0 + 32 * u < np ? __ldg(&pp_src[i0 + 32 * u]) : make_uint2(0u, 0u);
#pragma unroll
      for (int u = 0; u < kPairBatch; ++u) {
        a[u] = i0 + 32 * u < np ? label_of(pp[u].x) : 0;
        d[u] = i0 + 32 * u < np ? label_of(pp[u].y) : 0;
      }
#pragma unroll
      for (int u = 0; u < kPairBatch; ++u) {
        const int i = i0 + 32 * u;
        if (i >= np) continue;
        const unsigned long long key = final_key(bt.key_mode, fi, a[u], d[u]);
        uint32_t sl = warp_slot_of(key);
        for (int probe = 0; probe < kWarpProbes; ++probe) {
          const unsigned long long cur = HK[sl];
          if (cur == key) {
            ts.pool_slot[m.pbase + i] = HS[sl];
            if (keep_ad) ts.pool_ad[m.pbase + i] = make_int2(a[u], d[u]);
            break;
          }
          if (cur == ~0ull) break;  // inserted straight into the global set in pass 1
          sl = (sl + 1) & (kWarpHash - 1);
        }
      }
    }
    __syncwarp();  // the warp's set is reused by its next tile
  }
}

// Many-field batches: the first sorted pair of each field (its ids start there).
__global__ void k_field_starts(const unsigned long long *__restrict__ sorted, unsigned int m,
                               const unsigned int *m_dev, uint32_t *__restrict__ fstart) {
  if (m_dev) m = min(*m_dev, m);
  const unsigned int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const unsigned int f = (unsigned int)(sorted[i] >> 48);
  if (i == 0 || (unsigned int)(sorted[i - 1] >> 48) != f) fstart[f] = i;
}

// Per tile: stage the pair table -- each tile pair's (asc, desc) and MS id,
// read from the global pair set at the pair's slot -- and stream the labels
// out.  Each thread writes the run of kRun vertices it owned in the tile
// kernel (3D: the z-column (x0 + t % TX, y0 + t / TX, .); 2D: the y-run at
// x0 + lane + 32 (warp % 4)); its 16 pair numbers are one 32-byte vector.
// kFlat selects the 2D tiles, which follow the 3D ones (S: the 3D shape).
template <bool kFlat, bool kSingle, bool kInPool, class S>
__global__ void __launch_bounds__(kFlat ? k2Threads : S::Threads)
    k_tile_write(Batch bt, TiledScratch ts, RankScratch rs, const DevStatus *st) {
  constexpr int kThreads = kFlat ? k2Threads : S::Threads;
  // A replayed graph runs this kernel even when an earlier stage found its
  // buffers too small; the tile ranges and set slots are then not valid to
  // read, and the host runs the call again step by step.
  if (st->pool_overflow | st->hash_overflow | st->not_converged | st->bad_index | st->timeout |
      st->nan_flag)
    return;
  __shared__ int4 T[kStageCap];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t base = kFlat ? bt.tiles3 : 0;
  const long long count = kFlat ? bt.total_tiles - bt.tiles3 : bt.tiles3;
  unsigned int *ctr = ts.queue + (kFlat ? kQWrite2 : kQWrite3);
  __shared__ long long s_next;
  const bool dyn = bt.tune.dynamic != 0;
  for (long long k = queue_first(dyn, ctr, &s_next); k < count; k = queue_next(dyn, k, &s_next)) {
    queue_prefetch(dyn, ctr, &s_next);
    const int64_t gt = base + k;
    const int fi = kSingle ? 0 : field_of(bt, gt);
    const FieldDesc &fd = kSingle ? bt.f0 : bt.fields[fi];
    const TileGeom &g = fd.g;
    int64_t v0, stride;  // the run's first vertex and its step
    int n_here;
    bool col_in;
    if (kFlat) {
      int64_t x0, y0;
      tile_origin2(g, gt - fd.tile_base, &x0, &y0);
      const int64_t x = x0 + lane + 32 * (warp & 3), y = y0 + kRun * (warp >> 2);
      col_in = x < g.nx && y < g.ny;
      n_here = (int)std::min<int64_t>(kRun, g.ny - y);
      v0 = x + g.nx * y;
      stride = g.nx;
    } else {
      int64_t x0, y0, z0;
      tile_origin<S>(g, gt - fd.tile_base, &x0, &y0, &z0);
      const int64_t x = x0 + threadIdx.x % S::TX, y = y0 + threadIdx.x / S::TX;
      col_in = x < g.nx && y < g.ny;
      n_here = (int)std::min<int64_t>(S::TZ, g.nz - z0);
      stride = g.nx * g.ny;
      v0 = x + g.nx * y + stride * z0;
    }
    const TileMeta &m = ts.meta[gt];
    const unsigned long long b = m.pbase;
    const int cnt = m.npairs;
    const uint32_t *src = ts.pool_slot + b;
    const int2 *res = ts.pool_ad + b;  // resolved (asc, desc) of each tile pair
    const bool staged = cnt <= kStageCap;
    const bool batch = bt.key_mode == kKeyBatch;
    const int first = batch ? (int)ts.fstart[fi] : 0;
    uint4 q0 = make_uint4(0, 0, 0, 0), q1 = q0;
    if (col_in) {
      const uint4 *pid4 = reinterpret_cast<const uint4 *>(ts.pid + gt * (int64_t)kPidStride +
                                                          (int64_t)threadIdx.x * kRun);
      q0 = __ldcs(pid4);
      q1 = __ldcs(pid4 + 1);
    }
    // kInPool (a set of more than kSetInL2 entries): k_tile_pairs left each
    // resolved pair in its pool entry
    auto entry = [&](int i) {
      const uint32_t sl = __ldcs(src + i);
      if (kInPool) {
        const int2 ad = __ldcs(res + i);
        return make_int4(ad.x, ad.y, __ldg(&rs.table_vals[sl]) - first, 0);
      }
      const unsigned long long key = __ldg(&rs.table_keys[sl]);
      const int r = __ldg(&rs.table_vals[sl]) - first;
      return batch ? make_int4((int)((key >> 24) & 0xffffffull), (int)(key & 0xffffffull), r, 0)
                   : make_int4((int)(key >> 32), (int)(uint32_t)key, r, 0);
    };
    if (staged)
      for (int i = threadIdx.x; i < cnt; i += kThreads) T[i] = entry(i);
    __syncthreads();
    if (col_in) {
      int32_t *__restrict__ asc = fd.asc, *__restrict__ desc = fd.desc, *__restrict__ ms = fd.ms;
      const uint32_t w[8] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w};
#pragma unroll
      for (int j = 0; j < kRun; ++j) {
        if (j >= n_here) break;
        int id = (int)((w[j / 2] >> (16 * (j & 1))) & 0xffffu);
        if (id >= cnt) id = 0;  // cannot happen: every vertex's number is one of its tile's pairs
        const int4 t = staged ? T[id] : entry(id);
        const int64_t v = v0 + stride * j;
        __stcs(asc + v, t.x);
        __stcs(desc + v, t.y);
        __stcs(ms + v, t.z);
      }
    }
    __syncthreads();
  }
}

}  // namespace

bool tile_mode(const Batch &b) {
  return b.tune.resolve_mode == 0 || (b.tune.resolve_mode < 0 && b.total_tiles >= kTileModeMin);
}

namespace {

int sms() {
  int dev = 0, n = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n;
}

}  // namespace

TileGeom tile_geom(const int64_t dims[3], int shape3) {
  TileGeom g;
  g.nx = dims[0];
  g.ny = dims[1];
  g.nz = dims[2];
  g.flat = g.nz == 1 ? 1 : 0;
  const ShapeInfo si = shape_info(shape3);
  const int64_t tx = g.flat ? k2TX : si.tx, ty = g.flat ? k2TY : si.ty;
  g.tx = (g.nx + tx - 1) / tx;
  g.ty = (g.ny + ty - 1) / ty;
  g.tz = g.flat ? 1 : (g.nz + si.tz - 1) / si.tz;
  g.ntiles = g.tx * g.ty * g.tz;
  g.div_nx = FastDivU32((uint32_t)g.nx);
  g.div_ny = FastDivU32((uint32_t)g.ny);
  g.div_tx = FastDivU32((uint32_t)g.tx);
  g.div_ty = FastDivU32((uint32_t)g.ty);
  return g;
}

size_t tiled_scratch_bytes(long long total_tiles, int n_fields, unsigned long long pool_cap,
                           unsigned long long root_cap, int face_stride) {
  auto r = [](size_t b) { return (b + 255) & ~(size_t)255; };
  return r(256) + r((size_t)pool_cap * 8) + r((size_t)pool_cap * 4) + r((size_t)pool_cap * 8) +
         r((size_t)root_cap * 2) +
         r((size_t)root_cap * 4) +
         r((size_t)root_cap * 4) + r((size_t)total_tiles * sizeof(TileMeta)) + r((size_t)n_fields * 4) +
         r((size_t)total_tiles * face_stride * 4) + r((size_t)total_tiles * kPidStride * 2);
}

void tiled_scratch_carve(void *base, long long total_tiles, int n_fields,
                         unsigned long long pool_cap, unsigned long long root_cap, int face_stride,
                         TiledScratch *ts) {
  char *p = static_cast<char *>(base);
  auto take = [&](size_t bytes) {
    char *q = p;
    p += (bytes + 255) & ~(size_t)255;
    return q;
  };
  ts->counters = reinterpret_cast<unsigned long long *>(take(256));
  ts->queue = reinterpret_cast<unsigned int *>(ts->counters + 3);
  ts->pool_pair = reinterpret_cast<uint2 *>(take((size_t)pool_cap * 8));
  ts->pool_slot = reinterpret_cast<uint32_t *>(take((size_t)pool_cap * 4));
  ts->pool_ad = reinterpret_cast<int2 *>(take((size_t)pool_cap * 8));
  ts->root_box = reinterpret_cast<uint16_t *>(take((size_t)root_cap * 2));
  ts->root_tile = reinterpret_cast<uint32_t *>(take((size_t)root_cap * 4));
  ts->root_label = reinterpret_cast<int32_t *>(take((size_t)root_cap * 4));
  ts->meta = reinterpret_cast<TileMeta *>(take((size_t)total_tiles * sizeof(TileMeta)));
  ts->fstart = reinterpret_cast<uint32_t *>(take((size_t)n_fields * 4));
  ts->face = reinterpret_cast<uint32_t *>(take((size_t)total_tiles * face_stride * 4));
  ts->pid = reinterpret_cast<uint16_t *>(take((size_t)total_tiles * kPidStride * 2));
  ts->pool_cap = pool_cap;
  ts->root_cap = root_cap;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_tiled_fn() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {  // initialised once, thread-safe
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    const bool ok = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000,
                                                     cudaEnableDefault, &q) == cudaSuccess &&
                    q == cudaDriverEntryPointSuccess;
    cudaGetLastError();
    return ok ? reinterpret_cast<EncodeTiledFn>(p) : nullptr;
  }();
  return fn;
}

// A 3D (2D for flat fields) tensor map over a float32 field for the box
// load; false when the
// field's layout does not meet TMA's rules (16-byte aligned base and row /
// plane strides) or the driver entry point is missing.
bool make_box_map(const void *field, int dtype, const TileGeom &g, int shape3, CUtensorMap *map) {
  // float32 boxes start 4 values left of the tile, float16 boxes 8 (both 16 bytes)
  if (dtype != MS_F32 && dtype != MS_F16) return false;
  const cuuint64_t esz = dtype == MS_F16 ? 2 : 4;
  const int xo = dtype == MS_F16 ? 8 : kXO;
  const CUtensorMapDataType type =
      dtype == MS_F16 ? CU_TENSOR_MAP_DATA_TYPE_UINT16 : CU_TENSOR_MAP_DATA_TYPE_UINT32;
  if ((reinterpret_cast<uintptr_t>(field) & 15) != 0) return false;
  if ((g.nx * esz) % 16 != 0) return false;
  if (g.nx > (1ll << 31) || g.ny > (1ll << 31) || g.nz > (1ll << 31)) return false;
  EncodeTiledFn fn = encode_tiled_fn();
  if (!fn) return false;
  if (g.flat) {
    const cuuint64_t dims2[2] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny};
    const cuuint64_t strides2[1] = {(cuuint64_t)g.nx * esz};
    const cuuint32_t box2[2] = {(cuuint32_t)(k2TX + 2 * xo), k2EY};
    const cuuint32_t estr2[2] = {1, 1};
    return fn(map, type, 2, const_cast<void *>(field), dims2, strides2, box2, estr2,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
              CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, (cuuint64_t)g.nz};
  const cuuint64_t strides[2] = {(cuuint64_t)g.nx * esz, (cuuint64_t)(g.nx * g.ny) * esz};
  const ShapeInfo si = shape_info(shape3);
  const cuuint32_t box[3] = {(cuuint32_t)(si.tx + 2 * xo), (cuuint32_t)(si.ty + 2),
                             (cuuint32_t)(si.tz + 2)};
  const cuuint32_t estr[3] = {1, 1, 1};
  return fn(map, type, 3, const_cast<void *>(field), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

void make_field_desc(const void *field, int dtype, const int64_t dims[3], long long tile_base,
                     int32_t *asc, int32_t *desc, int32_t *ms, bool allow_tma, int shape3,
                     FieldDesc *fd, CUtensorMap *map) {
  fd->field = field;
  fd->asc = asc;
  fd->desc = desc;
  fd->ms = ms;
  fd->g = tile_geom(dims, shape3);
  fd->tile_base = tile_base;
  fd->dtype = dtype;
  memset(map, 0, sizeof(*map));
  fd->tma = (allow_tma && make_box_map(field, dtype, fd->g, shape3, map)) ? 1 : 0;
}

// Calls f with a value of the 3D shape type of id (the kernels' template
// argument).
template <class F>
cudaError_t with_shape(int id, F &&f) {
  switch (id) {
    case kShape64x8: return f(Shape64x8{});
    case kShape16x32: return f(Shape16x32{});
    case kShape16x16: return f(Shape16x16{});
    default: return f(Shape32x16{});
  }
}

namespace {
bool capturing(cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  return cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone;
}
}  // namespace

cudaError_t launch_tile_local(const Batch &b, const TiledScratch &ts, DevStatus *st,
                              cudaStream_t s) {
  // the pool and root counters and the work-queue counters after them
  cudaError_t e = cudaMemsetAsync(ts.counters, 0, 3 * sizeof(unsigned long long) + kQueues * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  if (b.tiles3 > 0) {
    e = with_shape(b.shape3, [&](auto shape) -> cudaError_t {
      using S = decltype(shape);
      constexpr int kSmem = 2 * S::Ext * 4;
      auto kern = b.n_fields == 1 ? k_tile_local<true, S> : k_tile_local<false, S>;
      if (!capturing(s)) {  // set by the step-by-step call that precedes every capture
        const cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem);
        if (r != cudaSuccess) return r;
      }
      // 512-thread shapes fit 2 CTAs an SM, 256-thread ones twice as many
      const int64_t per_sm = (int64_t)b.tune.tile_ctas * (512 / S::Threads);
      const int64_t grid = std::min<int64_t>(b.tiles3, (int64_t)sms() * per_sm);
      ++tl_launches;
      kern<<<(unsigned)grid, S::Threads, kSmem, s>>>(b, ts, st);
      return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
    // the 3D tiles' roots come first in the root list
    e = cudaMemcpyAsync(ts.counters + 2, ts.counters + 1, sizeof(unsigned long long),
                        cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
  }
  if (b.total_tiles > b.tiles3) {
    constexpr int kSmem2 = (k2KArea + k2PArea) * 4;
    auto kern = b.n_fields == 1 ? k_tile_local2<true> : k_tile_local2<false>;
    if (!capturing(s)) {
      e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmem2);
      if (e != cudaSuccess) return e;
    }
    const int64_t grid = std::min<int64_t>(b.total_tiles - b.tiles3, (int64_t)sms() * b.tune.tile_ctas);
    ++tl_launches;
    kern<<<(unsigned)grid, k2Threads, kSmem2, s>>>(b, ts, st);
    e = cudaGetLastError();
  }
  return e;
}

cudaError_t launch_chase_roots(const Batch &b, const TiledScratch &ts, const int2 *graph,
                               long long probe_stride, DevStatus *st, cudaStream_t s,
                               unsigned long long roots) {
  const bool tiles = tile_mode(b);
  cudaError_t e = cudaSuccess;
  if (tiles) e = cudaMemsetAsync(ts.queue + kQChase, 0, 2 * sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  for (int flat = 0; flat < 2; ++flat) {
    const long long n = flat ? b.total_tiles - b.tiles3 : b.tiles3;
    if (n == 0) continue;
    const size_t smem = (size_t)(flat ? k2Ext : shape_info(b.shape3).ext) * 4;
    // the probe samples every probe_stride-th root (flat) or tile (a tile a
    // warp): either way about kProbeRoots roots, as a tile holds about
    // nroots / tiles of them
    const long long stride = probe_stride;
    const long long work = tiles ? (stride > 0 ? (n + stride - 1) / stride : n) : 0;
    ++tl_launches;
    auto go = [&](auto kern) -> cudaError_t {
      if (!capturing(s)) {
        const cudaError_t r = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (r != cudaSuccess) return r;
      }
      // a tile a warp: up to chase_blocks blocks an SM, no more warps than
      // tiles; flat: every thread strides over the roots, so exactly the
      // blocks that are resident at once
      long long blocks;
      if (tiles) {
        blocks = std::max<long long>(1, std::min<long long>((long long)sms() * b.tune.chase_blocks,
                                                            (work + kChaseThreads / 32 - 1) / (kChaseThreads / 32)));
      } else {
        int per_sm = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kChaseThreads, smem) != cudaSuccess ||
            per_sm < 1)
          per_sm = 1;
        cudaGetLastError();
        blocks = (long long)sms() * std::min(per_sm, b.tune.chase_blocks);
        // no more blocks than the roots keep busy (kInFlight chases a thread):
        // small calls would otherwise spend their time building decode tables
        const unsigned long long bound = roots ? std::min(roots, ts.root_cap) : ts.root_cap;
        const unsigned long long items = stride > 0 ? bound / (unsigned long long)stride + 1 : bound;
        const unsigned long long per_block = (unsigned long long)kChaseThreads * kInFlight;
        blocks = std::max<long long>(
            1, std::min<long long>(blocks, (long long)((items + per_block - 1) / per_block)));
      }
      kern<<<(unsigned)blocks, kChaseThreads, smem, s>>>(b, ts, graph, stride, st);
      return cudaGetLastError();
    };
    const bool one = b.n_fields == 1;
    if (flat) {  // the 2D tiles' kernels do not depend on the 3D shape
      using S = Shape32x16;
      if (tiles)
        e = one ? go(k_chase_tiles<true, true, S>) : go(k_chase_tiles<true, false, S>);
      else
        e = one ? go(k_chase_flat<true, true, S>) : go(k_chase_flat<true, false, S>);
    } else {
      e = with_shape(b.shape3, [&](auto shape) -> cudaError_t {
        using S = decltype(shape);
        if (tiles)
          return one ? go(k_chase_tiles<false, true, S>) : go(k_chase_tiles<false, false, S>);
        return one ? go(k_chase_flat<false, true, S>) : go(k_chase_flat<false, false, S>);
      });
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_tile_pairs(const Batch &b, const TiledScratch &ts, const RankScratch &rs,
                              bool clear_table, DevStatus *st, cudaStream_t s,
                              unsigned long long pairs) {
  cudaError_t e = cudaSuccess;
  if (clear_table) e = cudaMemsetAsync(rs.table_keys, 0xff, (size_t)rs.capacity * 8, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ts.queue + kQPairs, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess || b.total_tiles == 0) return e;
  ++tl_launches;
  if (tile_mode(b)) {
    constexpr int kWarps = kPairThreads / 32;
    const long long blocks = std::min<long long>((b.total_tiles + kWarps - 1) / kWarps,
                                                 (long long)sms() * b.tune.pair_blocks);
    if (b.n_fields == 1)
      k_pairs_tiles<true><<<(unsigned)blocks, kPairThreads, 0, s>>>(b, ts, rs, st);
    else
      k_pairs_tiles<false><<<(unsigned)blocks, kPairThreads, 0, s>>>(b, ts, rs, st);
  } else {
    // every thread strides over the pool: the blocks resident at once
    auto kern = b.n_fields == 1 ? k_pairs_flat<true> : k_pairs_flat<false>;
    int per_sm = 1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kPairThreads, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    cudaGetLastError();
    const unsigned long long per_block = (unsigned long long)kPairThreads * kPairBatch;
    const long long blocks = (long long)std::max<unsigned long long>(
        1, std::min<unsigned long long>(((pairs ? std::min(pairs, ts.pool_cap) : ts.pool_cap) +
                                         per_block - 1) / per_block,
                                        (unsigned long long)sms() * std::min(per_sm, b.tune.pair_blocks)));
    kern<<<(unsigned)blocks, kPairThreads, 0, s>>>(b, ts, rs, st);
  }
  return cudaGetLastError();
}

namespace {
unsigned int graph_blocks(const Batch &b) {
  const long long n = face_graph_valid(b);
  long long blocks = (n + 255) / 256;
  const long long cap = (long long)sms() * 8;
  return (unsigned int)std::max<long long>(1, std::min(blocks, cap));
}
}  // namespace

cudaError_t launch_face_graph_build(const Batch &b, const TiledScratch &ts, int2 *graph,
                                    DevStatus *st, cudaStream_t s) {
  (void)st;
  ++tl_launches;
  return with_shape(b.shape3, [&](auto shape) -> cudaError_t {
    k_face_graph_build<decltype(shape)><<<graph_blocks(b), 256, 0, s>>>(b, ts, graph);
    return cudaGetLastError();
  });
}

cudaError_t launch_face_graph_rounds(const Batch &b, int2 *graph, int r0, int r1, DevStatus *st,
                                     cudaStream_t s) {
  for (int r = r0; r < r1; ++r) {
    ++tl_launches;
    k_face_graph_round<<<graph_blocks(b), 256, 0, s>>>(b, graph, r, st);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_field_starts(const Batch &b, const TiledScratch &ts, const RankScratch &rs,
                                unsigned int m, cudaStream_t s, const unsigned int *m_dev) {
  if (b.key_mode != kKeyBatch || m == 0) return cudaSuccess;
  ++tl_launches;
  k_field_starts<<<(m + 255) / 256, 256, 0, s>>>(rs.list, m, m_dev, ts.fstart);
  return cudaGetLastError();
}

cudaError_t launch_tile_write(const Batch &b, const TiledScratch &ts, const RankScratch &rs,
                              const DevStatus *st, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  const bool in_pool = rs.capacity > kSetInL2;  // as k_resolve_pairs decides on the device
  if (b.tiles3 > 0) {
    e = with_shape(b.shape3, [&](auto shape) -> cudaError_t {
      using S = decltype(shape);
      const int64_t per_sm = (int64_t)b.tune.write_ctas * (512 / S::Threads);
      const int64_t grid = std::min<int64_t>(b.tiles3, (int64_t)sms() * per_sm);
      const unsigned g = (unsigned)grid;
      ++tl_launches;
      if (b.n_fields == 1)
        if (in_pool)
          k_tile_write<false, true, true, S><<<g, S::Threads, 0, s>>>(b, ts, rs, st);
        else
          k_tile_write<false, true, false, S><<<g, S::Threads, 0, s>>>(b, ts, rs, st);
      else if (in_pool)
        k_tile_write<false, false, true, S><<<g, S::Threads, 0, s>>>(b, ts, rs, st);
      else
        k_tile_write<false, false, false, S><<<g, S::Threads, 0, s>>>(b, ts, rs, st);
      return cudaGetLastError();
    });
    if (e != cudaSuccess) return e;
  }
  if (b.total_tiles > b.tiles3) {
    const int64_t grid = std::min<int64_t>(b.total_tiles - b.tiles3, (int64_t)sms() * b.tune.write_ctas);
    ++tl_launches;
    using S = Shape32x16;  // unused by the 2D tiles
    if (b.n_fields == 1)
      if (in_pool)
        k_tile_write<true, true, true, S><<<(unsigned)grid, k2Threads, 0, s>>>(b, ts, rs, st);
      else
        k_tile_write<true, true, false, S><<<(unsigned)grid, k2Threads, 0, s>>>(b, ts, rs, st);
    else if (in_pool)
      k_tile_write<true, false, true, S><<<(unsigned)grid, k2Threads, 0, s>>>(b, ts, rs, st);
    else
      k_tile_write<true, false, false, S><<<(unsigned)grid, k2Threads, 0, s>>>(b, ts, rs, st);
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace msseg
