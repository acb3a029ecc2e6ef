// Shapes, scratch layout and launchers of the tiled segmentation (ms_tiled.cu).
#pragma once

#include <stdint.h>

#include <cuda.h>

#include <algorithm>

#include "fastdiv.h"
#include "ms_internal.cuh"

namespace msseg {

constexpr int kTZ = 16;   // tile depth: every 3D tile shape is TX x TY x kTZ
constexpr int kRun = 16;  // vertices per thread: a 3D tile's z-column, a 2D tile's y-run
// The staged box of a tile starts kXO values left of the tile (x0 - 4, a
// 16-byte boundary for float32 rows), so the tile's column lx sits at box
// column lx + kXO and the halo columns at kXO - 1 and kXO + TX.
constexpr int kXO = 4;
constexpr int32_t kExitFlag = (int32_t)0x80000000u;
constexpr int kStageCap = 2048;  // pair-table entries staged in smem

constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v >> 1); }

// A 3D tile shape: TX x TY x kTZ vertices and one thread per (x, y) column
// (thread t owns x = t % TX, y = t / TX, all kTZ planes).  The tile plus a
// one-vertex halo is staged in a box of EX x EY x EZ values.
template <int TX_, int TY_>
struct Shape3 {
  static constexpr int TX = TX_, TY = TY_, TZ = kTZ;
  static constexpr int Threads = TX * TY;
  static constexpr int EX = TX + 2 * kXO, EY = TY + 2, EZ = TZ + 2;
  static constexpr int Ext = EX * EY * EZ;
  static constexpr int TileV = TX * TY * TZ;
  static constexpr int Face = 2 * (TX * TY + TX * TZ + TY * TZ);  // face-root slots per tile
  static constexpr int Hash = TileV;  // the tile's pair set: a slot per vertex, never full
  static constexpr int HashBits = ilog2(Hash);
  static constexpr int BmW = (Ext + 31) / 32;  // words of a root bitmap over the box
  static constexpr int CX = TX + 1, CY = TY + 1;  // unit cubes along x and y
  static_assert(Threads % 32 == 0 && Threads <= 512, "whole warps, at most 512 threads");
  static_assert((1 << HashBits) == Hash, "tiles of a power-of-two size");
  static_assert(Threads * kRun == TileV, "one run of kRun per thread");
  static_assert(TX % 4 == 0, "box rows of whole 16-byte units");
  static_assert(2 * Ext < 65536 && Ext < 0x8000, "box indices (and root-list indices) fit");
  static_assert(CX * CY * (TZ + 1) <= Ext, "cube extrema fit the pointer area");
  static_assert(Hash + Hash / 2 <= Ext, "pair set and dense numbers fit the value area");
  static_assert(TileV + 4 * BmW <= Ext, "pair list and root bitmaps fit the pointer area");
  static_assert(BmW <= Threads, "two bitmap words per thread cover both root bitmaps");
  static_assert(Face < 4096 && TX < 128 && TY < 64, "the root-chase table's field widths");
};
// The shapes a call can take (Tuning::shape3); the first is the default.
using Shape32x16 = Shape3<32, 16>;
using Shape64x8 = Shape3<64, 8>;
using Shape16x32 = Shape3<16, 32>;
using Shape16x16 = Shape3<16, 16>;  // 4096 vertices: small fields
enum { kShape32x16 = 0, kShape64x8 = 1, kShape16x32 = 2, kShape16x16 = 3, kShapeCount = 4 };
struct ShapeInfo {
  int tx, ty, tz, threads, ext, face, tilev;
};
template <class S>
constexpr ShapeInfo info_of() {
  return ShapeInfo{S::TX, S::TY, S::TZ, S::Threads, S::Ext, S::Face, S::TileV};
}
inline ShapeInfo shape_info(int id) {
  switch (id) {
    case kShape64x8: return info_of<Shape64x8>();
    case kShape16x32: return info_of<Shape16x32>();
    case kShape16x16: return info_of<Shape16x16>();
    default: return info_of<Shape32x16>();
  }
}
constexpr int kExtMax = Shape16x32::Ext;  // the largest staged box of any shape
static_assert(kExtMax >= Shape32x16::Ext && kExtMax >= Shape64x8::Ext && kExtMax >= Shape16x16::Ext,
              "kExtMax bounds every shape");
constexpr int kPidStride = 8192;  // pair numbers stored per tile (the largest tile)

// 2D fields (nz = 1) use tiles of k2TX x k2TY vertices with 512 threads:
// thread (lane, warp) owns the y-run of 16 vertices at
// x = lane + 32 (warp % 4), y = 16 (warp / 4) + 0..15.  The staged box is the
// tile plus a one-vertex halo, x again from 4 values left of the tile.
constexpr int k2TX = 128, k2TY = 64;
constexpr int k2Threads = 512;
constexpr int k2EX = k2TX + 2 * kXO, k2EY = k2TY + 2;    // 136 x 66
constexpr int k2Ext = k2EX * k2EY;                       // 8976
constexpr int k2TileV = k2TX * k2TY;                     // 8192
constexpr int k2Face = 2 * (k2TX + k2TY);                // face-root slots of a 2D tile
constexpr int k2Hash = k2TileV;
constexpr int k2HashBits = ilog2(k2Hash);
constexpr int kBmW2 = (k2Ext + 31) / 32;  // words of a root bitmap over the 2D box
// Shared-memory areas of a 2D tile: the value area holds the extended box
// and, once the steepest step is done, the pair list and the root bitmaps;
// the pointer area holds the pointers and, once they are final, the pair set
// and its dense numbers.
constexpr int k2KArea = k2Ext > k2TileV + 4 * kBmW2 ? k2Ext : k2TileV + 4 * kBmW2;
constexpr int k2PArea = k2Ext > k2Hash + k2Hash / 2 ? k2Ext : k2Hash + k2Hash / 2;

static_assert(k2TileV == k2Threads * kRun, "one run of 16 per thread");
static_assert(k2TileV <= kPidStride, "a 2D tile's pair numbers fit its stride");
static_assert(k2Face <= Shape16x16::Face, "a 2D tile's face slots fit any shape's stride");
static_assert(2 * k2Ext < 65536, "root-list indices (dn roots, then up roots) fit 16 bits");
static_assert(kBmW2 <= k2Threads, "two bitmap words per thread cover both root bitmaps");
static_assert((k2KArea * 4) % 16 == 0, "the 2D pointer area starts 16-byte aligned");

struct TileGeom {
  int64_t nx, ny, nz;
  int64_t tx, ty, tz, ntiles;
  int flat;  // 1: nz = 1, 2D tiles of k2TX x k2TY
  FastDivU32 div_nx, div_ny, div_tx, div_ty;  // coordinates from linear indices
};

// One field of a (possibly one-field) batch, resident on the device.
struct FieldDesc {
  const void *field;
  int32_t *asc, *desc, *ms;
  TileGeom g;
  long long tile_base;  // global index of the field's first tile
  int dtype;
  int tma;              // 1: the batch's tmaps[field] describes this field
};

// Key layouts of the global pair set.
enum { kKeyOne = 0,     // one field: (asc << 32) | desc
       kKeyBatch = 1 };  // many fields, each N <= 2^24: (field << 48) | (asc << 24) | desc
constexpr int64_t kBatchMaxN = 1ll << 24;
constexpr int kBatchMaxFields = 1 << 16;

// Launch choices that change only scheduling, never results (picked by the
// batch autotuner; the defaults are the single-field choices).
struct Tuning {
  int tile_ctas = 2;     // tile kernels: CTAs per SM (2 fit an SM)
  int write_ctas = 4;    // write kernels: CTAs per SM
  int chase_blocks = 3;  // root chase: 512-thread blocks (16 warps) per SM
  int pair_blocks = 8;   // tile pairs: 256-thread blocks per SM
  int dynamic = 1;       // tile and write kernels: a work queue (1) or a static stride (0)
  int resolve_mode = -1;  // root chase and tile pairs: a tile a warp (0), flat over the root
                          // list and pair pool (1), or by tile count (-1, see tile_mode)
  int shape3 = kShape32x16;  // the 3D tiles' shape (a kShape* id)
};
// Calls with at least this many tiles resolve a tile a warp when the mode is
// left to the tile count: enough tiles keep every warp busy, and a warp then
// deduplicates its tile's pairs before the global set.  Fewer tiles resolve
// flat, which spreads a tile's roots and pairs over many warps.
constexpr long long kTileModeMin = 2048;

struct Batch;
bool tile_mode(const Batch &b);

struct Batch {
  const FieldDesc *fields;    // n_fields descriptors
  const CUtensorMap *tmaps;   // n_fields tensor maps (64-byte aligned)
  int n_fields;
  int key_mode;
  long long total_tiles;
  long long tiles3;  // tiles of the 3D fields, which come first; the rest are 2D
  FieldDesc f0;      // n_fields == 1: the descriptor itself, read from kernel parameters
  Tuning tune;
  int shape3;        // the 3D tiles' shape (the one their geometry was computed for)
  int face_stride;   // face slots per tile, 3D and 2D alike (the 3D shape's face count)
};

// Per-tile record of the tile pass: where the tile's pairs and roots start in
// the pair pool and the root list, and how many there are.
struct TileMeta {
  unsigned long long pbase;  // first pair-pool entry
  unsigned long long rbase;  // first root-list entry
  int npairs;                // distinct (dn-root, up-root) pairs of the tile
  int nd, nu;                // distinct dn roots, up roots (the root list holds dn, then up)
  int pad;
};

struct TiledScratch {
  unsigned long long *counters;  // [0] pairs reserved by all tiles, [1] roots, [2] roots of
                                 // the 3D tiles (which come first in the root list)
  unsigned int *queue;           // work-queue counters (kQueues)
  unsigned long long pool_cap;   // pair-pool entries
  unsigned long long root_cap;   // root-list entries
  uint2 *pool_pair;     // per tile pair: its dn root and up root (indices into the root list)
  uint32_t *pool_slot;  // per tile pair: slot of its (asc, desc) pair in the global pair set
  int2 *pool_ad;        // per tile pair: its (asc, desc), kept when the set exceeds kSetInL2 entries
  uint16_t *root_box;   // per tile root: its extended-box index | kUpRoot if an up root
  uint32_t *root_tile;  // per tile root: its tile (global index)
  int32_t *root_label;  // per tile root: the extremum its path reaches
  TileMeta *meta;       // per tile
  uint32_t *fstart;     // per field: index of its first pair in the sorted pair list
  uint32_t *face;       // per tile face_stride words: up-root | dn-root << 16 (box indices)
  uint16_t *pid;        // per tile kPidStride pair numbers; a thread's run of 16 is contiguous
};
// The root list: dn and up roots of a tile, the latter flagged.
constexpr uint16_t kUpRoot = 0x8000u;
static_assert(kExtMax < kUpRoot, "box indices leave the top bit free");
// Work-queue counters: tile pass 3D / 2D, write 3D / 2D, root chase 3D / 2D, tile pairs.
enum { kQTile3 = 0, kQTile2 = 1, kQWrite3 = 2, kQWrite2 = 3, kQChase = 4, kQChase2 = 5, kQPairs = 6,
       kQueues = 8 };

// Tile geometry of a field for the 3D shape shape3 (2D fields: 2D tiles).
TileGeom tile_geom(const int64_t dims[3], int shape3);
size_t tiled_scratch_bytes(long long total_tiles, int n_fields, unsigned long long pool_cap,
                           unsigned long long root_cap, int face_stride);
void tiled_scratch_carve(void *base, long long total_tiles, int n_fields,
                         unsigned long long pool_cap, unsigned long long root_cap, int face_stride,
                         TiledScratch *ts);
// Host side of a field descriptor (and its tensor map when TMA applies).
void make_field_desc(const void *field, int dtype, const int64_t dims[3], long long tile_base,
                     int32_t *asc, int32_t *desc, int32_t *ms, bool allow_tma, int shape3,
                     FieldDesc *fd, CUtensorMap *map);
// Tile pass: steepest neighbours, in-tile compression, the tile's distinct
// roots and pairs (counters[0] / [1] hold the pool and root-list totals).
cudaError_t launch_tile_local(const Batch &b, const TiledScratch &ts, DevStatus *st,
                              cudaStream_t s);
// Root chase: every tile root is followed from face to face (or looked up in
// the jumped face graph when `graph` is given) to the extremum it leads to.
// Probe form (probe_stride > 0): only every probe_stride-th root, at most
// kProbeHops hops a root, counting in st->pending the roots that need more
// and in st->sampled the roots sampled; no labels are stored.
constexpr int kProbeHops = 4;
// The probe runs when a call has at least kProbeMinRoots roots, on about
// kProbeRoots of them (every probe_stride-th root of the list).
constexpr unsigned long long kProbeMinRoots = 65536;
constexpr unsigned long long kProbeRoots = 16384;
// roots: an upper bound on the call's tile roots (0: the root list's capacity),
// which sizes the flat form's grid.
cudaError_t launch_chase_roots(const Batch &b, const TiledScratch &ts, const int2 *graph,
                               long long probe_stride, DevStatus *st, cudaStream_t s,
                               unsigned long long roots = 0);
// Tile pairs: each tile pair's (asc, desc) from its roots' labels, the tile's
// distinct pairs inserted into the global pair set (clear_table: reset it
// first), each tile pair's set slot stored.
// Pair sets of more entries than this (12 bytes each: beyond about a third of
// L2) are read in random order from DRAM; then the tile pairs also keep their
// (asc, desc) for the write kernel to read in order.
constexpr unsigned int kSetInL2 = 1u << 22;
// pairs: an upper bound on the call's tile pairs (0: the pool's capacity),
// which sizes the flat form's grid.
cudaError_t launch_tile_pairs(const Batch &b, const TiledScratch &ts, const RankScratch &rs,
                              bool clear_table, DevStatus *st, cudaStream_t s,
                              unsigned long long pairs = 0);

// The face graph: per face slot of every tile (face_stride slots per tile,
// 3D tiles first) the up and dn successor -- the global slot of the next
// face vertex on the path, or the extremum's vertex index | kSlotFinal.
constexpr uint32_t kSlotFinal = 0x80000000u;
inline long long face_graph_slots(const Batch &b) { return b.total_tiles * (long long)b.face_stride; }
// Builds the graph from the tiles' face roots, then pointer-jumps it in place
// until every entry is final (at most `rounds` rounds; rounds r use
// st->round_open[r]).  queue_rounds queues rounds [r0, r1).
cudaError_t launch_face_graph_build(const Batch &b, const TiledScratch &ts, int2 *graph,
                                    DevStatus *st, cudaStream_t s);
cudaError_t launch_face_graph_rounds(const Batch &b, int2 *graph, int r0, int r1, DevStatus *st,
                                     cudaStream_t s);
cudaError_t launch_field_starts(const Batch &b, const TiledScratch &ts, const RankScratch &rs,
                                unsigned int m, cudaStream_t s, const unsigned int *m_dev = nullptr);
cudaError_t launch_tile_write(const Batch &b, const TiledScratch &ts, const RankScratch &rs,
                              const DevStatus *st, cudaStream_t s);

}  // namespace msseg
