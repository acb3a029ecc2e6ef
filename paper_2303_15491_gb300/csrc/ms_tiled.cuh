// Shapes, scratch layout and launchers of the tiled segmentation (ms_tiled.cu).
#pragma once

#include <stdint.h>

#include <cuda.h>

#include <algorithm>

#include "fastdiv.h"
#include "ms_internal.cuh"

namespace msseg {

constexpr int kTX = 32, kTY = 16, kTZ = 16;               // tile, x fastest
constexpr int kThreads = kTX * kTY;                      // one thread per (x, y) column
// The tile plus a one-vertex halo is staged in a box of kEX x kEY x kEZ
// values whose x range starts 4 values left of the tile (x0 - 4, a 16-byte
// boundary for float32 rows), so the tile's column lx sits at box column
// lx + kXO and the halo columns at kXO - 1 and kXO + kTX.
constexpr int kXO = 4;
constexpr int kEX = kTX + 2 * kXO, kEY = kTY + 2, kEZ = kTZ + 2;  // 40 x 18 x 18
constexpr int kExt = kEX * kEY * kEZ;                    // 12960 < 2^16
constexpr int kTileV = kTX * kTY * kTZ;                  // 8192
constexpr int kFace = 2 * (kTX * kTY + kTX * kTZ + kTY * kTZ);  // face-root slots per tile
constexpr int kHashBits = 13;
constexpr int kHash = 1 << kHashBits;                    // >= kTileV: never overflows
constexpr int kStageCap = 2048;                          // pair-table entries staged in smem
constexpr int32_t kExitFlag = (int32_t)0x80000000u;

// 2D fields (nz = 1) use tiles of k2TX x k2TY vertices with the same 512
// threads: thread (lane, warp) owns the y-run of 16 vertices at
// x = lane + 32 (warp % 4), y = 16 (warp / 4) + 0..15.  The staged box is the
// tile plus a one-vertex halo, x again from 4 values left of the tile.
constexpr int k2TX = 128, k2TY = 64;
constexpr int k2EX = k2TX + 2 * kXO, k2EY = k2TY + 2;    // 136 x 66
constexpr int k2Ext = k2EX * k2EY;                       // 8976
constexpr int k2Face = 2 * (k2TX + k2TY);                // face-root slots of a 2D tile
constexpr int kRun = 16;                                 // vertices per thread, both shapes
// Words of the root bitmaps over a tile shape's extended box.
constexpr int kBmW3 = (kExt + 31) / 32;
constexpr int kBmW2 = (k2Ext + 31) / 32;
// Shared-memory areas of a 2D tile: the value area holds the extended box
// and, once the steepest step is done, the pair list and the root bitmaps;
// the pointer area holds the pointers and, once they are final, the pair set
// and its dense numbers.
constexpr int k2KArea = k2Ext > kTileV + 4 * kBmW2 ? k2Ext : kTileV + 4 * kBmW2;
constexpr int k2PArea = k2Ext > kHash + kHash / 2 ? k2Ext : kHash + kHash / 2;

static_assert(k2TX * k2TY == kTileV, "2D tiles hold as many vertices as 3D tiles");
static_assert(k2TX * k2TY == kThreads * kRun && kTZ == kRun, "one run of 16 per thread");
static_assert(k2Face <= kFace, "the face array has kFace slots per tile");
static_assert(kExt < 65536, "extended-box indices must fit 16 bits");
static_assert(2 * kExt < 65536, "root-list indices (dn roots, then up roots) fit 16 bits");
static_assert(kHash >= kTileV, "pair table must hold one pair per vertex");
static_assert((kTX + 1) * (kTY + 1) * (kTZ + 1) <= kExt, "cube extrema fit the pointer area");
static_assert(kHash + kHash / 2 <= kExt, "pair set and dense numbers fit the 3D value area");
static_assert(kTileV + 4 * kBmW3 <= kExt, "pair list and root bitmaps fit the 3D pointer area");
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
  uint32_t *face;       // per tile kFace words: up-root | dn-root << 16 (extended-box indices)
  uint16_t *pid;        // per tile kTileV pair numbers; the 16 of a thread's run are contiguous
};
// The root list: dn and up roots of a tile, the latter flagged.
constexpr uint16_t kUpRoot = 0x8000u;
static_assert(kExt < kUpRoot, "box indices leave the top bit free");
// Work-queue counters: tile pass 3D / 2D, write 3D / 2D, root chase 3D / 2D, tile pairs.
enum { kQTile3 = 0, kQTile2 = 1, kQWrite3 = 2, kQWrite2 = 3, kQChase = 4, kQChase2 = 5, kQPairs = 6,
       kQueues = 8 };

TileGeom tile_geom(const int64_t dims[3]);
size_t tiled_scratch_bytes(long long total_tiles, int n_fields, unsigned long long pool_cap,
                           unsigned long long root_cap);
void tiled_scratch_carve(void *base, long long total_tiles, int n_fields,
                         unsigned long long pool_cap, unsigned long long root_cap,
                         TiledScratch *ts);
// Host side of a field descriptor (and its tensor map when TMA applies).
void make_field_desc(const void *field, int dtype, const int64_t dims[3], long long tile_base,
                     int32_t *asc, int32_t *desc, int32_t *ms, bool allow_tma, FieldDesc *fd,
                     CUtensorMap *map);
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
cudaError_t launch_chase_roots(const Batch &b, const TiledScratch &ts, const int2 *graph,
                               long long probe_stride, DevStatus *st, cudaStream_t s);
// Tile pairs: each tile pair's (asc, desc) from its roots' labels, the tile's
// distinct pairs inserted into the global pair set (clear_table: reset it
// first), each tile pair's set slot stored.
// Pair sets of more entries than this (12 bytes each: beyond about a third of
// L2) are read in random order from DRAM; then the tile pairs also keep their
// (asc, desc) for the write kernel to read in order.
constexpr unsigned int kSetInL2 = 1u << 22;
cudaError_t launch_tile_pairs(const Batch &b, const TiledScratch &ts, const RankScratch &rs,
                              bool clear_table, DevStatus *st, cudaStream_t s);

// The face graph: per face slot of every tile (kFace slots per tile, 3D
// tiles first) the up and dn successor -- the global slot of the next face
// vertex on the path, or the extremum's vertex index | kSlotFinal.
constexpr uint32_t kSlotFinal = 0x80000000u;
inline long long face_graph_slots(const Batch &b) { return b.total_tiles * (long long)kFace; }
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
