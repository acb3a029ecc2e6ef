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
// The pointer area holds the extended box and, later, the candidate list and
// its 16-bit slots.
constexpr int k2PArea = k2Ext > kTileV + kTileV / 2 ? k2Ext : kTileV + kTileV / 2;

static_assert(k2TX * k2TY == kTileV, "2D tiles hold as many vertices as 3D tiles");
static_assert(k2TX * k2TY == kThreads * kRun && kTZ == kRun, "one run of 16 per thread");
static_assert(k2Face <= kFace, "the face array has kFace slots per tile");
static_assert(kHash <= k2Ext, "the 2D pair set fits the key area");
static_assert(kExt < 65536, "extended-box indices must fit 16 bits");
static_assert(kHash >= kTileV, "pair table must hold one pair per vertex");
static_assert(kHash <= kExt, "the pair set fits the key area");
static_assert((kTX + 1) * (kTY + 1) * (kTZ + 1) <= kExt, "cube extrema fit the pointer area");
static_assert(kTileV + kTileV / 2 <= kExt, "candidates (later the pair list) and their 16-bit slots fit the pointer area");

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
  int tile_ctas = 2;       // tile kernels: CTAs per SM (2 fit an SM)
  int write_ctas = 4;      // write kernels: CTAs per SM
  int resolve_blocks = 16;  // resolve: 256-thread blocks per SM
  int chase_hops = 16;     // budget of the first exit-chasing pass
  int dynamic = 1;         // tiles from a work queue (1) or a static stride (0)
};

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

struct TiledScratch {
  unsigned long long *pool_count;  // pairs reserved by all tiles
  unsigned int *queue;             // work-queue counters: tile 3D, tile 2D, write 3D, write 2D
  unsigned long long pool_cap;
  int2 *pool_roots;   // per tile pair: (dn-root, up-root), global index | kExitFlag if an exit;
                      // the resolved pair once resolved, if the set exceeds kSetInL2 entries
  uint32_t *pool_field;  // per tile pair: its field
  uint32_t *fstart;      // per field: index of its first pair in the sorted pair list
  uint32_t *pool_slot;  // per tile pair: slot of its (asc, desc) pair in the global pair set
  uint32_t *pending_list;  // tile pairs left by the budgeted chase (up to pending_cap)
  unsigned long long pending_cap;
  long long *tile_base;
  int32_t *tile_count;
  uint32_t *face;     // per tile kFace words: up-root | dn-root << 16 (extended-box indices)
  uint16_t *pid;      // per tile kTileV pair numbers; the 16 of column (lx, ly) are contiguous
};

TileGeom tile_geom(const int64_t dims[3]);
size_t tiled_scratch_bytes(long long total_tiles, int n_fields, unsigned long long pool_cap);
void tiled_scratch_carve(void *base, long long total_tiles, int n_fields,
                         unsigned long long pool_cap, TiledScratch *ts);
// Host side of a field descriptor (and its tensor map when TMA applies).
void make_field_desc(const void *field, int dtype, const int64_t dims[3], long long tile_base,
                     int32_t *asc, int32_t *desc, int32_t *ms, bool allow_tma, FieldDesc *fd,
                     CUtensorMap *map);
cudaError_t launch_tile_local(const Batch &b, const TiledScratch &ts, DevStatus *st,
                              cudaStream_t s);
// Exit resolution.  kChaseProbe chases the exits of a strided sample of the
// tile pairs (every `stride`-th) for at most kProbeHops face hops and only
// counts, in st->pending, the sampled pairs that need more: it decides
// between the two ways below.  kChaseBudget follows every pair's exits for at
// most Tuning::chase_hops hops, inserts the finished pairs and marks the others
// pending; kChasePending follows the pending pairs without a budget.
// kChaseGraph resolves every pair through the jumped face graph
// (launch_face_graph_*).  clear_table: reset the pair set first.
enum { kChaseProbe = 0, kChaseBudget = 1, kChasePending = 2, kChaseGraph = 3 };
// Pair sets of more entries than this (12 bytes each: beyond about a third of
// L2) are read in random order from DRAM; then k_resolve_pairs stores each
// resolved pair over its pool entry's roots and k_tile_write reads it there.
constexpr unsigned int kSetInL2 = 1u << 22;
constexpr int kProbeHops = 4;
// The probe samples about kProbeSample pairs, when there are kProbeMinPairs.
constexpr unsigned long long kProbeSample = 16384, kProbeMinPairs = 65536;
cudaError_t launch_resolve_pairs(const Batch &b, const TiledScratch &ts, const RankScratch &rs,
                                 unsigned long long npairs, int mode, const int2 *graph,
                                 unsigned long long stride, bool clear_table, DevStatus *st,
                                 cudaStream_t s);

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
