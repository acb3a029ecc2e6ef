// C ABI of libmsseg (declared in include/ms.h): context, argument checks,
// scratch memory and the order in which the steps of Sec. 4.2 are queued.
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "ms_internal.cuh"
#include "ms_tiled.cuh"

using namespace msseg;

// Sizes a step-by-step tiled call met (they size a captured replay).
struct RunInfo {
  unsigned long long npairs = 0;  // tile pairs
  unsigned long long nroots = 0;  // tile roots
  unsigned int m = 0;             // distinct (asc, desc) pairs
  bool use_graph = false;         // exits resolved through the face graph
  int rounds = 0;                 // face-graph rounds it took
};

// A repeated batch: its signature, tuning and captured pipeline.
struct BatchPlan {
  std::vector<int64_t> sig;
  bool tuned = false;
  Tuning tune;
  cudaGraphExec_t exec = nullptr;
  long long epoch = -1;      // ctx alloc_epoch the graph's buffers belong to
  long long launches = 0;    // kernels per replay
  std::vector<int> order;    // descriptor j describes field order[j]
  void *host_desc = nullptr;  // pinned copy of the descriptors the graph uploads
  size_t host_desc_bytes = 0;
  uint32_t *hfstart = nullptr;  // pinned: first sorted pair of each descriptor
  size_t hfstart_count = 0;
  int seen = 0;                   // consecutive calls with this signature
  long long stage_launches[3] = {};  // kernels per replay: tile_local, resolve, write
};

struct ms_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  DevStatus *dst = nullptr;  // device status block
  DevStatus *hst = nullptr;  // pinned host copy
  void *scratch = nullptr;   // pair-rank working memory
  size_t scratch_bytes = 0;
  void *io = nullptr;        // device buffers of ms_segment_host (and the first set of
  size_t io_bytes = 0;       // ms_segment_host_many)
  void *io2 = nullptr;       // the second buffer set of ms_segment_host_many
  size_t io2_bytes = 0;
  cudaStream_t up = nullptr, down = nullptr;  // ms_segment_host_many: upload / download streams
  cudaEvent_t ev_up[2] = {}, ev_comp[2] = {}, ev_down[2] = {};
  void *tscratch = nullptr;  // tiled path working memory
  size_t tscratch_bytes = 0;
  void *graph = nullptr;     // the face graph, built only for long exit chains
  size_t graph_bytes = 0;
  void *sxscratch = nullptr;  // index-pass block totals and bases
  size_t sxscratch_bytes = 0;
  void *slscratch = nullptr;  // z-slab pointer arrays (slab and its halo planes)
  size_t slscratch_bytes = 0;
  void *slmap = nullptr;      // published planes: their z and row, sorted by z
  size_t slmap_bytes = 0;
  void *pscratch = nullptr;   // persistence pairing working memory
  size_t pscratch_bytes = 0;
  void *pcount = nullptr;     // its pinned counter copy
  uint64_t pers_pairs_hint = 0;   // basin-pair capacity that sufficed last time
  uint64_t pers_minima_hint = 0;  // extremum capacity that sufficed last time
  unsigned long long *hcount = nullptr;  // pinned copies of the tile pass's pair and root counts
  unsigned long long pool_hint = 0;      // pair-pool capacity that sufficed last time
  unsigned long long root_hint = 0;      // root-list capacity that sufficed last time
  void *batch_dev = nullptr;             // field descriptors + tensor maps on the device
  size_t batch_dev_bytes = 0;
  void *batch_host = nullptr;            // their pinned staging copy
  size_t batch_host_bytes = 0;
  int64_t last_k = 0;
  long long alloc_epoch = 0;  // bumped whenever a device buffer is reallocated
  Tuning tune;                // launch choices without a tuned entry
  RunInfo run;                // sizes met by the last step-by-step tiled call
  BatchPlan plans[2];         // the last two batches: their tuning and captured graphs
  int plan_next = 0;          // the plan slot a new signature takes
  bool graphs_on = true;
  // profiler
  bool prof_on = false;
  ms_profile prof{};
  cudaEvent_t ev[MS_STAGE_COUNT][2] = {};
  bool ev_pending[MS_STAGE_COUNT] = {};
};

namespace msseg {
thread_local long long tl_launches = 0;
}

namespace {

constexpr int64_t kMaxVertices = 2147483647LL;

ms_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MS_OK;
  if (e == cudaErrorMemoryAllocation) return MS_ERR_OUT_OF_MEMORY;
  return MS_ERR_CUDA;
}

#define MS_TRY(expr)                       \
  do {                                     \
    ms_status _s = cuda_status((expr));    \
    if (_s != MS_OK) return _s;            \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

bool is_device_pointer(const void *p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

ms_status check_dims(const int64_t dims[3], int64_t *n_out) {
  if (!dims) return MS_ERR_INVALID_ARG;
  if (dims[0] < 1 || dims[1] < 1 || dims[2] < 1) return MS_ERR_INVALID_ARG;
  if (dims[0] > kMaxVertices || dims[1] > kMaxVertices || dims[2] > kMaxVertices)
    return MS_ERR_TOO_LARGE;
  const int64_t xy = dims[0] * dims[1];
  if (xy > kMaxVertices || xy * dims[2] > kMaxVertices) return MS_ERR_TOO_LARGE;
  *n_out = xy * dims[2];
  return MS_OK;
}

ms_status check_dtype(int dtype) {
  return (dtype == MS_F32 || dtype == MS_F16) ? MS_OK : MS_ERR_UNSUPPORTED_DTYPE;
}

int bit_width(int64_t x) {  // bits needed to hold values 0..x
  int b = 0;
  while (x > 0) {
    ++b;
    x >>= 1;
  }
  return b;
}

int round_cap(int64_t n) { return bit_width(n) + 2; }

ms_status reset_status(ms_ctx *c) {
  MS_TRY(cudaMemsetAsync(c->dst, 0, sizeof(DevStatus), c->stream));
  return MS_OK;
}

ms_status read_status(ms_ctx *c) {
  MS_TRY(cudaMemcpyAsync(c->hst, c->dst, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream));
  MS_TRY(cudaStreamSynchronize(c->stream));
  return MS_OK;
}

ms_status ensure_scratch(ms_ctx *c, size_t bytes) {
  if (c->scratch_bytes >= bytes) return MS_OK;
  ++c->alloc_epoch;
  if (c->scratch) {
    cudaStreamSynchronize(c->stream);
    cudaFree(c->scratch);
    c->scratch = nullptr;
    c->scratch_bytes = 0;
  }
  if (cudaMalloc(&c->scratch, bytes) != cudaSuccess) {
    cudaGetLastError();
    return MS_ERR_OUT_OF_MEMORY;
  }
  c->scratch_bytes = bytes;
  return MS_OK;
}

// The pair-rank working memory of a set of this capacity, carved.
ms_status rank_scratch_ready(ms_ctx *c, unsigned int cap, RankScratch *rs) {
  ms_status s = ensure_scratch(c, rank_scratch_bytes(cap));
  if (s != MS_OK) return s;
  rank_scratch_carve(c->scratch, cap, rs);
  return MS_OK;
}

unsigned int pow2_at_least(uint64_t x) {
  uint64_t p = 1024;
  while (p < x && p < (1ull << 31)) p <<= 1;
  return (unsigned int)p;
}

// Compression schedule: `first` rounds queued blind, then one status read;
// if the last round still had work, the rest of the cap is queued and read.
ms_status compress_pair(ms_ctx *c, int32_t *a, int32_t *b, int64_t n) {
  const int cap = round_cap(n);
  const int first = cap < 8 ? cap : 8;
  for (int r = 0; r < first; ++r) MS_TRY(launch_compress_round(a, b, n, 4, r, c->dst, c->stream));
  ms_status s = read_status(c);
  if (s != MS_OK) return s;
  if (c->hst->round_open[first - 1] == 0u) return MS_OK;
  for (int r = first; r < cap; ++r) MS_TRY(launch_compress_round(a, b, n, 4, r, c->dst, c->stream));
  s = read_status(c);
  if (s != MS_OK) return s;
  return c->hst->round_open[cap - 1] ? MS_ERR_NOT_CONVERGED : MS_OK;
}

// Dense pair ranks (Sec. 4.2.2).  `guess` is a first estimate of the number
// of distinct pairs; `bound` a hard upper bound.
ms_status rank_pairs(ms_ctx *c, const int32_t *asc, const int32_t *desc, int64_t n, int32_t *ms,
                     uint64_t guess, uint64_t bound) {
  if (n == 0) {
    c->last_k = 0;
    return MS_OK;
  }
  if (bound < 1) bound = 1;
  if (guess > bound) guess = bound;
  if (guess < 1) guess = 1;
  for (;;) {
    const unsigned int cap = pow2_at_least(2 * guess + 2);
    RankScratch rs;
    ms_status s = rank_scratch_ready(c, cap, &rs);
    if (s != MS_OK) return s;
    if (guess < bound) rs.probe_limit = kEstimateProbeLimit;
    MS_TRY(cudaMemsetAsync(&c->dst->n_unique, 0, sizeof(unsigned int), c->stream));
    MS_TRY(cudaMemsetAsync(&c->dst->hash_overflow, 0, sizeof(unsigned int), c->stream));
    MS_TRY(launch_pairs_insert(asc, desc, n, rs, c->dst, c->stream));
    s = read_status(c);
    if (s != MS_OK) return s;
    if (c->hst->bad_index) return MS_ERR_INVALID_ARG;
    if (c->hst->hash_overflow) {
      if (guess >= bound) return MS_ERR_CUDA;  // cannot happen: the bound is exact
      guess = guess * 4 < bound ? guess * 4 : bound;
      continue;
    }
    const unsigned int m = c->hst->n_unique;
    MS_TRY(launch_pairs_sort(rs, m, bit_width(n - 1), c->stream));
    MS_TRY(launch_pairs_assign(rs, m, c->stream));
    MS_TRY(launch_pairs_lookup(asc, desc, n, rs, ms, c->stream));
    s = read_status(c);
    if (s != MS_OK) return s;
    if (c->hst->timeout) return MS_ERR_TIMEOUT;
    c->last_k = m;
    return MS_OK;
  }
}

// Brackets one stage of a call with CUDA events on the context's stream
// (profiler on only); the elapsed times are collected by finish_profile once
// the call has synchronised.
struct StageTimer {
  ms_ctx *c;
  int stage;
  long long l0;
  StageTimer(ms_ctx *ctx, int st) : c(ctx), stage(st), l0(tl_launches) {
    if (c->prof_on) cudaEventRecord(c->ev[stage][0], c->stream);
  }
  void stop() {
    if (!c->prof_on) return;
    cudaEventRecord(c->ev[stage][1], c->stream);
    c->ev_pending[stage] = true;
    c->prof.stage_launches[stage] += tl_launches - l0;
  }
};

void finish_profile(ms_ctx *c, long long launches0) {
  if (!c->prof_on) return;
  cudaStreamSynchronize(c->stream);
  for (int s = 0; s < MS_STAGE_COUNT; ++s) {
    if (!c->ev_pending[s]) continue;
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, c->ev[s][0], c->ev[s][1]) == cudaSuccess) c->prof.stage_ms[s] += ms;
    c->ev_pending[s] = false;
  }
  cudaGetLastError();
  c->prof.calls += 1;
  c->prof.launches += tl_launches - launches0;
}

ms_status ensure_buffer(ms_ctx *c, void **buf, size_t *have, size_t bytes) {
  if (*have >= bytes) return MS_OK;
  ++c->alloc_epoch;
  if (*buf) {
    cudaStreamSynchronize(c->stream);
    cudaFree(*buf);
    *buf = nullptr;
    *have = 0;
  }
  if (cudaMalloc(buf, bytes) != cudaSuccess) {
    cudaGetLastError();
    return MS_ERR_OUT_OF_MEMORY;
  }
  *have = bytes;
  return MS_OK;
}

// Pointer-jumps the face graph until every entry is final: `first` rounds
// queued blind, one status read, then the rest of the cap if needed.
// Pointer-jumps the face graph until every entry is final: a few rounds
// queued blind, then one round at a time with a status read after each
// (rounds over large graphs cost far more than the read).
ms_status jump_face_graph(ms_ctx *c, const Batch &b, int2 *graph, long long slots) {
  const int cap = std::min(64, round_cap(slots));
  const int blind = std::min(cap, slots > (1ll << 24) ? 3 : 6);
  MS_TRY(cudaMemsetAsync(c->dst->round_open, 0, sizeof(c->dst->round_open), c->stream));
  MS_TRY(launch_face_graph_rounds(b, graph, 0, blind, c->dst, c->stream));
  ms_status s = read_status(c);
  if (s != MS_OK) return s;
  for (int r = blind;; ++r) {
    if (c->hst->round_open[r - 1] == 0u) {
      int used = r;  // the first round that left nothing open, counted from 1
      while (used > 1 && c->hst->round_open[used - 2] == 0u) --used;
      c->run.rounds = used;
      return MS_OK;
    }
    if (r == cap) return MS_ERR_NOT_CONVERGED;
    MS_TRY(launch_face_graph_rounds(b, graph, r, r + 1, c->dst, c->stream));
    s = read_status(c);
    if (s != MS_OK) return s;
  }
}

// The tiled path (ms_tiled.cu): tile-local steepest + compression + pair
// numbering, global resolution of tile exits and pair ranks, label write.
// One field of a segmentation request, as the tiled path sees it.
struct FieldArg {
  const void *field;
  const int64_t *dims;
  int dtype;
  int64_t n;
  int32_t *asc, *desc, *ms;
};

// The tiled path (ms_tiled.cu) over one field or a batch of fields: one
// launch per stage covers every tile of every field.  Batches key the global
// pair set by (field, asc, desc); each field's MS ids start at its first pair
// in the sorted set.  k_out[f] receives each field's region count.
// Descriptors and tensor maps of a field table, staged in pinned memory and
// copied to the device; fills b (tuning aside) and the field order.
struct Staged {
  Batch b;
  std::vector<int> order;
  int64_t total_n = 0, max_n = 0;
  size_t bytes = 0;  // descriptor bytes on the device
};

ms_status stage_fields(ms_ctx *c, const FieldArg *fa, int nf, int shape3, Staged *out) {
  const int key_mode = nf > 1 ? kKeyBatch : kKeyOne;
  const size_t desc_bytes = ((size_t)nf * sizeof(FieldDesc) + 127) & ~(size_t)127;
  const size_t bytes = desc_bytes + (size_t)nf * sizeof(CUtensorMap);
  ms_status s = ensure_buffer(c, &c->batch_dev, &c->batch_dev_bytes, bytes);
  if (s != MS_OK) return s;
  if (c->batch_host_bytes < bytes) {
    if (c->batch_host) {
      cudaStreamSynchronize(c->stream);
      cudaFreeHost(c->batch_host);
      c->batch_host = nullptr;
      c->batch_host_bytes = 0;
    }
    if (cudaMallocHost(&c->batch_host, bytes) != cudaSuccess) {
      cudaGetLastError();
      return MS_ERR_OUT_OF_MEMORY;
    }
    c->batch_host_bytes = bytes;
  }
  MS_TRY(cudaStreamSynchronize(c->stream));  // the staging buffer may still be in flight
  FieldDesc *hd = static_cast<FieldDesc *>(c->batch_host);
  CUtensorMap *hm = reinterpret_cast<CUtensorMap *>(static_cast<char *>(c->batch_host) + desc_bytes);
  // descriptor j describes field order[j]: the 3D fields first, then the 2D
  // ones, so that each tile shape's kernels cover one contiguous tile range
  std::vector<int> order;
  order.reserve(nf);
  for (int f = 0; f < nf; ++f)
    if (fa[f].dims[2] != 1) order.push_back(f);
  for (int f = 0; f < nf; ++f)
    if (fa[f].dims[2] == 1) order.push_back(f);
  long long total_tiles = 0, tiles3 = 0;
  int64_t total_n = 0, max_n = 0;
  for (int j = 0; j < nf; ++j) {
    const FieldArg &a = fa[order[j]];
    make_field_desc(a.field, a.dtype, a.dims, total_tiles, a.asc, a.desc, a.ms, true, shape3,
                    &hd[j], &hm[j]);
    total_tiles += hd[j].g.ntiles;
    if (!hd[j].g.flat) tiles3 = total_tiles;
    total_n += a.n;
    max_n = std::max(max_n, a.n);
  }
  MS_TRY(cudaMemcpyAsync(c->batch_dev, c->batch_host, bytes, cudaMemcpyHostToDevice, c->stream));
  Batch b;
  b.fields = static_cast<const FieldDesc *>(c->batch_dev);
  b.tmaps = reinterpret_cast<const CUtensorMap *>(static_cast<const char *>(c->batch_dev) + desc_bytes);
  b.n_fields = nf;
  b.key_mode = key_mode;
  b.total_tiles = total_tiles;
  b.tiles3 = tiles3;
  b.f0 = hd[0];
  b.shape3 = shape3;
  b.face_stride = shape_info(shape3).face;
  out->b = b;
  out->order = std::move(order);
  out->total_n = total_n;
  out->max_n = max_n;
  out->bytes = bytes;
  return MS_OK;
}

int pair_key_bits(const Staged &sf, int *raw_bits) {
  *raw_bits = sf.b.key_mode == kKeyBatch ? bit_width(sf.b.n_fields - 1) + 48 : 0;
  return sf.b.key_mode == kKeyBatch ? 0 : bit_width(sf.max_n - 1);
}

// The tiled path, step by step (host reads sizes and statuses in between).
ms_status segment_tiled(ms_ctx *c, const FieldArg *fa, int nf, int64_t *k_out,
                        const Tuning &tune) {
  Staged sf;
  ms_status s = stage_fields(c, fa, nf, tune.shape3, &sf);
  if (s != MS_OK) return s;
  Batch b = sf.b;
  b.tune = tune;
  const int key_mode = b.key_mode;
  const long long total_tiles = b.total_tiles;
  const int64_t total_n = sf.total_n;
  const std::vector<int> &order = sf.order;
  c->run = RunInfo{};

  // ---- tile pass; the pair pool and root list are sized from the last call,
  // exact on overflow
  const unsigned long long vslots = (unsigned long long)total_tiles * kPidStride;
  unsigned long long cap = c->pool_hint, rcap = c->root_hint;
  if (cap == 0) cap = std::max<unsigned long long>(1ull << 16, (unsigned long long)total_n / 4);
  if (rcap == 0) rcap = std::max<unsigned long long>(1ull << 16, (unsigned long long)total_n / 4);
  cap = std::min(cap, vslots);
  rcap = std::min(rcap, 2 * (unsigned long long)total_tiles * kExtMax);
  TiledScratch ts;
  unsigned long long npairs = 0, nroots = 0;
  for (;;) {
    s = reset_status(c);
    if (s != MS_OK) return s;
    s = ensure_buffer(c, &c->tscratch, &c->tscratch_bytes,
                      tiled_scratch_bytes(total_tiles, nf, cap, rcap, b.face_stride));
    if (s != MS_OK) return s;
    tiled_scratch_carve(c->tscratch, total_tiles, nf, cap, rcap, b.face_stride, &ts);
    if (tile_mode(b)) ts.root_tile = nullptr;  // only the flat resolution reads it
    StageTimer t0(c, MS_STAGE_TILE_LOCAL);
    MS_TRY(launch_tile_local(b, ts, c->dst, c->stream));
    t0.stop();
    MS_TRY(cudaMemcpyAsync(c->hcount, ts.counters, 2 * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, c->stream));
    s = read_status(c);
    if (s != MS_OK) return s;
    if (c->hst->nan_flag) return MS_ERR_NAN_INPUT;
    if (c->hst->timeout) return MS_ERR_TIMEOUT;
    npairs = c->hcount[0];
    nroots = c->hcount[1];
    if (!c->hst->pool_overflow) break;
    cap = std::max(cap, npairs);  // exact now
    rcap = std::max(rcap, nroots);
  }
  c->pool_hint = std::max(c->pool_hint, cap);
  c->root_hint = std::max(c->root_hint, rcap);

  // ---- every tile root followed to its extremum: face to face, or, where a
  // sample of the tiles shows long chains (smooth fields), through the face
  // graph, pointer-jumped in O(log) rounds over all face slots
  StageTimer t2(c, MS_STAGE_RESOLVE);
  const long long slots = face_graph_slots(b);
  bool use_graph = false;
  if (nroots >= kProbeMinRoots && slots < (1ll << 31)) {
    const long long stride = std::max<long long>(1, (long long)(nroots / kProbeRoots));
    MS_TRY(cudaMemsetAsync(&c->dst->pending, 0, 2 * sizeof(unsigned int), c->stream));
    MS_TRY(launch_chase_roots(b, ts, nullptr, stride, c->dst, c->stream, nroots));
    s = read_status(c);
    if (s != MS_OK) return s;
    use_graph = (unsigned long long)c->hst->pending * 8 > c->hst->sampled;
  }
  int2 *graph = nullptr;
  if (use_graph) {
    s = ensure_buffer(c, &c->graph, &c->graph_bytes, (size_t)slots * sizeof(int2));
    if (s != MS_OK) return s;
    graph = static_cast<int2 *>(c->graph);
    MS_TRY(launch_face_graph_build(b, ts, graph, c->dst, c->stream));
    s = jump_face_graph(c, b, graph, slots);
    if (s != MS_OK) return s;
    if (c->hst->bad_index) return MS_ERR_CUDA;  // an ill-formed face graph: cannot happen
  }
  MS_TRY(launch_chase_roots(b, ts, graph, 0, c->dst, c->stream, nroots));

  // ---- tile pairs into the global pair set, sized from the last call's
  // region count (or an eighth of the tile pairs), exact on overflow
  const uint64_t exact = 2 * npairs + 2;
  uint64_t want = c->last_k ? 2 * (uint64_t)c->last_k + 4096 : npairs / 8;
  if (want < (1u << 16)) want = 1u << 16;
  if (want > exact) want = exact;
  RankScratch rs;
  for (;;) {
    const unsigned int hcap = pow2_at_least(want);
    s = rank_scratch_ready(c, hcap, &rs);
    if (s != MS_OK) return s;
    if (want < exact) rs.probe_limit = kEstimateProbeLimit;
    MS_TRY(cudaMemsetAsync(&c->dst->n_unique, 0, sizeof(unsigned int), c->stream));
    MS_TRY(cudaMemsetAsync(&c->dst->hash_overflow, 0, sizeof(unsigned int), c->stream));
    MS_TRY(launch_tile_pairs(b, ts, rs, true, c->dst, c->stream, npairs));
    s = read_status(c);
    if (s != MS_OK) return s;
    if (c->hst->not_converged) return MS_ERR_NOT_CONVERGED;
    if (c->hst->bad_index) return MS_ERR_CUDA;  // a chase or a pair out of its tile: cannot happen
    if (!c->hst->hash_overflow) break;
    if (want >= exact) return MS_ERR_CUDA;  // cannot happen: the exact bound always fits
    want = exact;
  }
  const unsigned int m = c->hst->n_unique;
  c->run.npairs = npairs;
  c->run.nroots = nroots;
  c->run.m = m;
  c->run.use_graph = use_graph;
  {
    int raw = 0;
    const int kb = pair_key_bits(sf, &raw);
    MS_TRY(launch_pairs_sort(rs, m, kb, c->stream, raw));
  }
  MS_TRY(launch_pairs_assign(rs, m, c->stream));
  MS_TRY(launch_field_starts(b, ts, rs, m, c->stream));
  t2.stop();
  StageTimer t3(c, MS_STAGE_WRITE);
  MS_TRY(launch_tile_write(b, ts, rs, c->dst, c->stream));
  t3.stop();
  if (key_mode == kKeyBatch) {
    uint32_t *hf = reinterpret_cast<uint32_t *>(c->batch_host);  // reuse the staging buffer
    MS_TRY(cudaMemcpyAsync(hf, ts.fstart, (size_t)nf * 4, cudaMemcpyDeviceToHost, c->stream));
    MS_TRY(cudaStreamSynchronize(c->stream));
    for (int j = 0; j < nf; ++j) {
      const uint32_t end = j + 1 < nf ? hf[j + 1] : m;
      if (k_out) k_out[order[j]] = (int64_t)(end - hf[j]);
    }
  } else {
    if (k_out) k_out[0] = m;
  }
  s = read_status(c);  // synchronises; a sort wait that gave up left the labels unwritten
  if (s != MS_OK) return s;
  if (c->hst->timeout) return MS_ERR_TIMEOUT;
  c->last_k = m;
  return MS_OK;
}

ms_status segment_staged(ms_ctx *c, const void *field, const int64_t dims[3], int dtype,
                         int64_t n, int32_t *asc, int32_t *desc, int32_t *ms);

// 2D grids (nz = 1) take the tiled path with 2D tiles, grids at least
// kTZ / 2 planes deep the tiled path with 3D tiles; the few planes in
// between would leave most of every 32 x 16 x 16 tile empty, so they take
// the step-by-step path.
bool tiled_shape(const int64_t dims[3]) { return dims[2] == 1 || dims[2] >= kTZ / 2; }

ms_status run_batch(ms_ctx *c, const FieldArg *fa, int nf, int64_t *k_out);

ms_status segment_device(ms_ctx *c, const void *field, const int64_t dims[3], int dtype,
                         int64_t n, int32_t *asc, int32_t *desc, int32_t *ms) {
  if (tiled_shape(dims)) {
    const FieldArg fa{field, dims, dtype, n, asc, desc, ms};
    int64_t k = 0;
    const ms_status s = run_batch(c, &fa, 1, &k);
    if (s == MS_OK) c->last_k = k;
    return s;
  }
  return segment_staged(c, field, dims, dtype, n, asc, desc, ms);
}

ms_status segment_staged(ms_ctx *c, const void *field, const int64_t dims[3], int dtype,
                         int64_t n, int32_t *asc, int32_t *desc, int32_t *ms) {
  ms_status s = reset_status(c);
  if (s != MS_OK) return s;
  // up is built in place in desc and dn in asc: after compression each holds
  // the extremum its integral line reaches.
  StageTimer t0(c, MS_STAGE_TILE_LOCAL);
  MS_TRY(launch_steepest_simple(field, dims, dtype, desc, asc, c->dst, c->stream));
  t0.stop();
  StageTimer t1(c, MS_STAGE_RESOLVE);
  s = compress_pair(c, desc, asc, n);  // also reads the status block back
  t1.stop();
  if (c->hst->nan_flag) return MS_ERR_NAN_INPUT;
  if (s != MS_OK) return s;
  const uint64_t nmax = c->hst->n_max, nmin = c->hst->n_min;
  uint64_t bound = nmin * nmax;
  if (bound > (uint64_t)n) bound = (uint64_t)n;
  const uint64_t guess = 8 * (nmin + nmax) + 1024;
  StageTimer t2(c, MS_STAGE_WRITE);
  s = rank_pairs(c, asc, desc, n, ms, guess, bound);
  t2.stop();
  return s;
}

// Checks a field table and converts it; *batchable: the fields can share the
// tiled path's launches.
ms_status batch_args(int n_fields, const void *const *fields, const int64_t (*dims)[3],
                     const ms_dtype *dtypes, int32_t *const *asc, int32_t *const *desc,
                     int32_t *const *ms, std::vector<FieldArg> *out, bool *batchable) {
  if (n_fields < 0 || (n_fields > 0 && (!fields || !dims || !dtypes || !asc || !desc || !ms)))
    return MS_ERR_INVALID_ARG;
  std::vector<FieldArg> &fa = *out;
  fa.assign((size_t)n_fields, FieldArg{});
  *batchable = n_fields <= kBatchMaxFields;
  for (int f = 0; f < n_fields; ++f) {
    int64_t n = 0;
    ms_status s = check_dims(dims[f], &n);
    if (s != MS_OK) return s;
    s = check_dtype(dtypes[f]);
    if (s != MS_OK) return s;
    if (!is_device_pointer(fields[f]) || !is_device_pointer(asc[f]) || !is_device_pointer(desc[f]) ||
        !is_device_pointer(ms[f]))
      return MS_ERR_INVALID_ARG;
    if (asc[f] == desc[f] || asc[f] == ms[f] || desc[f] == ms[f]) return MS_ERR_INVALID_ARG;
    fa[f] = FieldArg{fields[f], dims[f], (int)dtypes[f], n, asc[f], desc[f], ms[f]};
    *batchable = *batchable && n <= kBatchMaxN && tiled_shape(dims[f]);
  }
  return MS_OK;
}

// ---- repeated batches: graph capture and replay --------------------------

std::vector<int64_t> batch_signature(const FieldArg *fa, int nf) {
  std::vector<int64_t> sig;
  sig.reserve(1 + (size_t)nf * 8);
  sig.push_back(nf);
  for (int f = 0; f < nf; ++f) {
    const FieldArg &a = fa[f];
    sig.insert(sig.end(), {(int64_t)(intptr_t)a.field, a.dims[0], a.dims[1], a.dims[2], a.dtype,
                           (int64_t)(intptr_t)a.asc, (int64_t)(intptr_t)a.desc,
                           (int64_t)(intptr_t)a.ms});
  }
  return sig;
}

void drop_graph(BatchPlan *p) {
  if (p->exec) cudaGraphExecDestroy(p->exec);
  p->exec = nullptr;
  p->epoch = -1;
}

void reset_plan(BatchPlan *p) {
  drop_graph(p);
  if (p->host_desc) cudaFreeHost(p->host_desc);
  if (p->hfstart) cudaFreeHost(p->hfstart);
  *p = BatchPlan{};
}

// Capture the whole tiled pipeline for these fields as one CUDA graph, sized
// from the step-by-step call that just ran (c->run) with margins; nothing in
// it reads back to the host but the final status block and field starts.
ms_status capture_plan(ms_ctx *c, BatchPlan &P, const FieldArg *fa, int nf) {
  drop_graph(&P);
  Staged sf;
  const Tuning tune = P.tuned ? P.tune : c->tune;
  ms_status s = stage_fields(c, fa, nf, tune.shape3, &sf);  // also leaves the descriptors on the device
  if (s != MS_OK) return s;
  Batch b = sf.b;
  b.tune = tune;
  const RunInfo run = c->run;
  // capacities: the sizes met, with margins; overflow is detected on the device
  unsigned long long pool_cap = run.npairs + run.npairs / 8 + 4096;
  pool_cap = std::min(pool_cap, (unsigned long long)b.total_tiles * kPidStride);
  unsigned long long root_cap = run.nroots + run.nroots / 8 + 4096;
  root_cap = std::min(root_cap, 2 * (unsigned long long)b.total_tiles * kExtMax);
  const unsigned int hcap = pow2_at_least(2ull * run.m + 4096);
  s = ensure_buffer(c, &c->tscratch, &c->tscratch_bytes,
                    tiled_scratch_bytes(b.total_tiles, nf, pool_cap, root_cap, b.face_stride));
  if (s != MS_OK) return s;
  RankScratch rs;
  s = rank_scratch_ready(c, hcap, &rs);
  if (s != MS_OK) return s;
  const long long slots = face_graph_slots(b);
  int2 *graph = nullptr;
  if (run.use_graph) {
    s = ensure_buffer(c, &c->graph, &c->graph_bytes, (size_t)slots * sizeof(int2));
    if (s != MS_OK) return s;
    graph = static_cast<int2 *>(c->graph);
  }
  TiledScratch ts;
  tiled_scratch_carve(c->tscratch, b.total_tiles, nf, pool_cap, root_cap, b.face_stride, &ts);
  if (tile_mode(b)) ts.root_tile = nullptr;
  if ((uint64_t)hcap < 2 * run.npairs + 2) rs.probe_limit = kEstimateProbeLimit;
  // the sort and rank launches are sized for this many distinct pairs; more
  // of them overflow the list on the device and the call runs step by step
  rs.max_unique = (unsigned int)std::min<uint64_t>(rs.max_unique, run.m + run.m / 4 + 4096);
  // pinned copies the graph reads from and writes to
  if (P.host_desc_bytes < sf.bytes) {
    if (P.host_desc) cudaFreeHost(P.host_desc);
    P.host_desc = nullptr;
    P.host_desc_bytes = 0;
    MS_TRY(cudaMallocHost(&P.host_desc, sf.bytes));
    P.host_desc_bytes = sf.bytes;
  }
  memcpy(P.host_desc, c->batch_host, sf.bytes);
  if (P.hfstart_count < (size_t)nf) {
    if (P.hfstart) cudaFreeHost(P.hfstart);
    P.hfstart = nullptr;
    P.hfstart_count = 0;
    MS_TRY(cudaMallocHost(reinterpret_cast<void **>(&P.hfstart), (size_t)nf * 4));
    P.hfstart_count = (size_t)nf;
  }
  P.order = sf.order;
  for (int i = 0; i < MS_STAGE_COUNT; ++i)  // the graph records the stage events
    for (int j = 0; j < 2; ++j)
      if (!c->ev[i][j]) MS_TRY(cudaEventCreate(&c->ev[i][j]));
  int raw = 0;
  const int kb = pair_key_bits(sf, &raw);
  const int rounds = std::max(3, run.rounds + 1);
  MS_TRY(cudaStreamSynchronize(c->stream));

  const long long l0 = tl_launches;
  MS_TRY(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
  auto enqueue = [&]() -> cudaError_t {
    cudaError_t e;
    // the descriptors, in case another call on this context replaced them
    if ((e = cudaMemcpyAsync(c->batch_dev, P.host_desc, sf.bytes, cudaMemcpyHostToDevice,
                             c->stream)) != cudaSuccess)
      return e;
    if ((e = cudaMemsetAsync(c->dst, 0, sizeof(DevStatus), c->stream)) != cudaSuccess) return e;
    // stage events as record nodes of the graph (external records; a plain
    // record during capture only orders the capture): a replay times its
    // stages like a call
    long long lc = tl_launches;
    if ((e = cudaEventRecordWithFlags(c->ev[MS_STAGE_TILE_LOCAL][0], c->stream, cudaEventRecordExternal)) != cudaSuccess) return e;
    if ((e = launch_tile_local(b, ts, c->dst, c->stream)) != cudaSuccess) return e;
    if ((e = cudaEventRecordWithFlags(c->ev[MS_STAGE_TILE_LOCAL][1], c->stream, cudaEventRecordExternal)) != cudaSuccess) return e;
    P.stage_launches[0] = tl_launches - lc;
    lc = tl_launches;
    if ((e = cudaEventRecordWithFlags(c->ev[MS_STAGE_RESOLVE][0], c->stream, cudaEventRecordExternal)) != cudaSuccess) return e;
    if (run.use_graph) {
      if ((e = launch_face_graph_build(b, ts, graph, c->dst, c->stream)) != cudaSuccess) return e;
      if ((e = launch_face_graph_rounds(b, graph, 0, rounds, c->dst, c->stream)) != cudaSuccess)
        return e;
    }
    if ((e = launch_chase_roots(b, ts, graph, 0, c->dst, c->stream)) != cudaSuccess) return e;
    if ((e = launch_tile_pairs(b, ts, rs, true, c->dst, c->stream)) != cudaSuccess) return e;
    if ((e = launch_pairs_sort(rs, rs.max_unique, kb, c->stream, raw, &c->dst->n_unique)) !=
        cudaSuccess)
      return e;
    if ((e = launch_pairs_assign(rs, rs.max_unique, c->stream, &c->dst->n_unique)) != cudaSuccess)
      return e;
    if ((e = launch_field_starts(b, ts, rs, rs.max_unique, c->stream, &c->dst->n_unique)) !=
        cudaSuccess)
      return e;
    if ((e = cudaEventRecordWithFlags(c->ev[MS_STAGE_RESOLVE][1], c->stream, cudaEventRecordExternal)) != cudaSuccess) return e;
    P.stage_launches[1] = tl_launches - lc;
    lc = tl_launches;
    if ((e = cudaEventRecordWithFlags(c->ev[MS_STAGE_WRITE][0], c->stream, cudaEventRecordExternal)) != cudaSuccess) return e;
    if ((e = launch_tile_write(b, ts, rs, c->dst, c->stream)) != cudaSuccess) return e;
    if ((e = cudaEventRecordWithFlags(c->ev[MS_STAGE_WRITE][1], c->stream, cudaEventRecordExternal)) != cudaSuccess) return e;
    P.stage_launches[2] = tl_launches - lc;
    if ((e = cudaMemcpyAsync(c->hst, c->dst, sizeof(DevStatus), cudaMemcpyDeviceToHost,
                             c->stream)) != cudaSuccess)
      return e;
    if (b.key_mode == kKeyBatch)
      e = cudaMemcpyAsync(P.hfstart, ts.fstart, (size_t)nf * 4, cudaMemcpyDeviceToHost, c->stream);
    return e;
  };
  const cudaError_t qe = enqueue();
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
  tl_launches = l0;  // capture launches nothing
  if (qe != cudaSuccess || ce != cudaSuccess || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    return MS_ERR_CUDA;
  }
  // kernel nodes per replay
  size_t nn = 0;
  cudaGraphGetNodes(g, nullptr, &nn);
  std::vector<cudaGraphNode_t> nodes(nn);
  cudaGraphGetNodes(g, nodes.data(), &nn);
  long long kernels = 0;
  for (cudaGraphNode_t n : nodes) {
    cudaGraphNodeType t;
    if (cudaGraphNodeGetType(n, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++kernels;
  }
  const cudaError_t ie = cudaGraphInstantiate(&P.exec, g, 0);
  cudaGraphDestroy(g);
  if (ie != cudaSuccess) {
    P.exec = nullptr;
    cudaGetLastError();
    return MS_ERR_CUDA;
  }
  P.launches = kernels;
  P.epoch = c->alloc_epoch;
  return MS_OK;
}

// Replay the captured pipeline.  *fallback: the sizes it was captured with no
// longer suffice (the caller runs the call step by step).
ms_status replay_plan(ms_ctx *c, BatchPlan &P, int nf, int64_t *k_out, bool *fallback) {
  *fallback = false;
  if (c->prof_on) cudaEventRecord(c->ev[MS_STAGE_GRAPH][0], c->stream);
  MS_TRY(cudaGraphLaunch(P.exec, c->stream));
  if (c->prof_on) {
    cudaEventRecord(c->ev[MS_STAGE_GRAPH][1], c->stream);
    c->ev_pending[MS_STAGE_GRAPH] = true;
    c->prof.stage_launches[MS_STAGE_GRAPH] += P.launches;
    const int st3[3] = {MS_STAGE_TILE_LOCAL, MS_STAGE_RESOLVE, MS_STAGE_WRITE};
    for (int i = 0; i < 3; ++i) {  // the graph recorded these stages' events
      c->ev_pending[st3[i]] = true;
      c->prof.stage_launches[st3[i]] += P.stage_launches[i];
    }
  }
  tl_launches += P.launches;
  MS_TRY(cudaStreamSynchronize(c->stream));
  const DevStatus &h = *c->hst;
  if (h.nan_flag) return MS_ERR_NAN_INPUT;
  if (h.timeout) return MS_ERR_TIMEOUT;
  if (h.pool_overflow || h.hash_overflow || h.not_converged || h.bad_index) {
    *fallback = true;
    return MS_OK;
  }
  const unsigned int m = h.n_unique;
  if (nf > 1) {
    for (int j = 0; j < nf; ++j) {
      const uint32_t end = j + 1 < nf ? P.hfstart[j + 1] : m;
      k_out[P.order[j]] = (int64_t)(end - P.hfstart[j]);
    }
  } else {
    k_out[0] = m;
  }
  c->last_k = m;
  return MS_OK;
}

// A batch through the tiled path: replayed from its graph when the same fields
// come again, else step by step (then captured for the next time).
// The plan of these fields: the slot holding their signature, else the older
// slot, reset for them (two buffer sets alternating -- ms_segment_host_many --
// keep both captured).
BatchPlan &plan_of(ms_ctx *c, std::vector<int64_t> sig) {
  for (BatchPlan &P : c->plans)
    if (P.sig == sig) return P;
  BatchPlan &P = c->plans[c->plan_next];
  c->plan_next ^= 1;
  reset_plan(&P);
  P.sig = std::move(sig);
  return P;
}

ms_status run_batch(ms_ctx *c, const FieldArg *fa, int nf, int64_t *k_out) {
  BatchPlan &P = plan_of(c, batch_signature(fa, nf));
  ++P.seen;
  if (c->graphs_on && P.exec && P.epoch == c->alloc_epoch) {
    bool fallback = false;
    const ms_status s = replay_plan(c, P, nf, k_out, &fallback);
    if (s != MS_OK || !fallback) return s;
    drop_graph(&P);
  }
  const ms_status s = segment_tiled(c, fa, nf, k_out, P.tuned ? P.tune : c->tune);
  if (s != MS_OK) return s;
  // capture once the same fields come a second time (one-off calls never pay for it)
  if (c->graphs_on && !P.exec && P.seen >= 2 && capture_plan(c, P, fa, nf) != MS_OK) drop_graph(&P);
  return MS_OK;
}

}  // namespace

namespace msseg {

size_t ctx_resident_bytes(const ms_ctx *c) {
  return c->scratch_bytes + c->io_bytes + c->io2_bytes + c->tscratch_bytes + c->graph_bytes +
         c->sxscratch_bytes + c->pscratch_bytes + c->slscratch_bytes + c->slmap_bytes +
         c->batch_dev_bytes + sizeof(DevStatus);
}

void ctx_release_scratch(ms_ctx *c) {
  DeviceGuard g(c->device);
  cudaStreamSynchronize(c->stream);
  for (BatchPlan &P : c->plans) drop_graph(&P);
  void **bufs[] = {&c->scratch, &c->io,       &c->io2,    &c->tscratch, &c->graph,
                   &c->sxscratch, &c->pscratch, &c->slscratch, &c->slmap, &c->batch_dev};
  size_t *sizes[] = {&c->scratch_bytes,   &c->io_bytes,        &c->io2_bytes,
                     &c->tscratch_bytes,  &c->graph_bytes,     &c->sxscratch_bytes,
                     &c->pscratch_bytes,  &c->slscratch_bytes, &c->slmap_bytes,
                     &c->batch_dev_bytes};
  for (int i = 0; i < 10; ++i) {
    if (*bufs[i]) cudaFree(*bufs[i]);
    *bufs[i] = nullptr;
    *sizes[i] = 0;
  }
  ++c->alloc_epoch;
  cudaGetLastError();
}

}  // namespace msseg

extern "C" {

const char *ms_status_string(ms_status s) {
  switch (s) {
    case MS_OK: return "MS_OK";
    case MS_ERR_INVALID_ARG: return "MS_ERR_INVALID_ARG";
    case MS_ERR_UNSUPPORTED_DTYPE: return "MS_ERR_UNSUPPORTED_DTYPE";
    case MS_ERR_TOO_LARGE: return "MS_ERR_TOO_LARGE";
    case MS_ERR_NAN_INPUT: return "MS_ERR_NAN_INPUT";
    case MS_ERR_OUT_OF_MEMORY: return "MS_ERR_OUT_OF_MEMORY";
    case MS_ERR_CUDA: return "MS_ERR_CUDA";
    case MS_ERR_NOT_CONVERGED: return "MS_ERR_NOT_CONVERGED";
    case MS_ERR_TIMEOUT: return "MS_ERR_TIMEOUT";
    case MS_ERR_BUSY: return "MS_ERR_BUSY";
  }
  return "MS_ERR_UNKNOWN";
}

ms_status ms_create(ms_ctx **out, int device, void *cuda_stream) {
  if (!out) return MS_ERR_INVALID_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return MS_ERR_CUDA;
  }
  if (device < 0 || device >= ndev) return MS_ERR_INVALID_ARG;
  DeviceGuard g(device);
  ms_ctx *c = new (std::nothrow) ms_ctx();
  if (!c) return MS_ERR_OUT_OF_MEMORY;
  c->device = device;
  ms_status s = MS_OK;
  if (cuda_stream) {
    c->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    s = cuda_status(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    c->own_stream = s == MS_OK;
  }
  if (s == MS_OK) s = cuda_status(cudaMalloc(&c->dst, sizeof(DevStatus)));
  if (s == MS_OK) s = cuda_status(cudaMallocHost(&c->hst, sizeof(DevStatus)));
  if (s == MS_OK) s = cuda_status(cudaMallocHost(&c->hcount, 2 * sizeof(unsigned long long)));
  if (s != MS_OK) {
    ms_destroy(c);
    return s;
  }
  *out = c;
  return MS_OK;
}

ms_status ms_destroy(ms_ctx *c) {
  if (!c) return MS_OK;
  DeviceGuard g(c->device);
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->scratch) cudaFree(c->scratch);
  if (c->io) cudaFree(c->io);
  if (c->tscratch) cudaFree(c->tscratch);
  if (c->graph) cudaFree(c->graph);
  if (c->sxscratch) cudaFree(c->sxscratch);
  if (c->pscratch) cudaFree(c->pscratch);
  if (c->slscratch) cudaFree(c->slscratch);
  if (c->slmap) cudaFree(c->slmap);
  if (c->pcount) cudaFreeHost(c->pcount);
  if (c->batch_dev) cudaFree(c->batch_dev);
  if (c->batch_host) cudaFreeHost(c->batch_host);
  if (c->hcount) cudaFreeHost(c->hcount);
  if (c->dst) cudaFree(c->dst);
  if (c->hst) cudaFreeHost(c->hst);
  for (int i = 0; i < MS_STAGE_COUNT; ++i)
    for (int j = 0; j < 2; ++j)
      if (c->ev[i][j]) cudaEventDestroy(c->ev[i][j]);
  for (int i = 0; i < 2; ++i) {
    if (c->ev_up[i]) cudaEventDestroy(c->ev_up[i]);
    if (c->ev_comp[i]) cudaEventDestroy(c->ev_comp[i]);
    if (c->ev_down[i]) cudaEventDestroy(c->ev_down[i]);
  }
  if (c->up) cudaStreamDestroy(c->up);
  if (c->down) cudaStreamDestroy(c->down);
  if (c->io2) cudaFree(c->io2);
  for (BatchPlan &P : c->plans) reset_plan(&P);
  if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
  delete c;
  return MS_OK;
}

ms_status ms_last_region_count(const ms_ctx *c, int64_t *k) {
  if (!c || !k) return MS_ERR_INVALID_ARG;
  *k = c->last_k;
  return MS_OK;
}

ms_status ms_segment(ms_ctx *c, const void *field, const int64_t dims[3], ms_dtype dtype,
                     int32_t *out_asc, int32_t *out_desc, int32_t *out_ms) {
  if (!c) return MS_ERR_INVALID_ARG;
  int64_t n = 0;
  ms_status s = check_dims(dims, &n);
  if (s != MS_OK) return s;
  s = check_dtype(dtype);
  if (s != MS_OK) return s;
  DeviceGuard g(c->device);
  if (!is_device_pointer(field) || !is_device_pointer(out_asc) || !is_device_pointer(out_desc) ||
      !is_device_pointer(out_ms))
    return MS_ERR_INVALID_ARG;
  if (out_asc == out_desc || out_asc == out_ms || out_desc == out_ms) return MS_ERR_INVALID_ARG;
  const long long l0 = tl_launches;
  s = segment_device(c, field, dims, dtype, n, out_asc, out_desc, out_ms);
  if (s == MS_OK) finish_profile(c, l0);
  return s;
}

ms_status ms_segment_staged(ms_ctx *c, const void *field, const int64_t dims[3], ms_dtype dtype,
                            int32_t *out_asc, int32_t *out_desc, int32_t *out_ms) {
  if (!c) return MS_ERR_INVALID_ARG;
  int64_t n = 0;
  ms_status s = check_dims(dims, &n);
  if (s != MS_OK) return s;
  s = check_dtype(dtype);
  if (s != MS_OK) return s;
  DeviceGuard g(c->device);
  if (!is_device_pointer(field) || !is_device_pointer(out_asc) || !is_device_pointer(out_desc) ||
      !is_device_pointer(out_ms))
    return MS_ERR_INVALID_ARG;
  if (out_asc == out_desc || out_asc == out_ms || out_desc == out_ms) return MS_ERR_INVALID_ARG;
  const long long l0 = tl_launches;
  s = segment_staged(c, field, dims, dtype, n, out_asc, out_desc, out_ms);
  if (s == MS_OK) finish_profile(c, l0);
  return s;
}

ms_status ms_segment_batch(ms_ctx *c, int n_fields, const void *const *fields,
                           const int64_t (*dims)[3], const ms_dtype *dtypes, int32_t *const *asc,
                           int32_t *const *desc, int32_t *const *ms, int64_t *k_out) {
  if (!c || n_fields < 0) return MS_ERR_INVALID_ARG;
  if (n_fields == 0) return MS_OK;
  DeviceGuard g(c->device);
  std::vector<FieldArg> fa;
  bool batchable = false;
  {
    const ms_status s = batch_args(n_fields, fields, dims, dtypes, asc, desc, ms, &fa, &batchable);
    if (s != MS_OK) return s;
  }
  const long long l0 = tl_launches;
  ms_status s = MS_OK;
  int64_t total_k = 0;
  if (batchable) {
    std::vector<int64_t> k((size_t)n_fields, 0);
    s = run_batch(c, fa.data(), n_fields, k.data());
    for (int f = 0; f < n_fields && s == MS_OK; ++f) {
      if (k_out) k_out[f] = k[f];
      total_k += k[f];
    }
  } else {
    for (int f = 0; f < n_fields && s == MS_OK; ++f) {
      s = segment_device(c, fa[f].field, fa[f].dims, fa[f].dtype, fa[f].n, fa[f].asc, fa[f].desc,
                         fa[f].ms);
      if (s == MS_OK) {
        if (k_out) k_out[f] = c->last_k;
        total_k += c->last_k;
      }
    }
  }
  if (s == MS_OK) {
    c->last_k = total_k;
    finish_profile(c, l0);
  }
  return s;
}

ms_status ms_simplex_index(ms_ctx *c, const int32_t *labels, const int64_t dims[3], int mode,
                           uint8_t *codes, int64_t *cell_offsets, int64_t *total) {
  if (!c || !labels || (mode != 0 && mode != 1)) return MS_ERR_INVALID_ARG;
  int64_t n = 0;
  ms_status s = check_dims(dims, &n);
  if (s != MS_OK) return s;
  DeviceGuard g(c->device);
  const bool flat = dims[2] == 1;
  const int64_t cz = flat ? 1 : dims[2] - 1;
  const int64_t cells = (dims[0] > 1 && dims[1] > 1 && cz > 0) ? (dims[0] - 1) * (dims[1] - 1) * cz : 0;
  if (cells == 0) {
    if (total) *total = 0;
    return MS_OK;
  }
  if (!is_device_pointer(labels) || !is_device_pointer(codes) || !is_device_pointer(cell_offsets))
    return MS_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(codes) & 15) || (reinterpret_cast<uintptr_t>(cell_offsets) & 7))
    return MS_ERR_INVALID_ARG;
  s = ensure_buffer(c, &c->sxscratch, &c->sxscratch_bytes, simplex_scratch_bytes(cells));
  if (s != MS_OK) return s;
  const long long l0 = tl_launches;
  unsigned long long *tot_dev = nullptr;
  int64_t nc = 0;
  s = reset_status(c);
  if (s != MS_OK) return s;
  StageTimer t0(c, MS_STAGE_TILE_LOCAL);
  MS_TRY(launch_simplex_index(labels, dims, mode, codes, cell_offsets, c->sxscratch, &tot_dev, &nc,
                              c->dst, c->stream));
  t0.stop();
  MS_TRY(cudaMemcpyAsync(c->hcount, tot_dev, sizeof(unsigned long long), cudaMemcpyDeviceToHost,
                         c->stream));
  s = read_status(c);  // synchronises the stream
  if (s != MS_OK) return s;
  if (c->hst->timeout) return MS_ERR_TIMEOUT;
  if (total) *total = (int64_t)*c->hcount;
  finish_profile(c, l0);
  return MS_OK;
}

ms_status ms_simplex_geometry(ms_ctx *c, const int32_t *labels, const int64_t dims[3], int mode,
                              const int64_t *cell_offsets, int64_t total, float *points,
                              int32_t *pairs) {
  if (!c || !labels || (mode != 0 && mode != 1) || total < 0) return MS_ERR_INVALID_ARG;
  int64_t n = 0;
  ms_status s = check_dims(dims, &n);
  if (s != MS_OK) return s;
  DeviceGuard g(c->device);
  const bool flat = dims[2] == 1;
  const int64_t cz = flat ? 1 : dims[2] - 1;
  const int64_t cells = (dims[0] > 1 && dims[1] > 1 && cz > 0) ? (dims[0] - 1) * (dims[1] - 1) * cz : 0;
  if (cells == 0) return total == 0 ? MS_OK : MS_ERR_INVALID_ARG;
  if (!is_device_pointer(labels) || !is_device_pointer(cell_offsets) ||
      (total > 0 && !is_device_pointer(points)) || (pairs && !is_device_pointer(pairs)))
    return MS_ERR_INVALID_ARG;
  if ((reinterpret_cast<uintptr_t>(points) & 3) || (reinterpret_cast<uintptr_t>(pairs) & 3) ||
      (reinterpret_cast<uintptr_t>(cell_offsets) & 7))
    return MS_ERR_INVALID_ARG;
  const long long l0 = tl_launches;
  s = reset_status(c);
  if (s != MS_OK) return s;
  StageTimer t0(c, MS_STAGE_WRITE);
  MS_TRY(launch_simplex_geometry(labels, dims, mode, cell_offsets, total, points, pairs, c->dst,
                                 c->stream));
  t0.stop();
  s = read_status(c);
  if (s != MS_OK) return s;
  if (c->hst->bad_index) return MS_ERR_INVALID_ARG;  // offsets or total do not match the labels
  finish_profile(c, l0);
  return MS_OK;
}

ms_status ms_persistence(ms_ctx *c, const void *field, const int64_t dims[3], ms_dtype dtype,
                         const int32_t *labels, int direction, int32_t *extremum, int32_t *death,
                         int64_t capacity, ms_persistence_info *info) {
  if (!c || !field || !labels || (direction != 1 && direction != -1) || capacity < 0)
    return MS_ERR_INVALID_ARG;
  int64_t n = 0;
  ms_status s = check_dims(dims, &n);
  if (s != MS_OK) return s;
  s = check_dtype(dtype);
  if (s != MS_OK) return s;
  DeviceGuard g(c->device);
  if (!is_device_pointer(field) || !is_device_pointer(labels)) return MS_ERR_INVALID_ARG;
  if (capacity > 0 && (!is_device_pointer(extremum) || !is_device_pointer(death)))
    return MS_ERR_INVALID_ARG;
  const uintptr_t align = dtype == MS_F16 ? 1 : 3;
  if ((reinterpret_cast<uintptr_t>(field) & align) || (reinterpret_cast<uintptr_t>(labels) & 3) ||
      (reinterpret_cast<uintptr_t>(extremum) & 3) || (reinterpret_cast<uintptr_t>(death) & 3))
    return MS_ERR_INVALID_ARG;
  if (!c->pcount) {
    if (cudaMallocHost(&c->pcount, persist_counters_bytes()) != cudaSuccess) {
      cudaGetLastError();
      return MS_ERR_OUT_OF_MEMORY;
    }
  }
  // capacities: first from the last call (within this field's bounds), else
  // from the field's size; grown by 4x while a pass reports them full
  const uint64_t pair_bound = std::min<uint64_t>(1ull << 30, (uint64_t)n * (dims[2] > 1 ? 7 : 3));
  const uint64_t min_bound = (uint64_t)n;
  uint64_t pairs = std::max<uint64_t>(c->pers_pairs_hint, std::max<int64_t>(4096, n / 32));
  uint64_t minima = std::max<uint64_t>(c->pers_minima_hint, std::max<int64_t>(1024, n / 32));
  pairs = std::max<uint64_t>(1, std::min(pairs, pair_bound));
  minima = std::max<uint64_t>(1, std::min(minima, min_bound));
  const long long l0 = tl_launches;
  for (;;) {
    s = ensure_buffer(c, &c->pscratch, &c->pscratch_bytes, persist_scratch_bytes(pairs, minima));
    if (s != MS_OK) return s;
    PersistCall P{};
    P.field = field;
    P.dtype = dtype;
    P.labels = labels;
    for (int i = 0; i < 3; ++i) P.dims[i] = dims[i];
    P.n = n;
    P.direction = direction;
    P.extremum = extremum;
    P.death = death;
    P.capacity = capacity;
    P.max_pairs = pairs;
    P.max_minima = minima;
    P.min_rounds = 4;
    PersistOutcome o;
    StageTimer t0(c, MS_STAGE_RESOLVE);
    MS_TRY(persist_run(P, c->pscratch, c->pcount, c->stream, &o));
    t0.stop();
    switch (o.kind) {
      case PersistOutcome::kNan:
        return MS_ERR_NAN_INPUT;
      case PersistOutcome::kBadLabels:
        return MS_ERR_INVALID_ARG;
      case PersistOutcome::kGrow:
        if (o.n_minima > minima) minima = std::min(min_bound, std::max(minima * 4, o.n_minima));
        if (o.pairs_full) {
          if (pairs >= pair_bound) return MS_ERR_TOO_LARGE;
          pairs = std::min(pair_bound, std::max(pairs * 4, o.n_pairs));
        }
        continue;
      case PersistOutcome::kTooSmall:
        if (info) {
          *info = ms_persistence_info{};
          info->n_extrema = (int64_t)o.n_minima;
          info->basin_edges = (int64_t)o.n_pairs;
        }
        return MS_ERR_TOO_LARGE;
      case PersistOutcome::kDone:
        break;
    }
    c->pers_pairs_hint = pairs;
    c->pers_minima_hint = minima;
    if (info) {
      *info = ms_persistence_info{};
      info->n_extrema = (int64_t)o.n_minima;
      info->basin_edges = (int64_t)o.n_pairs;
      info->rounds = o.rounds;
      info->finish_edges = (int64_t)o.finish_edges;
    }
    finish_profile(c, l0);
    return MS_OK;
  }
}

ms_status ms_slab_local(ms_ctx *c, const void *field, const int64_t dims[3], ms_dtype dtype,
                        int64_t z0, int64_t z1, int32_t *out_asc, int32_t *out_desc) {
  if (!c || !field || !out_asc || !out_desc || out_asc == out_desc) return MS_ERR_INVALID_ARG;
  int64_t n = 0;
  ms_status s = check_dims(dims, &n);
  if (s != MS_OK) return s;
  s = check_dtype(dtype);
  if (s != MS_OK) return s;
  if (z0 < 0 || z1 <= z0 || z1 > dims[2]) return MS_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  if (!is_device_pointer(field) || !is_device_pointer(out_asc) || !is_device_pointer(out_desc))
    return MS_ERR_INVALID_ARG;
  const int64_t nxy = dims[0] * dims[1];
  const int64_t lo = z0 > 0 ? 1 : 0, hi = z1 < dims[2] ? 1 : 0, owned = z1 - z0;
  const int64_t ext_dims[3] = {dims[0], dims[1], owned + lo + hi};
  const int64_t n_ext = ext_dims[2] * nxy;
  s = ensure_buffer(c, &c->slscratch, &c->slscratch_bytes, (size_t)n_ext * 8);
  if (s != MS_OK) return s;
  int32_t *up = static_cast<int32_t *>(c->slscratch), *dn = up + n_ext;
  const long long l0 = tl_launches;
  s = reset_status(c);
  if (s != MS_OK) return s;
  StageTimer t0(c, MS_STAGE_TILE_LOCAL);
  MS_TRY(launch_steepest_simple(field, ext_dims, dtype, up, dn, c->dst, c->stream));
  MS_TRY(launch_slab_halo_self(up, dn, nxy, lo, owned, hi, c->stream));
  t0.stop();
  StageTimer t1(c, MS_STAGE_RESOLVE);
  s = compress_pair(c, up, dn, n_ext);  // also reads the status block back
  t1.stop();
  if (c->hst->nan_flag) return MS_ERR_NAN_INPUT;
  if (s != MS_OK) return s;
  MS_TRY(launch_slab_encode(up, dn, nxy, lo, owned, (z0 - lo) * nxy, out_asc, out_desc, c->stream));
  MS_TRY(cudaStreamSynchronize(c->stream));
  finish_profile(c, l0);
  return MS_OK;
}

ms_status ms_slab_resolve(ms_ctx *c, const int64_t dims[3], int32_t *rows, const int64_t *plane_z,
                          int n_planes, int32_t *asc, int32_t *desc, int64_t n_owned) {
  if (!c || n_planes < 0 || n_owned < 0 || (n_planes > 0 && (!rows || !plane_z)) ||
      (n_owned > 0 && (!asc || !desc)))
    return MS_ERR_INVALID_ARG;
  int64_t n = 0;
  ms_status s = check_dims(dims, &n);
  if (s != MS_OK) return s;
  DeviceGuard g(c->device);
  if ((n_planes > 0 && !is_device_pointer(rows)) ||
      (n_owned > 0 && (!is_device_pointer(asc) || !is_device_pointer(desc))))
    return MS_ERR_INVALID_ARG;
  const int64_t nxy = dims[0] * dims[1];
  if ((int64_t)n_planes * 2 * nxy > kMaxVertices) return MS_ERR_TOO_LARGE;
  // the planes' z, sorted, each with its row
  std::vector<std::pair<long long, int>> zr((size_t)n_planes);
  for (int i = 0; i < n_planes; ++i) {
    if (plane_z[i] < 0 || plane_z[i] >= dims[2]) return MS_ERR_INVALID_ARG;
    zr[(size_t)i] = {(long long)plane_z[i], i};
  }
  std::sort(zr.begin(), zr.end());
  for (int i = 1; i < n_planes; ++i)
    if (zr[(size_t)i].first == zr[(size_t)i - 1].first) return MS_ERR_INVALID_ARG;
  const size_t zbytes = (size_t)n_planes * 8;
  s = ensure_buffer(c, &c->slmap, &c->slmap_bytes, zbytes + (size_t)n_planes * 4 + 16);
  if (s != MS_OK) return s;
  long long *zs = static_cast<long long *>(c->slmap);
  int *slot = reinterpret_cast<int *>(static_cast<char *>(c->slmap) + zbytes);
  if (n_planes > 0) {
    std::vector<long long> hz((size_t)n_planes);
    std::vector<int> hs((size_t)n_planes);
    for (int i = 0; i < n_planes; ++i) {
      hz[(size_t)i] = zr[(size_t)i].first;
      hs[(size_t)i] = zr[(size_t)i].second;
    }
    MS_TRY(cudaMemcpyAsync(zs, hz.data(), zbytes, cudaMemcpyHostToDevice, c->stream));
    MS_TRY(cudaMemcpyAsync(slot, hs.data(), (size_t)n_planes * 4, cudaMemcpyHostToDevice, c->stream));
  }
  const long long l0 = tl_launches;
  s = reset_status(c);
  if (s != MS_OK) return s;
  StageTimer t0(c, MS_STAGE_RESOLVE);
  // an exit chain visits each row entry at most once: jumping with doubling
  // ends within ceil(log2(entries)) + 2 rounds
  const int cap = n_planes > 0 ? round_cap((int64_t)n_planes * 2 * nxy) : 0;
  for (int r = 0; r < cap; ++r)
    MS_TRY(launch_slab_rows_round(rows, n_planes, nxy, n, zs, slot, c->dst, r, c->stream));
  MS_TRY(launch_slab_apply(asc, desc, n_owned, rows, nxy, n, zs, slot, n_planes, c->dst, c->stream));
  t0.stop();
  s = read_status(c);
  if (s != MS_OK) return s;
  if (c->hst->bad_index) return MS_ERR_INVALID_ARG;
  if (cap > 0 && c->hst->round_open[cap - 1]) return MS_ERR_NOT_CONVERGED;
  finish_profile(c, l0);
  return MS_OK;
}

ms_status ms_slab_pairs(ms_ctx *c, const int32_t *asc, const int32_t *desc, int64_t n,
                        int64_t n_labels, uint64_t *keys, int64_t capacity, int64_t *m) {
  if (!c || n < 0 || capacity < 0 || n_labels < 1 || n_labels > kMaxVertices || n > kMaxVertices ||
      (n > 0 && (!asc || !desc)))
    return MS_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  if (n == 0) {
    if (m) *m = 0;
    return MS_OK;
  }
  if (!is_device_pointer(asc) || !is_device_pointer(desc) || (capacity > 0 && !is_device_pointer(keys)))
    return MS_ERR_INVALID_ARG;
  const long long l0 = tl_launches;
  uint64_t guess = std::min<uint64_t>((uint64_t)n, (uint64_t)n / 16 + 1024);
  for (;;) {
    const unsigned int cap = pow2_at_least(2 * guess + 2);
    RankScratch rs;
    ms_status s = rank_scratch_ready(c, cap, &rs);
    if (s != MS_OK) return s;
    if (guess < (uint64_t)n) rs.probe_limit = kEstimateProbeLimit;
    s = reset_status(c);
    if (s != MS_OK) return s;
    MS_TRY(launch_pairs_insert(asc, desc, n, rs, c->dst, c->stream, n_labels));
    s = read_status(c);
    if (s != MS_OK) return s;
    if (c->hst->bad_index) return MS_ERR_INVALID_ARG;
    if (c->hst->hash_overflow) {
      if (guess >= (uint64_t)n) return MS_ERR_CUDA;  // cannot happen: n is a bound
      guess = std::min<uint64_t>((uint64_t)n, guess * 4);
      continue;
    }
    const unsigned int mu = c->hst->n_unique;
    if (m) *m = mu;
    if ((int64_t)mu > capacity) return MS_ERR_TOO_LARGE;
    MS_TRY(launch_pairs_sort(rs, mu, bit_width(n_labels - 1), c->stream));
    MS_TRY(cudaMemcpyAsync(keys, rs.list, (size_t)mu * 8, cudaMemcpyDeviceToDevice, c->stream));
    s = read_status(c);
    if (s != MS_OK) return s;
    if (c->hst->timeout) return MS_ERR_TIMEOUT;
    finish_profile(c, l0);
    return MS_OK;
  }
}

ms_status ms_slab_rank(ms_ctx *c, const int32_t *asc, const int32_t *desc, int64_t n,
                       int64_t n_labels, const uint64_t *keys, int64_t n_keys, int32_t *ms,
                       int64_t *k) {
  if (!c || n < 0 || n_keys < 0 || n_labels < 1 || n_labels > kMaxVertices || n > kMaxVertices ||
      n_keys > (1ll << 30) || (n > 0 && (!asc || !desc || !ms)) || (n_keys > 0 && !keys))
    return MS_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  if ((n > 0 && (!is_device_pointer(asc) || !is_device_pointer(desc) || !is_device_pointer(ms))) ||
      (n_keys > 0 && !is_device_pointer(keys)))
    return MS_ERR_INVALID_ARG;
  if (n > 0 && n_keys == 0) return MS_ERR_INVALID_ARG;  // the slab's own pairs are missing
  const long long l0 = tl_launches;
  const unsigned int cap = pow2_at_least(2 * (uint64_t)n_keys + 2);
  RankScratch rs;
  ms_status s = rank_scratch_ready(c, cap, &rs);
  if (s != MS_OK) return s;
  s = reset_status(c);
  if (s != MS_OK) return s;
  MS_TRY(launch_keys_insert(reinterpret_cast<const unsigned long long *>(keys), n_keys, n_labels, rs,
                            c->dst, c->stream));
  s = read_status(c);
  if (s != MS_OK) return s;
  if (c->hst->bad_index) return MS_ERR_INVALID_ARG;
  if (c->hst->hash_overflow) return MS_ERR_CUDA;  // cannot happen: sized from n_keys
  const unsigned int mu = c->hst->n_unique;
  MS_TRY(launch_pairs_sort(rs, mu, bit_width(n_labels - 1), c->stream));
  MS_TRY(launch_pairs_assign(rs, mu, c->stream));
  MS_TRY(launch_pairs_lookup(asc, desc, n, rs, ms, c->stream));
  MS_TRY(launch_check_nonneg(ms, n, c->dst, c->stream));
  s = read_status(c);
  if (s != MS_OK) return s;
  if (c->hst->bad_index) return MS_ERR_INVALID_ARG;  // a pair missing from the keys
  if (c->hst->timeout) return MS_ERR_TIMEOUT;
  c->last_k = mu;
  if (k) *k = mu;
  finish_profile(c, l0);
  return MS_OK;
}

ms_status ms_set_tuning(ms_ctx *c, const ms_tuning *t) {
  if (!c || !t) return MS_ERR_INVALID_ARG;
  if (t->tile_ctas < 1 || t->tile_ctas > 4 || t->write_ctas < 1 || t->write_ctas > 16 ||
      t->chase_blocks < 1 || t->chase_blocks > 4 || t->pair_blocks < 1 || t->pair_blocks > 16 ||
      t->dynamic < 0 || t->dynamic > 1 || t->resolve_mode < -1 || t->resolve_mode > 1 ||
      t->shape3 < 0 || t->shape3 >= kShapeCount)
    return MS_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  Tuning u;
  u.tile_ctas = t->tile_ctas;
  u.write_ctas = t->write_ctas;
  u.chase_blocks = t->chase_blocks;
  u.pair_blocks = t->pair_blocks;
  u.dynamic = t->dynamic;
  u.resolve_mode = t->resolve_mode;
  u.shape3 = t->shape3;
  c->tune = u;
  for (BatchPlan &P : c->plans)
    if (!P.tuned) drop_graph(&P);
  return MS_OK;
}

ms_status ms_get_tuning(const ms_ctx *c, ms_tuning *t) {
  if (!c || !t) return MS_ERR_INVALID_ARG;
  *t = ms_tuning{};
  t->tile_ctas = c->tune.tile_ctas;
  t->write_ctas = c->tune.write_ctas;
  t->chase_blocks = c->tune.chase_blocks;
  t->pair_blocks = c->tune.pair_blocks;
  t->dynamic = c->tune.dynamic;
  t->resolve_mode = c->tune.resolve_mode;
  t->shape3 = c->tune.shape3;
  return MS_OK;
}

ms_status ms_batch_graphs(ms_ctx *c, int on) {
  if (!c) return MS_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  c->graphs_on = on != 0;
  if (!c->graphs_on)
    for (BatchPlan &P : c->plans) drop_graph(&P);
  return MS_OK;
}

ms_status ms_batch_autotune(ms_ctx *c, int n_fields, const void *const *fields,
                            const int64_t (*dims)[3], const ms_dtype *dtypes, int32_t *const *asc,
                            int32_t *const *desc, int32_t *const *ms, ms_tuning *out) {
  if (!c || n_fields <= 0) return MS_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  std::vector<FieldArg> fa;
  bool batchable = false;
  ms_status s = batch_args(n_fields, fields, dims, dtypes, asc, desc, ms, &fa, &batchable);
  if (s != MS_OK) return s;
  if (!batchable) return MS_ERR_INVALID_ARG;
  BatchPlan &P = plan_of(c, batch_signature(fa.data(), n_fields));
  drop_graph(&P);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  MS_TRY(cudaEventCreate(&e0));
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return MS_ERR_CUDA;
  }
  std::vector<int64_t> k((size_t)n_fields, 0);
  const bool prof = c->prof_on;
  c->prof_on = false;  // candidates are not profiled calls
  // median of three timed step-by-step runs (after one untimed run)
  auto time_of = [&](const Tuning &t, double *ms_out) -> ms_status {
    std::vector<float> v;
    for (int r = 0; r < 4; ++r) {
      cudaEventRecord(e0, c->stream);
      const ms_status st = segment_tiled(c, fa.data(), n_fields, k.data(), t);
      if (st != MS_OK) return st;
      cudaEventRecord(e1, c->stream);
      if (cudaEventSynchronize(e1) != cudaSuccess) return MS_ERR_CUDA;
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (r > 0) v.push_back(ms);
    }
    std::sort(v.begin(), v.end());
    *ms_out = v[v.size() / 2];
    return MS_OK;
  };
  Tuning best = c->tune;
  double t_default = 0, t_best = 0;
  s = time_of(best, &t_default);
  t_best = t_default;
  struct Knob {
    int Tuning::*field;
    std::vector<int> values;
  };
  const Knob knobs[] = {{&Tuning::shape3, {kShape32x16, kShape64x8, kShape16x32, kShape16x16}},
                        {&Tuning::dynamic, {1, 0}},
                        {&Tuning::tile_ctas, {2, 1}},
                        {&Tuning::write_ctas, {2, 4, 8}},
                        {&Tuning::chase_blocks, {3, 2}},
                        {&Tuning::pair_blocks, {8, 4}},
                        {&Tuning::resolve_mode, {-1, 0, 1}}};
  for (const Knob &kn : knobs) {
    if (s != MS_OK) break;
    const int start = best.*(kn.field);
    for (int v : kn.values) {
      if (v == start) continue;
      Tuning t = best;
      t.*(kn.field) = v;
      double tm = 0;
      s = time_of(t, &tm);
      if (s != MS_OK) break;
      if (tm < 0.98 * t_best) {
        best = t;
        t_best = tm;
      }
    }
  }
  c->prof_on = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (s != MS_OK) return s;
  P.tune = best;
  P.tuned = true;
  // leave the outputs as the chosen choices compute them (identical anyway)
  s = segment_tiled(c, fa.data(), n_fields, k.data(), best);
  if (s != MS_OK) return s;
  if (out) {
    out->tile_ctas = best.tile_ctas;
    out->write_ctas = best.write_ctas;
    out->chase_blocks = best.chase_blocks;
    out->pair_blocks = best.pair_blocks;
    out->resolve_mode = best.resolve_mode;
    out->dynamic = best.dynamic;
    out->shape3 = best.shape3;
    out->default_ms = t_default;
    out->best_ms = t_best;
  }
  int64_t total = 0;
  for (int64_t x : k) total += x;
  c->last_k = total;
  return MS_OK;
}

ms_status ms_segment_host(ms_ctx *c, const void *host_field, const int64_t dims[3],
                          ms_dtype dtype, int32_t *host_asc, int32_t *host_desc,
                          int32_t *host_ms) {
  if (!c || !host_field || !host_asc || !host_desc || !host_ms) return MS_ERR_INVALID_ARG;
  int64_t n = 0;
  ms_status s = check_dims(dims, &n);
  if (s != MS_OK) return s;
  s = check_dtype(dtype);
  if (s != MS_OK) return s;
  DeviceGuard g(c->device);
  const size_t esz = dtype == MS_F16 ? 2 : 4;
  const size_t fbytes = ((size_t)n * esz + 255) & ~(size_t)255;
  const size_t lbytes = ((size_t)n * 4 + 255) & ~(size_t)255;
  const size_t need = fbytes + 3 * lbytes;
  if (c->io_bytes < need) {
    if (c->io) {
      cudaStreamSynchronize(c->stream);
      cudaFree(c->io);
      c->io = nullptr;
      c->io_bytes = 0;
    }
    if (cudaMalloc(&c->io, need) != cudaSuccess) {
      cudaGetLastError();
      return MS_ERR_OUT_OF_MEMORY;
    }
    c->io_bytes = need;
  }
  char *base = static_cast<char *>(c->io);
  void *dfield = base;
  int32_t *dasc = reinterpret_cast<int32_t *>(base + fbytes);
  int32_t *ddesc = reinterpret_cast<int32_t *>(base + fbytes + lbytes);
  int32_t *dms = reinterpret_cast<int32_t *>(base + fbytes + 2 * lbytes);
  const long long l0 = tl_launches;
  StageTimer th(c, MS_STAGE_H2D);
  MS_TRY(cudaMemcpyAsync(dfield, host_field, (size_t)n * esz, cudaMemcpyHostToDevice, c->stream));
  th.stop();
  s = segment_device(c, dfield, dims, dtype, n, dasc, ddesc, dms);
  if (s != MS_OK) return s;
  StageTimer td(c, MS_STAGE_D2H);
  MS_TRY(cudaMemcpyAsync(host_asc, dasc, (size_t)n * 4, cudaMemcpyDeviceToHost, c->stream));
  MS_TRY(cudaMemcpyAsync(host_desc, ddesc, (size_t)n * 4, cudaMemcpyDeviceToHost, c->stream));
  MS_TRY(cudaMemcpyAsync(host_ms, dms, (size_t)n * 4, cudaMemcpyDeviceToHost, c->stream));
  td.stop();
  MS_TRY(cudaStreamSynchronize(c->stream));
  finish_profile(c, l0);
  return MS_OK;
}

ms_status ms_segment_host_many(ms_ctx *c, int n_fields, const void *const *host_fields,
                               const int64_t (*dims)[3], const ms_dtype *dtypes,
                               int32_t *const *host_asc, int32_t *const *host_desc,
                               int32_t *const *host_ms, int64_t *k_out) {
  if (!c || n_fields < 0) return MS_ERR_INVALID_ARG;
  if (n_fields == 0) return MS_OK;
  if (!host_fields || !dims || !dtypes || !host_asc || !host_desc || !host_ms)
    return MS_ERR_INVALID_ARG;
  std::vector<int64_t> nv((size_t)n_fields);
  size_t need = 0;
  for (int f = 0; f < n_fields; ++f) {
    ms_status s = check_dims(dims[f], &nv[f]);
    if (s != MS_OK) return s;
    s = check_dtype(dtypes[f]);
    if (s != MS_OK) return s;
    if (!host_fields[f] || !host_asc[f] || !host_desc[f] || !host_ms[f]) return MS_ERR_INVALID_ARG;
    const size_t esz = dtypes[f] == MS_F16 ? 2 : 4;
    const size_t fb = ((size_t)nv[f] * esz + 255) & ~(size_t)255;
    const size_t lb = ((size_t)nv[f] * 4 + 255) & ~(size_t)255;
    need = std::max(need, fb + 3 * lb);
  }
  DeviceGuard g(c->device);
  ms_status s = ensure_buffer(c, &c->io, &c->io_bytes, need);
  if (s == MS_OK && n_fields > 1) s = ensure_buffer(c, &c->io2, &c->io2_bytes, need);
  if (s != MS_OK) return s;
  if (!c->up) MS_TRY(cudaStreamCreateWithFlags(&c->up, cudaStreamNonBlocking));
  if (!c->down) MS_TRY(cudaStreamCreateWithFlags(&c->down, cudaStreamNonBlocking));
  for (int i = 0; i < 2; ++i) {
    if (!c->ev_up[i]) MS_TRY(cudaEventCreateWithFlags(&c->ev_up[i], cudaEventDisableTiming));
    if (!c->ev_comp[i]) MS_TRY(cudaEventCreateWithFlags(&c->ev_comp[i], cudaEventDisableTiming));
    if (!c->ev_down[i]) MS_TRY(cudaEventCreateWithFlags(&c->ev_down[i], cudaEventDisableTiming));
  }
  // the buffers of set `slot` for field f
  struct Io {
    void *field;
    int32_t *asc, *desc, *ms;
  };
  auto io_of = [&](int slot, int f) {
    const size_t esz = dtypes[f] == MS_F16 ? 2 : 4;
    const size_t fb = ((size_t)nv[f] * esz + 255) & ~(size_t)255;
    const size_t lb = ((size_t)nv[f] * 4 + 255) & ~(size_t)255;
    char *base = static_cast<char *>(slot ? c->io2 : c->io);
    return Io{base, reinterpret_cast<int32_t *>(base + fb), reinterpret_cast<int32_t *>(base + fb + lb),
              reinterpret_cast<int32_t *>(base + fb + 2 * lb)};
  };
  // field f's upload into set f % 2, once field f - 2 (the set's last user) is downloaded
  auto upload = [&](int f) -> cudaError_t {
    const int slot = f & 1;
    cudaError_t e = cudaSuccess;
    if (f >= 2) e = cudaStreamWaitEvent(c->up, c->ev_down[slot], 0);
    const size_t esz = dtypes[f] == MS_F16 ? 2 : 4;
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(io_of(slot, f).field, host_fields[f], (size_t)nv[f] * esz,
                          cudaMemcpyHostToDevice, c->up);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_up[slot], c->up);
    return e;
  };
  auto drain = [&]() {
    cudaStreamSynchronize(c->up);
    cudaStreamSynchronize(c->down);
    cudaStreamSynchronize(c->stream);
  };
  // the streams of a previous call on this context are idle: each call drains them
  const long long l0 = tl_launches;
  cudaError_t e = upload(0);
  for (int f = 0; f < n_fields && e == cudaSuccess; ++f) {
    if (f + 1 < n_fields) e = upload(f + 1);  // overlaps field f's segmentation and downloads
    if (e != cudaSuccess) break;
    const int slot = f & 1;
    const Io io = io_of(slot, f);
    e = cudaStreamWaitEvent(c->stream, c->ev_up[slot], 0);
    if (e != cudaSuccess) break;
    s = segment_device(c, io.field, dims[f], (int)dtypes[f], nv[f], io.asc, io.desc, io.ms);
    if (s != MS_OK) {
      drain();
      return s;
    }
    if (k_out) k_out[f] = c->last_k;
    e = cudaEventRecord(c->ev_comp[slot], c->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->down, c->ev_comp[slot], 0);
    const size_t lbytes = (size_t)nv[f] * 4;
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_asc[f], io.asc, lbytes, cudaMemcpyDeviceToHost, c->down);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_desc[f], io.desc, lbytes, cudaMemcpyDeviceToHost, c->down);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_ms[f], io.ms, lbytes, cudaMemcpyDeviceToHost, c->down);
    if (e == cudaSuccess) e = cudaEventRecord(c->ev_down[slot], c->down);
  }
  drain();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_status(e);
  }
  finish_profile(c, l0);
  return MS_OK;
}

ms_status ms_order_keys(ms_ctx *c, const void *field, int64_t n, ms_dtype dtype, uint32_t *keys) {
  if (!c || n < 0) return MS_ERR_INVALID_ARG;
  if (n > kMaxVertices) return MS_ERR_TOO_LARGE;
  ms_status s = check_dtype(dtype);
  if (s != MS_OK) return s;
  DeviceGuard g(c->device);
  if (n == 0) return MS_OK;
  if (!is_device_pointer(field) || !is_device_pointer(keys)) return MS_ERR_INVALID_ARG;
  s = reset_status(c);
  if (s != MS_OK) return s;
  MS_TRY(launch_order_keys(field, n, dtype, keys, c->dst, c->stream));
  s = read_status(c);
  if (s != MS_OK) return s;
  return c->hst->nan_flag ? MS_ERR_NAN_INPUT : MS_OK;
}

ms_status ms_steepest(ms_ctx *c, const void *field, const int64_t dims[3], ms_dtype dtype,
                      int32_t *up, int32_t *dn) {
  if (!c) return MS_ERR_INVALID_ARG;
  int64_t n = 0;
  ms_status s = check_dims(dims, &n);
  if (s != MS_OK) return s;
  s = check_dtype(dtype);
  if (s != MS_OK) return s;
  DeviceGuard g(c->device);
  if (!is_device_pointer(field) || !is_device_pointer(up) || !is_device_pointer(dn) || up == dn)
    return MS_ERR_INVALID_ARG;
  s = reset_status(c);
  if (s != MS_OK) return s;
  MS_TRY(launch_steepest_simple(field, dims, dtype, up, dn, c->dst, c->stream));
  s = read_status(c);
  if (s != MS_OK) return s;
  return c->hst->nan_flag ? MS_ERR_NAN_INPUT : MS_OK;
}

ms_status ms_compress(ms_ctx *c, int32_t *ptr, int64_t n) {
  if (!c || n < 0) return MS_ERR_INVALID_ARG;
  if (n > kMaxVertices) return MS_ERR_TOO_LARGE;
  DeviceGuard g(c->device);
  if (n == 0) return MS_OK;
  if (!is_device_pointer(ptr)) return MS_ERR_INVALID_ARG;
  ms_status s = reset_status(c);
  if (s != MS_OK) return s;
  MS_TRY(launch_check_range(ptr, n, c->dst, c->stream));
  s = read_status(c);
  if (s != MS_OK) return s;
  if (c->hst->bad_index) return MS_ERR_INVALID_ARG;
  return compress_pair(c, ptr, nullptr, n);
}

ms_status ms_pair_rank(ms_ctx *c, const int32_t *asc, const int32_t *desc, int64_t n,
                       int32_t *ms, int64_t *k_out) {
  if (!c || n < 0) return MS_ERR_INVALID_ARG;
  if (n > kMaxVertices) return MS_ERR_TOO_LARGE;
  DeviceGuard g(c->device);
  if (n > 0 && (!is_device_pointer(asc) || !is_device_pointer(desc) || !is_device_pointer(ms)))
    return MS_ERR_INVALID_ARG;
  ms_status s = reset_status(c);
  if (s != MS_OK) return s;
  const uint64_t guess = (uint64_t)(n < (1 << 16) ? n : (1 << 16));
  s = rank_pairs(c, asc, desc, n, ms, guess, (uint64_t)n);
  if (s == MS_OK && k_out) *k_out = c->last_k;
  return s;
}

ms_status ms_profile_enable(ms_ctx *c, int on) {
  if (!c) return MS_ERR_INVALID_ARG;
  DeviceGuard g(c->device);
  if (on) {
    for (int i = 0; i < MS_STAGE_COUNT; ++i)
      for (int j = 0; j < 2; ++j)
        if (!c->ev[i][j]) MS_TRY(cudaEventCreate(&c->ev[i][j]));
  }
  c->prof = ms_profile{};
  for (int i = 0; i < MS_STAGE_COUNT; ++i) c->ev_pending[i] = false;
  c->prof_on = on != 0;
  return MS_OK;
}

ms_status ms_profile_read(const ms_ctx *c, ms_profile *out) {
  if (!c || !out) return MS_ERR_INVALID_ARG;
  *out = c->prof;
  return MS_OK;
}

const char *ms_profile_stage_name(int stage) {
  static const char *names[MS_STAGE_COUNT] = {"tile_local", "resolve", "write",
                                              "h2d",        "d2h",     "graph"};
  return (stage >= 0 && stage < MS_STAGE_COUNT) ? names[stage] : "?";
}

}  // extern "C"
