/*
 * ms.h -- C ABI of the GB300 (sm_103a) piecewise-linear Morse-Smale
 * segmentation library (libmsseg.so).
 *
 * What it computes (paper: "Parallel Computation of Piecewise Linear
 * Morse-Smale Segmentations", arXiv 2303.15491):
 *
 *   Input  (Sec. 3.1): a scalar field f on the vertices of a regular grid of
 *          nx*ny*nz vertices, linearly interpolated on the grid's implicit
 *          Freudenthal triangulation (each cell cut along its
 *          (0,0,0)->(1,1,1) diagonal; in 2D the (x,y)->(x+1,y+1) diagonal
 *          drawn in Fig. 1).  Vertex (x,y,z) has index v = x + nx*(y + ny*z).
 *          N(v), the vertices sharing an edge with v, are the grid points at
 *          offsets +-(1,0,0), +-(0,1,0), +-(0,0,1), +-(1,1,0), +-(1,0,1),
 *          +-(0,1,1), +-(1,1,1) that lie inside the box (14 in the interior
 *          of a 3D grid, 6 in 2D).
 *   Order  (Sec. 4.1): vertices are compared by (f value, index); equal
 *          values (including -0.0 and +0.0) are ordered by index, the
 *          smaller index being lower.  NaN values are rejected.
 *   up/dn  (Sec. 4.2.1): up(v) is the highest vertex of N(v) u {v}, dn(v)
 *          the lowest; a vertex with up(v) == v is a maximum, dn(v) == v a
 *          minimum.
 *   labels (Sec. 3.3, 3.4, 4.2.1): desc(v) is the maximum reached by
 *          following up from v (path compression until every pointer is at
 *          its fixed point), asc(v) the minimum reached by following dn.
 *          Following the paper's naming, the DEScending segmentation holds
 *          the maxima and the ASCending one the minima (Sec. 4.2, Fig. 1).
 *          Labels are the extremum's vertex index.
 *   MS id  (Sec. 3.4, 4.2.2): vertices with the same (asc, desc) pair form
 *          one MS region; ms(v) is the 0-based rank of v's pair among the K
 *          distinct pairs that occur, sorted lexicographically with asc
 *          first.
 *
 * Conventions for every entry point:
 *   - dims = {nx, ny, nz}, each >= 1, N = nx*ny*nz <= 2^31 - 1 (otherwise
 *     MS_ERR_TOO_LARGE).  A 2D field is nz == 1; the 3D stencil clipped to
 *     the box is then exactly the 2D one.
 *   - Pointers named field / out_* / ptr / keys / asc / desc / ms are DEVICE
 *     pointers (cudaMalloc'd or managed) owned by the caller, unless the
 *     function name ends in _host.  The library owns only its scratch memory
 *     and never frees caller memory.  Fields are densely packed, x fastest.
 *   - Every call is ordered on the context's stream and returns after the
 *     work has completed, with a status.  On error the outputs are
 *     unspecified.  A context is not thread-safe: use one per host thread.
 */
#ifndef MS_H_
#define MS_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ms_ctx ms_ctx;

typedef enum { MS_F32 = 0, MS_F16 = 1 } ms_dtype;

typedef enum {
  MS_OK = 0,
  MS_ERR_INVALID_ARG = 1,       /* null pointer, dims < 1, host pointer where a device one is needed */
  MS_ERR_UNSUPPORTED_DTYPE = 2, /* dtype not MS_F32 / MS_F16 */
  MS_ERR_TOO_LARGE = 3,         /* N > 2^31 - 1 or a size beyond a stated maximum */
  MS_ERR_NAN_INPUT = 4,         /* the field holds a NaN */
  MS_ERR_OUT_OF_MEMORY = 5,     /* scratch allocation failed */
  MS_ERR_CUDA = 6,              /* a CUDA runtime call or kernel launch failed */
  MS_ERR_NOT_CONVERGED = 7,     /* path compression hit its round cap (input is not a forest) */
  MS_ERR_TIMEOUT = 8,           /* a bounded wait gave up */
  MS_ERR_BUSY = 9               /* a server slot or budget is not available */
} ms_status;

/* Human-readable name of a status.  Never NULL; static storage. */
const char *ms_status_string(ms_status s);

/* Create a context on CUDA device `device`.  cuda_stream is a cudaStream_t
 * to run on (borrowed, not destroyed by ms_destroy), or NULL for a stream
 * the context creates and owns.  *out is set only on MS_OK. */
ms_status ms_create(ms_ctx **out, int device, void *cuda_stream);

/* Release the context's stream (if owned) and scratch memory.  NULL is a
 * no-op. */
ms_status ms_destroy(ms_ctx *ctx);

/* Full segmentation (Sec. 4.2): order keys, steepest neighbours, path
 * compression, MS ids.  field: N values of `dtype`; out_asc, out_desc,
 * out_ms: int32[N] each (distinct, non-overlapping, 4-byte aligned).
 * Repeated calls on the same buffers replay a captured CUDA graph (see
 * ms_segment_batch); the results are the same either way.
 * Errors: MS_ERR_INVALID_ARG, MS_ERR_UNSUPPORTED_DTYPE, MS_ERR_TOO_LARGE,
 * MS_ERR_NAN_INPUT, MS_ERR_OUT_OF_MEMORY, MS_ERR_CUDA, MS_ERR_NOT_CONVERGED. */
ms_status ms_segment(ms_ctx *ctx, const void *field, const int64_t dims[3], ms_dtype dtype,
                     int32_t *out_asc, int32_t *out_desc, int32_t *out_ms);

/* Many segmentations in one call (ensemble members, time steps): fields[f]
 * with dims[f] and dtypes[f] -> asc[f], desc[f], ms[f], exactly as n_fields
 * separate ms_segment calls would give them.  All pointer arrays are HOST
 * arrays of n_fields DEVICE pointers; k_out (may be NULL) is a host array of
 * n_fields that receives each field's region count K.  When every field has
 * at most 2^24 vertices and is 2D (nz = 1) or has at least 8 planes, all
 * fields go through one launch per stage (tiles of all fields in one work
 * queue, one global pair set keyed by field); otherwise the fields are
 * segmented one after the other.
 * Repeats (here and in ms_segment): a call with the same fields as the call
 * before (same pointers, dims and dtypes) runs step by step, records the sizes
 * it met and captures the whole pipeline (sized from them, with margins) in a
 * CUDA graph; later calls with the same fields replay it with one host
 * synchronisation.  A replay whose sizes no longer suffice (the fields'
 * contents changed) is detected on the device and the call runs step by step
 * again, so results never depend on the path taken.
 * A NaN in any field fails the whole call (MS_ERR_NAN_INPUT).
 * ms_last_region_count then returns the sum of the fields' K. */
ms_status ms_segment_batch(ms_ctx *ctx, int n_fields, const void *const *fields,
                           const int64_t (*dims)[3], const ms_dtype *dtypes, int32_t *const *asc,
                           int32_t *const *desc, int32_t *const *ms, int64_t *k_out);

/* The same segmentation computed by the four step kernels below, one after
 * the other, each through global memory (slower than ms_segment; kept as an
 * independent GPU cross-check of the fused path).  Same arguments, outputs
 * and errors as ms_segment. */
ms_status ms_segment_staged(ms_ctx *ctx, const void *field, const int64_t dims[3], ms_dtype dtype,
                            int32_t *out_asc, int32_t *out_desc, int32_t *out_ms);

/* The same segmentation from and to HOST memory: copies the field to the
 * device, segments it and copies the three label arrays back, all on the
 * context's stream (pinned host buffers make the copies asynchronous DMA;
 * pageable ones also work).  Device buffers are the context's scratch. */
ms_status ms_segment_host(ms_ctx *ctx, const void *host_field, const int64_t dims[3],
                          ms_dtype dtype, int32_t *host_asc, int32_t *host_desc,
                          int32_t *host_ms);

/* Many segmentations from and to HOST memory, pipelined: field f is copied
 * to the device while field f - 1 is segmented and field f - 2's labels are
 * copied back, so the host link carries uploads and downloads at once (two
 * device buffer sets, one upload and one download stream besides the
 * context's).  Arguments per field as ms_segment_host; k_out[f] (may be NULL)
 * receives each field's region count.  Returns after every field's labels
 * are in host memory, or at the first failing field (later fields' outputs
 * are then undefined).  Host buffers should be pinned: pageable memory makes
 * the copies synchronous and removes the overlap. */
ms_status ms_segment_host_many(ms_ctx *ctx, int n_fields, const void *const *host_fields,
                               const int64_t (*dims)[3], const ms_dtype *dtypes,
                               int32_t *const *host_asc, int32_t *const *host_desc,
                               int32_t *const *host_ms, int64_t *k_out);

/* K, the number of MS regions found by the last successful ms_segment /
 * ms_segment_host / ms_pair_rank on this context (0 before any). */
ms_status ms_last_region_count(const ms_ctx *ctx, int64_t *k);

/* ---- the four steps of the path, callable one at a time ----------------- */

/* Step 1 (Sec. 4.1 order field, without the sort): keys[v] is a uint32 such
 * that (keys[u], u) < (keys[w], w) exactly when u is lower than w in the
 * (value, index) order: IEEE bits with -0.0 mapped to +0.0, the sign bit
 * flipped for positives and all bits flipped for negatives (fp16 values are
 * widened exactly to fp32 first).  n = number of values.  MS_ERR_NAN_INPUT
 * if any value is NaN (keys then unspecified). */
ms_status ms_order_keys(ms_ctx *ctx, const void *field, int64_t n, ms_dtype dtype,
                        uint32_t *keys);

/* Step 2 (Sec. 4.2.1 first step): up[v] / dn[v] = index of the highest /
 * lowest vertex of N(v) u {v}.  up and dn: int32[N], distinct buffers. */
ms_status ms_steepest(ms_ctx *ctx, const void *field, const int64_t dims[3], ms_dtype dtype,
                      int32_t *up, int32_t *dn);

/* Step 3 (Sec. 4.2.1 path compression, Fig. 3): replaces ptr[v] by
 * ptr[ptr[v]] until every entry is a fixed point, in place.  ptr: int32[n]
 * forming a forest whose roots are self-pointers (as up / dn are).  Entries
 * outside [0, n) give MS_ERR_INVALID_ARG; a cycle gives
 * MS_ERR_NOT_CONVERGED after ceil(log2 n) + 2 doubling rounds. */
ms_status ms_compress(ms_ctx *ctx, int32_t *ptr, int64_t n);

/* Step 4 (Sec. 4.2.2): ms[v] = rank of (asc[v], desc[v]) among the distinct
 * pairs, lexicographic with asc first; *k_out (may be NULL) = K.  asc, desc
 * values must lie in [0, n) (else MS_ERR_INVALID_ARG). */
ms_status ms_pair_rank(ms_ctx *ctx, const int32_t *asc, const int32_t *desc, int64_t n,
                       int32_t *ms, int64_t *k_out);


/* Launch choices of the batched path; they change scheduling only, never
 * results.  The library has no counterpart in the paper for them. */
typedef struct {
  int tile_ctas;      /* tile kernels: CTAs per SM (1 or 2) */
  int write_ctas;     /* label-writing kernels: CTAs per SM */
  int chase_blocks;   /* root chase: 512-thread blocks (warps take tiles) per SM */
  int pair_blocks;    /* tile pairs: 256-thread blocks per SM */
  int dynamic;        /* 1: tiles taken from a work queue; 0: static stride */
  int resolve_mode;   /* exits and pairs: -1 by tile count, 0 a tile a warp, 1 flat */
  int shape3;         /* 3D tile shape (x * y * z vertices): 0 32x16x16 (the default),
                         1 64x8x16, 2 16x32x16, 3 16x16x16 */
  double default_ms;  /* ms_batch_autotune: time of the default choices */
  double best_ms;     /* ms_batch_autotune: time of the chosen ones */
} ms_tuning;

/* Time the batched path on these fields (arguments as ms_segment_batch; the
 * outputs are written) under candidate launch choices -- the tile shape
 * first, then one knob at a time, keeping a change only if it is at least
 * 2 % faster -- and keep the fastest for later calls with the same fields
 * (ms_segment_batch, or ms_segment for one field).  *out (may be NULL)
 * receives the choice.  MS_ERR_INVALID_ARG if the fields do not take the
 * batched path. */
ms_status ms_batch_autotune(ms_ctx *ctx, int n_fields, const void *const *fields,
                            const int64_t (*dims)[3], const ms_dtype *dtypes,
                            int32_t *const *asc, int32_t *const *desc, int32_t *const *ms,
                            ms_tuning *out);

/* The choices calls on this context take when no ms_batch_autotune entry
 * covers their fields (the timing fields are ignored / zero).  Setting them
 * drops captured graphs of untuned calls.  MS_ERR_INVALID_ARG for a choice
 * out of range (tile_ctas 1..4, write_ctas 1..16, chase_blocks 1..4,
 * pair_blocks 1..16, dynamic 0..1, resolve_mode -1..1, shape3 0..3). */
ms_status ms_set_tuning(ms_ctx *ctx, const ms_tuning *t);
ms_status ms_get_tuning(const ms_ctx *ctx, ms_tuning *t);

/* Enable (on != 0, the default) or disable graph capture and replay of
 * repeated calls (ms_segment, ms_segment_batch) on this context. */
ms_status ms_batch_graphs(ms_ctx *ctx, int on);

/* ---- after the segmentation: the marching triangles / tetrahedra index pass - */

/* Sec. 4.3 (multi-label marching triangles and tetrahedra), the pass before
 * the separating geometry: for every simplex of the triangulation the binary
 * code of its label configuration (Fig. 4, Tab. 1) and, per cell, where the
 * cell's separating elements start in the output.
 *   Cells: (x, y[, z]) with x < nx-1, y < ny-1 (, z < nz-1), linear index
 *   c = x + (nx-1)(y + (ny-1) z); a 2D grid (nz = 1) has (nx-1)(ny-1) cells.
 *   Simplices: each cell is cut along its (0,..,0)->(1,..,1) diagonal into
 *   one simplex per axis order -- 2D: 2c (x then y), 2c+1 (y then x); 3D:
 *   6c + p with p = 0..5 for xyz, xzy, yxz, yzx, zxy, zyx.  The vertices
 *   a, b, c(, d) of a simplex are its corners in stepping order.
 *   Code: a gets local label 0; each later vertex takes the local label of
 *   the first earlier vertex with an equal label, else its own position;
 *   triangle code = b << 2 | c, tetrahedron code = b << 4 | c << 2 | d.
 *   Elements (Figs. 5, 6): a triangle with 2 labels is cut by 1 segment, with
 *   3 by 3; a tetrahedron whose labels split 3+1 by 1 triangle, 2+2 by 2,
 *   2+1+1 by 5, 1+1+1+1 by 12.
 * labels: int32[nx*ny*nz] (any segmentation: ms, asc or desc ids) on the
 * device; mode: which elements are counted -- 0 region separators (the counts
 * above), 1 region boundaries (one per simplex whose labels split 3+1, 2D:
 * 2+1; see ms_simplex_geometry); codes: uint8[cells * (2 or 6)] on the
 * device, 16-byte aligned; cell_offsets: int64[cells] on the device, the
 * exclusive prefix sum of the cells' element counts; *total (host, may be
 * NULL): the element total.  Grids without cells (an extent of 1 other than
 * nz) give *total = 0 and touch no output.  One kernel launch: tiles of
 * cells find their offset bases from the earlier tiles' totals (a bounded
 * wait; MS_ERR_TIMEOUT if it runs out).  Errors: MS_ERR_INVALID_ARG,
 * MS_ERR_TOO_LARGE, MS_ERR_OUT_OF_MEMORY, MS_ERR_TIMEOUT, MS_ERR_CUDA. */
ms_status ms_simplex_index(ms_ctx *ctx, const int32_t *labels, const int64_t dims[3], int mode,
                           uint8_t *codes, int64_t *cell_offsets, int64_t *total);

/* Sec. 4.3, the region-separating geometry, written where ms_simplex_index
 * (same labels, dims and mode) put each cell's elements.
 *   mode 0, region separators (Figs. 5, 6): triangle, 2 labels: the segment
 *   joining the midpoints of the lone corner's edges; 3 labels: segments from
 *   the centre to the midpoints of ab, bc, ac.  Tetrahedron, 3+1: the
 *   triangle of the midpoints of the lone corner's edges; 2+2 ({p0,p1} holds
 *   corner a, {q0,q1} the rest): (p0q0, p0q1, p1q0), (p0q1, p1q0, p1q1);
 *   2+1+1 (pair P < Q, singles R < S, T1 / T2 the centres of faces PRS /
 *   QRS): (T1,T2,PR), (T2,PR,QR), (T1,T2,RS), (T1,T2,PS), (T2,PS,QS); four
 *   labels: (centre, face centre, edge midpoint) for the faces abc, abd,
 *   acd, bcd and each face's edges in the order first-second, first-third,
 *   second-third.  An element separates the labels at the ends of its
 *   midpoint's edge (the first midpoint's, for 3+1 / 2+2 / 2+1 elements).
 *   mode 1, region boundaries: the triangle (2D: edge) of the corners that
 *   share the label all but one corner carry, in chain order; it separates
 *   that label from the remaining corner's.
 * Points are grid coordinates, float32: a midpoint is (u+v)/2, a face
 * centre (u+v+w)/3, the centre the corners' sum / 4, each coordinate's sum
 * formed exactly and divided once, rounded to nearest.
 * points: float[total * 3 * 3] (3D: three xyz points per triangle) or
 * float[total * 2 * 2] (2D: two xy points per segment), device; pairs:
 * int32[total * 2] (smaller label first), device, or NULL.  total: the value
 * ms_simplex_index returned.  MS_ERR_INVALID_ARG also when the offsets or
 * total do not match the labels (nothing is written outside the ranges). */
ms_status ms_simplex_geometry(ms_ctx *ctx, const int32_t *labels, const int64_t dims[3], int mode,
                              const int64_t *cell_offsets, int64_t total, float *points,
                              int32_t *pairs);

/* ---- after the segmentation: persistence pairs of the extrema ----------------- */

/* Sec. 4.1 (topological simplification by persistence, with the thresholds of
 * Sec. 6): the 0-dimensional persistence pairs of the minima (direction -1)
 * or maxima (+1), computed from the basins of a segmentation of the same
 * field -- the ascending labels (out_asc of ms_segment) for minima, the
 * descending ones (out_desc) for maxima.
 *   Vertices enter in increasing (value, index) order for minima, decreasing
 *   for maxima (Sec. 4.1's total order); a vertex with no earlier neighbour
 *   starts a component, its extremum; a vertex joining several components
 *   ends all but the one whose extremum entered first (the elder rule), and
 *   each ended extremum dies at that vertex.  The extremum that enters first
 *   never dies.  Its persistence is |f(death) - f(extremum)|.
 * field, dims, dtype: as ms_segment (device).  labels: int32[n], device; every
 * label must be an extremum's own label (labels[labels[v]] == labels[v]),
 * else MS_ERR_INVALID_ARG.  extremum, death: int32[capacity], device; pair i
 * is (extremum[i], death[i]) with the extrema in increasing vertex index and
 * death -1 for the one that never dies.  *info (host, may be NULL) receives
 * the counts; n_extrema is set also when it exceeds capacity
 * (MS_ERR_TOO_LARGE, nothing written), so capacity 0 asks for the count.
 * The labels are trusted to be the segmentation of this field: other labels
 * give other pairs, never an out-of-range access.  Errors: MS_ERR_INVALID_ARG,
 * MS_ERR_UNSUPPORTED_DTYPE, MS_ERR_TOO_LARGE (also more than 2^30 distinct
 * basin pairs), MS_ERR_NAN_INPUT, MS_ERR_OUT_OF_MEMORY, MS_ERR_CUDA. */
typedef struct {
  int64_t n_extrema;    /* pairs (extrema) */
  int64_t basin_edges;  /* distinct pairs of adjacent basins */
  int32_t rounds;       /* parallel merge rounds that ran */
  int32_t pad;
  int64_t finish_edges; /* edges left to the one-thread finish in entry order (0: none) */
} ms_persistence_info;

ms_status ms_persistence(ms_ctx *ctx, const void *field, const int64_t dims[3], ms_dtype dtype,
                         const int32_t *labels, int direction, int32_t *extremum, int32_t *death,
                         int64_t capacity, ms_persistence_info *info);

/* ---- one field over several processes: z-slabs ------------------------------- */

/* The paper leaves computing one field on many nodes to future work (Sec. 8).
 * These four calls split Sec. 4.2's steps by z-slab so that each process (one
 * GPU each) segments its slab and the processes exchange two small messages:
 *   1. ms_slab_local on every slab; each publishes the asc / desc labels of
 *      its first and last owned planes (those another slab's lines can
 *      enter) -- planes z0 (if z0 > 0) and z1 - 1 (if z1 < nz);
 *   2. all-gather of those rows; ms_slab_resolve on every slab;
 *   3. ms_slab_pairs on every slab; all-gather of the pair lists;
 *      ms_slab_rank on every slab.
 * Labels and MS ids then equal ms_segment's on the whole field, vertex for
 * vertex.  Every buffer is in the calling process's device memory: gathered
 * data is copied in before a call reads it. */

/* Steepest steps and pointer jumping inside one slab (Sec. 4.2.1).
 * dims: the whole field's (nx, ny, nz); the slab owns planes [z0, z1).
 * field: the slab's planes plus one halo plane on each side that exists --
 * planes [z0 - (z0 > 0), z1 + (z1 < nz)) -- device.  out_asc, out_desc:
 * int32[(z1 - z0) nx ny], device: for each owned vertex the global index of
 * the extremum its line reaches inside the slab, or -(h + 1) where the line
 * leaves the slab at global vertex h (a halo vertex).  Errors as
 * ms_segment. */
ms_status ms_slab_local(ms_ctx *ctx, const void *field, const int64_t dims[3], ms_dtype dtype,
                        int64_t z0, int64_t z1, int32_t *out_asc, int32_t *out_desc);

/* Resolves exits.  rows: int32[n_planes][2][nx ny] on the device, the
 * published rows of all slabs ([plane][0] asc, [plane][1] desc), rewritten in
 * place; plane_z: int64[n_planes] on the host, each row's global z (distinct).
 * asc, desc: int32[n_owned] on the device, this slab's ms_slab_local output,
 * rewritten with every exit replaced by the extremum its line reaches.
 * MS_ERR_INVALID_ARG if an exit points into a plane that is not among the
 * rows (or the rows hold an index out of range); MS_ERR_NOT_CONVERGED if the
 * rows hold a cycle. */
ms_status ms_slab_resolve(ms_ctx *ctx, const int64_t dims[3], int32_t *rows, const int64_t *plane_z,
                          int n_planes, int32_t *asc, int32_t *desc, int64_t n_owned);

/* The distinct (asc, desc) pairs of n resolved vertices, as keys
 * (asc << 32) | desc in increasing order, into keys (uint64[capacity],
 * device); *m receives the count (also on MS_ERR_TOO_LARGE, when it exceeds
 * capacity and nothing is written).  Labels must lie in [0, n_labels). */
ms_status ms_slab_pairs(ms_ctx *ctx, const int32_t *asc, const int32_t *desc, int64_t n,
                        int64_t n_labels, uint64_t *keys, int64_t capacity, int64_t *m);

/* MS ids (Sec. 4.2.2) of n resolved vertices: the rank of each vertex's pair
 * among the distinct keys of all slabs (keys: every slab's ms_slab_pairs
 * output, concatenated, n_keys <= 2^30, device).  ms: int32[n], device; *k
 * (may be NULL): the number of distinct pairs of the whole field.
 * MS_ERR_INVALID_ARG if a vertex's pair is missing from the keys. */
ms_status ms_slab_rank(ms_ctx *ctx, const int32_t *asc, const int32_t *desc, int64_t n,
                       int64_t n_labels, const uint64_t *keys, int64_t n_keys, int32_t *ms,
                       int64_t *k);

/* ---- serving ---------------------------------------------------------------- */

/* A request loop for segmentations of mixed sizes.  The server owns n_slots
 * worker threads, each with its own context (stream and resident scratch) on
 * `device`, so requests run concurrently and their kernels overlap on the GPU.
 * budget_bytes bounds what the server's requests hold on the device: the
 * scratch each slot keeps between requests (measured after every request)
 * plus, for each running request, its field and three label arrays and the
 * growth of its slot's scratch (estimated at 10 bytes per vertex).  A
 * submitted request waits until a slot is idle and that much fits in what the
 * budget has left; among waiting requests the first that fits is admitted (one
 * passed over 8 times is admitted next, once it fits), except that requests of
 * at least 2^25 vertices -- each fills the GPU by itself -- run one at a time.
 * When a waiting request does not fit and no request is running, idle slots
 * free their scratch; a slot whose scratch outgrew its estimate frees it after
 * the request.  Results are exactly those of ms_segment. */
typedef struct ms_server ms_server;

typedef struct {
  uint64_t admitted, completed, queued; /* requests */
  size_t bytes_in_use;                  /* slots' resident scratch + running requests' charges */
  size_t peak_bytes;                    /* the largest bytes_in_use so far */
  size_t budget_bytes;
  uint64_t launches;                    /* kernel launches of completed requests */
  size_t resident_bytes;                /* device bytes the slots' contexts hold now */
} ms_server_info;

/* n_slots in [1, 64], budget_bytes > 0.  *out is set only on MS_OK. */
ms_status ms_server_create(ms_server **out, int device, size_t budget_bytes, int n_slots);

/* Queue one segmentation (arguments as ms_segment, device pointers).  The
 * field must already hold its values -- the server's streams do not wait on
 * the caller's -- and all four buffers must stay valid and untouched until the
 * request completes.  *ticket identifies it.  A request whose
 * estimate exceeds the whole budget is refused with MS_ERR_TOO_LARGE. */
ms_status ms_server_submit(ms_server *srv, const void *field, const int64_t dims[3],
                           ms_dtype dtype, int32_t *out_asc, int32_t *out_desc, int32_t *out_ms,
                           uint64_t *ticket);

/* Wait up to timeout_ms (< 0: no limit) for a request.  MS_OK: it completed,
 * *result (may be NULL) holds its status, *k_out its region count and
 * *latency_ms the time from submission to completion (both may be NULL); the
 * ticket is then released.  MS_ERR_TIMEOUT: still running (wait again).
 * MS_ERR_INVALID_ARG: unknown ticket. */
ms_status ms_server_wait(ms_server *srv, uint64_t ticket, int64_t timeout_ms, ms_status *result,
                         int64_t *k_out, double *latency_ms);

ms_status ms_server_stats(ms_server *srv, ms_server_info *out);

/* Finish every submitted request, then stop the workers and free the
 * contexts.  NULL is a no-op. */
ms_status ms_server_destroy(ms_server *srv);

/* ---- step 4 without allocation --------------------------------------------- */

/* Largest n that ms_pair_rank_noalloc accepts (64^3 vertices). */
#define MS_NOALLOC_MAX_N 262144

/* MS ids exactly as ms_pair_rank computes them, for callers that cannot
 * allocate device memory -- code running where a memory pool or framework
 * owns the whole device, or a latency-critical loop that cannot afford the
 * synchronisation and possible failure of cudaMalloc.  The paper has no
 * counterpart: this is an interface convenience, not part of the method.
 *
 * asc, desc: int32[n] device arrays with values in [0, n); ms: int32[n]
 * device output; *k_out (may be NULL) receives K; cuda_stream: the stream to
 * run on (NULL = the legacy default stream).  Needs no ms_ctx.  n above
 * MS_NOALLOC_MAX_N gives MS_ERR_TOO_LARGE, values outside [0, n)
 * MS_ERR_INVALID_ARG.  The call returns after its work has completed.
 *
 * Its working memory is one static device array of about 10.3 MB inside the
 * library (hash set, sort buffers and a status block), which every GPU that
 * loads the library holds until the process exits; the call itself performs
 * no cudaMalloc / cudaFree and calls no allocating routine.  The first call
 * on a device looks the array's device address up (cudaGetSymbolAddress) and
 * caches it for the device's current context, so make that first call before
 * any stream capture on the device; the cache is keyed by the context's id
 * (cuCtxGetId), and a call made in a new context (for example after
 * cudaDeviceReset) looks the address up again, which again must happen
 * outside a stream capture.  Every call reuses the same array: the call clears what must start
 * empty, but calls that overlap on the GPU (two streams, two threads) race on
 * it and must be serialised by the caller. */
ms_status ms_pair_rank_noalloc(const int32_t *asc, const int32_t *desc, int64_t n, int32_t *ms,
                               int64_t *k_out, void *cuda_stream);

/* ---- measurement ---------------------------------------------------------- */

/* Stages of one segmentation, as timed by the profiler.  For ms_segment:
 *   TILE_LOCAL  one kernel: order keys, steepest neighbours, path compression
 *               inside each tile, numbering of each tile's (asc, desc) root pairs
 *   RESOLVE     exits followed across tiles, global pair set, sort, MS ids
 *   WRITE       one kernel: the three label arrays streamed out
 * For ms_segment_staged the same three slots hold steepest neighbours, the
 * compression rounds and the pair ranking. */
typedef enum {
  MS_STAGE_TILE_LOCAL = 0,
  MS_STAGE_RESOLVE = 1,
  MS_STAGE_WRITE = 2,
  MS_STAGE_H2D = 3, /* ms_segment_host: field upload */
  MS_STAGE_D2H = 4, /* ms_segment_host: label download */
  MS_STAGE_GRAPH = 5, /* ms_segment_batch: a whole replayed CUDA graph */
  MS_STAGE_COUNT = 6
} ms_stage;

typedef struct {
  int64_t calls;                   /* segmentations since the profiler was enabled */
  int64_t launches;                /* CUDA kernels this library launched in them */
  int64_t stage_launches[8];       /* kernels per stage */
  double stage_ms[8];              /* summed device time per stage (CUDA events on the
                                      context's stream) */
} ms_profile;

/* Enable (on != 0) or disable the per-stage profiler of a context; enabling
 * resets its counters.  With the profiler on, each stage of a call is
 * bracketed by CUDA events on the context's stream and their elapsed times
 * are summed when the call completes.  Off by default. */
ms_status ms_profile_enable(ms_ctx *ctx, int on);

/* Copy the profiler's counters (zeros if it was never enabled). */
ms_status ms_profile_read(const ms_ctx *ctx, ms_profile *out);

/* Name of a stage ("tile_local", "resolve", "write", "h2d", "d2h", "graph");
 * "?" if out of range. */
const char *ms_profile_stage_name(int stage);

#ifdef __cplusplus
}
#endif
#endif /* MS_H_ */
