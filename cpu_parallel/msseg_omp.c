/* The paper's CPU-parallel segmentation scheme (Sec. 4.2), with OpenMP: the
 * CPU-parallel baseline of the measurements.  It is neither the GPU path nor
 * the oracle (shares no code with either) and runs on all host cores.
 *
 *  - Order (Sec. 4.1): vertices ordered by (value, index); values compared as
 *    reals through an order-preserving integer key (-0 folded onto +0, NaN
 *    rejected).
 *  - Neighbours: the Freudenthal triangulation of the grid (cells cut along
 *    their (0,0,0)->(1,1,1) diagonal): u and v share an edge iff v - u is a
 *    non-zero vector with all components in {0, 1} or all in {0, -1}.
 *  - First step (Sec. 4.2.1): every vertex gets its largest and its smallest
 *    neighbour (itself for a maximum / minimum), both directions at once; the
 *    vertices are split evenly over the threads, and every thread keeps the
 *    vertices it found not yet converged in its own active list L0.
 *  - Second step: each thread independently replaces dsc(v) by dsc(dsc(v))
 *    (and asc likewise) for the vertices of its list; a vertex stays active
 *    (list L1) while dsc(v) or asc(v) is not yet an extremum; then L0 = L1,
 *    until the list is empty.  Threads read pointers other threads are
 *    updating: every value read lies on the same path to the same extremum,
 *    so the order changes the number of iterations, not the result.
 *  - MS ids (Sec. 4.2.2): vertices with equal (asc, desc) share a region; the
 *    id is the pair's dense rank among the distinct pairs, asc first (each
 *    thread collects its distinct pairs in a hash set, the union is sorted,
 *    every vertex looks its pair up). */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OMP_OK = 0, OMP_ERR_NAN = 1, OMP_ERR_ARG = 2, OMP_ERR_MEMORY = 3 };

static inline uint32_t order_key(float f) {
  uint32_t b;
  memcpy(&b, &f, sizeof b);
  if (b == 0x80000000u) b = 0; /* -0 == +0 */
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

static inline int is_nan(float f) {
  uint32_t b;
  memcpy(&b, &f, sizeof b);
  return (b & 0x7f800000u) == 0x7f800000u && (b & 0x007fffffu) != 0;
}

static inline int32_t load(const int32_t *p) { return __atomic_load_n(p, __ATOMIC_RELAXED); }
static inline void store(int32_t *p, int32_t v) { __atomic_store_n(p, v, __ATOMIC_RELAXED); }

static int cmp_u64(const void *a, const void *b) {
  const uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
  return x < y ? -1 : (x > y);
}

/* open-addressing set of 64-bit pair keys, grown at half load */
typedef struct {
  uint64_t *slot;
  size_t cap, n;
} pair_set;

static const uint64_t kEmptyKey = ~0ull;

static int set_init(pair_set *s, size_t cap) {
  s->cap = cap;
  s->n = 0;
  s->slot = (uint64_t *)malloc(cap * sizeof(uint64_t));
  if (!s->slot) return 0;
  for (size_t i = 0; i < cap; ++i) s->slot[i] = kEmptyKey;
  return 1;
}

static inline size_t set_hash(uint64_t k, size_t mask) {
  k ^= k >> 31;
  k *= 0x9e3779b97f4a7c15ull;
  k ^= k >> 29;
  return (size_t)k & mask;
}

static int set_add(pair_set *s, uint64_t k);

static int set_grow(pair_set *s) {
  pair_set t;
  if (!set_init(&t, s->cap * 2)) return 0;
  for (size_t i = 0; i < s->cap; ++i)
    if (s->slot[i] != kEmptyKey && !set_add(&t, s->slot[i])) return 0;
  free(s->slot);
  *s = t;
  return 1;
}

static int set_add(pair_set *s, uint64_t k) {
  if (2 * (s->n + 1) > s->cap && !set_grow(s)) return 0;
  size_t i = set_hash(k, s->cap - 1);
  while (s->slot[i] != kEmptyKey) {
    if (s->slot[i] == k) return 1;
    i = (i + 1) & (s->cap - 1);
  }
  s->slot[i] = k;
  ++s->n;
  return 1;
}

/* field: float32[nx*ny*nz], x fastest; asc, desc, ms: int32[n]; *k_out: the
 * region count; threads <= 0: OpenMP's default.  Returns OMP_OK or an error. */
int msseg_omp_segment(const float *field, int64_t nx, int64_t ny, int64_t nz, int32_t *asc,
                      int32_t *desc, int32_t *ms, int64_t *k_out, int threads) {
  if (!field || !asc || !desc || !ms || !k_out || nx < 1 || ny < 1 || nz < 1) return OMP_ERR_ARG;
  const int64_t n = nx * ny * nz;
  if (n > 2147483647LL) return OMP_ERR_ARG;
  if (threads <= 0) threads = omp_get_max_threads();
  /* the 14 Freudenthal offsets: components all in {0,1} or all in {0,-1} */
  int off[14][3], no = 0;
  for (int s = 1; s >= -1; s -= 2)
    for (int m = 1; m < 8; ++m) {
      off[no][0] = s * (m & 1);
      off[no][1] = s * ((m >> 1) & 1);
      off[no][2] = s * ((m >> 2) & 1);
      ++no;
    }
  int status = OMP_OK;
  uint64_t **uniq = (uint64_t **)calloc((size_t)threads, sizeof(uint64_t *));
  size_t *nuniq = (size_t *)calloc((size_t)threads, sizeof(size_t));
  if (!uniq || !nuniq) {
    free(uniq);
    free(nuniq);
    return OMP_ERR_MEMORY;
  }
  uint64_t *all = NULL;
  size_t k = 0;
#pragma omp parallel num_threads(threads)
  {
    const int t = omp_get_thread_num(), nt = omp_get_num_threads();
    const int64_t lo = n * t / nt, hi = n * (t + 1) / nt;
    int32_t *list0 = (int32_t *)malloc((size_t)(hi - lo + 1) * sizeof(int32_t));
    int32_t *list1 = (int32_t *)malloc((size_t)(hi - lo + 1) * sizeof(int32_t));
    int local = list0 && list1 ? OMP_OK : OMP_ERR_MEMORY;
    int64_t n0 = 0;
    /* ---- first step: largest and smallest neighbour */
    for (int64_t v = lo; v < hi && local == OMP_OK; ++v) {
      const int64_t x = v % nx, y = (v / nx) % ny, z = v / (nx * ny);
      const float fv = field[v];
      if (is_nan(fv)) {
        local = OMP_ERR_NAN;
        break;
      }
      const uint32_t kv = order_key(fv);
      uint32_t kmax = kv, kmin = kv;
      int64_t vmax = v, vmin = v;
      for (int i = 0; i < 14; ++i) {
        const int64_t ux = x + off[i][0], uy = y + off[i][1], uz = z + off[i][2];
        if (ux < 0 || uy < 0 || uz < 0 || ux >= nx || uy >= ny || uz >= nz) continue;
        const int64_t u = ux + nx * (uy + ny * uz);
        const float fu = field[u];
        if (is_nan(fu)) {
          local = OMP_ERR_NAN;
          break;
        }
        const uint32_t ku = order_key(fu);
        if (ku > kmax || (ku == kmax && u > vmax)) kmax = ku, vmax = u;
        if (ku < kmin || (ku == kmin && u < vmin)) kmin = ku, vmin = u;
      }
      store(&desc[v], (int32_t)vmax);
      store(&asc[v], (int32_t)vmin);
      if (vmax != v || vmin != v) list0[n0++] = (int32_t)v;
    }
    if (local != OMP_OK) {
#pragma omp atomic write
      status = local;
    }
#pragma omp barrier
    /* ---- second step: path compression over the thread's active list */
    if (status == OMP_OK) {
      while (n0 > 0) {
        int64_t n1 = 0;
        for (int64_t i = 0; i < n0; ++i) {
          const int32_t v = list0[i];
          const int32_t d = load(&desc[v]), a = load(&asc[v]);
          const int32_t dd = load(&desc[d]), aa = load(&asc[a]);
          if (dd != d) store(&desc[v], dd);
          if (aa != a) store(&asc[v], aa);
          /* converged once the pointer is at an extremum (a self-pointer) */
          if (load(&desc[dd]) != dd || load(&asc[aa]) != aa) list1[n1++] = v;
        }
        int32_t *tmp = list0;
        list0 = list1;
        list1 = tmp;
        n0 = n1;
      }
    }
    free(list0);
    free(list1);
#pragma omp barrier
    /* ---- MS ids: distinct pairs of the thread's vertices */
    if (status == OMP_OK) {
      pair_set set;
      if (!set_init(&set, 1024)) {
#pragma omp atomic write
        status = OMP_ERR_MEMORY;
      } else {
        for (int64_t v = lo; v < hi; ++v) {
          const uint64_t key = ((uint64_t)(uint32_t)asc[v] << 32) | (uint32_t)desc[v];
          if (!set_add(&set, key)) {
#pragma omp atomic write
            status = OMP_ERR_MEMORY;
            break;
          }
        }
        uint64_t *mine = (uint64_t *)malloc((set.n + 1) * sizeof(uint64_t));
        size_t m = 0;
        if (mine)
          for (size_t i = 0; i < set.cap; ++i)
            if (set.slot[i] != kEmptyKey) mine[m++] = set.slot[i];
        free(set.slot);
        uniq[t] = mine;
        nuniq[t] = m;
        if (!mine) {
#pragma omp atomic write
          status = OMP_ERR_MEMORY;
        }
      }
    }
#pragma omp barrier
#pragma omp single
    {
      if (status == OMP_OK) {
        size_t total = 0;
        for (int i = 0; i < nt; ++i) total += nuniq[i];
        all = (uint64_t *)malloc((total + 1) * sizeof(uint64_t));
        if (!all) {
          status = OMP_ERR_MEMORY;
        } else {
          size_t p = 0;
          for (int i = 0; i < nt; ++i) {
            memcpy(all + p, uniq[i], nuniq[i] * sizeof(uint64_t));
            p += nuniq[i];
          }
          qsort(all, total, sizeof(uint64_t), cmp_u64);
          for (size_t i = 0; i < total; ++i)
            if (k == 0 || all[i] != all[k - 1]) all[k++] = all[i];
        }
      }
    }
    /* (implicit barrier of single) every vertex looks its pair up */
    if (status == OMP_OK) {
      for (int64_t v = lo; v < hi; ++v) {
        const uint64_t key = ((uint64_t)(uint32_t)asc[v] << 32) | (uint32_t)desc[v];
        size_t l = 0, r = k;
        while (l < r) {
          const size_t mid = (l + r) / 2;
          if (all[mid] < key)
            l = mid + 1;
          else
            r = mid;
        }
        ms[v] = (int32_t)l;
      }
    }
  }
  for (int i = 0; i < threads; ++i) free(uniq[i]);
  free(uniq);
  free(nuniq);
  free(all);
  *k_out = (int64_t)k;
  return status;
}

int msseg_omp_max_threads(void) { return omp_get_max_threads(); }
