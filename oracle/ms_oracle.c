/*
 * Plain, single-threaded CPU oracle of the vertex-based piecewise-linear
 * Morse-Smale (MS) segmentation of a scalar field on a regular grid.
 *
 * TEST INFRASTRUCTURE.  This file exists to check the CUDA path; it is not
 * part of the product.  Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark may build, load or call it.  It shares no
 * code, header, table or helper with the CUDA library.
 *
 * Every function follows a definition of the paper written out directly,
 * with no blocking, fusion or reordering:
 *
 *   order       Sec. 3.1 + Sec. 4.1: vertices are totally ordered by
 *               (f value, vertex index); ties in f go to the index, the
 *               smaller index being lower.  Values are compared as real
 *               numbers (float32/float16 inputs are widened exactly to
 *               double), so -0.0 and +0.0 tie and are split by the index.
 *   neighbours  Sec. 4.2: N(v) = the vertices joined to v by an edge of the
 *               triangulation.  The triangulation of the grid is the
 *               Freudenthal (Kuhn) one whose 2D form is drawn in Fig. 1:
 *               each cell is cut into simplices along its (0,..,0)->(1,..,1)
 *               diagonal, so u and v share an edge iff u - v is a non-zero
 *               vector with all components in {0, 1} or all in {0, -1}.
 *   steepest    Sec. 3.3 + Sec. 4.2: up(v) is the highest vertex of
 *               N(v) u {v}, dn(v) the lowest; up(v) == v iff v is a
 *               maximum, dn(v) == v iff v is a minimum.
 *   extremities Sec. 3.3 + Sec. 3.4: the forward integral line of v follows
 *               up until it stops at a maximum M (the "descending"
 *               segmentation label, Sec. 4.2), the backward one follows dn to
 *               a minimum m (the "ascending" label).  Computed by walking
 *               the line and memoising every vertex on it.  The label is the
 *               extremum's linear vertex index.
 *   MS id       Sec. 3.4 + Sec. 4.2.2: v1 ~ v2 iff (m, M) agree; the id of a
 *               vertex is the 0-based rank of its (m, M) pair among all
 *               distinct pairs that occur, sorted with m first.
 *   links       Sec. 3.2: lower/upper link of a vertex, their Euler
 *               characteristic and number of connected components
 *               (Banchoff's classification), from an explicit enumeration of
 *               the simplices of the triangulation.
 *   persistence Sec. 4.1 (simplification by persistence) + Sec. 6
 *               (thresholds): the 0-dimensional persistence pairs of the
 *               extrema -- sublevel-set components for minima, superlevel-set
 *               components for maxima, the elder rule at every merge.
 *   simplify    Sec. 4.1 + Sec. 6 again: the order after removing the
 *               extrema whose persistence is below a threshold, in the
 *               reading stated at ms_oracle_simplify (the paper names the
 *               operation and its thresholds, not its procedure).
 *
 * Vertex numbering: v = x + nx*(y + ny*z), x fastest (Fig. 1 numbers the
 * nodes of its grid along x first).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

enum { OR_F32 = 0, OR_F16 = 1, OR_F64 = 2 };
enum { OR_OK = 0, OR_ERR_NAN = 1, OR_ERR_ARG = 2, OR_ERR_NOMEM = 3, OR_ERR_CYCLE = 4 };

typedef struct {
  const void *data;
  int dtype;
  int64_t nx, ny, nz, n;
} field_t;

/* IEEE 754 binary16 -> double, written from the format's definition:
 * sign, 5-bit biased exponent (bias 15), 10-bit fraction; subnormals have
 * an implicit leading 0 and exponent -14. */
static double half_to_double(uint16_t h) {
  int s = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
  double v;
  if (e == 0)
    v = ldexp((double)m, -24);
  else if (e == 31)
    v = m ? NAN : INFINITY;
  else
    v = ldexp((double)(m + 1024), e - 25);
  return s ? -v : v;
}

static double value_at(const field_t *F, int64_t v) {
  switch (F->dtype) {
    case OR_F32: return (double)((const float *)F->data)[v];
    case OR_F16: return half_to_double(((const uint16_t *)F->data)[v]);
    default: return ((const double *)F->data)[v];
  }
}

/* u is lower than w in the total order of Sec. 4.1. */
static int lower(const field_t *F, int64_t u, int64_t w) {
  double a = value_at(F, u), b = value_at(F, w);
  if (a < b) return 1;
  if (a > b) return 0;
  return u < w;
}

static int make_field(field_t *F, const void *data, int dtype, const int64_t dims[3]) {
  if (!data || !dims || dims[0] < 1 || dims[1] < 1 || dims[2] < 1) return OR_ERR_ARG;
  if (dtype != OR_F32 && dtype != OR_F16 && dtype != OR_F64) return OR_ERR_ARG;
  F->data = data;
  F->dtype = dtype;
  F->nx = dims[0];
  F->ny = dims[1];
  F->nz = dims[2];
  F->n = dims[0] * dims[1] * dims[2];
  return OR_OK;
}

/* N(v): every grid vertex u != v with u - v in {0,1}^3 or v - u in {0,1}^3,
 * inside the box.  Returns the count (at most 14) and writes the indices in
 * increasing offset-loop order. */
static int neighbours_of(const field_t *F, int64_t v, int64_t *out) {
  int64_t x = v % F->nx, y = (v / F->nx) % F->ny, z = v / (F->nx * F->ny);
  int c = 0;
  for (int dz = -1; dz <= 1; ++dz)
    for (int dy = -1; dy <= 1; ++dy)
      for (int dx = -1; dx <= 1; ++dx) {
        if (!dx && !dy && !dz) continue;
        int nonneg = dx >= 0 && dy >= 0 && dz >= 0;
        int nonpos = dx <= 0 && dy <= 0 && dz <= 0;
        if (!nonneg && !nonpos) continue;
        int64_t X = x + dx, Y = y + dy, Z = z + dz;
        if (X < 0 || Y < 0 || Z < 0 || X >= F->nx || Y >= F->ny || Z >= F->nz) continue;
        out[c++] = X + F->nx * (Y + F->ny * Z);
      }
  return c;
}

int ms_oracle_neighbors(const int64_t dims[3], int64_t v, int64_t *out) {
  field_t F;
  static const float dummy = 0.f;
  if (make_field(&F, &dummy, OR_F32, dims) != OR_OK || v < 0 || v >= F.n) return -1;
  return neighbours_of(&F, v, out);
}

/* Highest (dir > 0) or lowest (dir < 0) vertex of N(v) u {v}. */
static int64_t steepest_at(const field_t *F, int64_t v, int dir) {
  int64_t nb[14];
  int c = neighbours_of(F, v, nb);
  int64_t best = v;
  for (int i = 0; i < c; ++i) {
    if (dir > 0) {
      if (lower(F, best, nb[i])) best = nb[i];
    } else {
      if (lower(F, nb[i], best)) best = nb[i];
    }
  }
  return best;
}

static int has_nan(const field_t *F) {
  for (int64_t v = 0; v < F->n; ++v)
    if (isnan(value_at(F, v))) return 1;
  return 0;
}

int ms_oracle_steepest(const void *field, int dtype, const int64_t dims[3], int32_t *up,
                       int32_t *dn) {
  field_t F;
  int st = make_field(&F, field, dtype, dims);
  if (st) return st;
  if (has_nan(&F)) return OR_ERR_NAN;
  for (int64_t v = 0; v < F.n; ++v) {
    up[v] = (int32_t)steepest_at(&F, v, +1);
    dn[v] = (int32_t)steepest_at(&F, v, -1);
  }
  return OR_OK;
}

/* Follow the line v -> ptr(v) -> ... to its fixed point, for every v,
 * memoising each vertex of a walked line so that each vertex is visited
 * once.  Fails (instead of looping) if a walk is longer than n steps. */
int ms_oracle_follow(const int32_t *ptr, int64_t n, int32_t *out) {
  int64_t *stack = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  if (!stack) return OR_ERR_NOMEM;
  for (int64_t v = 0; v < n; ++v) out[v] = -1;
  for (int64_t v = 0; v < n; ++v) {
    if (out[v] >= 0) continue;
    int64_t top = 0, w = v;
    while (out[w] < 0 && ptr[w] != w) {
      if (top >= n) {
        free(stack);
        return OR_ERR_CYCLE;
      }
      stack[top++] = w;
      w = ptr[w];
    }
    int32_t root = out[w] >= 0 ? out[w] : (int32_t)w;
    out[w] = root;
    while (top > 0) out[stack[--top]] = root;
  }
  free(stack);
  return OR_OK;
}

/* The same fixed point, walking every vertex's line independently. */
int ms_oracle_follow_brute(const int32_t *ptr, int64_t n, int32_t *out) {
  for (int64_t v = 0; v < n; ++v) {
    int64_t w = v, steps = 0;
    while (ptr[w] != w) {
      w = ptr[w];
      if (++steps > n) return OR_ERR_CYCLE;
    }
    out[v] = (int32_t)w;
  }
  return OR_OK;
}

/* Walk the integral line of one vertex straight from the field: returns the
 * extremum reached (dir > 0: maximum, dir < 0: minimum) and its number of
 * steps, or -1 if more than max_steps steps are taken. */
int64_t ms_oracle_walk(const void *field, int dtype, const int64_t dims[3], int64_t v, int dir,
                       int64_t max_steps, int64_t *steps_out) {
  field_t F;
  if (make_field(&F, field, dtype, dims) || v < 0 || v >= F.n) return -1;
  int64_t steps = 0, w = v;
  for (;;) {
    int64_t s = steepest_at(&F, w, dir);
    if (s == w) break;
    w = s;
    if (++steps > max_steps) return -1;
  }
  if (steps_out) *steps_out = steps;
  return w;
}

/* up(v) and dn(v) of single vertices, evaluated straight from the field. */
int ms_oracle_steepest_at(const void *field, int dtype, const int64_t dims[3], const int64_t *vs,
                          int64_t count, int32_t *up, int32_t *dn) {
  field_t F;
  int st = make_field(&F, field, dtype, dims);
  if (st) return st;
  for (int64_t i = 0; i < count; ++i) {
    if (vs[i] < 0 || vs[i] >= F.n) return OR_ERR_ARG;
    up[i] = (int32_t)steepest_at(&F, vs[i], +1);
    dn[i] = (int32_t)steepest_at(&F, vs[i], -1);
  }
  return OR_OK;
}

static int cmp_i64(const void *a, const void *b) {
  int64_t x = *(const int64_t *)a, y = *(const int64_t *)b;
  return (x > y) - (x < y);
}

/* Dense rank of the (m, M) pair of every vertex among the distinct pairs,
 * lexicographic with m first.  Returns the number of distinct pairs K, or
 * -1 on allocation failure. */
int64_t ms_oracle_ms_rank(const int32_t *asc, const int32_t *desc, int64_t n, int32_t *ms) {
  if (n <= 0) return 0;
  int64_t *key = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int64_t *uniq = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  if (!key || !uniq) {
    free(key);
    free(uniq);
    return -1;
  }
  for (int64_t v = 0; v < n; ++v) {
    key[v] = (int64_t)asc[v] * n + (int64_t)desc[v];
    uniq[v] = key[v];
  }
  qsort(uniq, (size_t)n, sizeof(int64_t), cmp_i64);
  int64_t k = 0;
  for (int64_t i = 0; i < n; ++i)
    if (i == 0 || uniq[i] != uniq[k - 1]) uniq[k++] = uniq[i];
  for (int64_t v = 0; v < n; ++v) {
    int64_t lo = 0, hi = k; /* first index with uniq[i] >= key[v] */
    while (lo < hi) {
      int64_t mid = lo + (hi - lo) / 2;
      if (uniq[mid] < key[v])
        lo = mid + 1;
      else
        hi = mid;
    }
    ms[v] = (int32_t)lo;
  }
  free(key);
  free(uniq);
  return k;
}

/* The whole segmentation of one field: up/dn (may be NULL), the ascending
 * labels (minimum reached), the descending labels (maximum reached), the MS
 * ids and their count. */
int ms_oracle_segment(const void *field, int dtype, const int64_t dims[3], int32_t *asc,
                      int32_t *desc, int32_t *ms, int64_t *k_out, int32_t *up_out,
                      int32_t *dn_out) {
  field_t F;
  int st = make_field(&F, field, dtype, dims);
  if (st) return st;
  if (F.n > INT32_MAX) return OR_ERR_ARG;
  int32_t *up = up_out ? up_out : (int32_t *)malloc(sizeof(int32_t) * (size_t)F.n);
  int32_t *dn = dn_out ? dn_out : (int32_t *)malloc(sizeof(int32_t) * (size_t)F.n);
  if (!up || !dn) {
    if (!up_out) free(up);
    if (!dn_out) free(dn);
    return OR_ERR_NOMEM;
  }
  st = ms_oracle_steepest(field, dtype, dims, up, dn);
  if (!st) st = ms_oracle_follow(up, F.n, desc);
  if (!st) st = ms_oracle_follow(dn, F.n, asc);
  if (!st) {
    int64_t k = ms_oracle_ms_rank(asc, desc, F.n, ms);
    if (k < 0)
      st = OR_ERR_NOMEM;
    else if (k_out)
      *k_out = k;
  }
  if (!up_out) free(up);
  if (!dn_out) free(dn);
  return st;
}

/* ---------------------------------------------------------------------
 * Links (Sec. 3.2).  The triangulation is enumerated explicitly: over the
 * axes of extent >= 2 (d of them), every grid cell with minimum corner c is
 * cut into d! simplices, one per ordering (a_1..a_d) of the axes, with
 * vertices c, c+e_a1, c+e_a1+e_a2, ..., c+e_a1+..+e_ad.  The link of v is
 * the set of faces, not containing v, of the simplices containing v.
 * --------------------------------------------------------------------- */
typedef struct {
  int64_t v[3];
  int k; /* number of vertices, 1..3 */
} lsimp_t;

static int cmp_lsimp(const void *a, const void *b) {
  const lsimp_t *p = (const lsimp_t *)a, *q = (const lsimp_t *)b;
  if (p->k != q->k) return p->k - q->k;
  for (int i = 0; i < p->k; ++i)
    if (p->v[i] != q->v[i]) return p->v[i] < q->v[i] ? -1 : 1;
  return 0;
}

static int64_t uf_find(int64_t *par, int64_t i) {
  while (par[i] != i) i = par[i];
  return i;
}

/* Per vertex, into out[5*v .. 5*v+4]: chi(Lk-), chi(Lk+), number of
 * connected components of Lk- and of Lk+, and 1 if v is interior to the
 * box in every axis of extent >= 2.  Also returns, through link_out (may be
 * NULL, 14 entries per vertex, -1 padded), the vertex set of Lk(v). */
int ms_oracle_link_stats(const void *field, int dtype, const int64_t dims[3], int32_t *out,
                         int64_t *link_out) {
  field_t F;
  int st = make_field(&F, field, dtype, dims);
  if (st) return st;
  if (has_nan(&F)) return OR_ERR_NAN;
  int64_t ext[3] = {F.nx, F.ny, F.nz};
  int axes[3], d = 0;
  for (int a = 0; a < 3; ++a)
    if (ext[a] >= 2) axes[d++] = a;
  /* orderings of the active axes */
  int perms[6][3], np = 0;
  if (d == 0) {
    np = 0;
  } else if (d == 1) {
    perms[0][0] = 0;
    np = 1;
  } else if (d == 2) {
    perms[0][0] = 0; perms[0][1] = 1;
    perms[1][0] = 1; perms[1][1] = 0;
    np = 2;
  } else {
    int p[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    memcpy(perms, p, sizeof(p));
    np = 6;
  }
  lsimp_t buf[8 * 6 * 7];
  for (int64_t v = 0; v < F.n; ++v) {
    int64_t p[3] = {v % F.nx, (v / F.nx) % F.ny, v / (F.nx * F.ny)};
    int nb = 0;
    for (int s = 0; s < (1 << d); ++s) {
      int64_t c[3] = {p[0], p[1], p[2]};
      int ok = 1;
      for (int i = 0; i < d; ++i) {
        int a = axes[i];
        if (s & (1 << i)) c[a] -= 1;
        if (c[a] < 0 || c[a] > ext[a] - 2) ok = 0;
      }
      if (!ok) continue;
      for (int q = 0; q < np; ++q) {
        /* chain vertices of this simplex */
        int64_t chain[4][3];
        memcpy(chain[0], c, sizeof(c));
        for (int j = 1; j <= d; ++j) {
          memcpy(chain[j], chain[j - 1], sizeof(c));
          chain[j][axes[perms[q][j - 1]]] += 1;
        }
        int at = -1;
        for (int j = 0; j <= d; ++j)
          if (chain[j][0] == p[0] && chain[j][1] == p[1] && chain[j][2] == p[2]) at = j;
        if (at < 0) continue;
        int64_t opp[3];
        int m = 0;
        for (int j = 0; j <= d; ++j)
          if (j != at) opp[m++] = chain[j][0] + F.nx * (chain[j][1] + F.ny * chain[j][2]);
        /* all non-empty faces of the opposite simplex */
        for (int sub = 1; sub < (1 << m); ++sub) {
          lsimp_t t;
          t.k = 0;
          for (int j = 0; j < m; ++j)
            if (sub & (1 << j)) t.v[t.k++] = opp[j];
          for (int i = 1; i < t.k; ++i) /* sort the face's vertices */
            for (int j = i; j > 0 && t.v[j - 1] > t.v[j]; --j) {
              int64_t tmp = t.v[j];
              t.v[j] = t.v[j - 1];
              t.v[j - 1] = tmp;
            }
          for (int j = t.k; j < 3; ++j) t.v[j] = -1;
          buf[nb++] = t;
        }
      }
    }
    qsort(buf, (size_t)nb, sizeof(lsimp_t), cmp_lsimp);
    int nu = 0;
    for (int i = 0; i < nb; ++i)
      if (nu == 0 || cmp_lsimp(&buf[i], &buf[nu - 1]) != 0) buf[nu++] = buf[i];
    /* Euler characteristics and components of the lower and upper links */
    int chi_lo = 0, chi_up = 0;
    int64_t lv[14];
    int nlv = 0;
    for (int i = 0; i < nu; ++i) {
      int all_lo = 1, all_up = 1;
      for (int j = 0; j < buf[i].k; ++j) {
        if (!lower(&F, buf[i].v[j], v)) all_lo = 0;
        if (!lower(&F, v, buf[i].v[j])) all_up = 0;
      }
      int sign = (buf[i].k % 2 == 1) ? 1 : -1;
      if (all_lo) chi_lo += sign;
      if (all_up) chi_up += sign;
      if (buf[i].k == 1 && nlv < 14) lv[nlv++] = buf[i].v[0];
    }
    int comps[2] = {0, 0};
    for (int side = 0; side < 2; ++side) {
      int64_t par[14];
      int in[14];
      for (int i = 0; i < nlv; ++i) {
        par[i] = i;
        in[i] = side == 0 ? lower(&F, lv[i], v) : lower(&F, v, lv[i]);
      }
      for (int i = 0; i < nu; ++i) {
        if (buf[i].k != 2) continue;
        int a = -1, b = -1;
        for (int j = 0; j < nlv; ++j) {
          if (lv[j] == buf[i].v[0]) a = j;
          if (lv[j] == buf[i].v[1]) b = j;
        }
        if (a < 0 || b < 0 || !in[a] || !in[b]) continue;
        int64_t ra = uf_find(par, a), rb = uf_find(par, b);
        if (ra != rb) par[ra] = rb;
      }
      for (int i = 0; i < nlv; ++i)
        if (in[i] && uf_find(par, i) == i) comps[side]++;
    }
    int interior = 1;
    for (int i = 0; i < d; ++i) {
      int a = axes[i];
      if (p[a] == 0 || p[a] == ext[a] - 1) interior = 0;
    }
    out[5 * v + 0] = chi_lo;
    out[5 * v + 1] = chi_up;
    out[5 * v + 2] = comps[0];
    out[5 * v + 3] = comps[1];
    out[5 * v + 4] = interior;
    if (link_out) {
      for (int i = 0; i < 14; ++i) link_out[14 * v + i] = i < nlv ? lv[i] : -1;
    }
  }
  return OR_OK;
}

/* ---- the index pass of the multi-label marching triangles / tetrahedra --
 *
 * Sec. 4.3 (region-separating geometry).  Every simplex of the triangulation
 * whose vertices carry more than one label is split; the pass that precedes
 * the geometry computes, per simplex, a binary code of its label
 * configuration and the number of separating elements it produces, and the
 * exclusive prefix sum of those numbers (where each cell's output starts).
 *
 * Simplices: the Freudenthal cells are cut along the (0,..,0)->(1,..,1)
 * diagonal into one simplex per order in which the axes are stepped.
 *   2D: cell (x, y), x < nx-1, y < ny-1, index c = x + (nx-1) y, triangles
 *       t = 2c + p, p = 0: x then y, p = 1: y then x.
 *   3D: cell (x, y, z), index c = x + (nx-1)(y + (ny-1) z), tetrahedra
 *       t = 6c + p with axis orders p = 0: xyz, 1: xzy, 2: yxz, 3: yzx,
 *       4: zxy, 5: zyx.
 * The vertices a, b, c (, d) of a simplex are its chain in stepping order,
 * which is also increasing vertex index.
 *
 * Code (Sec. 4.3, Fig. 4, Tab. 1): the first vertex gets local label 0; each
 * later vertex gets the local label of the first earlier vertex with the same
 * label, or its own position (1, 2, 3) if none has it.  Triangle code =
 * b << 2 | c (3 bits); tetrahedron code = b << 4 | c << 2 | d (5 bits).
 * Separating elements per code (Figs. 5 and 6): a triangle with two labels is
 * cut by one segment, with three by three segments meeting at its centre; a
 * tetrahedron whose labels split 1 + 3 is cut by one triangle, 2 + 2 by two,
 * with three labels by five and with four labels by twelve.
 */

static int tri_code(int32_t la, int32_t lb, int32_t lc) {
  const int b = lb == la ? 0 : 1;
  const int c = lc == la ? 0 : (lc == lb ? b : 2);
  return (b << 2) | c;
}

static int tri_count(int code) {
  int32_t l[3] = {0, code >> 2, code & 3};
  int distinct = 1;
  if (l[1] != l[0]) ++distinct;
  if (l[2] != l[0] && l[2] != l[1]) ++distinct;
  return distinct == 1 ? 0 : distinct == 2 ? 1 : 3;
}

static int tet_code(const int32_t *lab) {
  int loc[4];
  for (int k = 0; k < 4; ++k) {
    loc[k] = k;
    for (int j = 0; j < k; ++j)
      if (lab[j] == lab[k]) {
        loc[k] = loc[j];
        break;
      }
  }
  return (loc[1] << 4) | (loc[2] << 2) | loc[3];
}

static int tet_count(int code) {
  const int loc[4] = {0, code >> 4, (code >> 2) & 3, code & 3};
  int size[4] = {0, 0, 0, 0};
  for (int k = 0; k < 4; ++k) size[loc[k]]++;
  int distinct = 0, largest = 0;
  for (int k = 0; k < 4; ++k)
    if (size[k]) {
      ++distinct;
      if (size[k] > largest) largest = size[k];
    }
  if (distinct == 1) return 0;
  if (distinct == 2) return largest == 3 ? 1 : 2;
  return distinct == 3 ? 5 : 12;
}

/* Code and element count of one label configuration (for the pins). */
int ms_oracle_simplex_code(int nverts, const int32_t *labels, int *count) {
  if (nverts == 3) {
    const int code = tri_code(labels[0], labels[1], labels[2]);
    *count = tri_count(code);
    return code;
  }
  if (nverts == 4) {
    const int code = tet_code(labels);
    *count = tet_count(code);
    return code;
  }
  return -1;
}

/* codes: one byte per simplex; cell_offsets: per cell, the exclusive prefix
 * sum over cells of the cell's element count (sum over its simplices);
 * *total: the sum over all cells.  Grids with a dimension of extent 1 other
 * than nz (2D is nz == 1) have no cells. */
int ms_oracle_simplex_count_mode(int nverts, const int32_t *labels, int mode);
static int count_of_mode(int nverts, const int32_t *labels, int mode);

int ms_oracle_simplex_index_mode(const int32_t *labels, const int64_t dims[3], int mode,
                                 uint8_t *codes, int64_t *cell_offsets, int64_t *total);

int ms_oracle_simplex_index(const int32_t *labels, const int64_t dims[3], uint8_t *codes,
                            int64_t *cell_offsets, int64_t *total) {
  return ms_oracle_simplex_index_mode(labels, dims, 0, codes, cell_offsets, total);
}

/* mode 0: separator elements per cell; mode 1: boundary elements */
int ms_oracle_simplex_index_mode(const int32_t *labels, const int64_t dims[3], int mode,
                                 uint8_t *codes, int64_t *cell_offsets, int64_t *total) {
  if (mode != 0 && mode != 1) return OR_ERR_ARG;
  const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
  if (nx < 1 || ny < 1 || nz < 1) return OR_ERR_ARG;
  const int two_d = nz == 1;
  const int64_t cx = nx - 1, cy = ny - 1, cz = two_d ? 1 : nz - 1;
  int64_t run = 0;
  if (cx > 0 && cy > 0 && cz > 0) {
    for (int64_t z = 0; z < cz; ++z)
      for (int64_t y = 0; y < cy; ++y)
        for (int64_t x = 0; x < cx; ++x) {
          const int64_t c = x + cx * (y + cy * z);
          const int64_t v0 = x + nx * (y + ny * z);
          int cell_count = 0;
          if (two_d) {
            const int64_t step[2][2] = {{1, nx}, {nx, 1}};
            for (int p = 0; p < 2; ++p) {
              const int64_t va = v0, vb = va + step[p][0], vc = vb + step[p][1];
              const int code = tri_code(labels[va], labels[vb], labels[vc]);
              codes[2 * c + p] = (uint8_t)code;
              const int32_t lab3[3] = {labels[va], labels[vb], labels[vc]};
              cell_count += mode == 0 ? tri_count(code) : count_of_mode(3, lab3, 1);
            }
          } else {
            const int64_t ax[3] = {1, nx, nx * ny};
            const int order[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
            for (int p = 0; p < 6; ++p) {
              int32_t lab[4];
              int64_t v = v0;
              lab[0] = labels[v];
              for (int k = 0; k < 3; ++k) {
                v += ax[order[p][k]];
                lab[k + 1] = labels[v];
              }
              const int code = tet_code(lab);
              codes[6 * c + p] = (uint8_t)code;
              cell_count += mode == 0 ? tet_count(code) : count_of_mode(4, lab, 1);
            }
          }
          cell_offsets[c] = run;
          run += cell_count;
        }
  }
  *total = run;
  return OR_OK;
}

/* ---- the geometry pass of the multi-label marching triangles / tetrahedra --
 *
 * Sec. 4.3 ("Region Separating Geometries"), after the index pass:
 *
 *  mode 0, region separators (Figs. 5, 6): in a simplex with several labels,
 *   triangle, labels 2+1: one segment joining the midpoints of the two edges at
 *     the lone vertex; 3 labels: three segments from the triangle's centre to
 *     its edge midpoints (ab, bc, ac);
 *   tetrahedron, 3+1: the triangle of the midpoints of the three edges at the
 *     lone vertex; 2+2 (pairs {p1,p2}, {q1,q2}): the quad of the midpoints of
 *     the four edges between the pairs, as triangles (p1q1, p1q2, p2q1),
 *     (p1q2, p2q1, p2q2); 2+1+1 (pair P < Q, singles R < S): with T1, T2 the
 *     centres of the faces PRS, QRS: (T1,T2,PR), (T2,PR,QR), (T1,T2,RS),
 *     (T1,T2,PS), (T2,PS,QS); four labels: from the tetrahedron's centre C,
 *     for each face (abc, abd, acd, bcd) with centre T and each of its edges
 *     e (in the order ab, ac, ad, bc, bd, cd): (C, T, e).
 *   Each element separates the labels at the two ends of its first edge
 *   midpoint's edge; the pair is stored smaller label first.
 *  mode 1, region boundaries: a tetrahedron with exactly three vertices of one
 *   label gives the triangle of those three vertices (stored in chain order),
 *   separating (that label, the fourth vertex's label), smaller first; a
 *   triangle (2D) with exactly two vertices of one label gives that edge.
 *
 * Element order: cells in index order, simplices in chain order p, elements
 * in the order above.  Points are grid coordinates (x, y[, z]) in float32:
 * a midpoint is (u + v) / 2, a face centre (u + v + w) / 3, the tetrahedron
 * centre the sum of its corners / 4: each coordinate is the exact sum S of
 * the corners' integer coordinates divided by the corner count n, rounded
 * once to the nearest float32 (ties to even).  It is computed as
 * (float)((double)S / n): for n = 1, 2, 4 the double quotient is exact; for
 * n = 3, S / 3 is an integer (exact) or differs from every float32 rounding
 * midpoint m by at least 2^(E-25) / 3 (S and 3m are both multiples of
 * 2^(E-25), E the exponent of S / 3), far more than the double rounding
 * error 2^(E-53), so rounding the double to float32 rounds S / 3 itself.
 */

typedef struct {
  float *pos;      /* dim floats per point */
  int32_t *pairs;  /* 2 per element (may be NULL) */
  int dim, npts;   /* coordinates per point, points per element */
  int64_t at;      /* next element */
} geo_out;

/* The mean of n corner coordinates whose exact sum is sum (n in 1..4),
 * rounded once to float32 (see above). */
float ms_oracle_coord_mean(int64_t sum, int n) { return (float)((double)sum / (double)n); }

static void geo_point(geo_out *o, int k, const int64_t (*c)[3], const int *ids, int nids) {
  for (int d = 0; d < o->dim; ++d) {
    int64_t sum = 0;
    for (int i = 0; i < nids; ++i) sum += c[ids[i]][d];
    o->pos[(o->at * o->npts + k) * o->dim + d] = ms_oracle_coord_mean(sum, nids);
  }
}

static void geo_pair(geo_out *o, int32_t l1, int32_t l2) {
  if (o->pairs) {
    o->pairs[2 * o->at] = l1 < l2 ? l1 : l2;
    o->pairs[2 * o->at + 1] = l1 < l2 ? l2 : l1;
  }
}

/* one element whose points are the centroids of the index sets ids[k] */
static void geo_elem(geo_out *o, const int64_t (*c)[3], const int (*ids)[4], const int *nids,
                     int32_t l1, int32_t l2) {
  for (int k = 0; k < o->npts; ++k) geo_point(o, k, c, ids[k], nids[k]);
  geo_pair(o, l1, l2);
  o->at++;
}

static void tri_separators(geo_out *o, const int64_t (*c)[3], const int32_t *lab) {
  const int code = tri_code(lab[0], lab[1], lab[2]);
  const int b = code >> 2, cc = code & 3;
  if (code == 0) return;
  if (code == 6) {
    const int e[3][2] = {{0, 1}, {1, 2}, {0, 2}};
    for (int k = 0; k < 3; ++k) {
      const int ids[2][4] = {{0, 1, 2}, {e[k][0], e[k][1]}};
      const int n[2] = {3, 2};
      geo_elem(o, c, ids, n, lab[e[k][0]], lab[e[k][1]]);
    }
    return;
  }
  /* two labels: the lone vertex */
  const int loc[3] = {0, b, cc};
  int lone = -1;
  for (int k = 0; k < 3; ++k) {
    int same = 0;
    for (int j = 0; j < 3; ++j) same += loc[j] == loc[k];
    if (same == 1) lone = k;
  }
  int oth[2], no = 0;
  for (int k = 0; k < 3; ++k)
    if (k != lone) oth[no++] = k;
  const int ids[2][4] = {{lone, oth[0]}, {lone, oth[1]}};
  const int n[2] = {2, 2};
  geo_elem(o, c, ids, n, lab[lone], lab[oth[0]]);
}

static void tet_separators(geo_out *o, const int64_t (*c)[3], const int32_t *lab) {
  const int code = tet_code(lab);
  const int loc[4] = {0, code >> 4, (code >> 2) & 3, code & 3};
  int size[4] = {0, 0, 0, 0};
  for (int k = 0; k < 4; ++k) size[loc[k]]++;
  int classes = 0;
  for (int k = 0; k < 4; ++k) classes += size[k] > 0;
  const int n3[3] = {2, 2, 2};
  if (classes == 1) return;
  if (classes == 2) {
    int big = 0;
    for (int k = 0; k < 4; ++k)
      if (size[k] > size[big]) big = k;
    if (size[big] == 3) {
      int lone = 0, oth[3], no = 0;
      for (int k = 0; k < 4; ++k) {
        if (loc[k] != big) lone = k;
        else oth[no++] = k;
      }
      const int ids[3][4] = {{lone, oth[0]}, {lone, oth[1]}, {lone, oth[2]}};
      geo_elem(o, c, ids, n3, lab[lone], lab[oth[0]]);
    } else {
      int p[2], q[2], np = 0, nq = 0;
      for (int k = 0; k < 4; ++k) {
        if (loc[k] == 0) p[np++] = k;
        else q[nq++] = k;
      }
      const int t1[3][4] = {{p[0], q[0]}, {p[0], q[1]}, {p[1], q[0]}};
      const int t2[3][4] = {{p[0], q[1]}, {p[1], q[0]}, {p[1], q[1]}};
      geo_elem(o, c, t1, n3, lab[p[0]], lab[q[0]]);
      geo_elem(o, c, t2, n3, lab[p[0]], lab[q[1]]);
    }
    return;
  }
  if (classes == 3) {
    int P = -1, Q = -1, R = -1, S = -1;
    for (int k = 0; k < 4; ++k) {
      if (size[loc[k]] == 2) {
        if (P < 0) P = k;
        else Q = k;
      } else {
        if (R < 0) R = k;
        else S = k;
      }
    }
    const int n[3] = {3, 3, 2}, nb[3] = {3, 2, 2};
    {
      const int ids[3][4] = {{P, R, S}, {Q, R, S}, {P, R}};  /* T1, T2, PR */
      geo_elem(o, c, ids, n, lab[P], lab[R]);
    }
    {
      const int ids[3][4] = {{Q, R, S}, {P, R}, {Q, R}};  /* T2, PR, QR */
      geo_elem(o, c, ids, nb, lab[P], lab[R]);
    }
    {
      const int ids[3][4] = {{P, R, S}, {Q, R, S}, {R, S}};  /* T1, T2, RS */
      geo_elem(o, c, ids, n, lab[R], lab[S]);
    }
    {
      const int ids[3][4] = {{P, R, S}, {Q, R, S}, {P, S}};  /* T1, T2, PS */
      geo_elem(o, c, ids, n, lab[P], lab[S]);
    }
    {
      const int ids[3][4] = {{Q, R, S}, {P, S}, {Q, S}};  /* T2, PS, QS */
      geo_elem(o, c, ids, nb, lab[P], lab[S]);
    }
    return;
  }
  /* four labels */
  const int faces[4][3] = {{0, 1, 2}, {0, 1, 3}, {0, 2, 3}, {1, 2, 3}};
  for (int f = 0; f < 4; ++f) {
    const int e[3][2] = {{faces[f][0], faces[f][1]}, {faces[f][0], faces[f][2]},
                         {faces[f][1], faces[f][2]}};
    for (int k = 0; k < 3; ++k) {
      const int ids[3][4] = {{0, 1, 2, 3}, {faces[f][0], faces[f][1], faces[f][2]}, {e[k][0], e[k][1]}};
      const int n[3] = {4, 3, 2};
      geo_elem(o, c, ids, n, lab[e[k][0]], lab[e[k][1]]);
    }
  }
}

static void boundaries(geo_out *o, const int64_t (*c)[3], const int32_t *lab, int nv) {
  /* the vertices sharing a label that exactly nv - 1 of them carry */
  for (int lone = 0; lone < nv; ++lone) {
    int same = 0;
    for (int k = 0; k < nv; ++k)
      if (k != lone && lab[k] == lab[(lone + 1) % nv]) ++same;
    int all_same = same == nv - 1, lone_differs = lab[lone] != lab[(lone + 1) % nv];
    if (all_same && lone_differs) {
      int ids[3][4], n[3], m = 0;
      for (int k = 0; k < nv; ++k)
        if (k != lone) {
          ids[m][0] = k;
          n[m++] = 1;
        }
      geo_elem(o, c, ids, n, lab[(lone + 1) % nv], lab[lone]);
      return;
    }
  }
}

static int count_of_mode(int nverts, const int32_t *labels, int mode) {
  return ms_oracle_simplex_count_mode(nverts, labels, mode);
}

int ms_oracle_simplex_count_mode(int nverts, const int32_t *labels, int mode) {
  int cnt = 0;
  if (mode == 0) {
    ms_oracle_simplex_code(nverts, labels, &cnt);
    return cnt;
  }
  for (int lone = 0; lone < nverts; ++lone) {
    int same = 0;
    for (int k = 0; k < nverts; ++k)
      if (k != lone && labels[k] == labels[(lone + 1) % nverts]) ++same;
    if (same == nverts - 1 && labels[lone] != labels[(lone + 1) % nverts]) return 1;
  }
  return 0;
}

/* Elements of every simplex in order (see above); pos: total * npts * dim
 * floats, pairs: total * 2 int32 (may be NULL).  *total receives the count;
 * with pos == NULL only the count is computed. */
int ms_oracle_simplex_geometry(const int32_t *labels, const int64_t dims[3], int mode, float *pos,
                               int32_t *pairs, int64_t *total) {
  const int64_t nx = dims[0], ny = dims[1], nz = dims[2];
  if (nx < 1 || ny < 1 || nz < 1 || (mode != 0 && mode != 1)) return OR_ERR_ARG;
  const int two_d = nz == 1;
  const int64_t cx = nx - 1, cy = ny - 1, cz = two_d ? 1 : nz - 1;
  geo_out o;
  o.pos = pos;
  o.pairs = pairs;
  o.dim = two_d ? 2 : 3;
  o.npts = two_d ? 2 : 3;
  o.at = 0;
  int64_t count = 0;
  if (cx > 0 && cy > 0 && cz > 0) {
    for (int64_t z = 0; z < cz; ++z)
      for (int64_t y = 0; y < cy; ++y)
        for (int64_t x = 0; x < cx; ++x) {
          const int nv = two_d ? 3 : 4;
          const int np = two_d ? 2 : 6;
          const int order[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
          for (int p = 0; p < np; ++p) {
            int64_t c[4][3];
            int32_t lab[4];
            int64_t pt[3] = {x, y, z};
            for (int k = 0; k < nv; ++k) {
              if (k > 0) pt[two_d ? (p == 0 ? k - 1 : 2 - k) : order[p][k - 1]] += 1;
              c[k][0] = pt[0];
              c[k][1] = pt[1];
              c[k][2] = pt[2];
              lab[k] = labels[pt[0] + nx * (pt[1] + ny * pt[2])];
            }
            if (!pos) {
              count += ms_oracle_simplex_count_mode(nv, lab, mode);
              continue;
            }
            if (mode == 1)
              boundaries(&o, (const int64_t(*)[3])c, lab, nv);
            else if (two_d)
              tri_separators(&o, (const int64_t(*)[3])c, lab);
            else
              tet_separators(&o, (const int64_t(*)[3])c, lab);
          }
        }
  }
  *total = pos ? o.at : count;
  return OR_OK;
}

/* ---- 0-dimensional persistence of the extrema --------------------------------
 *
 * The paper removes non-persistent critical points by topological
 * simplification before segmenting (Sec. 4.1) and quotes persistence
 * thresholds for its runs (Sec. 6); the pairing that decides which extrema a
 * threshold removes is the persistence pairing of the sublevel-set components
 * (minima) or superlevel-set components (maxima), written out here from its
 * textbook definition on the vertex-edge graph of the triangulation:
 *
 *   vertices enter one at a time in the order of Sec. 4.1 (increasing for
 *   minima, decreasing for maxima); a vertex with no earlier neighbour starts
 *   a component -- it is an extremum, born there; a vertex with earlier
 *   neighbours joins their components, and where it joins several, every
 *   component but the one whose extremum entered first ends there (the elder
 *   rule): its extremum dies at that vertex.  The extremum that entered first
 *   of a connected grid never dies.
 *
 * direction -1: minima, +1: maxima.  extremum / death: int32[n] (at most one
 * pair per vertex); pair i = (extremum[i], death[i]), death -1 for the one
 * that never dies, pairs in increasing extremum index; *npairs receives the
 * count.  The persistence of a pair is |f(death) - f(extremum)|. */
typedef struct {
  double value;
  int64_t index;
} ordered_t;

static int cmp_ordered(const void *a, const void *b) {
  const ordered_t *x = (const ordered_t *)a, *y = (const ordered_t *)b;
  if (x->value < y->value) return -1;
  if (x->value > y->value) return 1;
  return x->index < y->index ? -1 : (x->index > y->index);
}

/* root of v's component, compressing the path on the way */
static int64_t uf_root(int64_t *parent, int64_t v) {
  int64_t r = v;
  while (parent[r] != r) r = parent[r];
  while (parent[v] != r) {
    const int64_t next = parent[v];
    parent[v] = r;
    v = next;
  }
  return r;
}

int ms_oracle_persistence(const void *field, int dtype, const int64_t dims[3], int direction,
                          int32_t *extremum, int32_t *death, int64_t *npairs) {
  field_t F;
  int st = make_field(&F, field, dtype, dims);
  if (st != OR_OK) return st;
  if ((direction != 1 && direction != -1) || !extremum || !death || !npairs) return OR_ERR_ARG;
  if (F.n > 2147483647LL) return OR_ERR_ARG;
  if (has_nan(&F)) return OR_ERR_NAN;
  const int64_t n = F.n;
  ordered_t *ord = (ordered_t *)malloc(sizeof(ordered_t) * (size_t)n);
  int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);     /* entry step of a vertex */
  int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int64_t *eldest = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);  /* a root's first extremum */
  int32_t *dies = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);    /* per extremum, or -2 */
  if (!ord || !pos || !parent || !eldest || !dies) {
    free(ord);
    free(pos);
    free(parent);
    free(eldest);
    free(dies);
    return OR_ERR_NOMEM;
  }
  for (int64_t v = 0; v < n; ++v) {
    ord[v].value = value_at(&F, v);
    ord[v].index = v;
    dies[v] = -2; /* not an extremum */
  }
  qsort(ord, (size_t)n, sizeof(ordered_t), cmp_ordered);
  for (int64_t s = 0; s < n; ++s) {
    const int64_t v = ord[direction < 0 ? s : n - 1 - s].index;
    pos[v] = s;
  }
  for (int64_t v = 0; v < n; ++v) parent[v] = -1; /* not entered yet */
  for (int64_t s = 0; s < n; ++s) {
    const int64_t v = ord[direction < 0 ? s : n - 1 - s].index;
    int64_t nb[14], roots[14];
    const int c = neighbours_of(&F, v, nb);
    int nr = 0;
    for (int i = 0; i < c; ++i) {
      if (parent[nb[i]] < 0) continue; /* enters later */
      const int64_t r = uf_root(parent, nb[i]);
      int seen = 0;
      for (int j = 0; j < nr; ++j) seen |= roots[j] == r;
      if (!seen) roots[nr++] = r;
    }
    if (nr == 0) { /* an extremum: a new component */
      parent[v] = v;
      eldest[v] = v;
      dies[v] = -1;
      continue;
    }
    /* the component whose extremum entered first survives */
    int keep = 0;
    for (int j = 1; j < nr; ++j)
      if (pos[eldest[roots[j]]] < pos[eldest[roots[keep]]]) keep = j;
    const int64_t root = roots[keep];
    for (int j = 0; j < nr; ++j) {
      if (j == keep) continue;
      dies[eldest[roots[j]]] = (int32_t)v;
      parent[roots[j]] = root;
    }
    parent[v] = root;
  }
  int64_t k = 0;
  for (int64_t v = 0; v < n; ++v)
    if (dies[v] != -2) {
      extremum[k] = (int32_t)v;
      death[k] = dies[v];
      ++k;
    }
  *npairs = k;
  free(ord);
  free(pos);
  free(parent);
  free(eldest);
  free(dies);
  return OR_OK;
}

/* ---- simplification of the order ----------------------------------------
 * Sec. 4.1 simplifies the field before segmenting it, removing the extrema
 * whose persistence lies below a threshold (Sec. 6 quotes the thresholds);
 * the paper does not spell out the procedure.  This follows the reading
 * written down for it, one pass per extremum type (minima on sublevel sets,
 * then maxima on superlevel sets, each on the order the previous pass left):
 *   1. the pairs of the pass by the elder rule on the current order (as in
 *      ms_oracle_persistence);
 *   2. an extremum m paired with d is removed when |value(d) - value(m)| is
 *      below the threshold; its region R(m) is m's component among the
 *      vertices that enter before d;
 *   3. regions are nested or disjoint; each vertex takes the outermost
 *      removed region that contains it.  The vertices of a region take d's
 *      value and enter right after d, before any vertex that entered after d,
 *      in order of their breadth-first distance from d inside the region and
 *      then of their vertex index.
 * A minima pass leaves exactly the minima of persistence >= threshold, but
 * the maxima pass after it can leave new minima: a flattened maximum region
 * that reaches the box boundary can hold a vertex with no lower neighbour
 * (the one farthest from d), of persistence 0.  So with both kinds the passes
 * alternate until a maxima pass removes nothing (on random fields: two rounds,
 * at most three); the order then has no extremum of either kind below the
 * threshold.  A vertex region that d does not reach, or two regions that
 * overlap without nesting, would contradict the reading: OR_ERR_REGIONS.
 * rank[v]: the position of v in the simplified order, ascending (0 .. n-1);
 * value[v]: the value it carries; removed[0], removed[1]: the minima and the
 * maxima removed, removed[2]: the rounds run.  which: 1 one minima pass, 2 one
 * maxima pass, 3 both kinds, alternating (minima first). */
enum { OR_ERR_REGIONS = 5 };
static const int64_t kSimplifyRounds = 256;

typedef struct {
  int64_t k0, k1, k2;
} skey_t;

static int cmp_skey(const void *a, const void *b) {
  const skey_t *x = (const skey_t *)a, *y = (const skey_t *)b;
  if (x->k0 != y->k0) return x->k0 < y->k0 ? -1 : 1;
  if (x->k1 != y->k1) return x->k1 < y->k1 ? -1 : 1;
  return x->k2 < y->k2 ? -1 : (x->k2 > y->k2);
}

/* entry step of v in a pass: ascending rank for minima, descending for maxima */
static int64_t entry_of(const int64_t *rank, int64_t n, int dir, int64_t v) {
  return dir < 0 ? rank[v] : n - 1 - rank[v];
}

static int simplify_pass(const field_t *F, int64_t *rank, double *val, int dir, double threshold,
                         int64_t *removed) {
  const int64_t n = F->n;
  int64_t *byent = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int64_t *eldest = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int64_t *death = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int64_t *owner = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int64_t *dist = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
  skey_t *keys = (skey_t *)malloc(sizeof(skey_t) * (size_t)n);
  int st = OR_OK;
  if (!byent || !parent || !eldest || !death || !owner || !dist || !queue || !keys) {
    st = OR_ERR_NOMEM;
    goto done;
  }
  for (int64_t v = 0; v < n; ++v) {
    byent[entry_of(rank, n, dir, v)] = v;
    parent[v] = -1; /* not entered yet */
    death[v] = -2;  /* not an extremum */
    owner[v] = -1;
    dist[v] = -1;
  }
  /* 1. elder rule over the entry order */
  for (int64_t s = 0; s < n; ++s) {
    const int64_t v = byent[s];
    int64_t nb[14], roots[14];
    const int c = neighbours_of(F, v, nb);
    int nr = 0;
    for (int i = 0; i < c; ++i) {
      if (parent[nb[i]] < 0) continue;
      const int64_t r = uf_root(parent, nb[i]);
      int seen = 0;
      for (int j = 0; j < nr; ++j) seen |= roots[j] == r;
      if (!seen) roots[nr++] = r;
    }
    if (nr == 0) {
      parent[v] = v;
      eldest[v] = v;
      death[v] = -1;
      continue;
    }
    int keep = 0;
    for (int j = 1; j < nr; ++j)
      if (entry_of(rank, n, dir, eldest[roots[j]]) < entry_of(rank, n, dir, eldest[roots[keep]])) keep = j;
    for (int j = 0; j < nr; ++j) {
      if (j == keep) continue;
      death[eldest[roots[j]]] = v;
      parent[roots[j]] = roots[keep];
    }
    parent[v] = roots[keep];
  }
  /* 2. the removed extrema, latest death first (outer regions before the
   * regions nested in them); keys[] holds (-entry(d), m) for the sort */
  int64_t nrm = 0;
  for (int64_t m = 0; m < n; ++m) {
    const int64_t d = death[m];
    if (d < 0 || !(fabs(val[d] - val[m]) < threshold)) continue;
    keys[nrm].k0 = -entry_of(rank, n, dir, d);
    keys[nrm].k1 = m;
    keys[nrm].k2 = 0;
    ++nrm;
  }
  qsort(keys, (size_t)nrm, sizeof(skey_t), cmp_skey);
  *removed = nrm;
  /* 3. regions: claimed outermost first, then breadth-first distances from d */
  for (int64_t i = 0; i < nrm; ++i) {
    const int64_t m = keys[i].k1, d = death[m], sd = entry_of(rank, n, dir, d);
    if (owner[m] >= 0) continue; /* inside a region claimed already */
    int64_t head = 0, tail = 0;
    owner[m] = m;
    queue[tail++] = m;
    while (head < tail) {
      const int64_t x = queue[head++];
      int64_t nb[14];
      const int c = neighbours_of(F, x, nb);
      for (int j = 0; j < c; ++j) {
        const int64_t w = nb[j];
        if (entry_of(rank, n, dir, w) >= sd || owner[w] == m) continue;
        if (owner[w] >= 0) { /* regions that overlap without nesting */
          st = OR_ERR_REGIONS;
          goto done;
        }
        owner[w] = m;
        queue[tail++] = w;
      }
    }
    const int64_t size = tail;
    head = tail = 0;
    dist[d] = 0;
    queue[tail++] = d;
    while (head < tail) {
      const int64_t x = queue[head++];
      int64_t nb[14];
      const int c = neighbours_of(F, x, nb);
      for (int j = 0; j < c; ++j) {
        const int64_t w = nb[j];
        if (owner[w] != m || dist[w] >= 0) continue;
        dist[w] = dist[x] + 1;
        queue[tail++] = w;
      }
    }
    dist[d] = -1;
    if (tail - 1 != size) { /* a region that d does not reach */
      st = OR_ERR_REGIONS;
      goto done;
    }
  }
  /* the new entry order */
  for (int64_t v = 0; v < n; ++v) {
    if (owner[v] >= 0) {
      const int64_t d = death[owner[v]];
      keys[v].k0 = entry_of(rank, n, dir, d);
      keys[v].k1 = dist[v];
    } else {
      keys[v].k0 = entry_of(rank, n, dir, v);
      keys[v].k1 = 0;
    }
    keys[v].k2 = v;
  }
  qsort(keys, (size_t)n, sizeof(skey_t), cmp_skey);
  for (int64_t v = 0; v < n; ++v)
    if (owner[v] >= 0) val[v] = val[death[owner[v]]];
  for (int64_t s = 0; s < n; ++s) rank[keys[s].k2] = dir < 0 ? s : n - 1 - s;
done:
  free(byent);
  free(parent);
  free(eldest);
  free(death);
  free(owner);
  free(dist);
  free(queue);
  free(keys);
  return st;
}

int ms_oracle_simplify(const void *field, int dtype, const int64_t dims[3], double threshold, int which,
                       int64_t *rank, double *value, int64_t *removed) {
  field_t F;
  int st = make_field(&F, field, dtype, dims);
  if (st != OR_OK) return st;
  if (which < 1 || which > 3 || !rank || !value || !removed || threshold != threshold) return OR_ERR_ARG;
  if (has_nan(&F)) return OR_ERR_NAN;
  const int64_t n = F.n;
  ordered_t *ord = (ordered_t *)malloc(sizeof(ordered_t) * (size_t)n);
  if (!ord) return OR_ERR_NOMEM;
  for (int64_t v = 0; v < n; ++v) {
    ord[v].value = value_at(&F, v);
    ord[v].index = v;
    value[v] = ord[v].value;
  }
  qsort(ord, (size_t)n, sizeof(ordered_t), cmp_ordered);
  for (int64_t s = 0; s < n; ++s) rank[ord[s].index] = s;
  free(ord);
  removed[0] = removed[1] = removed[2] = 0;
  for (int64_t round = 0;; ++round) {
    if (round == kSimplifyRounds) return OR_ERR_CYCLE;
    int64_t rm[2] = {0, 0};
    if (which & 1) st = simplify_pass(&F, rank, value, -1, threshold, &rm[0]);
    if (st == OR_OK && (which & 2)) st = simplify_pass(&F, rank, value, 1, threshold, &rm[1]);
    if (st != OR_OK) return st;
    removed[0] += rm[0];
    removed[1] += rm[1];
    removed[2] = round + 1;
    /* a minima pass leaves only minima of persistence >= threshold; when the
     * maxima pass after it removes nothing, neither kind is left below it */
    if (which != 3 || rm[1] == 0) break;
  }
  return OR_OK;
}
