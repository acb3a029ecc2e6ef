"""Pins of the CPU oracle against facts fixed by the paper and by
mathematics -- never against the oracle itself.

* Fig. 1 worked example (values, descending / ascending / MS labels).
* Fig. 3 path-compression chain.
* Brute force on tiny grids: the paper's literal recipe (Sec. 4.1: sort the
  vertices into an order field, then Sec. 4.2: step to the neighbour of
  largest order value), with the neighbour sets taken from an explicit
  enumeration of the triangulation's simplices.
* Closed forms: monotone ramp, constant field (index tie-break), paraboloid.
* Invariants: Euler sums of lower/upper links (Sec. 3.2), extrema <-> empty
  lower/upper links, Alexander duality at interior 3D vertices, point
  reflection duality, plane embeddings, MS id properties.
"""
import itertools

import numpy as np
import pytest

import oracle
import synthfields as sf


# ---------------------------------------------------------------- helpers
def kuhn_edges(dims):
    """Edge set of the Freudenthal/Kuhn triangulation, by enumerating every
    simplex: each cell [c, c+1]^d (over axes of extent >= 2) is split into d!
    simplices c -> c+e_a1 -> c+e_a1+e_a2 -> ... (one per axis ordering); an
    edge joins any two vertices of a simplex."""
    nx, ny, nz = dims
    ext = (nx, ny, nz)
    axes = [a for a in range(3) if ext[a] >= 2]
    lin = lambda p: p[0] + nx * (p[1] + ny * p[2])
    edges = set()
    ranges = [range(ext[a] - 1) if a in axes else range(1) for a in range(3)]
    for c in itertools.product(*ranges):
        for perm in itertools.permutations(axes):
            chain = [list(c)]
            for a in perm:
                q = list(chain[-1])
                q[a] += 1
                chain.append(q)
            ids = [lin(p) for p in chain]
            for i in range(len(ids)):
                for j in range(i + 1, len(ids)):
                    edges.add((min(ids[i], ids[j]), max(ids[i], ids[j])))
    nbrs = {v: set() for v in range(nx * ny * nz)}
    for a, b in edges:
        nbrs[a].add(b)
        nbrs[b].add(a)
    return nbrs


def literal_segmentation(field):
    """Sec. 4.1 + 4.2 read literally, in pure Python: sort the vertices by
    (value, index) into the order field fbar, point every vertex at the
    neighbour of largest (smallest) fbar if that beats its own, walk each
    vertex independently to the end, then rank the distinct (min, max) pairs."""
    f = np.asarray(field, dtype=np.float64)
    if f.ndim == 2:
        f = f[None]
    nz, ny, nx = f.shape
    vals = f.reshape(-1)
    n = vals.size
    order = np.lexsort((np.arange(n), vals))  # primary key value, ties by index
    fbar = np.empty(n, np.int64)
    fbar[order] = np.arange(n)
    nb = kuhn_edges((nx, ny, nz))
    up = list(range(n))
    dn = list(range(n))
    for v in range(n):
        for u in nb[v]:
            if fbar[u] > fbar[up[v]]:
                up[v] = u
            if fbar[u] < fbar[dn[v]]:
                dn[v] = u

    def end(p, v):
        while p[v] != v:
            v = p[v]
        return v

    desc = [end(up, v) for v in range(n)]
    asc = [end(dn, v) for v in range(n)]
    pairs = sorted(set(zip(asc, desc)))
    rank = {p: i for i, p in enumerate(pairs)}
    ms = [rank[p] for p in zip(asc, desc)]
    return dict(up=np.array(up), dn=np.array(dn), desc=np.array(desc), asc=np.array(asc),
                ms=np.array(ms), K=len(pairs))


TINY_DIMS = [(1, 1, 1), (2, 1, 1), (5, 1, 1), (1, 6, 1), (4, 4, 1), (7, 5, 1), (3, 1, 4),
             (1, 3, 5), (2, 2, 2), (3, 3, 3), (4, 3, 2), (5, 4, 6), (2, 7, 3)]


# ---------------------------------------------------------------- Fig. 1 / Fig. 3
def test_fig1_worked_example(golden):
    g = golden("fig1_4x4.txt")
    nx, ny, nz = g["dims"]
    f = np.array(g["values"], np.float32).reshape(nz, ny, nx)
    r = oracle.segment(f)
    assert r["desc"].tolist() == g["desc"]
    assert r["asc"].tolist() == g["asc"]
    assert r["ms"].tolist() == g["ms"]
    assert r["K"] == g["K"][0]


def test_fig1_other_diagonal_disagrees(golden):
    """The figure fixes the diagonal orientation: mirroring x (which turns
    the (x,y)-(x+1,y+1) diagonals into the other family) must change the
    labels that the figure prints."""
    g = golden("fig1_4x4.txt")
    f = np.array(g["values"], np.float32).reshape(4, 4)
    r = oracle.segment(np.ascontiguousarray(f[:, ::-1]))
    back = lambda a: np.asarray(a).reshape(4, 4)[:, ::-1].reshape(-1)
    remap = lambda lab: np.array([(l // 4) * 4 + 3 - l % 4 for l in lab])
    assert back(remap(r["asc"])).tolist() != g["asc"] or back(remap(r["desc"])).tolist() != g["desc"]


def test_fig3_chain(golden):
    g = golden("fig3_chain7.txt")
    f = np.array(g["values"], np.float32).reshape(1, 1, -1)
    r = oracle.segment(f)
    assert r["up"].tolist() == g["up"]
    assert r["desc"].tolist() == g["desc"]
    assert r["asc"].tolist() == g["asc"]
    assert r["K"] == 1


# ---------------------------------------------------------------- brute force
@pytest.mark.parametrize("dims", [(4, 4, 1), (3, 3, 3), (4, 3, 2), (3, 1, 4), (5, 4, 6)])
def test_neighbours_match_triangulation(dims):
    nb = kuhn_edges(dims)
    for v in range(int(np.prod(dims))):
        assert oracle.neighbors(dims, v) == sorted(nb[v]), v


@pytest.mark.parametrize("dims", TINY_DIMS)
@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("levels", [0, 3])
def test_brute_force_literal(dims, seed, levels):
    """The oracle equals the literal order-field recipe on tiny grids, with
    distinct values (levels == 0) and with heavy ties (3 levels)."""
    nx, ny, nz = dims
    if levels:
        f = sf.random_ties(dims, seed, levels=levels)
    else:
        f = sf.rng_for(seed).standard_normal((nz, ny, nx)).astype(np.float32)
    r = oracle.segment(f)
    b = literal_segmentation(f)
    for k in ("up", "dn", "desc", "asc", "ms"):
        assert r[k].tolist() == b[k].tolist(), k
    assert r["K"] == b["K"]


@pytest.mark.parametrize("seed", range(4))
def test_memoised_follow_equals_independent_walks(seed):
    f = sf.smoothed_noise((17, 13, 11), seed, sigma=1.5, radius=6)
    up, dn = oracle.steepest(f)
    assert oracle.follow(up).tolist() == oracle.follow(up, brute=True).tolist()
    assert oracle.follow(dn).tolist() == oracle.follow(dn, brute=True).tolist()


def test_walk_from_field_matches_segment():
    f = sf.gaussian_sum((20, 18, 16), 3)
    r = oracle.segment(f)
    for v in range(0, f.size, 97):
        assert oracle.walk(f, v, +1)[0] == r["desc"][v]
        assert oracle.walk(f, v, -1)[0] == r["asc"][v]
    vs = np.arange(0, f.size, 31)
    up, dn = oracle.steepest_at(f, vs)
    assert up.tolist() == r["up"][vs].tolist() and dn.tolist() == r["dn"][vs].tolist()


# ---------------------------------------------------------------- closed forms
@pytest.mark.parametrize("dims", [(9, 1, 1), (6, 5, 1), (5, 6, 7), (1, 1, 1)])
def test_monotone_ramp(dims):
    f = sf.ramp(dims)
    r = oracle.segment(f)
    n = f.size
    assert (r["desc"] == n - 1).all() and (r["asc"] == 0).all()
    assert r["K"] == 1 and (r["ms"] == 0).all()


@pytest.mark.parametrize("dims", [(7, 1, 1), (5, 4, 1), (4, 5, 6)])
def test_constant_field_index_tiebreak(dims):
    """All values tie, so the order is the index order: the larger index is
    higher (Sec. 4.1, ties resolved by index)."""
    f = sf.constant(dims, 2.5)
    r = oracle.segment(f)
    assert (r["desc"] == f.size - 1).all() and (r["asc"] == 0).all()


@pytest.mark.parametrize("dims,centre", [((9, 9, 9), (4, 4, 4)), ((11, 7, 8), (3, 5, 2)),
                                         ((12, 9, 1), (5, 4, 0))])
def test_paraboloid(dims, centre):
    nx, ny, nz = dims
    f = sf.paraboloid(dims, centre, dtype=np.float64)
    r = oracle.segment(f)
    c = centre[0] + nx * (centre[1] + ny * centre[2])
    assert (r["desc"] == c).all()
    corners = set()
    for z in {0, nz - 1}:
        for y in {0, ny - 1}:
            for x in {0, nx - 1}:
                corners.add(x + nx * (y + ny * z))
    minima = set(np.flatnonzero(r["dn"] == np.arange(f.size)).tolist())
    assert minima == corners


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("dims", [(6, 5, 4), (7, 7, 7), (9, 8, 1), (5, 1, 6), (8, 1, 1)])
@pytest.mark.parametrize("kind", ["noise", "ties"])
def test_link_euler_sums_and_extrema(dims, kind):
    """Sec. 3.2: sum over vertices of (1 - chi(lower link)) is the Euler
    characteristic of the box, 1; same for the upper link.  v is a minimum
    (dn(v) == v) iff its lower link is empty, a maximum iff its upper link is
    empty."""
    f = sf.smoothed_noise(dims, 5, sigma=1.0, radius=4) if kind == "noise" else sf.random_ties(dims, 5)
    st, links = oracle.link_stats(f, with_links=True)
    assert int((1 - st[:, 0]).sum()) == 1
    assert int((1 - st[:, 1]).sum()) == 1
    up, dn = oracle.steepest(f)
    idx = np.arange(f.size)
    assert ((dn == idx) == (st[:, 2] == 0)).all()
    assert ((up == idx) == (st[:, 3] == 0)).all()
    # the link's vertex set is the neighbour set N(v)
    for v in range(0, f.size, 7):
        lv = sorted(x for x in links[v] if x >= 0)
        assert lv == oracle.neighbors(dims, v)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_banchoff_alternating_sum_3d(seed):
    """Interior 3D vertices: 1 - chi(Lk-) = c+ - c- (Alexander duality on the
    link sphere), i.e. a 1-saddle of multiplicity c- - 1 and a 2-saddle of
    multiplicity c+ - 1; with the boundary terms the alternating sum
    minima - 1-saddles + 2-saddles - maxima is the box's Euler number 1."""
    f = sf.smoothed_noise((10, 9, 8), seed, sigma=1.2, radius=5)
    st = oracle.link_stats(f)
    inner = st[:, 4] == 1
    cl, cu = st[inner, 2], st[inner, 3]
    assert ((1 - st[inner, 0]) == (cu - cl)).all()
    n_min = int((cl == 0).sum())
    n_max = int((cu == 0).sum())
    s1 = int(np.maximum(cl - 1, 0).sum())
    s2 = int(np.maximum(cu - 1, 0).sum())
    boundary = int((1 - st[~inner, 0]).sum())
    assert n_min - s1 + s2 - n_max + boundary == 1
    assert n_min > 0 and n_max > 0 and s1 + s2 > 0


@pytest.mark.parametrize("dims", [(6, 5, 4), (9, 7, 1), (5, 5, 5)])
@pytest.mark.parametrize("kind", ["noise", "ties"])
def test_point_reflection_duality(dims, kind):
    """f'(p) = -f(mirror p), mirror = all axes reversed (index N-1-v): the
    stencil is point symmetric and the order reverses exactly, ties included,
    so desc'(p) = N-1-asc(mirror p)."""
    f = sf.smoothed_noise(dims, 2, sigma=1.0, radius=4) if kind == "noise" else sf.random_ties(dims, 2)
    g = np.ascontiguousarray(-f[::-1, ::-1, ::-1])
    a, b = oracle.segment(f), oracle.segment(g)
    n = f.size
    assert (b["desc"] == (n - 1 - a["asc"][::-1])).all()
    assert (b["asc"] == (n - 1 - a["desc"][::-1])).all()


def test_plane_embeddings_agree():
    """A 2D field laid out as (nx, ny, 1) or as (nx, 1, nz) has the same
    vertex numbering and the same triangulation, so the same labels."""
    f2 = sf.smoothed_noise((13, 11, 1), 4, sigma=1.0, radius=4)[0]
    a = oracle.segment(f2)
    b = oracle.segment(f2.reshape(11, 1, 13))
    for k in ("asc", "desc", "ms"):
        assert (a[k] == b[k]).all()


def test_ms_id_properties():
    f = sf.gaussian_sum((24, 20, 16), 1)
    r = oracle.segment(f)
    k = r["K"]
    assert sorted(set(r["ms"].tolist())) == list(range(k))
    pairs = sorted(set(zip(r["asc"].tolist(), r["desc"].tolist())))
    assert len(pairs) == k
    for i, (a, d) in enumerate(pairs):
        sel = (r["asc"] == a) & (r["desc"] == d)
        assert (r["ms"][sel] == i).all()
    # labels are extrema
    assert (r["up"][r["desc"]] == r["desc"]).all() and (r["dn"][r["asc"]] == r["asc"]).all()


# ---------------------------------------------------------------- values
def test_signed_zero_ties_by_index():
    f = np.array([[0.0, -0.0, 0.0, -0.0, 0.0]], np.float32)
    r = oracle.segment(f)
    assert (r["desc"] == 4).all() and (r["asc"] == 0).all()


def test_denormals_and_infinities_compare_exactly():
    tiny = np.float32(1.4e-45)  # smallest positive subnormal
    f = np.array([[-np.inf, 0.0, tiny, 2 * tiny, np.inf, 3 * tiny]], np.float32)
    r = oracle.segment(f)
    assert r["up"].tolist() == [1, 2, 3, 4, 4, 4]
    assert r["dn"].tolist() == [0, 0, 1, 2, 3, 5]


def test_fp16_equals_exact_widening():
    f16 = sf.random_ties((9, 8, 7), 3, levels=5).astype(np.float16) * np.float16(0.1)
    a = oracle.segment(f16)
    b = oracle.segment(f16.astype(np.float32))
    c = oracle.segment(f16.astype(np.float64))
    for k in ("asc", "desc", "ms"):
        assert (a[k] == b[k]).all() and (a[k] == c[k]).all()
    # subnormal halves are distinct and ordered
    h = np.array([[0, 1, 2, 3]], np.uint16).view(np.float16)
    assert oracle.segment(h)["up"].tolist() == [1, 2, 3, 3]


def test_nan_rejected():
    f = np.zeros((3, 4), np.float32)
    f[1, 2] = np.nan
    with pytest.raises(ValueError):
        oracle.segment(f)
