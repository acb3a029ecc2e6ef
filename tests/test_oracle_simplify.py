"""Pins of the oracle's simplification of the order (`oracle.simplify`): the
persistence-based removal of extrema that Sec. 4.1 runs before segmenting
(thresholds: Sec. 6), in the reading the oracle states -- per pass, every
extremum whose pair has persistence below the threshold is removed, its
region (its component among the vertices entered before its death vertex d)
takes d's value and enters right after d, nearer vertices (breadth-first
steps from d inside the region) first, then lower indices; minima and maxima
passes alternate until a maxima pass removes nothing.

Checked against: a chain worked by hand; an independent brute-force
restatement of the reading on tiny grids (components recomputed from scratch
at every step, no union-find); and the properties the reading guarantees."""
import itertools

import numpy as np
import pytest

import oracle
import synthfields as sf

# ---- a chain worked by hand -------------------------------------------------
# values 0, 3, 1, 4, 2.5, 6, 5, 7 at x = 0..7 (a path graph).  Minima 0, 2, 4, 6.
# Sublevel entry order: v0 v2 v4 v1 v3 v6 v5 v7; v1 joins {v0} and {v2}: v2 dies
# at v1 (persistence 2); v3 joins {v0 v1 v2} and {v4}: v4 dies at v3 (1.5); v5
# joins {v6} to the rest: v6 dies at v5 (1).
# Threshold 1.6: v4 and v6 go.  R(v4) = {v4} (its component before v3 enters),
# R(v6) = {v6}.  v4 takes value 4 and enters right after v3, v6 takes 6 and
# enters right after v5: order v0 v2 v1 v3 v4 v5 v6 v7.  The maxima pass on it
# pairs v1 (value 3) with v2 (value 1): persistence 2, kept.
# Threshold 2.5: v2 goes too, R(v2) = {v2} after v1: the order becomes the
# chain's own, one minimum and one maximum.
CHAIN = np.array([[0, 3, 1, 4, 2.5, 6, 5, 7]], np.float32)


def test_chain_worked_by_hand():
    r = oracle.simplify(CHAIN, 0.0)
    assert r["rank"].ravel().tolist() == [0, 3, 1, 4, 2, 6, 5, 7]
    assert r["removed_minima"] == 0 and r["removed_maxima"] == 0
    r = oracle.simplify(CHAIN, 1.6)
    assert r["rank"].ravel().tolist() == [0, 2, 1, 3, 4, 5, 6, 7]
    assert r["value"].ravel().tolist() == [0, 3, 1, 4, 4, 6, 6, 7]
    assert (r["removed_minima"], r["removed_maxima"]) == (2, 0)
    r = oracle.simplify(CHAIN, 2.5)
    assert r["rank"].ravel().tolist() == list(range(8))
    assert r["value"].ravel().tolist() == [0, 3, 3, 4, 4, 6, 6, 7]
    assert (r["removed_minima"], r["removed_maxima"]) == (3, 0)


def test_nested_regions_worked_by_hand():
    # values 0, 6, 2, 4, 3, 5, 1, 7.  Sublevel entry: v0 v6 v2 v4 v3 v5 v1 v7.
    # v3 joins {v2} and {v4}: v4 dies at v3 (persistence 1); v5 joins {v2 v3 v4}
    # and {v6}: v2 dies at v5 (3, v6 is older); v1 joins {v0} and the rest: v6
    # dies at v1 (5).  Threshold 3.5 removes v4 and v2; R(v4) = {v4} lies inside
    # R(v2) = {v2 v3 v4} (v2's component before v5 enters), so the outer region
    # decides: v2, v3, v4 take value 5 and enter right after v5 by distance
    # from it: v4 (1), v3 (2), v2 (3).  Order: v0 v6 v5 v4 v3 v2 v1 v7.  The
    # maxima pass on it pairs v1 with v6 (persistence 5): nothing removed.
    f = np.array([[0, 6, 2, 4, 3, 5, 1, 7]], np.float32)
    r = oracle.simplify(f, 3.5)
    assert r["rank"].ravel().tolist() == [0, 6, 5, 4, 3, 2, 1, 7]
    assert r["value"].ravel().tolist() == [0, 6, 5, 5, 5, 5, 1, 7]
    assert (r["removed_minima"], r["removed_maxima"], r["rounds"]) == (2, 0, 1)


def test_single_vertex():
    r = oracle.simplify(np.array([[4.0]], np.float32), 1.0)
    assert r["rank"].tolist() == [[0]] and r["value"].tolist() == [[4.0]]
    assert (r["removed_minima"], r["removed_maxima"]) == (0, 0)


def test_maxima_flattened_below_their_death():
    # 5 0 5: maxima v0, v2 (v2 is higher: equal values, higher index); v0 dies
    # at v1 with persistence 5.  Above 5 it is removed: it takes value 0 and
    # enters right after v1 in descending order, i.e. just below v1 -- it
    # becomes the minimum, v1 is no longer one.
    f = np.array([[5, 0, 5]], np.float32)
    r = oracle.simplify(f, 6.0, 2)
    assert r["rank"].ravel().tolist() == [0, 1, 2]
    assert r["value"].ravel().tolist() == [0, 0, 5]
    assert (r["removed_minima"], r["removed_maxima"]) == (0, 1)


# ---- an independent restatement for tiny grids ----------------------------
def nbrs(dims, v):
    nx, ny, nz = dims
    x, y, z = v % nx, (v // nx) % ny, v // (nx * ny)
    out = []
    for dx, dy, dz in itertools.product((-1, 0, 1), repeat=3):
        if (dx, dy, dz) == (0, 0, 0):
            continue
        if not (min(dx, dy, dz) >= 0 or max(dx, dy, dz) <= 0):
            continue
        X, Y, Z = x + dx, y + dy, z + dz
        if 0 <= X < nx and 0 <= Y < ny and 0 <= Z < nz:
            out.append(X + nx * (Y + ny * Z))
    return out


def component(dims, start, allowed):
    seen, todo = {start}, [start]
    while todo:
        x = todo.pop()
        for w in nbrs(dims, x):
            if w in allowed and w not in seen:
                seen.add(w)
                todo.append(w)
    return seen


def brute_pass(dims, order, val, thr):
    """One pass over `order` (the entry order of the pass: a list of
    vertices).  Returns the new entry order, the new values and the count of
    removed extrema."""
    n = len(order)
    ent = {v: s for s, v in enumerate(order)}
    # pairs from scratch: at each step, the components of the entered vertices
    death = {}
    for s, v in enumerate(order):
        before = set(order[:s])
        comps = []
        for w in nbrs(dims, v):
            if w in before and not any(w in c for c in comps):
                comps.append(component(dims, w, before))
        if not comps:
            death[v] = -1
            continue
        firsts = [min(c, key=lambda u: ent[u]) for c in comps]
        old = min(firsts, key=lambda u: ent[u])
        for m in firsts:
            if m != old:
                death[m] = v
    rm = [m for m, d in death.items() if d >= 0 and abs(val[d] - val[m]) < thr]
    region = {m: component(dims, m, set(order[:ent[death[m]]])) for m in rm}
    owner = {}
    for m in sorted(rm, key=lambda m: -ent[death[m]]):  # outermost first
        for u in region[m]:
            owner.setdefault(u, m)
    key = {}
    for v in range(n):
        if v in owner:
            m = owner[v]
            d = death[m]
            dist = {d: 0}
            frontier = [d]
            while v not in dist:  # breadth-first from d inside the region of m
                nxt = []
                for x in frontier:
                    for w in nbrs(dims, x):
                        if owner.get(w) == m and w not in dist:
                            dist[w] = dist[x] + 1
                            nxt.append(w)
                frontier = nxt
            key[v] = (ent[d], dist[v], v)
        else:
            key[v] = (ent[v], 0, v)
    new_order = sorted(range(n), key=lambda v: key[v])
    new_val = list(val)
    for v, m in owner.items():
        new_val[v] = val[death[m]]
    return new_order, new_val, len(rm)


def brute_simplify(field, thr, which):
    dims = (field.shape[-1], field.shape[-2] if field.ndim > 1 else 1, field.shape[0] if field.ndim == 3 else 1)
    val = [float(x) for x in field.ravel()]
    asc = sorted(range(len(val)), key=lambda v: (val[v], v))
    removed = [0, 0]
    while True:
        rm = [0, 0]
        if which & 1:
            asc, val, rm[0] = brute_pass(dims, asc, val, thr)
        if which & 2:
            desc, val, rm[1] = brute_pass(dims, asc[::-1], val, thr)
            asc = desc[::-1]
        removed[0] += rm[0]
        removed[1] += rm[1]
        if which != 3 or rm[1] == 0:
            break
    rank = np.empty(len(val), np.int64)
    rank[asc] = np.arange(len(val))
    return rank, np.array(val), removed


@pytest.mark.parametrize("case", range(24))
def test_brute_force_on_tiny_grids(case):
    rng = np.random.default_rng(100 + case)
    shape = [(5, 6), (3, 4, 3), (1, 9), (4, 4, 2)][case % 4]
    f = rng.standard_normal(shape).astype(np.float32)
    if case % 3 == 0:
        f = np.round(f * 2) / 2  # ties: equal values split by the index
    span = float(f.max() - f.min())
    which = (1, 2, 3)[case % 3]
    for thr in (0.1 * span, 0.4 * span, 2 * span):
        r = oracle.simplify(f, thr, which)
        rank, val, removed = brute_simplify(f, thr, which)
        assert np.array_equal(r["rank"].ravel(), rank), (shape, thr, which)
        assert np.array_equal(r["value"].ravel(), val), (shape, thr, which)
        assert [r["removed_minima"], r["removed_maxima"]] == removed


# ---- what the reading guarantees -------------------------------------------
def extrema_of(rank):
    up, dn = oracle.steepest(rank.astype(np.float64))
    v = np.arange(up.size)
    return set(v[dn == v].tolist()), set(v[up == v].tolist())


def below(rank, value, thr, direction):
    p = oracle.persistence(rank.astype(np.float64), direction)
    v = value.ravel()
    return [int(m) for m, d in zip(p["extremum"], p["death"]) if d >= 0 and abs(v[d] - v[m]) < thr]


def fields():
    rng = np.random.default_rng(7)
    yield "white 2D", rng.standard_normal((24, 20)).astype(np.float32)
    yield "white 3D", rng.standard_normal((10, 9, 8)).astype(np.float32)
    yield "smooth 3D", sf.smoothed_noise((16, 14, 12), 3, sigma=1.5)
    yield "quantised 2D", sf.quantize_levels(sf.smoothed_noise((30, 20, 1), 4, sigma=2.0), 6)
    yield "fp16 3D", sf.smoothed_noise((12, 10, 9), 5, sigma=1.5).astype(np.float16)


@pytest.mark.parametrize("name,f", list(fields()))
def test_minima_pass_keeps_exactly_the_persistent_minima(name, f):
    span = float(f.max()) - float(f.min())
    p = oracle.persistence(f, -1)
    vals = f.ravel().astype(np.float64)
    for thr in (0.05 * span, 0.3 * span, 3 * span):
        kept = {int(m) for m, d in zip(p["extremum"], p["death"]) if d < 0 or abs(vals[d] - vals[m]) >= thr}
        r = oracle.simplify(f, thr, 1)
        mins, _ = extrema_of(r["rank"])
        assert mins == kept, (name, thr)
        assert r["removed_minima"] == p["extremum"].size - len(kept)
        assert (r["value"].ravel() >= vals).all()  # a minima pass only raises values
        assert sorted(r["rank"].ravel().tolist()) == list(range(f.size))


@pytest.mark.parametrize("name,f", list(fields()))
def test_both_kinds_end_above_the_threshold(name, f):
    span = float(f.max()) - float(f.min())
    vals = f.ravel().astype(np.float64)
    r0 = oracle.simplify(f, 0.0)
    assert np.array_equal(r0["rank"].ravel(), np.argsort(np.argsort(vals, kind="stable"), kind="stable"))
    for thr in (0.05 * span, 0.3 * span):
        r = oracle.simplify(f, thr)
        assert not below(r["rank"], r["value"], thr, -1), (name, thr)
        assert not below(r["rank"], r["value"], thr, 1), (name, thr)
        assert 1 <= r["rounds"] <= 8
    r = oracle.simplify(f, 3 * span)
    mins, maxs = extrema_of(r["rank"])
    assert len(mins) == 1 and len(maxs) == 1


def test_maxima_pass_only_lowers_values():
    f = sf.smoothed_noise((14, 12, 10), 9, sigma=1.5)
    span = float(f.max() - f.min())
    r = oracle.simplify(f, 0.3 * span, 2)
    assert (r["value"].ravel() <= f.ravel().astype(np.float64)).all()
    _, maxs = extrema_of(r["rank"])
    p = oracle.persistence(f, 1)
    vals = f.ravel().astype(np.float64)
    kept = {int(m) for m, d in zip(p["extremum"], p["death"]) if d < 0 or abs(vals[d] - vals[m]) >= 0.3 * span}
    assert maxs == kept


def test_errors():
    f = np.zeros((3, 3), np.float32)
    with pytest.raises(ValueError):
        oracle.simplify(f, 1.0, 0)
    with pytest.raises(ValueError):
        oracle.simplify(f, float("nan"), 3)
    g = f.copy()
    g[1, 1] = np.nan
    with pytest.raises(ValueError, match="NaN"):
        oracle.simplify(g, 1.0, 3)
