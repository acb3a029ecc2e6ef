"""Pins of the oracle's 0-dimensional persistence pairing of the extrema
(``oracle.persistence``), the pairing by which the paper's topological
simplification (Sec. 4.1; thresholds in Sec. 6) removes extrema: a chain
worked by hand, brute force from the definition on tiny grids (an extremum
dies at the first vertex whose entry connects its component to an earlier
vertex), the extremum sets of the steepest step, and point-reflection
duality between maxima and minima."""
from collections import deque

import numpy as np
import pytest

import oracle


def order_positions(f, direction):
    """Entry step of every vertex: increasing (value, index) for minima,
    the reverse for maxima."""
    flat = f.reshape(-1).astype(np.float64)
    order = np.lexsort((np.arange(flat.size), flat))
    if direction > 0:
        order = order[::-1]
    pos = np.empty(flat.size, np.int64)
    pos[order] = np.arange(flat.size)
    return order, pos


def brute_pairs(f, dims, direction):
    order, pos = order_positions(f, direction)
    up, dn = oracle.steepest(f)
    ext = np.flatnonzero((dn if direction < 0 else up) == np.arange(f.size))
    nbrs = [oracle.neighbors(dims, v) for v in range(f.size)]
    deaths = []
    for m in ext:
        death = -1
        for r in range(pos[m], f.size):
            seen, q, found = {int(m)}, deque([int(m)]), False
            while q and not found:
                v = q.popleft()
                for u in nbrs[v]:
                    if pos[u] <= r and u not in seen:
                        if pos[u] < pos[m]:
                            found = True
                            break
                        seen.add(u)
                        q.append(u)
            if found:
                death = int(order[r])
                break
        deaths.append(death)
    return ext.astype(np.int32), np.array(deaths, np.int32)


def test_chain_worked_by_hand(golden):
    g = golden("persistence_chain7.txt")
    f = np.array(g["values"], np.float32).reshape(1, 1, 7)
    mn, mx = oracle.persistence(f, -1), oracle.persistence(f, 1)
    assert mn["extremum"].tolist() == g["min_extremum"] and mn["death"].tolist() == g["min_death"]
    assert mx["extremum"].tolist() == g["max_extremum"] and mx["death"].tolist() == g["max_death"]


@pytest.mark.parametrize("dims", [(4, 3, 1), (3, 3, 2), (5, 2, 2), (6, 1, 1), (2, 2, 3), (4, 4, 2)])
@pytest.mark.parametrize("levels", [3, 1 << 20])
@pytest.mark.parametrize("seed", range(3))
def test_brute_force_from_the_definition(dims, levels, seed):
    g = np.random.default_rng(seed * 131 + levels % 97 + dims[0])
    f = g.integers(0, levels, size=dims[::-1]).astype(np.float32)
    for direction in (-1, 1):
        got = oracle.persistence(f, direction)
        ext, death = brute_pairs(f, dims, direction)
        assert np.array_equal(got["extremum"], ext), (dims, direction)
        assert np.array_equal(got["death"], death), (dims, direction)


@pytest.mark.parametrize("dims", [(30, 24, 18), (120, 90, 1)])
def test_extrema_and_ordering(dims):
    f = np.random.default_rng(7).standard_normal(dims[::-1]).astype(np.float32)
    up, dn = oracle.steepest(f)
    for direction, ptr in ((-1, dn), (1, up)):
        p = oracle.persistence(f, direction)
        assert np.array_equal(p["extremum"], np.flatnonzero(ptr == np.arange(f.size)))
        assert (p["death"] == -1).sum() == 1  # a connected grid: one survivor
        _, pos = order_positions(f, direction)
        alive = p["death"] >= 0
        assert (pos[p["death"][alive]] > pos[p["extremum"][alive]]).all()
        # the survivor entered first: the global extremum
        assert pos[p["extremum"][~alive][0]] == 0


@pytest.mark.parametrize("dims", [(9, 7, 5), (13, 11, 1)])
def test_point_reflection_duality(dims):
    """f'(p) = -f(mirror p) with vertex v -> N-1-v reverses the (value,
    index) order exactly, so the maxima pairs of f are the minima pairs of
    f' mirrored."""
    g = np.random.default_rng(11)
    f = g.integers(0, 5, size=dims[::-1]).astype(np.float32)
    n = f.size
    fr = -f.reshape(-1)[::-1].reshape(f.shape).copy()
    mx = oracle.persistence(f, 1)
    mn = oracle.persistence(fr, -1)
    mirrored = sorted(zip((n - 1 - mn["extremum"]).tolist(),
                          [d if d < 0 else n - 1 - d for d in mn["death"].tolist()]))
    assert mirrored == list(zip(mx["extremum"].tolist(), mx["death"].tolist()))


def test_nan_rejected():
    f = np.zeros((3, 3, 3), np.float32)
    f[1, 1, 1] = np.nan
    with pytest.raises(Exception):
        oracle.persistence(f, -1)


def basin_graph_pairs(f, dims):
    """The same pairing computed the way a data-parallel pass can: from the
    ascending segmentation (every vertex's minimum), every edge of the
    triangulation between two basins becomes active when its later endpoint
    enters; taking the active edges in entry order and merging basins with
    the elder rule gives each minimum's death vertex."""
    _, pos = order_positions(f, -1)
    asc = oracle.segment(f)["asc"]
    n = f.size
    best = {}  # (basin a, basin b) -> (activation step, entering vertex)
    for v in range(n):
        for u in oracle.neighbors(dims, v):
            if u <= v or asc[u] == asc[v]:
                continue
            a, b = sorted((int(asc[u]), int(asc[v])))
            w = max(pos[u], pos[v])
            if (a, b) not in best or w < best[(a, b)][0]:
                best[(a, b)] = (w, u if pos[u] > pos[v] else v)
    parent = {m: m for m in set(asc.tolist())}

    def root(x):
        while parent[x] != x:
            x = parent[x]
        return x

    death = {m: -1 for m in parent}
    for (a, b), (w, v) in sorted(best.items(), key=lambda kv: kv[1][0]):
        ra, rb = root(a), root(b)
        if ra == rb:
            continue
        young, old = (ra, rb) if pos[ra] > pos[rb] else (rb, ra)  # a root is its component's eldest
        death[young] = v
        parent[young] = old
    ext = np.array(sorted(death), np.int32)
    return ext, np.array([death[m] for m in ext], np.int32)


@pytest.mark.parametrize("dims", [(9, 8, 7), (20, 15, 1), (6, 5, 4)])
@pytest.mark.parametrize("levels", [4, 1 << 20])
def test_basin_graph_formulation_agrees(dims, levels):
    """Sublevel-set components at any step are unions of (parts of) basins
    joined by active basin-boundary edges -- every entered vertex reaches its
    minimum by steepest descent inside the sublevel set -- so the merges
    happen exactly when boundary edges become active.  Checked against the
    oracle's pairing, with and without ties."""
    f = np.random.default_rng(levels % 1000 + dims[0]).integers(0, levels, size=dims[::-1]).astype(np.float32)
    p = oracle.persistence(f, -1)
    ext, death = basin_graph_pairs(f, dims)
    assert np.array_equal(p["extremum"], ext)
    assert np.array_equal(p["death"], death)


def staircase(k_steps, wall=10000.0):
    f = np.empty(2 * k_steps + 1, np.float32)
    f[0::2] = np.arange(k_steps + 1)
    f[1::2] = wall - np.arange(k_steps)
    return f.reshape(1, -1)


@pytest.mark.parametrize("steps", [1, 2, 5, 50])
def test_staircase_closed_form(steps):
    """Minima at x = 2k with value k, walls at x = 2k + 1 with value W - k.
    Walls enter lowest first, i.e. from the right: the wall at 2k - 1 joins
    minimum k to minimum k - 1's component, so minimum k dies there.  For
    maxima the valleys enter highest first, from the right: the valley at 2k
    joins wall k to wall k - 1's component, so wall k dies at 2k."""
    f = staircase(steps)
    mn, mx = oracle.persistence(f, -1), oracle.persistence(f, 1)
    assert mn["extremum"].tolist() == list(range(0, 2 * steps + 1, 2))
    assert mn["death"].tolist() == [-1] + [2 * k - 1 for k in range(1, steps + 1)]
    assert mx["extremum"].tolist() == list(range(1, 2 * steps, 2))
    assert mx["death"].tolist() == [-1] + [2 * k for k in range(1, steps)]
