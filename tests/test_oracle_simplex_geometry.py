"""Pins of the oracle's geometry pass (Sec. 4.3, region separators and region
boundaries): the elements drawn in Figs. 5 and 6, planes whose separating
geometry is known in closed form, counts that agree with the index pass, and
closed, hole-free separating surfaces."""
import collections
import itertools
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
# the chain of tetrahedron 0 of a cell (steps x, y, z) and of triangle 0 (x, y)
TET0 = np.array([[0, 0, 0], [1, 0, 0], [1, 1, 0], [1, 1, 1]], np.float64)
TRI0 = np.array([[0, 0], [1, 0], [1, 1]], np.float64)


def _point(name, corners):
    idx = {"A": 0, "B": 1, "C": 2, "D": 3}
    if name == "C":
        return corners.mean(0)
    if name == "O":
        return corners[:3].mean(0)
    if name.startswith("T"):
        return corners[[idx[ch] for ch in name[1:]]].mean(0)
    return corners[[idx[ch] for ch in name]].mean(0)


def _drawn():
    out = []
    with open(os.path.join(GOLDEN, "fig5_6_separators.txt")) as fh:
        for ln in fh:
            if not ln.strip() or ln.startswith("#"):
                continue
            head, elems = ln.split(":", 1)
            kind, *labels = head.split()
            out.append((kind, [int(v) for v in labels],
                        [e.split() for e in elems.split("|")]))
    return out


@pytest.mark.parametrize("case", range(8))
def test_drawn_elements(case):
    kind, labels, elems = _drawn()[case]
    if kind == "tri":
        # labels on (0,0), (1,0), (0,1), (1,1) so that triangle 0 is a, b, c
        grid = np.array([labels[0], labels[1], 9, labels[2]], np.int32)
        r = oracle.simplex_geometry(grid, (2, 2, 1))
        corners = TRI0
    else:
        grid = np.full(8, 9, np.int32)
        for k, v in zip((0, 1, 3, 7), labels):  # corners of the xyz chain
            grid[k] = v
        r = oracle.simplex_geometry(grid, (2, 2, 2))
        corners = TET0
    got = r["pos"][:len(elems)].astype(np.float64)
    want = np.array([[_point(p, corners) for p in e] for e in elems])
    assert np.allclose(got, want, atol=1e-6), (kind, labels, got, want)


def _areas(pos):
    if pos.shape[2] == 2:
        return np.linalg.norm(pos[:, 1] - pos[:, 0], axis=1)
    return 0.5 * np.linalg.norm(np.cross(pos[:, 1] - pos[:, 0], pos[:, 2] - pos[:, 0]), axis=1)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_plane_split_3d(axis):
    dims = (6, 5, 7)
    nx, ny, nz = dims
    coords = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")[::-1]
    k = 3
    lab = np.where(coords[axis] >= k, 11, 4).astype(np.int32)
    cross = {0: (ny - 1) * (nz - 1), 1: (nx - 1) * (nz - 1), 2: (nx - 1) * (ny - 1)}[axis]
    sep = oracle.simplex_geometry(lab, dims, 0)
    assert np.all(sep["pos"][:, :, axis] == k - 0.5)  # on the plane between the regions
    assert np.isclose(_areas(sep["pos"]).sum(), cross)
    assert (sep["pairs"] == [4, 11]).all()
    bnd = oracle.simplex_geometry(lab, dims, 1)
    assert set(np.unique(bnd["pos"][:, :, axis])) == {k - 1.0, float(k)}
    assert np.isclose(_areas(bnd["pos"]).sum(), 2 * cross)  # each region's face once


def test_plane_split_2d():
    nx, ny = 9, 6
    lab = (np.arange(nx)[None, :] >= 4).astype(np.int32).repeat(ny, 0)
    sep = oracle.simplex_geometry(lab, (nx, ny, 1), 0)
    assert np.all(sep["pos"][:, :, 0] == 3.5) and np.isclose(_areas(sep["pos"]).sum(), ny - 1)
    bnd = oracle.simplex_geometry(lab, (nx, ny, 1), 1)
    assert np.isclose(_areas(bnd["pos"]).sum(), 2 * (ny - 1))


@pytest.mark.parametrize("dims", [(6, 5, 4), (8, 7, 1), (3, 3, 3)])
@pytest.mark.parametrize("mode", [0, 1])
def test_counts_agree_with_the_index_pass(dims, mode):
    g = np.random.default_rng(5)
    lab = g.integers(0, 4, size=int(np.prod(dims))).astype(np.int32)
    assert oracle.simplex_geometry(lab, dims, mode)["total"] == oracle.simplex_index(lab, dims, mode)["total"]


def _edge_use(pos):
    use = collections.Counter()
    for tri in pos:
        for i, j in ((0, 1), (1, 2), (0, 2)):
            a, b = tuple(tri[i]), tuple(tri[j])
            use[(min(a, b), max(a, b))] += 1
    return use


@pytest.mark.parametrize("levels", [2, 3, 5])
def test_separators_are_closed(levels):
    """Inside the box every edge of the separating surface is shared by two
    triangles where two regions meet, and by at least two where more meet
    (no holes); edges on the box's faces may be used once."""
    dims = (7, 6, 5)
    nx, ny, nz = dims
    g = np.random.default_rng(levels)
    lab = g.integers(0, levels, size=nx * ny * nz).astype(np.int32)
    pos = oracle.simplex_geometry(lab, dims, 0)["pos"]
    hi = np.array([nx - 1, ny - 1, nz - 1], np.float32)
    for (a, b), n in _edge_use(pos).items():
        a, b = np.array(a), np.array(b)
        on_face = any((a[d] == b[d] == 0) or (a[d] == b[d] == hi[d]) for d in range(3))
        if on_face:
            continue
        if levels == 2:
            assert n == 2, (a, b, n)
        else:
            assert n >= 2, (a, b, n)


def _f32_nearest(q):
    """The float32 nearest to the positive rational q, ties to even, by
    integer arithmetic (no floating-point step)."""
    from fractions import Fraction
    q = Fraction(q)
    e = q.numerator.bit_length() - q.denominator.bit_length()
    if Fraction(2) ** e > q:
        e -= 1
    m = q / Fraction(2) ** (e - 23)  # in [2^23, 2^24)
    r = m.numerator // m.denominator
    rem = m - r
    if rem > Fraction(1, 2) or (rem == Fraction(1, 2) and r % 2 == 1):
        r += 1
    return float(r) * 2.0 ** (e - 23)


def test_coordinate_mean_is_one_rounding_of_the_exact_quotient():
    """Sec. 4.3 centres and midpoints: a point coordinate is the exact mean of
    its corners' integer coordinates rounded once to float32.  Checked against
    rational arithmetic for sums past 2^24, where rounding the sum to float
    first would round twice (it does so for some of these cases)."""
    from fractions import Fraction
    g = np.random.default_rng(2024)
    cases = [(s, n) for n in (1, 2, 3, 4) for s in g.integers(1, 1 << 33, 400, dtype=np.int64)]
    # sums just past powers of two and odd sums near 2^24..2^26 (thirds land
    # between float32 neighbours there)
    for b in (24, 25, 26, 30, 33):
        for d in range(-7, 8):
            for n in (2, 3, 4):
                cases.append((int((1 << b) + d), n))
    twice = 0
    for s, n in cases:
        s = int(s)
        want = _f32_nearest(Fraction(s, n))
        assert oracle.coord_mean(s, n) == want, (s, n)
        twice += float(np.float32(np.float32(s) / np.float32(n))) != want
    assert twice > 0  # the cases include ones where two roundings differ
