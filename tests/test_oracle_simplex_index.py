"""Pins of the oracle's index pass for the multi-label marching triangles /
tetrahedra (Sec. 4.3): the codes against Tab. 1 and Fig. 4, the element
counts against the drawings of Figs. 5 and 6, and the totals of label fields
whose separating geometry is known in closed form."""
import itertools
import os

import numpy as np
import pytest

import oracle

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _rows(name):
    with open(os.path.join(GOLDEN, name)) as fh:
        return [ln.split() for ln in fh if ln.strip() and not ln.startswith("#")]


def test_tab1_codes_are_exactly_the_valid_ones():
    rows = _rows("tab1_tet_codes.txt")
    table = {int(r[1]): (int(r[2]), tuple(int(v) for v in r[3:7])) for r in rows}
    assert all(int(r[0], 2) == int(r[1]) for r in rows)  # the binary and integer columns agree
    seen = {}
    for labels in itertools.product(range(4), repeat=4):
        code, _ = oracle.simplex_code(list(labels))
        seen.setdefault(code, labels)
        nlab, local = table[code]  # KeyError: a code the table does not list
        assert len(set(labels)) == nlab, (labels, code)
        # the local labels of the table reproduce the equality pattern
        for i in range(4):
            for j in range(4):
                assert (labels[i] == labels[j]) == (local[i] == local[j]), (labels, code)
    assert set(seen) == set(table)  # all 15 appear


def test_fig4_triangle_codes():
    # Fig. 4: b is 1 iff it differs from a; c is 0 if equal to a, 1 if equal
    # to b (only possible when b is 1), else 2; the five valid codes.
    expect = {(0, 0, 0): 0, (0, 0, 1): 2, (0, 1, 0): 4, (0, 1, 1): 5, (0, 1, 2): 6}
    codes = set()
    for labels in itertools.product(range(3), repeat=3):
        code, _ = oracle.simplex_code(list(labels))
        pattern = tuple(sorted(set(labels)).index(v) for v in labels)
        first = {}
        canon = tuple(first.setdefault(v, len(first)) for v in labels)
        assert code == expect[canon], (labels, pattern, code)
        codes.add(code)
    assert codes == {0, 2, 4, 5, 6}


def test_element_counts_of_figs_5_and_6():
    rows = _rows("fig5_6_element_counts.txt")
    decode_tri = lambda c: [0, c >> 2, c & 3]
    decode_tet = lambda c: [0, c >> 4, (c >> 2) & 3, c & 3]
    for kind, code, count in rows:
        code, count = int(code), int(count)
        labels = decode_tri(code) if kind == "tri" else decode_tet(code)
        got_code, got_count = oracle.simplex_code(labels)
        assert got_code == code and got_count == count, (kind, code, got_count)


@pytest.mark.parametrize("dims", [(5, 4, 3), (2, 2, 2), (7, 3, 6)])
def test_plane_split_closed_form_3d(dims):
    # labels 0 on x < k, 1 beyond: each cell across the plane holds two
    # tetrahedra with x stepped first (1 + 3 split), two with x second
    # (2 + 2) and two with x last (3 + 1): 1 + 1 + 2 + 2 + 1 + 1 = 8 triangles
    nx, ny, nz = dims
    x = np.arange(nx)[None, None, :].repeat(ny, 1).repeat(nz, 0)
    y = np.arange(ny)[None, :, None].repeat(nx, 2).repeat(nz, 0)
    z = np.arange(nz)[:, None, None].repeat(ny, 1).repeat(nx, 2)
    for axis_vals, others in ((x, (ny - 1) * (nz - 1)), (y, (nx - 1) * (nz - 1)),
                              (z, (nx - 1) * (ny - 1))):
        k = max(1, axis_vals.max() // 2)
        lab = (axis_vals >= k).astype(np.int32) * 7 + 3
        r = oracle.simplex_index(lab, dims)
        assert r["total"] == 8 * others


def test_plane_split_closed_form_2d():
    nx, ny = 9, 6
    lab = (np.arange(nx)[None, :] >= 4).astype(np.int32).repeat(ny, 0)
    assert oracle.simplex_index(lab, (nx, ny, 1))["total"] == 2 * (ny - 1)
    lab = (np.arange(ny)[:, None] >= 2).astype(np.int32).repeat(nx, 1)
    assert oracle.simplex_index(lab, (nx, ny, 1))["total"] == 2 * (nx - 1)


@pytest.mark.parametrize("dims", [(4, 3, 5), (6, 5, 1)])
def test_constant_and_all_distinct(dims):
    n = int(np.prod(dims))
    cells, per = oracle.simplex_cells(dims)
    r = oracle.simplex_index(np.full(n, 4, np.int32), dims)
    assert r["total"] == 0 and not r["codes"].any()
    r = oracle.simplex_index(np.arange(n, dtype=np.int32), dims)
    full = 27 if per == 6 else 6
    assert (r["codes"] == full).all()
    assert r["total"] == cells * (per * (12 if per == 6 else 3))


def test_offsets_are_the_prefix_sum_of_cell_counts():
    rng = np.random.default_rng(3)
    for dims in [(6, 5, 4), (9, 7, 1)]:
        lab = rng.integers(0, 3, size=int(np.prod(dims))).astype(np.int32)
        r = oracle.simplex_index(lab, dims)
        cells, per = oracle.simplex_cells(dims)
        counts = np.array([sum(oracle.simplex_code(
            [0, c >> 4, (c >> 2) & 3, c & 3] if per == 6 else [0, c >> 2, c & 3])[1]
            for c in r["codes"][i * per:(i + 1) * per]) for i in range(cells)])
        assert r["cell_offsets"][0] == 0
        assert np.array_equal(np.diff(r["cell_offsets"]), counts[:-1])
        assert r["total"] == counts.sum()


def test_simplex_vertices_follow_the_kuhn_chains():
    # a label that differs only at the far corner (1,1,1) of a single cell
    # touches all 6 tetrahedra as their last vertex: each is a 3 + 1 split
    lab = np.zeros(8, np.int32)
    lab[7] = 1
    r = oracle.simplex_index(lab, (2, 2, 2))
    assert list(r["codes"]) == [3] * 6 and r["total"] == 6
    # the corner (1,0,0) is the second vertex of the two x-first chains only
    lab = np.zeros(8, np.int32)
    lab[1] = 1
    r = oracle.simplex_index(lab, (2, 2, 2))
    assert list(r["codes"]) == [16, 16, 0, 0, 0, 0]
    # 2D: the corner (1,0) is in the x-first triangle only
    lab = np.array([0, 1, 0, 0], np.int32)
    r = oracle.simplex_index(lab, (2, 2, 1))
    assert list(r["codes"]) == [4, 0]
