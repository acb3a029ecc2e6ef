"""The marching triangles / tetrahedra index pass on the GPU (ms_simplex_index)
against the oracle: every code and every cell offset, on label fields from
real segmentations, random labels with many ties, and edge shapes."""
import numpy as np
import pytest

import oracle
import paper_2303_15491_gb300 as ms
import synthfields as sf
from gpu_util import gpu_segment

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    h = ms.ms_create(0)
    yield h
    ms.ms_destroy(h)


def gpu_index(ctx, labels, dims):
    cells, per = ms.simplex_cells(dims)
    lab = torch.from_numpy(np.ascontiguousarray(labels, dtype=np.int32).reshape(-1)).cuda()
    codes = torch.full((max(cells * per, 1),), 255, dtype=torch.uint8, device="cuda")
    offs = torch.full((max(cells, 1),), -1, dtype=torch.int64, device="cuda")
    total = ms.ms_simplex_index(ctx, lab, dims, codes, offs)
    return codes[:cells * per].cpu().numpy(), offs[:cells].cpu().numpy(), total


def check(ctx, labels, dims, what):
    ref = oracle.simplex_index(labels, dims)
    codes, offs, total = gpu_index(ctx, labels, dims)
    assert total == ref["total"], f"{what}: total {total} != {ref['total']}"
    for name, a, b in (("codes", codes, ref["codes"]), ("offsets", offs, ref["cell_offsets"])):
        if not np.array_equal(a, b):
            bad = np.flatnonzero(a != b)
            raise AssertionError(f"{what}: {name} differ at {bad.size}, first {bad[:6]}: "
                                 f"{a[bad[:6]]} vs {b[bad[:6]]}")


@pytest.mark.parametrize("dims", [(40, 36, 30), (33, 17, 9), (2, 2, 2), (300, 200, 1), (2, 2, 1),
                                  (257, 3, 1), (5, 70, 41)])
def test_on_segmentation_labels(ctx, dims):
    f = sf.smoothed_noise(dims, 17, sigma=2.0)
    if dims[2] == 1:
        f = f[0]
    asc, desc, m, _ = gpu_segment(ctx, f)
    for name, lab in (("ms", m), ("asc", asc), ("desc", desc)):
        check(ctx, lab, dims, f"{dims} {name}")


@pytest.mark.parametrize("dims", [(31, 29, 27), (129, 65, 1), (64, 64, 64)])
@pytest.mark.parametrize("levels", [2, 4, 1 << 30])
def test_random_labels(ctx, dims, levels):
    g = np.random.default_rng(levels % 1000 + dims[0])
    lab = g.integers(0, levels, size=int(np.prod(dims))).astype(np.int32)
    check(ctx, lab, dims, f"{dims} levels {levels}")


@pytest.mark.parametrize("dims", [(1, 5, 5), (5, 1, 5), (7, 1, 1), (1, 1, 1), (6, 6, 2)])
def test_degenerate_shapes(ctx, dims):
    lab = np.arange(int(np.prod(dims)), dtype=np.int32) % 3
    check(ctx, lab, dims, f"degenerate {dims}")


def test_constant_and_distinct_totals(ctx):
    dims = (50, 40, 30)
    n = 50 * 40 * 30
    assert gpu_index(ctx, np.zeros(n, np.int32), dims)[2] == 0
    cells = 49 * 39 * 29
    assert gpu_index(ctx, np.arange(n, dtype=np.int32), dims)[2] == cells * 6 * 12


def test_errors(ctx):
    lab = torch.zeros(27, dtype=torch.int32, device="cuda")
    codes = torch.zeros(64, dtype=torch.uint8, device="cuda")
    offs = torch.zeros(8, dtype=torch.int64, device="cuda")
    with pytest.raises(ms.MSError) as e:  # codes not 16-byte aligned
        ms.ms_simplex_index(ctx, lab, (3, 3, 3), codes[1:], offs)
    assert e.value.name == "MS_ERR_INVALID_ARG"
    with pytest.raises(ms.MSError) as e:  # host labels
        ms.ms_simplex_index(ctx, np.zeros(27, np.int32), (3, 3, 3), codes, offs)
    assert e.value.name == "MS_ERR_INVALID_ARG"
    with pytest.raises(ms.MSError) as e:
        ms.ms_simplex_index(ctx, lab, (0, 3, 3), codes, offs)
    assert e.value.name == "MS_ERR_INVALID_ARG"


def test_offsets_only_8_byte_aligned(ctx):
    """Offsets at an address that is 8- but not 16-byte aligned take the
    scalar stores; every offset still equals the oracle's and nothing before
    the array is touched."""
    dims = (37, 23, 19)
    lab = np.random.default_rng(4).integers(0, 3, int(np.prod(dims))).astype(np.int32)
    ref = oracle.simplex_index(lab, dims)
    cells, per = ms.simplex_cells(dims)
    codes = torch.empty(cells * per, dtype=torch.uint8, device="cuda")
    offs = torch.full((cells + 1,), -1, dtype=torch.int64, device="cuda")
    total = ms.ms_simplex_index(ctx, torch.from_numpy(lab).cuda(), dims, codes, offs[1:])
    assert offs[1:].data_ptr() % 16 == 8
    assert total == ref["total"]
    assert np.array_equal(offs[1:].cpu().numpy(), ref["cell_offsets"])
    assert int(offs[0]) == -1
    assert np.array_equal(codes.cpu().numpy(), ref["codes"])


@pytest.mark.slow
def test_full_size_512(ctx):
    """512^3 MS labels of the smoothed-noise workload: the codes of sampled
    cells against the oracle (from their corner labels), and every offset
    against the prefix-sum property with element counts per code taken from
    the drawings of Figs. 5-6."""
    import os
    from test_gpu_fullsize import cached
    f = cached("noise512", lambda: sf.smoothed_noise((512, 512, 512), 0, sigma=4.0, radius=16))
    dims = (512, 512, 512)
    asc, desc, m, k = ms.segment(ctx, torch.from_numpy(f).cuda())
    del asc, desc
    cells, per = ms.simplex_cells(dims)
    codes = torch.empty(cells * per, dtype=torch.uint8, device="cuda")
    offs = torch.empty(cells, dtype=torch.int64, device="cuda")
    total = ms.ms_simplex_index(ctx, m, dims, codes, offs)
    # sampled cells: codes from the oracle on the cell's own 2x2x2 corners
    g = np.random.default_rng(5)
    lab = m.view(512, 512, 512)
    for c in g.integers(0, cells, size=3000):
        x, y, z = c % 511, (c // 511) % 511, c // (511 * 511)
        corner = lab[z:z + 2, y:y + 2, x:x + 2].cpu().numpy()
        ref = oracle.simplex_index(corner, (2, 2, 2))
        assert np.array_equal(codes[c * 6:(c + 1) * 6].cpu().numpy(), ref["codes"]), c
    # offsets: exclusive prefix sums of per-cell counts
    table = torch.zeros(32, dtype=torch.int64, device="cuda")
    with open(os.path.join(os.path.dirname(__file__), "golden", "fig5_6_element_counts.txt")) as fh:
        for ln in fh:
            if ln.startswith("tet"):
                _, code, cnt = ln.split()
                table[int(code)] = int(cnt)
    counts = table[codes.to(torch.int64)].view(cells, 6).sum(1)
    assert int(offs[0]) == 0
    assert bool(torch.equal(offs[1:] - offs[:-1], counts[:-1]))
    assert total == int(offs[-1] + counts[-1])


# ---------------------------------------------------------------- geometry
def gpu_geometry(ctx, labels, dims, mode):
    cells, per = ms.simplex_cells(dims)
    lab = torch.from_numpy(np.ascontiguousarray(labels, dtype=np.int32).reshape(-1)).cuda()
    codes = torch.empty(max(cells * per, 1), dtype=torch.uint8, device="cuda")
    offs = torch.empty(max(cells, 1), dtype=torch.int64, device="cuda")
    total = ms.ms_simplex_index(ctx, lab, dims, codes, offs, mode)
    dim = 2 if dims[2] == 1 else 3
    pts = torch.full((max(total, 1), dim, dim), float("nan"), dtype=torch.float32, device="cuda")
    pairs = torch.full((max(total, 1), 2), -1, dtype=torch.int32, device="cuda")
    ms.ms_simplex_geometry(ctx, lab, dims, offs, total, pts, pairs, mode)
    return total, pts[:total].cpu().numpy(), pairs[:total].cpu().numpy(), offs[:cells].cpu().numpy()


@pytest.mark.parametrize("dims", [(30, 26, 22), (2, 2, 2), (140, 90, 1), (33, 17, 9)])
@pytest.mark.parametrize("mode", [0, 1])
def test_geometry_matches_oracle(ctx, dims, mode):
    f = sf.smoothed_noise(dims, 23, sigma=2.0)
    if dims[2] == 1:
        f = f[0]
    _, _, m, _ = gpu_segment(ctx, f)
    for name, lab in (("ms", m), ("random 4", np.random.default_rng(1).integers(0, 4, m.size))):
        ref = oracle.simplex_geometry(lab, dims, mode)
        iref = oracle.simplex_index(lab, dims, mode)
        total, pts, pairs, offs = gpu_geometry(ctx, lab, dims, mode)
        assert total == ref["total"] == iref["total"]
        assert np.array_equal(offs, iref["cell_offsets"])
        assert np.array_equal(pts, ref["pos"]), f"{dims} {name} mode {mode}: points differ"
        assert np.array_equal(pairs, ref["pairs"]), f"{dims} {name} mode {mode}: pairs differ"


def test_geometry_rejects_a_wrong_total(ctx):
    dims = (10, 9, 8)
    lab = np.random.default_rng(2).integers(0, 3, 720).astype(np.int32)
    cells, per = ms.simplex_cells(dims)
    dl = torch.from_numpy(lab).cuda()
    codes = torch.empty(cells * per, dtype=torch.uint8, device="cuda")
    offs = torch.empty(cells, dtype=torch.int64, device="cuda")
    total = ms.ms_simplex_index(ctx, dl, dims, codes, offs)
    pts = torch.empty((total, 3, 3), dtype=torch.float32, device="cuda")
    with pytest.raises(ms.MSError) as e:
        ms.ms_simplex_geometry(ctx, dl, dims, offs, total - 1, pts)
    assert e.value.name == "MS_ERR_INVALID_ARG"
    ms.ms_simplex_geometry(ctx, dl, dims, offs, total, pts)  # without pairs


@pytest.mark.parametrize("dims", [(140, 90, 1), (30, 26, 22)])
def test_geometry_points_not_16_byte_aligned(ctx, dims):
    """Points at an address 4 bytes past a 16-byte boundary (the stores then
    go through the window word by word at the ends): bit-exact all the same,
    and the word before the array untouched."""
    lab = np.random.default_rng(6).integers(0, 4, int(np.prod(dims))).astype(np.int32)
    ref = oracle.simplex_geometry(lab, dims, 0)
    cells, per = ms.simplex_cells(dims)
    dl = torch.from_numpy(lab).cuda()
    codes = torch.empty(cells * per, dtype=torch.uint8, device="cuda")
    offs = torch.empty(cells, dtype=torch.int64, device="cuda")
    total = ms.ms_simplex_index(ctx, dl, dims, codes, offs)
    dim = 2 if dims[2] == 1 else 3
    buf = torch.full((total * dim * dim + 4,), float("nan"), dtype=torch.float32, device="cuda")
    pts = buf[1:1 + total * dim * dim].view(total, dim, dim)
    assert pts.data_ptr() % 16 == 4
    ms.ms_simplex_geometry(ctx, dl, dims, offs, total, pts)
    assert np.array_equal(pts.cpu().numpy(), ref["pos"])
    assert torch.isnan(buf[0]) and bool(torch.isnan(buf[1 + total * dim * dim:]).all())


@pytest.mark.parametrize("dims", [((1 << 21) - 3, 2, 1), ((1 << 21) + 5, 2, 1), ((1 << 21) - 3, 2, 2),
                                  ((6 << 20) + 3, 2, 1)])
def test_geometry_far_coordinates(ctx, dims):
    """Coordinates up to 2^21 - 3 (the largest whose corner sums the kernel
    converts without a division), past 2^21 (the division path) and past
    2^24 / 3 (sums of three corners beyond 2^24, where rounding the sum before
    dividing would round twice): points bit-exact with the oracle, whose
    coordinate rounding is pinned to exact rational arithmetic.  Sparse labels
    keep the element count small; triples of labels give the face and
    triangle centres (thirds)."""
    g = np.random.default_rng(dims[0] % 97 + dims[2])
    n = int(np.prod(dims))
    lab = np.zeros(n, np.int32)
    hit = g.random(n) < 0.03
    lab[hit] = g.integers(1, 4, int(hit.sum()))
    ref = oracle.simplex_geometry(lab, dims, 0)
    total, pts, pairs, _ = gpu_geometry(ctx, lab, dims, 0)
    assert total == ref["total"] > 0
    far = pts.reshape(total, -1)[:, 0] > (1 << 20)
    assert far.any()
    assert np.array_equal(pts, ref["pos"]), f"{dims}: points differ"
    assert np.array_equal(pairs, ref["pairs"]), f"{dims}: pairs differ"


@pytest.mark.slow
def test_geometry_full_size_512(ctx):
    """Region separators of the 512^3 MS labels, in the launch the index512
    bench times: for sampled cells, the elements at the cell's offsets equal
    the oracle's on the cell's own 2x2x2 corners, shifted to the cell (each
    local coordinate k/n becomes (n o + k)/n rounded, from the exact fraction)."""
    from test_gpu_fullsize import cached
    f = cached("noise512", lambda: sf.smoothed_noise((512, 512, 512), 0, sigma=4.0, radius=16))
    dims = (512, 512, 512)
    _, _, m, _ = ms.segment(ctx, torch.from_numpy(f).cuda())
    cells, per = ms.simplex_cells(dims)
    codes = torch.empty(cells * per, dtype=torch.uint8, device="cuda")
    offs = torch.empty(cells, dtype=torch.int64, device="cuda")
    total = ms.ms_simplex_index(ctx, m, dims, codes, offs)
    del codes
    pts = torch.empty((total, 3, 3), dtype=torch.float32, device="cuda")
    pairs = torch.empty((total, 2), dtype=torch.int32, device="cuda")
    ms.ms_simplex_geometry(ctx, m, dims, offs, total, pts, pairs)
    frac = {float(np.float32(k / n)): (k, n) for n in (1, 2, 3, 4) for k in range(n + 1)}
    lab = m.view(512, 512, 512)
    g = np.random.default_rng(8)
    seen = 0
    for c in g.integers(0, cells, size=2000):
        x, y, z = c % 511, (c // 511) % 511, c // (511 * 511)
        ref = oracle.simplex_geometry(lab[z:z + 2, y:y + 2, x:x + 2].cpu().numpy(), (2, 2, 2), 0)
        a = int(offs[c])
        b = int(offs[c + 1]) if c + 1 < cells else total
        assert b - a == ref["total"], c
        if a == b:
            continue
        seen += 1
        assert np.array_equal(pairs[a:b].cpu().numpy(), ref["pairs"]), c
        want = np.empty_like(ref["pos"])
        base = np.array([x, y, z], np.int64)
        for idx in np.ndindex(*ref["pos"].shape):
            k, n = frac[float(ref["pos"][idx])]
            want[idx] = np.float32((n * int(base[idx[-1]]) + k) / n)
        assert np.array_equal(pts[a:b].cpu().numpy(), want), c
    assert seen > 500
