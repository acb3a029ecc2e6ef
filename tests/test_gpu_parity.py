"""GPU parity: every step of the path, called through the C ABI, against the
CPU oracle on the same seeded inputs.  Labels are integers, so the bar is
bit-exact equality everywhere."""
import numpy as np
import pytest

import oracle
import paper_2303_15491_gb300 as ms
import synthfields as sf
from gpu_util import assert_same_labels, gpu_segment, to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    h = ms.ms_create(0)
    yield h
    ms.ms_destroy(h)


def run_and_compare(ctx, f, what=""):
    ref = oracle.segment(f)
    assert_same_labels(gpu_segment(ctx, f), ref, what)
    return ref


# ------------------------------------------------------------- worked examples
def test_fig1(ctx, golden):
    g = golden("fig1_4x4.txt")
    f = np.array(g["values"], np.float32).reshape(4, 4)
    asc, desc, m, k = gpu_segment(ctx, f)
    assert desc.tolist() == g["desc"] and asc.tolist() == g["asc"]
    assert m.tolist() == g["ms"] and k == g["K"][0]


def test_fig3_chain(ctx, golden):
    g = golden("fig3_chain7.txt")
    f = np.array(g["values"], np.float32).reshape(1, 1, 7)
    dev = to_dev(f)
    up = torch.empty(7, dtype=torch.int32, device="cuda")
    dn = torch.empty_like(up)
    ms.ms_steepest(ctx, dev, (7, 1, 1), ms.MS_F32, up, dn)
    assert up.cpu().tolist() == g["up"]
    ms.ms_compress(ctx, up, 7)
    assert up.cpu().tolist() == g["desc"]


# ------------------------------------------------------------- step 1: keys
@pytest.mark.parametrize("dtype", [np.float32, np.float16])
def test_order_keys_are_the_value_index_order(ctx, dtype):
    g = sf.rng_for(11)
    vals = g.standard_normal(50000).astype(dtype)
    vals[:200] = 0.0
    vals[200:400] = -0.0
    vals[400:410] = np.inf
    vals[410:420] = -np.inf
    info = np.finfo(dtype)
    vals[420:440] = info.smallest_subnormal * np.arange(20)
    vals[440:460] = -info.smallest_subnormal * np.arange(20)
    vals[460:2000] = np.round(vals[460:2000])  # many exact ties
    g.shuffle(vals)
    keys = torch.empty(vals.size, dtype=torch.int32, device="cuda")
    ms.ms_order_keys(ctx, to_dev(vals), vals.size, ms.MS_F16 if dtype == np.float16 else ms.MS_F32, keys)
    k = keys.cpu().numpy().view(np.uint32).astype(np.int64)
    idx = np.arange(vals.size)
    by_value = np.lexsort((idx, vals.astype(np.float64)))  # Sec. 4.1: value, then index
    by_key = np.lexsort((idx, k))
    assert np.array_equal(by_value, by_key)


def test_order_keys_reject_nan(ctx):
    v = np.ones(1000, np.float32)
    v[777] = np.nan
    keys = torch.empty(1000, dtype=torch.int32, device="cuda")
    with pytest.raises(ms.MSError) as e:
        ms.ms_order_keys(ctx, to_dev(v), 1000, ms.MS_F32, keys)
    assert e.value.name == "MS_ERR_NAN_INPUT"


# ------------------------------------------------------------- step 2: steepest
STEEP_DIMS = [(1, 1, 1), (2, 1, 1), (33, 1, 1), (1, 40, 1), (31, 17, 1), (64, 64, 1), (2, 2, 2),
              (33, 9, 5), (1, 7, 9), (8, 1, 13), (37, 29, 23), (64, 16, 40), (130, 3, 2)]


@pytest.mark.parametrize("dims", STEEP_DIMS)
@pytest.mark.parametrize("kind", ["noise", "ties", "const"])
def test_steepest_matches_oracle(ctx, dims, kind):
    if kind == "noise":
        f = sf.smoothed_noise(dims, 3, sigma=1.5, radius=6)
    elif kind == "ties":
        f = sf.random_ties(dims, 3, levels=4)
    else:
        f = sf.constant(dims, -0.0)
    up_ref, dn_ref = oracle.steepest(f)
    n = f.size
    up = torch.empty(n, dtype=torch.int32, device="cuda")
    dn = torch.empty_like(up)
    ms.ms_steepest(ctx, to_dev(f), dims, ms.MS_F32, up, dn)
    assert np.array_equal(up.cpu().numpy(), up_ref)
    assert np.array_equal(dn.cpu().numpy(), dn_ref)


# ------------------------------------------------------------- step 3: compression
@pytest.mark.parametrize("n", [1, 7, 1000, 1 << 20])
def test_compress_long_chain(ctx, n):
    """Fig. 3 stretched: one chain 0 -> 1 -> ... -> n-1."""
    p = torch.arange(1, n + 1, dtype=torch.int32, device="cuda")
    p[-1] = n - 1
    ms.ms_compress(ctx, p, n)
    assert bool((p == n - 1).all())


@pytest.mark.parametrize("seed", [0, 1])
def test_compress_matches_oracle(ctx, seed):
    f = sf.smoothed_noise((70, 50, 30), seed, sigma=3.0, radius=12)
    up, dn = oracle.steepest(f)
    for ptr in (up, dn):
        d = torch.from_numpy(ptr.copy()).cuda()
        ms.ms_compress(ctx, d, ptr.size)
        assert np.array_equal(d.cpu().numpy(), oracle.follow(ptr))


def test_compress_random_deep_forest(ctx):
    g = sf.rng_for(5)
    n = 200000
    perm = g.permutation(n)
    parent = np.empty(n, np.int32)
    # a random recursive tree over a random vertex order: deep chains of mixed length
    parent[perm[0]] = perm[0]
    choose = (np.arange(1, n) * g.uniform(0.9, 1.0, n - 1)).astype(np.int64)
    parent[perm[1:]] = perm[choose]
    d = torch.from_numpy(parent.copy()).cuda()
    ms.ms_compress(ctx, d, n)
    assert np.array_equal(d.cpu().numpy(), oracle.follow(parent))


def test_compress_rejects_out_of_range(ctx):
    p = torch.tensor([0, 5, 1], dtype=torch.int32, device="cuda")
    with pytest.raises(ms.MSError) as e:
        ms.ms_compress(ctx, p, 3)
    assert e.value.name == "MS_ERR_INVALID_ARG"


def test_compress_cycle_is_not_converged(ctx):
    """A 2-cycle is not a forest; the round cap ends the work with a status."""
    p = torch.tensor([1, 0, 2], dtype=torch.int32, device="cuda")
    with pytest.raises(ms.MSError) as e:
        ms.ms_compress(ctx, p, 3)
    assert e.value.name == "MS_ERR_NOT_CONVERGED"


# ------------------------------------------------------------- step 4: MS ids
@pytest.mark.parametrize("n,levels", [(1, 1), (5000, 3), (300000, 50), (300000, 300000),
                                      (2000000, 40000), (6000000, 6000000)])
def test_pair_rank_matches_oracle(ctx, n, levels):
    g = sf.rng_for(n + levels)
    a = g.integers(0, min(levels, n), n).astype(np.int32)
    d = (g.integers(0, min(levels, n), n).astype(np.int32) * 7919 % n).astype(np.int32)
    ref, k_ref = oracle.ms_rank(a, d)
    out = torch.empty(n, dtype=torch.int32, device="cuda")
    k = ms.ms_pair_rank(ctx, torch.from_numpy(a).cuda(), torch.from_numpy(d).cuda(), n, out)
    assert k == k_ref
    assert np.array_equal(out.cpu().numpy(), ref)


# ------------------------------------------------------------- the whole path
@pytest.mark.parametrize("seed", range(5))
def test_segment_gaussian_sum_64(ctx, seed):
    """The 64^3 small case: 8 Gaussians + 1e-3 noise, seeds 0..4."""
    f = sf.gaussian_sum((64, 64, 64), seed)
    run_and_compare(ctx, f, f"gauss64 seed {seed}")


SEG_DIMS = [(1, 1, 1), (3, 1, 1), (1, 1, 9), (5, 5, 1), (2, 2, 2), (2, 3, 2), (17, 2, 31),
            (33, 33, 1), (65, 7, 3), (40, 41, 42), (129, 66, 10), (255, 1, 77), (300, 257, 1)]


@pytest.mark.parametrize("dims", SEG_DIMS)
@pytest.mark.parametrize("kind", ["noise", "ties", "ramp", "const"])
def test_segment_shapes_and_kinds(ctx, dims, kind):
    if kind == "noise":
        f = sf.smoothed_noise(dims, 7, sigma=2.0, radius=8)
    elif kind == "ties":
        f = sf.random_ties(dims, 7, levels=3)
    elif kind == "ramp":
        f = sf.ramp(dims)
    else:
        f = sf.constant(dims, 3.0)
    run_and_compare(ctx, f, f"{kind} {dims}")


# rows of whole 16-byte units (nx a multiple of 8) take TMA boxes, the others plain loads
@pytest.mark.parametrize("dims", [(48, 40, 36), (513, 300, 1), (520, 300, 1), (52, 33, 20),
                                  (136, 70, 40)])
def test_segment_fp16(ctx, dims):
    f = sf.smoothed_noise(dims, 9, sigma=2.0, radius=8).astype(np.float16)
    run_and_compare(ctx, f, f"fp16 {dims}")
    q = sf.quantize_levels(sf.smoothed_noise(dims, 9, sigma=2.0, radius=8), 64).astype(np.float16)
    run_and_compare(ctx, q, f"fp16 quantised {dims}")


def test_segment_quantised_ties_midsize(ctx):
    """Several tiles with a ragged tail, 256-level ties (the 2b variant's
    statistics at a size the oracle finishes in seconds)."""
    f = sf.quantize_levels(sf.smoothed_noise((160, 144, 136), 0, sigma=4.0))
    run_and_compare(ctx, f, "quantised 160x144x136")


def test_segment_smoothed_noise_midsize(ctx):
    f = sf.smoothed_noise((160, 144, 136), 1, sigma=4.0)
    run_and_compare(ctx, f, "noise 160x144x136")


def test_segment_broad_ramp_long_paths(ctx):
    f = sf.broad_gaussians_ramp((150, 140, 130), 2, sigma=60.0)
    ref = run_and_compare(ctx, f, "broad ramp")
    assert ref["K"] >= 1


def test_segment_is_deterministic(ctx):
    f = sf.quantize_levels(sf.smoothed_noise((90, 80, 70), 4, sigma=3.0))
    a = gpu_segment(ctx, f)
    for _ in range(3):
        b = gpu_segment(ctx, f)
        for x, y in zip(a[:3], b[:3]):
            assert np.array_equal(x, y)
        assert a[3] == b[3]


def test_segment_host_buffers(ctx):
    f = sf.gaussian_sum((50, 60, 70), 8)
    ref = oracle.segment(f)
    n = f.size
    asc = np.empty(n, np.int32)
    desc = np.empty(n, np.int32)
    m = np.empty(n, np.int32)
    ms.ms_segment_host(ctx, f, (50, 60, 70), ms.MS_F32, asc, desc, m)
    assert_same_labels((asc, desc, m, ms.ms_last_region_count(ctx)), ref, "host")


# ------------------------------------------------------------- errors
def test_nan_input(ctx):
    f = sf.gaussian_sum((20, 20, 20), 0)
    f[3, 4, 5] = np.nan
    with pytest.raises(ms.MSError) as e:
        gpu_segment(ctx, f)
    assert e.value.name == "MS_ERR_NAN_INPUT"
    # the context stays usable
    run_and_compare(ctx, sf.gaussian_sum((20, 20, 20), 0), "after NaN")


def test_invalid_arguments(ctx):
    f = to_dev(np.zeros((4, 4, 4), np.float32))
    out = [torch.empty(64, dtype=torch.int32, device="cuda") for _ in range(3)]
    host = np.zeros(64, np.int32)

    def status(fn):
        with pytest.raises(ms.MSError) as e:
            fn()
        return e.value.name

    assert status(lambda: ms.ms_segment(ctx, f, (4, 4, 4), ms.MS_F32, host, out[1], out[2])) == \
        "MS_ERR_INVALID_ARG"
    assert status(lambda: ms.ms_segment(ctx, f, (4, 0, 4), ms.MS_F32, *out)) == "MS_ERR_INVALID_ARG"
    assert status(lambda: ms.ms_segment(ctx, f, (4, 4, 4), 7, *out)) == "MS_ERR_UNSUPPORTED_DTYPE"
    assert status(lambda: ms.ms_segment(ctx, f, (4, 4, 4), ms.MS_F32, out[0], out[0], out[2])) == \
        "MS_ERR_INVALID_ARG"
    assert status(lambda: ms.ms_segment(ctx, f, (1 << 16, 1 << 16, 1), ms.MS_F32, *out)) == \
        "MS_ERR_TOO_LARGE"
    assert status(lambda: ms.ms_segment(ctx, f, (1 << 31, 1, 1), ms.MS_F32, *out)) == \
        "MS_ERR_TOO_LARGE"
    ms.ms_segment(ctx, f, (4, 4, 4), ms.MS_F32, *out)  # still usable
    assert ms.ms_last_region_count(ctx) == 1


def test_borrowed_stream(ctx):
    s = torch.cuda.Stream()
    h = ms.ms_create(0, s)
    try:
        f = sf.gaussian_sum((30, 20, 10), 2)
        assert_same_labels(gpu_segment(h, f), oracle.segment(f), "borrowed stream")
    finally:
        ms.ms_destroy(h)


@pytest.mark.parametrize("dims", [(40, 41, 42), (64, 64, 64), (300, 257, 1)])
def test_staged_path_matches_oracle(ctx, dims):
    """The step-by-step GPU path (ms_segment_staged) is an independent GPU
    form of the same method; it must agree with the oracle too."""
    f = sf.smoothed_noise(dims, 12, sigma=2.5, radius=10)
    ref = oracle.segment(f)
    dev = to_dev(f)
    n = f.size
    out = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(3)]
    ms.ms_segment_staged(ctx, dev, dims, ms.MS_F32, *out)
    got = tuple(o.cpu().numpy() for o in out) + (ms.ms_last_region_count(ctx),)
    assert_same_labels(got, ref, f"staged {dims}")


@pytest.mark.parametrize("dims", [(32, 16, 16), (33, 17, 17), (31, 15, 15), (64, 32, 48),
                                  (97, 50, 35), (32, 16, 1), (1, 16, 16), (32, 1, 16)])
def test_tile_boundaries(ctx, dims):
    """Exact tile multiples, one past, one short, and flat boxes: paths that
    cross tile faces, edges and corners."""
    for seed, f in enumerate([sf.smoothed_noise(dims, 21, sigma=3.0, radius=12),
                              sf.random_ties(dims, 22, levels=2),
                              sf.broad_gaussians_ramp(dims, 23, sigma=20.0)]):
        run_and_compare(ctx, f, f"tile boundary {dims} case {seed}")


@pytest.mark.parametrize("seed", [0, 1])
def test_interior_tiles_signed_zero_and_subnormals(ctx, seed):
    """Tiles whose halo lies inside the field compare raw float values; the
    order there must still tie -0 with +0 (broken by index) and order
    subnormals exactly.  The grid has interior and boundary tiles."""
    dims = (100, 52, 50)
    g = sf.rng_for(100 + seed)
    tiny = np.float32(1.4e-45)
    f = (g.integers(-3, 4, size=(50, 52, 100)).astype(np.float32) * tiny)
    zeros = g.uniform(size=f.shape) < 0.3
    f[zeros] = np.where(g.uniform(size=zeros.sum()) < 0.5, np.float32(0.0), np.float32(-0.0))
    run_and_compare(ctx, f, f"subnormal/zero field seed {seed}")
    # the same with infinities sprinkled in
    inf = g.uniform(size=f.shape) < 0.01
    f[inf] = np.where(g.uniform(size=inf.sum()) < 0.5, np.float32(np.inf), np.float32(-np.inf))
    run_and_compare(ctx, f, f"subnormal/zero/inf field seed {seed}")


def test_nan_in_interior_tile(ctx):
    f = sf.smoothed_noise((100, 52, 50), 3, sigma=3.0)
    f[25, 26, 50] = np.nan
    with pytest.raises(ms.MSError) as e:
        gpu_segment(ctx, f)
    assert e.value.name == "MS_ERR_NAN_INPUT"


def zigzag_field(nx=64, ny=40, nz=40, x0=31):
    """A strictly increasing path that steps +(1,1,0) and (-1,0,-1) in turn,
    so it crosses the x tile face between x0 and x0+1 at every step (about
    2 min(ny, nz) crossings of the same two tiles, far more than there are
    tiles), on a low smooth background."""
    f = sf.smoothed_noise((nx, ny, nz), 41, sigma=2.0) - np.float32(1000.0)
    x, y, z = x0, 0, nz - 1
    k = 0
    while True:
        f[z, y, x] = k
        k += 1
        if k % 2 == 1:
            x, y = x + 1, y + 1
        else:
            x, z = x - 1, z - 1
        if y >= ny or z < 0:
            break
    return f


@pytest.mark.parametrize("sign", [1, -1])
def test_paths_reentering_the_same_tiles(ctx, sign):
    """A steepest path may leave and re-enter the same tiles many times: the
    number of face hops is not bounded by the tile count."""
    f = zigzag_field()
    if sign < 0:  # the same path for steepest descent
        f = -f
    run_and_compare(ctx, f, f"zigzag path sign {sign}")


def test_small_grid_with_more_face_hops_than_tiles(ctx):
    # 18^3 has 4 tiles; a descending path of this seeded field changes tiles 5 times
    f = sf.smoothed_noise((18, 18, 18), 109732, sigma=2.5)
    run_and_compare(ctx, f, "18^3 smoothed noise")


# 2D grids (nz = 1) take 128 x 64 tiles: exact multiples, one past, one
# short, many tiles, single rows and columns, and widths that are not a
# multiple of 4 (no box loads).
FLAT_DIMS = [(128, 64, 1), (129, 65, 1), (127, 63, 1), (256, 128, 1), (301, 200, 1), (4, 4, 1),
             (1000, 3, 1), (3, 1000, 1), (1, 5000, 1), (5000, 1, 1), (515, 390, 1)]


@pytest.mark.parametrize("dims", FLAT_DIMS)
def test_flat_tiles(ctx, dims):
    for case, f in enumerate([sf.smoothed_noise(dims, 51, sigma=3.0, radius=12),
                              sf.random_ties(dims, 52, levels=2),
                              sf.broad_gaussians_ramp(dims, 53, sigma=40.0)]):
        run_and_compare(ctx, f, f"flat {dims} case {case}")


def test_flat_long_paths_across_many_tiles(ctx):
    f = sf.broad_gaussians_ramp((1500, 1100, 1), 54, sigma=300.0)
    run_and_compare(ctx, f, "flat broad ramp")


@pytest.mark.parametrize("seed", [0, 1])
def test_flat_interior_tiles_signed_zero_subnormals_inf(ctx, seed):
    """2D tiles whose halo lies inside the field compare raw values."""
    g = sf.rng_for(200 + seed)
    tiny = np.float32(1.4e-45)
    f = g.integers(-3, 4, size=(200, 400)).astype(np.float32) * tiny
    zeros = g.uniform(size=f.shape) < 0.3
    f[zeros] = np.where(g.uniform(size=zeros.sum()) < 0.5, np.float32(0.0), np.float32(-0.0))
    run_and_compare(ctx, f, f"flat subnormal/zero seed {seed}")
    inf = g.uniform(size=f.shape) < 0.01
    f[inf] = np.where(g.uniform(size=inf.sum()) < 0.5, np.float32(np.inf), np.float32(-np.inf))
    run_and_compare(ctx, f, f"flat subnormal/zero/inf seed {seed}")


def test_flat_nan_in_interior_tile(ctx):
    f = sf.smoothed_noise((400, 200, 1), 5, sigma=3.0)
    f[0, 100, 200] = np.nan
    with pytest.raises(ms.MSError) as e:
        gpu_segment(ctx, f)
    assert e.value.name == "MS_ERR_NAN_INPUT"


def test_flat_tiles_equal_staged_path(ctx):
    f = sf.smoothed_noise((700, 333, 1), 55, sigma=4.0)
    dev = to_dev(f)
    n = f.size
    tiled = ms.segment(ctx, dev)
    outs = [torch.empty(n, dtype=torch.int32, device="cuda") for _ in range(3)]
    ms.ms_segment_staged(ctx, dev, (700, 333, 1), ms.MS_F32, *outs)
    for a, b in zip(tiled[:3], outs):
        assert torch.equal(a, b)
    assert tiled[3] == ms.ms_last_region_count(ctx)


def test_repeated_calls_replay_and_follow_new_contents(ctx):
    """ms_segment on the same buffers: the third call replays the captured
    graph; changing the field's contents in place (many more regions) is
    caught and the call runs step by step; results always match the oracle."""
    dims = (70, 60, 50)
    smooth = sf.broad_gaussians_ramp(dims, 91, sigma=25.0)
    noisy = sf.smoothed_noise(dims, 92, sigma=1.0)
    dev = to_dev(smooth)
    outs = [torch.empty(smooth.size, dtype=torch.int32, device="cuda") for _ in range(3)]
    ms.ms_profile_enable(ctx, True)
    for f in (smooth, smooth, smooth, noisy, noisy, noisy, smooth):
        dev.copy_(torch.from_numpy(np.ascontiguousarray(f)))
        torch.cuda.synchronize()
        ms.ms_segment(ctx, dev, dims, ms.MS_F32, *outs)
        got = tuple(o.cpu().numpy() for o in outs) + (ms.ms_last_region_count(ctx),)
        assert_same_labels(got, oracle.segment(f), "repeated call")
    prof = ms.ms_profile_read(ctx)
    ms.ms_profile_enable(ctx, False)
    assert prof["stages"]["graph"]["launches"] > 0
