"""Persistence pairs of the extrema on the GPU (ms_persistence, Sec. 4.1)
against the oracle's elder-rule pairing, pair for pair: every extremum and
every death vertex, for minima (asc labels) and maxima (desc labels), on
tiny grids through 256^3, with value ties, in fp32 and fp16, and on
staircases whose merge order defeats the parallel rounds (the in-order
finish then does the rest)."""
import numpy as np
import pytest

import oracle
import paper_2303_15491_gb300 as ms
import synthfields as sf
from gpu_util import to_dev

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    h = ms.ms_create(0)
    yield h
    ms.ms_destroy(h)


def gpu_pairs(ctx, f, direction, labels=None):
    dev = to_dev(f)
    if labels is None:
        asc, desc, _, _ = ms.segment(ctx, dev)
        labels = asc if direction < 0 else desc
    ext, death, info = ms.persistence(ctx, dev, labels, direction)
    return ext.cpu().numpy(), death.cpu().numpy(), info


def check(ctx, f, what, directions=(-1, 1)):
    infos = []
    for d in directions:
        ext, death, info = gpu_pairs(ctx, f, d)
        ref = oracle.persistence(f, d)
        assert info["n_extrema"] == ref["extremum"].size, (what, d)
        assert np.array_equal(ext, ref["extremum"]), (what, d)
        if not np.array_equal(death, ref["death"]):
            bad = np.flatnonzero(death != ref["death"])
            raise AssertionError(f"{what} dir {d}: {bad.size} deaths differ, extrema "
                                 f"{ext[bad[:6]]}: got {death[bad[:6]]} want {ref['death'][bad[:6]]}")
        assert np.count_nonzero(death == -1) == 1
        infos.append(info)
    return infos


def staircase(k_steps, wall=10000.0):
    """1D chain: minima at x = 2k with value k, walls at x = 2k + 1 with value
    wall - k.  The lowest wall separates the two youngest minima, so every
    basin's earliest edge leads to a younger one."""
    f = np.empty(2 * k_steps + 1, np.float32)
    f[0::2] = np.arange(k_steps + 1)
    f[1::2] = wall - np.arange(k_steps)
    return f


def test_chain_worked_by_hand(ctx, golden):
    g = golden("persistence_chain7.txt")
    f = np.array(g["values"], np.float32).reshape(1, 7)
    for d, key in ((-1, "min"), (1, "max")):
        ext, death, _ = gpu_pairs(ctx, f, d)
        assert ext.tolist() == g[f"{key}_extremum"] and death.tolist() == g[f"{key}_death"]


@pytest.mark.parametrize("dims", [(1, 1, 1), (2, 1, 1), (7, 1, 1), (4, 3, 1), (3, 3, 2), (5, 2, 2),
                                  (2, 2, 3), (9, 7, 5), (33, 17, 1), (17, 9, 6)])
@pytest.mark.parametrize("levels", [2, 3, 1 << 20])
def test_tiny_grids_with_ties(ctx, dims, levels):
    g = np.random.default_rng(dims[0] * 7 + dims[1] * 3 + levels % 101)
    shape = dims[::-1] if dims[2] > 1 else dims[1::-1]
    f = g.integers(0, levels, size=shape).astype(np.float32)
    check(ctx, f, f"{dims} levels {levels}")


@pytest.mark.parametrize("dims", [(64, 64, 64), (96, 80, 72), (512, 384, 1)])
def test_gaussian_sums(ctx, dims):
    f = sf.gaussian_sum(dims, 3)
    if dims[2] == 1:
        f = f[0]
    infos = check(ctx, f, f"gaussians {dims}")
    assert all(i["finish_edges"] == 0 for i in infos)


@pytest.mark.parametrize("n", [128, 256])
def test_smoothed_noise(ctx, n):
    f = sf.smoothed_noise((n, n, n), 5, sigma=4.0, radius=16)
    infos = check(ctx, f, f"noise {n}^3")
    assert infos[0]["n_extrema"] > 100 and infos[0]["basin_edges"] > infos[0]["n_extrema"]


def test_quantised_noise_256(ctx):
    f = sf.quantize_levels(sf.smoothed_noise((256, 256, 256), 6, sigma=4.0, radius=16), 64)
    check(ctx, f, "quantised 256^3")


@pytest.mark.parametrize("shape", [(1024, 768), (80, 72, 64)])
def test_white_noise(ctx, shape):
    f = np.random.default_rng(9).standard_normal(shape).astype(np.float32)
    infos = check(ctx, f, f"white {shape}")
    assert infos[0]["rounds"] >= 3


@pytest.mark.parametrize("dims", [(48, 40, 36), (120, 90, 1)])
def test_float16_field(ctx, dims):
    f = sf.smoothed_noise(dims, 2, sigma=2.0).astype(np.float16)
    check(ctx, f, f"fp16 {dims}")


def test_oracle_labels_give_the_same_pairs(ctx):
    f = sf.smoothed_noise((60, 50, 40), 8, sigma=3.0)
    ref = oracle.segment(f)
    for d, name in ((-1, "asc"), (1, "desc")):
        lab = torch.from_numpy(ref[name].astype(np.int32)).cuda()
        ext, death, _ = gpu_pairs(ctx, f, d, labels=lab)
        want = oracle.persistence(f, d)
        assert np.array_equal(ext, want["extremum"]) and np.array_equal(death, want["death"])


@pytest.mark.parametrize("steps", [3, 40, 3000])
def test_staircase_finishes_in_entry_order(ctx, steps):
    f = staircase(steps).reshape(1, -1)
    infos = check(ctx, f, f"staircase {steps}")
    if steps >= 40:
        assert all(i["finish_edges"] > 0 for i in infos), infos


def test_staircase_with_noise_runs_rounds_then_finishes(ctx):
    """Noise wells inside every step merge in the parallel rounds; the
    staircase itself is left to the finish."""
    g = np.random.default_rng(4)
    base = staircase(600)
    f = (np.repeat(base[None, :], 6, axis=0) + g.uniform(0, 0.4, (6, base.size))).astype(np.float32)
    infos = check(ctx, f, "staircase + noise")
    assert all(i["rounds"] >= 4 and i["finish_edges"] > 0 for i in infos), infos


def test_repeated_calls_and_sizes(ctx):
    """A large call, then a small one on the same context (capacities kept
    from the first), then the large one again."""
    big = sf.smoothed_noise((128, 96, 80), 1, sigma=2.0)
    small = sf.gaussian_sum((20, 18, 16), 2)
    for f in (big, small, big):
        check(ctx, f, f"{f.shape}", directions=(-1,))


def test_capacity_query_and_errors(ctx):
    f = sf.smoothed_noise((40, 30, 20), 3, sigma=2.0)
    dev = to_dev(f)
    asc, desc, _, _ = ms.segment(ctx, dev)
    dims, dt = ms.dims_of(f), ms.dtype_code(f)
    n_min = oracle.persistence(f, -1)["extremum"].size
    with pytest.raises(ms.MSError) as e:
        ms.ms_persistence(ctx, dev, dims, dt, asc, -1, None, None, 0)
    assert e.value.name == "MS_ERR_TOO_LARGE" and e.value.info["n_extrema"] == n_min
    ext = torch.empty(n_min, dtype=torch.int32, device="cuda")
    dth = torch.empty_like(ext)
    info = ms.ms_persistence(ctx, dev, dims, dt, asc, -1, ext, dth, n_min)
    assert info["n_extrema"] == n_min
    for direction in (0, 2):
        with pytest.raises(ms.MSError, match="INVALID_ARG"):
            ms.ms_persistence(ctx, dev, dims, dt, asc, direction, ext, dth, n_min)
    # a label that is not an extremum's own label
    bad = asc.clone()
    v = int(torch.nonzero(asc != torch.arange(asc.numel(), device="cuda", dtype=torch.int32))[0])
    bad[int(asc[v])] = v
    with pytest.raises(ms.MSError, match="INVALID_ARG"):
        ms.ms_persistence(ctx, dev, dims, dt, bad, -1, ext, dth, n_min)
    # labels out of range
    bad = asc.clone()
    bad[5] = asc.numel()
    with pytest.raises(ms.MSError, match="INVALID_ARG"):
        ms.ms_persistence(ctx, dev, dims, dt, bad, -1, ext, dth, n_min)
    # a NaN in the field
    g = dev.clone()
    g.view(-1)[7] = float("nan")
    with pytest.raises(ms.MSError, match="NAN_INPUT"):
        ms.ms_persistence(ctx, g, dims, dt, asc, -1, ext, dth, n_min)
    # host pointers
    with pytest.raises(ms.MSError, match="INVALID_ARG"):
        ms.ms_persistence(ctx, f, dims, dt, asc, -1, ext, dth, n_min)
