"""Batched segmentation: many fields of uneven, non-cubic shapes (float32 and
float16, smoothed noise and Gaussian sums) in one ms_segment_batch call must
give, field by field, exactly the oracle's labels -- and exactly what separate
ms_segment calls give."""
import numpy as np
import pytest

import oracle
import paper_2303_15491_gb300 as ms
import synthfields as sf
from gpu_util import assert_same_labels

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    h = ms.ms_create(0)
    yield h
    ms.ms_destroy(h)


def run_batch(ctx, fields):
    devs = [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in fields]
    outs = [[torch.empty(f.size, dtype=torch.int32, device="cuda") for _ in range(3)] for f in fields]
    dims = [ms.dims_of(f) for f in fields]
    dts = [ms.dtype_code(f) for f in fields]
    ks = ms.ms_segment_batch(ctx, devs, dims, dts, [o[0] for o in outs], [o[1] for o in outs],
                             [o[2] for o in outs])
    return [(o[0].cpu().numpy(), o[1].cpu().numpy(), o[2].cpu().numpy(), k) for o, k in zip(outs, ks)]


def small_batch(n, seed):
    specs = sf.batch_specs(n, seed=seed, lo=16, hi=72)
    return [sf.batch_field(s) for s in specs]


@pytest.mark.parametrize("seed", [0, 1])
def test_batch_matches_oracle(ctx, seed):
    fields = small_batch(14, seed)
    assert {f.dtype for f in fields} == {np.dtype(np.float32), np.dtype(np.float16)}
    for i, (f, got) in enumerate(zip(fields, run_batch(ctx, fields))):
        assert_same_labels(got, oracle.segment(f), f"batch field {i} {f.shape} {f.dtype}")


def test_batch_equals_single_calls_and_is_deterministic(ctx):
    fields = small_batch(9, 5) + [sf.quantize_levels(sf.smoothed_noise((40, 33, 20), 3, sigma=3.0), 16)]
    a = run_batch(ctx, fields)
    b = run_batch(ctx, fields)
    for f, x, y in zip(fields, a, b):
        dev = torch.from_numpy(np.ascontiguousarray(f)).cuda()
        single = ms.segment(ctx, dev)
        for u, v, w in zip(x[:3], y[:3], single[:3]):
            assert np.array_equal(u, v) and np.array_equal(u, w.cpu().numpy())
        assert x[3] == y[3] == single[3]


def test_batch_with_flat_field_falls_back(ctx):
    fields = small_batch(4, 7) + [sf.smoothed_noise((50, 40, 1), 2, sigma=2.0)]
    for f, got in zip(fields, run_batch(ctx, fields)):
        assert_same_labels(got, oracle.segment(f), f"mixed batch {f.shape}")


def test_batch_nan_fails_whole_call(ctx):
    fields = small_batch(4, 9)
    fields[2] = fields[2].copy()
    fields[2].flat[7] = np.nan
    with pytest.raises(ms.MSError) as e:
        run_batch(ctx, fields)
    assert e.value.name == "MS_ERR_NAN_INPUT"


def test_batch_region_count_sum(ctx):
    fields = small_batch(6, 11)
    res = run_batch(ctx, fields)
    assert ms.ms_last_region_count(ctx) == sum(r[3] for r in res)


def test_batch_with_many_distinct_pairs(ctx):
    """Barely smoothed noise: a large share of the tile pairs are distinct
    final pairs, so the first (estimated) pair-set size is too small and the
    call must retry with the exact bound -- correctly and quickly."""
    fields = [sf.smoothed_noise((48, 40, 36), s, sigma=0.6, radius=2) for s in range(6)]
    fresh = ms.ms_create(0)  # no size hint from earlier calls
    try:
        for f, got in zip(fields, run_batch(fresh, fields)):
            assert_same_labels(got, oracle.segment(f), f"noisy batch {f.shape}")
    finally:
        ms.ms_destroy(fresh)


def test_single_field_many_distinct_pairs(ctx):
    f = sf.smoothed_noise((96, 80, 72), 8, sigma=0.5, radius=2)
    fresh = ms.ms_create(0)
    try:
        dev = torch.from_numpy(f).cuda()
        got = ms.segment(fresh, dev)
        got = (got[0].cpu().numpy(), got[1].cpu().numpy(), got[2].cpu().numpy(), got[3])
        assert_same_labels(got, oracle.segment(f), "noisy single field")
    finally:
        ms.ms_destroy(fresh)


def test_batch_mixed_2d_and_3d_fields(ctx):
    """2D fields (2D tiles) interleaved with 3D ones in one batch: the host
    groups them by tile shape, and each field's labels and region count must
    still come back in the caller's order."""
    three = small_batch(5, 21)
    two = [sf.smoothed_noise((300, 200, 1), 31, sigma=3.0)[0],
           sf.random_ties((129, 65, 1), 32, levels=3)[0],
           sf.smoothed_noise((64, 64, 1), 33, sigma=2.0)[0].astype(np.float16),
           sf.broad_gaussians_ramp((500, 70, 1), 34, sigma=50.0)[0]]
    fields = [two[0], three[0], three[1], two[1], three[2], two[2], three[3], three[4], two[3]]
    res = run_batch(ctx, fields)
    for i, (f, got) in enumerate(zip(fields, res)):
        assert_same_labels(got, oracle.segment(f), f"mixed batch field {i} {f.shape} {f.dtype}")
    assert ms.ms_last_region_count(ctx) == sum(r[3] for r in res)


def test_batch_long_paths_mixed_shapes(ctx):
    """Smooth fields (long steepest paths through many tiles, resolved through
    the face graph) batched with noise fields, in both tile shapes."""
    fields = [sf.broad_gaussians_ramp((150, 140, 130), 61, sigma=60.0),
              sf.smoothed_noise((70, 50, 40), 62, sigma=3.0),
              sf.broad_gaussians_ramp((1500, 1100, 1), 63, sigma=300.0)[0],
              sf.broad_gaussians_ramp((90, 200, 30), 64, sigma=40.0).astype(np.float16)]
    res = run_batch(ctx, fields)
    for i, (f, got) in enumerate(zip(fields, res)):
        assert_same_labels(got, oracle.segment(f), f"long-path batch field {i} {f.shape} {f.dtype}")


def _dev_batch(fields):
    devs = [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in fields]
    outs = [[torch.full((f.size,), -5, dtype=torch.int32, device="cuda") for _ in range(3)]
            for f in fields]
    return devs, outs


def _call(ctx, fields, devs, outs):
    ks = ms.ms_segment_batch(ctx, devs, [ms.dims_of(f) for f in fields],
                             [ms.dtype_code(f) for f in fields], [o[0] for o in outs],
                             [o[1] for o in outs], [o[2] for o in outs])
    return [(o[0].cpu().numpy(), o[1].cpu().numpy(), o[2].cpu().numpy(), k) for o, k in zip(outs, ks)]


def test_repeated_batch_replays_a_graph(ctx):
    """The same fields again: the second and third calls replay the captured
    graph (one graph stage per call), with the oracle's results."""
    fields = small_batch(10, 41) + [sf.smoothed_noise((200, 150, 1), 42, sigma=3.0)[0]]
    devs, outs = _dev_batch(fields)
    refs = [oracle.segment(f) for f in fields]
    ms.ms_profile_enable(ctx, True)
    for call in range(3):
        for o in outs:
            for t in o:
                t.fill_(-5)
        torch.cuda.synchronize()
        got = _call(ctx, fields, devs, outs)
        for i, (g, r) in enumerate(zip(got, refs)):
            assert_same_labels(g, r, f"call {call} field {i}")
    prof = ms.ms_profile_read(ctx)
    ms.ms_profile_enable(ctx, False)
    assert prof["calls"] == 3
    assert prof["stages"]["graph"]["launches"] > 0  # calls 2 and 3 replayed


def test_replay_after_contents_change(ctx):
    """Same pointers, new contents with many more regions than the graph was
    sized for: the replay detects it and the call runs step by step."""
    smooth = [sf.broad_gaussians_ramp((64, 48, 40), 50 + i, sigma=30.0) for i in range(4)]
    noisy = [sf.smoothed_noise((64, 48, 40), 60 + i, sigma=1.0) for i in range(4)]
    devs, outs = _dev_batch(smooth)
    for _ in range(2):  # step by step, then a replay
        _call(ctx, smooth, devs, outs)
    for d, f in zip(devs, noisy):
        d.copy_(torch.from_numpy(f))
    torch.cuda.synchronize()
    for call in range(2):
        got = _call(ctx, noisy, devs, outs)
        for i, (f, g) in enumerate(zip(noisy, got)):
            assert_same_labels(g, oracle.segment(f), f"changed contents call {call} field {i}")
    for d, f in zip(devs, smooth):  # and back
        d.copy_(torch.from_numpy(f))
    torch.cuda.synchronize()
    got = _call(ctx, smooth, devs, outs)
    for i, (f, g) in enumerate(zip(smooth, got)):
        assert_same_labels(g, oracle.segment(f), f"restored contents field {i}")


def test_graphs_off_and_autotune(ctx):
    fields = small_batch(8, 71)
    devs, outs = _dev_batch(fields)
    refs = [oracle.segment(f) for f in fields]
    ms.ms_batch_graphs(ctx, False)
    try:
        for _ in range(2):
            for i, (g, r) in enumerate(zip(_call(ctx, fields, devs, outs), refs)):
                assert_same_labels(g, r, f"graphs off field {i}")
    finally:
        ms.ms_batch_graphs(ctx, True)
    t = ms.ms_batch_autotune(ctx, devs, [ms.dims_of(f) for f in fields],
                             [ms.dtype_code(f) for f in fields], [o[0] for o in outs],
                             [o[1] for o in outs], [o[2] for o in outs])
    assert t["tile_ctas"] in (1, 2) and t["write_ctas"] in (2, 4, 8) and t["dynamic"] in (0, 1)
    assert t["chase_blocks"] in (2, 3) and t["pair_blocks"] in (4, 8) and t["resolve_mode"] in (-1, 0, 1)
    assert t["shape3"] in ms.TILE_SHAPES
    assert 0 < t["best_ms"] <= t["default_ms"]
    for call in range(3):  # tuned, then captured and replayed with the tuning
        for i, (g, r) in enumerate(zip(_call(ctx, fields, devs, outs), refs)):
            assert_same_labels(g, r, f"tuned call {call} field {i}")


def test_replay_reports_nan(ctx):
    fields = small_batch(4, 81)
    devs, outs = _dev_batch(fields)
    for _ in range(2):
        _call(ctx, fields, devs, outs)
    flat = devs[1].view(-1)
    flat[flat.numel() // 3] = float("nan")
    torch.cuda.synchronize()
    with pytest.raises(ms.MSError) as e:
        _call(ctx, fields, devs, outs)
    assert e.value.name == "MS_ERR_NAN_INPUT"
