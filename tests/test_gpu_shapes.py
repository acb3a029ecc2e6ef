"""Every 3D tile shape (ms_tuning.shape3: 32x16x16, 64x8x16, 16x32x16 and
the small-field 16x16x16) forced on a context and checked against the
oracle, label for label: single fields whose extents are and are not
multiples of the tile, ties, fp16, many distinct pairs, long paths through
many tiles (the face graph), batches mixing 3D and 2D fields, and the
captured graph's replays."""
import numpy as np
import pytest

import oracle
import paper_2303_15491_gb300 as ms
import synthfields as sf
from gpu_util import assert_same_labels

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

SHAPES = sorted(ms.TILE_SHAPES)


@pytest.fixture(scope="module", params=SHAPES, ids=lambda s: "x".join(map(str, ms.TILE_SHAPES[s])))
def shaped(request):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    h = ms.ms_create(0)
    ms.ms_set_tuning(h, shape3=request.param)
    assert ms.ms_get_tuning(h)["shape3"] == request.param
    yield h
    ms.ms_destroy(h)


def run(ctx, fields, calls=1):
    devs = [torch.from_numpy(np.ascontiguousarray(f)).cuda() for f in fields]
    outs = [[torch.full((f.size,), -7, dtype=torch.int32, device="cuda") for _ in range(3)]
            for f in fields]
    res = None
    for _ in range(calls):
        ks = ms.ms_segment_batch(ctx, devs, [ms.dims_of(f) for f in fields],
                                 [ms.dtype_code(f) for f in fields], [o[0] for o in outs],
                                 [o[1] for o in outs], [o[2] for o in outs])
        res = [(o[0].cpu().numpy(), o[1].cpu().numpy(), o[2].cpu().numpy(), k)
               for o, k in zip(outs, ks)]
    return res


SINGLE = {
    "exact": lambda: sf.smoothed_noise((64, 32, 32), 1, sigma=2.0),
    "ragged": lambda: sf.smoothed_noise((70, 37, 41), 2, sigma=2.0),
    "thin": lambda: sf.smoothed_noise((200, 9, 10), 3, sigma=1.5),
    "ties": lambda: sf.quantize_levels(sf.smoothed_noise((48, 40, 36), 4, sigma=2.5), 8),
    "fp16": lambda: sf.smoothed_noise((40, 44, 24), 5, sigma=2.0).astype(np.float16),
    "white": lambda: np.random.default_rng(6).standard_normal((33, 70, 65)).astype(np.float32),
    "long_paths": lambda: sf.broad_gaussians_ramp((130, 120, 110), 7, sigma=50.0),
}


@pytest.mark.parametrize("kind", sorted(SINGLE))
def test_single_fields(shaped, kind):
    f = SINGLE[kind]()
    got = run(shaped, [f], calls=3)[0]  # step by step, captured, replayed
    assert_same_labels(got, oracle.segment(f), f"{kind} {f.shape}")


def test_segment_call_takes_the_shape(shaped):
    f = sf.smoothed_noise((90, 50, 30), 8, sigma=2.0)
    dev = torch.from_numpy(f).cuda()
    for _ in range(3):
        asc, desc, m, k = ms.segment(shaped, dev)
    assert_same_labels((asc.cpu().numpy(), desc.cpu().numpy(), m.cpu().numpy(), k),
                       oracle.segment(f), "ms_segment")


def test_mixed_batch(shaped):
    fields = [sf.batch_field(s) for s in sf.batch_specs(10, seed=9, lo=16, hi=90)]
    fields += [sf.smoothed_noise((300, 200, 1), 10, sigma=3.0)[0],
               sf.broad_gaussians_ramp((60, 50, 40), 11, sigma=25.0)]
    for i, (f, got) in enumerate(zip(fields, run(shaped, fields, calls=2))):
        assert_same_labels(got, oracle.segment(f), f"batch field {i} {f.shape} {f.dtype}")


def test_tuning_choices_are_checked():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    h = ms.ms_create(0)
    try:
        for bad in ({"shape3": 4}, {"shape3": -1}, {"tile_ctas": 0}, {"resolve_mode": 2}):
            with pytest.raises(ms.MSError, match="INVALID_ARG"):
                ms.ms_set_tuning(h, **bad)
        assert ms.ms_get_tuning(h)["shape3"] == 0
    finally:
        ms.ms_destroy(h)
