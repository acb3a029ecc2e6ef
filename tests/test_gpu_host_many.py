"""The pipelined host path (ms_segment_host_many): fields of mixed sizes and
dtypes, copied in from and out to pinned host memory while their neighbours
are segmented -- every field's labels and region count equal the oracle's,
and a repeated call (two captured plans, one a buffer set) gives the same."""
import numpy as np
import pytest

import oracle
import paper_2303_15491_gb300 as ms
import synthfields as sf
from gpu_util import assert_same_labels

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _fields():
    out = [sf.smoothed_noise((40, 36, 33), 5, sigma=2.5),
           np.ascontiguousarray(sf.smoothed_noise((300, 170, 1), 6, sigma=3.0)[0]),
           sf.quantize_levels(sf.smoothed_noise((48, 40, 24), 7, sigma=3.0), 16).astype(np.float16),
           sf.gaussian_sum((33, 47, 29), 8),
           sf.smoothed_noise((40, 36, 33), 9, sigma=2.5)]
    return [np.ascontiguousarray(f) for f in out]


def test_host_many_matches_oracle_twice():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    fields = _fields()
    refs = [oracle.segment(f) for f in fields]
    hf = [torch.from_numpy(f).pin_memory() for f in fields]
    outs = [[torch.full((f.size,), -5, dtype=torch.int32).pin_memory() for _ in range(3)] for f in fields]
    ctx = ms.ms_create(0)
    try:
        for call in range(3):  # step by step, captured, replayed
            ks = ms.ms_segment_host_many(ctx, hf, [ms.dims_of(f) for f in fields],
                                         [ms.dtype_code(f) for f in fields], [o[0] for o in outs],
                                         [o[1] for o in outs], [o[2] for o in outs])
            for i, (f, o, r, k) in enumerate(zip(fields, outs, refs, ks)):
                got = tuple(x.numpy() for x in o) + (k,)
                assert_same_labels(got, r, f"call {call} field {i} {f.shape} {f.dtype}")
                for x in o:
                    x.fill_(-5)
    finally:
        ms.ms_destroy(ctx)


def test_host_many_same_field_repeated():
    """One host field segmented many times in a row (the end-to-end bench's
    pattern): the two buffer sets alternate; every result is the oracle's."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    f = sf.smoothed_noise((64, 64, 48), 11, sigma=3.0)
    ref = oracle.segment(f)
    h = torch.from_numpy(f).pin_memory()
    n = 5
    outs = [[torch.empty(f.size, dtype=torch.int32).pin_memory() for _ in range(3)] for _ in range(n)]
    ctx = ms.ms_create(0)
    try:
        ks = ms.ms_segment_host_many(ctx, [h] * n, [ms.dims_of(f)] * n, [0] * n, [o[0] for o in outs],
                                     [o[1] for o in outs], [o[2] for o in outs])
    finally:
        ms.ms_destroy(ctx)
    for o, k in zip(outs, ks):
        assert_same_labels(tuple(x.numpy() for x in o) + (k,), ref, "repeated field")
