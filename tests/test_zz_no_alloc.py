"""ms_pair_rank_noalloc -- the pair-ranking step for callers that cannot
allocate device memory (its working memory is a static array inside the
library) -- must give exactly the dense pair ranks of the oracle, and what
ms_pair_rank gives.  Two calls in a row on different inputs check that the
shared array is cleared between calls.

This file sorts last so that a run stopping at the first failure has already
run every other test; it also passes alone in a fresh process."""
import numpy as np
import pytest

import oracle
import paper_2303_15491_gb300 as ms
import synthfields as sf

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _labels(n, levels, seed):
    g = sf.rng_for(seed)
    a = g.integers(0, levels, n).astype(np.int32)
    d = ((g.integers(0, levels, n).astype(np.int64) * 7919) % n).astype(np.int32)
    return torch.from_numpy(a).cuda(), torch.from_numpy(d).cuda()


def test_noalloc_matches_oracle_two_calls():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = ms.ms_create(0)
    try:
        cases = [(ms.MS_NOALLOC_MAX_N, 5000, 1), (100000, 200, 2)]
        for n, levels, seed in cases:  # two calls in a row on the shared array
            a, d = _labels(n, levels, seed)
            ref = torch.empty(n, dtype=torch.int32, device="cuda")
            k_ref = ms.ms_pair_rank(ctx, a, d, n, ref)
            out = torch.full((n,), -7, dtype=torch.int32, device="cuda")
            k = ms.ms_pair_rank_noalloc(a, d, n, out)
            torch.cuda.synchronize()
            want, k_want = oracle.ms_rank(a.cpu().numpy(), d.cpu().numpy())
            assert k == k_want
            assert np.array_equal(out.cpu().numpy(), want)
            assert k_ref == k_want and torch.equal(out, ref)
    finally:
        ms.ms_destroy(ctx)


def test_noalloc_rejects_oversize_and_bad_labels():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = ms.MS_NOALLOC_MAX_N + 1
    a = torch.zeros(n, dtype=torch.int32, device="cuda")
    with pytest.raises(ms.MSError) as e:
        ms.ms_pair_rank_noalloc(a, a, n, a.clone())
    assert e.value.name == "MS_ERR_TOO_LARGE"
    bad = torch.tensor([0, 9, 1], dtype=torch.int32, device="cuda")
    with pytest.raises(ms.MSError) as e:
        ms.ms_pair_rank_noalloc(bad, bad, 3, torch.empty_like(bad))
    assert e.value.name == "MS_ERR_INVALID_ARG"
