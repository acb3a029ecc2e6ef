"""Shared helpers of the GPU tests: run the library through its C ABI on
torch device memory, and compare against the CPU oracle."""
import numpy as np

import paper_2303_15491_gb300 as ms


def to_dev(field_np):
    import torch

    return torch.from_numpy(np.ascontiguousarray(field_np)).cuda()


def gpu_segment(ctx, field_np):
    """asc, desc, ms (numpy int32) and K from ms_segment on the device."""
    f = to_dev(field_np)
    asc, desc, m, k = ms.segment(ctx, f)
    return asc.cpu().numpy(), desc.cpu().numpy(), m.cpu().numpy(), k


def assert_same_labels(got, ref, what=""):
    asc, desc, m, k = got
    assert k == ref["K"], f"{what}: K {k} != {ref['K']}"
    for name, a in (("asc", asc), ("desc", desc), ("ms", m)):
        b = ref[name]
        if not np.array_equal(a, b):
            bad = np.flatnonzero(a != b)
            raise AssertionError(f"{what}: {name} differs at {bad.size} vertices, first {bad[:8]} "
                                 f"got {a[bad[:8]]} want {b[bad[:8]]}")
