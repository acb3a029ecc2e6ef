"""The CPU-parallel baseline (the paper's per-thread active-list scheme with
OpenMP, ``cpu_parallel``): labels and region counts equal to the oracle's on
fields with and without ties, 2D and 3D, degenerate shapes, and any thread
count -- the order in which threads compress paths changes the iterations,
not the result (Sec. 4.2.1)."""
import numpy as np
import pytest

import cpu_parallel
import oracle
import synthfields as sf


def same(got, ref, what):
    assert got["K"] == ref["K"], f"{what}: K {got['K']} != {ref['K']}"
    for k in ("asc", "desc", "ms"):
        assert np.array_equal(got[k], ref[k]), f"{what}: {k} differs"


@pytest.mark.parametrize("dims", [(40, 36, 30), (33, 17, 9), (100, 80, 1), (2, 2, 2), (1, 1, 1),
                                  (7, 1, 1), (1, 5, 5), (257, 3, 1)])
@pytest.mark.parametrize("threads", [1, 3, 8])
def test_matches_oracle(dims, threads):
    f = sf.smoothed_noise(dims, 5, sigma=2.0)
    if dims[2] == 1:
        f = f[0]
    same(cpu_parallel.segment(f, threads), oracle.segment(f), f"{dims} x{threads}")


@pytest.mark.parametrize("threads", [2, 16])
def test_ties_and_signed_zero(threads):
    g = np.random.default_rng(3)
    f = g.integers(-2, 3, size=(12, 20, 24)).astype(np.float32)
    f[f == 0] = np.where(g.random(int((f == 0).sum())) < 0.5, -0.0, 0.0).astype(np.float32)
    same(cpu_parallel.segment(f, threads), oracle.segment(f), "ties")
    const = np.zeros((5, 6, 7), np.float32)
    same(cpu_parallel.segment(const, threads), oracle.segment(const), "constant")


def test_more_threads_than_vertices():
    f = np.arange(6, dtype=np.float32).reshape(1, 2, 3)
    same(cpu_parallel.segment(f, 32), oracle.segment(f), "tiny")


def test_nan_is_rejected():
    f = sf.smoothed_noise((8, 8, 8), 1, sigma=1.0)
    f[3, 4, 5] = np.nan
    with pytest.raises(RuntimeError):
        cpu_parallel.segment(f, 4)
