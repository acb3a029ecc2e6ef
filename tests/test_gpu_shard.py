"""The z-slab path on one GPU: a field split into 2-5 slabs, each slab's
phases run through the library's slab calls in one process (the gathers are
concatenations), and the slabs' asc, desc and MS labels together equal the
oracle's segmentation of the whole field, vertex for vertex.  Also the slab
calls' argument checks."""
import numpy as np
import pytest

import oracle
import paper_2303_15491_gb300 as ms
import synthfields as sf
from gpu_util import to_dev
from paper_2303_15491_gb300 import shard

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    h = ms.ms_create(0)
    yield h
    ms.ms_destroy(h)


def run_slabs(ctx, f, n_slabs):
    dims, dt = ms.dims_of(f), ms.dtype_code(f)
    ops = shard.CudaSlabOps(ctx)
    jobs = []
    for r in range(n_slabs):
        z0, z1 = shard.slab_bounds(dims[2], n_slabs, r)
        h0, h1 = shard.halo_bounds(dims[2], z0, z1)
        jobs.append(shard.SlabJob(ops, to_dev(f[h0:h1]), dims, dt, z0, z1))
    pub = [j.publish() for j in jobs]
    rows = torch.cat([p[0] for p in pub])
    zs = torch.cat([p[1] for p in pub])
    keys = torch.cat([j.resolve(rows.clone(), zs) for j in jobs])
    outs = [j.finish(keys) for j in jobs]
    return [np.concatenate([o[i].cpu().numpy() for o in outs]) for i in range(3)], [o[3] for o in outs]


def ramp_noise(dims, amp=0.5):
    f = sf.ramp(dims)
    return (f + np.random.default_rng(2).uniform(0, amp, f.shape)).astype(np.float32)


@pytest.mark.parametrize("n_slabs", [2, 3, 5])
@pytest.mark.parametrize("kind", ["noise", "ties", "white", "ramp"])
def test_slabs_equal_the_whole_field(ctx, kind, n_slabs):
    dims = (48, 40, 37)
    f = {"noise": lambda: sf.smoothed_noise(dims, 3, sigma=3.0),
         "ties": lambda: sf.quantize_levels(sf.smoothed_noise(dims, 4, sigma=3.0), 8),
         "white": lambda: np.random.default_rng(5).standard_normal(dims[::-1]).astype(np.float32),
         "ramp": lambda: ramp_noise(dims)}[kind]()
    (asc, desc, m), ks = run_slabs(ctx, f, n_slabs)
    ref = oracle.segment(f)
    assert all(k == ref["K"] for k in ks)
    for name, got in (("asc", asc), ("desc", desc), ("ms", m)):
        if not np.array_equal(got, ref[name]):
            bad = np.flatnonzero(got != ref[name])
            raise AssertionError(f"{kind}/{n_slabs}: {name} differs at {bad.size}, first {bad[:6]}")


def test_one_plane_slabs_and_fp16(ctx):
    dims = (33, 21, 6)
    f = sf.smoothed_noise(dims, 8, sigma=2.0).astype(np.float16)
    (asc, desc, m), ks = run_slabs(ctx, f, 6)  # every slab one plane deep
    ref = oracle.segment(f)
    assert np.array_equal(asc, ref["asc"]) and np.array_equal(desc, ref["desc"])
    assert np.array_equal(m, ref["ms"]) and ks[0] == ref["K"]


def test_single_slab_is_the_whole_field(ctx):
    f = sf.gaussian_sum((40, 30, 20), 1)
    (asc, desc, m), ks = run_slabs(ctx, f, 1)
    ref = oracle.segment(f)
    assert np.array_equal(asc, ref["asc"]) and np.array_equal(m, ref["ms"]) and ks[0] == ref["K"]


def test_exit_codes_point_into_the_halo(ctx):
    """Before resolution an owned vertex holds an owned extremum or -(h+1)
    with h in a halo plane."""
    dims = (20, 16, 12)
    f = ramp_noise(dims, amp=0.2)
    z0, z1 = 4, 8
    h0, h1 = shard.halo_bounds(dims[2], z0, z1)
    asc, desc = shard.CudaSlabOps(ctx).local(to_dev(f[h0:h1]), dims, 0, z0, z1)
    nxy = dims[0] * dims[1]
    for lab in (asc.cpu().numpy(), desc.cpu().numpy()):
        own = lab[lab >= 0]
        assert ((own >= z0 * nxy) & (own < z1 * nxy)).all()
        h = -lab[lab < 0].astype(np.int64) - 1
        assert h.size > 0 and np.isin(h // nxy, [z0 - 1, z1]).all()


def test_slab_call_errors(ctx):
    dims = (8, 8, 8)
    f = to_dev(sf.smoothed_noise(dims, 1, sigma=1.5))
    a = torch.empty(8 * 8 * 4, dtype=torch.int32, device="cuda")
    d = torch.empty_like(a)
    for z0, z1 in ((4, 4), (-1, 3), (5, 9)):
        with pytest.raises(ms.MSError, match="INVALID_ARG"):
            ms.ms_slab_local(ctx, f, dims, 0, z0, z1, a, d)
    ms.ms_slab_local(ctx, f[0:5], dims, 0, 0, 4, a, d)
    # an exit into a plane that no row covers
    rows = torch.zeros((1, 2, 64), dtype=torch.int32, device="cuda")
    if (a < 0).any():
        with pytest.raises(ms.MSError, match="INVALID_ARG"):
            ms.ms_slab_resolve(ctx, dims, rows, [0], a.clone(), d.clone(), a.numel())
    with pytest.raises(ms.MSError, match="INVALID_ARG"):  # repeated plane
        ms.ms_slab_resolve(ctx, dims, torch.zeros((2, 2, 64), dtype=torch.int32, device="cuda"),
                           [3, 3], a.clone(), d.clone(), a.numel())
    # a cycle in the rows: plane 4 points to plane 3 and back
    rows = torch.empty((2, 2, 64), dtype=torch.int32, device="cuda")
    rows[0] = -(4 * 64 + torch.arange(64, device="cuda", dtype=torch.int32)) - 1
    rows[1] = -(3 * 64 + torch.arange(64, device="cuda", dtype=torch.int32)) - 1
    with pytest.raises(ms.MSError, match="NOT_CONVERGED"):
        ms.ms_slab_resolve(ctx, dims, rows, [3, 4], a.clone(), d.clone(), 0)
    # a pair missing from the keys
    good_a = torch.zeros(4, dtype=torch.int32, device="cuda")
    good_d = torch.full((4,), 7, dtype=torch.int32, device="cuda")
    keys = torch.tensor([(0 << 32) | 6], dtype=torch.int64, device="cuda")
    m = torch.empty(4, dtype=torch.int32, device="cuda")
    with pytest.raises(ms.MSError, match="INVALID_ARG"):
        ms.ms_slab_rank(ctx, good_a, good_d, 4, 512, keys, 1, m)
    keys = torch.tensor([7, 6], dtype=torch.int64, device="cuda")
    assert ms.ms_slab_rank(ctx, good_a, good_d, 4, 512, keys, 2, m) == 2
    assert m.tolist() == [1, 1, 1, 1]
    # labels out of range
    with pytest.raises(ms.MSError, match="INVALID_ARG"):
        ms.ms_slab_rank(ctx, good_a, good_d, 4, 7, keys, 2, m)
    with pytest.raises(ms.MSError) as e:
        ms.ms_slab_pairs(ctx, good_a, good_d, 4, 512, keys, 0)
    assert e.value.count == 1
