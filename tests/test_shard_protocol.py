"""The z-slab exchange protocol (paper_2303_15491_gb300.shard) on CPU ranks:
world-size 2 and 3 gloo process groups run ``segment_sharded`` -- the
phases, the published planes, the variable-size all-gathers -- with the slab
steps written out here on the host (the oracle's steepest step on the slab
and its halo, pointer doubling, exits followed through the gathered rows),
and the slabs' labels together must equal the oracle's segmentation of the
whole field, vertex for vertex."""
import os
import socket

import numpy as np
import pytest

import oracle
import synthfields as sf

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_2303_15491_gb300 import shard  # noqa: E402


class HostSlabOps:
    """The slab steps on the host, from their definitions."""

    def local(self, field_ext, dims, dtype, z0, z1):
        nx, ny, nz = dims
        nxy = nx * ny
        f = np.asarray(field_ext)
        lo = 1 if z0 > 0 else 0
        owned = z1 - z0
        up, dn = oracle.steepest(f)
        up, dn = up.astype(np.int64), dn.astype(np.int64)
        halo = np.r_[np.arange(lo * nxy), np.arange((lo + owned) * nxy, f.size)].astype(np.int64)
        up[halo] = halo
        dn[halo] = halo
        for p in (up, dn):
            while True:
                q = p[p]
                if np.array_equal(q, p):
                    break
                p[:] = q
        base = (z0 - lo) * nxy
        sl = slice(lo * nxy, (lo + owned) * nxy)

        def encode(r):
            g = r + base
            out = np.where((r < lo * nxy) | (r >= (lo + owned) * nxy), -g - 1, g)
            return torch.from_numpy(out.astype(np.int32))

        return encode(dn[sl]), encode(up[sl])

    def resolve(self, dims, rows, plane_z, asc, desc):
        nxy = dims[0] * dims[1]
        r = rows.numpy()
        slot = {z: i for i, z in enumerate(plane_z)}

        def follow(code, kind):
            h = -int(code) - 1
            return r[slot[h // nxy], kind, h % nxy]

        for _ in range(r.size + 1):
            neg = np.argwhere(r < 0)
            if neg.size == 0:
                break
            for p, kind, xy in neg:
                r[p, kind, xy] = follow(r[p, kind, xy], kind)
        for kind, lab in ((0, asc.numpy()), (1, desc.numpy())):
            for i in np.flatnonzero(lab < 0):
                lab[i] = follow(lab[i], kind)
            assert (lab >= 0).all()

    def pairs(self, asc, desc, n_labels):
        key = (asc.numpy().astype(np.int64) << 32) | desc.numpy().astype(np.int64)
        return torch.from_numpy(np.unique(key))

    def rank(self, asc, desc, n_labels, keys):
        u = np.unique(keys.numpy())
        key = (asc.numpy().astype(np.int64) << 32) | desc.numpy().astype(np.int64)
        return torch.from_numpy(np.searchsorted(u, key).astype(np.int32)), int(u.size)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def make_field(kind, dims):
    if kind == "noise":
        return sf.smoothed_noise(dims, 4, sigma=2.0)
    if kind == "ties":
        return sf.quantize_levels(sf.smoothed_noise(dims, 5, sigma=2.0), 6)
    if kind == "ramp":  # lines run the whole depth of the field, through every slab
        f = sf.ramp(dims)
        return (f + np.random.default_rng(1).uniform(0, 0.5, f.shape)).astype(np.float32)
    raise ValueError(kind)


def _rank_main(rank, world, port, kind, dims, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        f = make_field(kind, dims)
        nz = dims[2]
        z0, z1 = shard.slab_bounds(nz, world, rank)
        h0, h1 = shard.halo_bounds(nz, z0, z1)
        asc, desc, m, k = shard.segment_sharded(HostSlabOps(), f[h0:h1], dims, 0, z0, z1)
        out[rank] = (asc.numpy().copy(), desc.numpy().copy(), m.numpy().copy(), k)
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,kind,dims", [(2, "noise", (14, 12, 17)), (2, "ties", (9, 11, 10)),
                                             (3, "ramp", (7, 6, 13))])
def test_gloo_ranks_match_the_whole_field(world, kind, dims):
    port = _free_port()
    ctx = mp.get_context("spawn")
    manager = ctx.Manager()
    out = manager.dict()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, kind, dims, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(240)
        assert p.exitcode == 0
    ref = oracle.segment(make_field(kind, dims))
    got = [out[r] for r in range(world)]
    assert all(g[3] == ref["K"] for g in got)
    for i, name in enumerate(("asc", "desc", "ms")):
        assert np.array_equal(np.concatenate([g[i] for g in got]), ref[name]), name


def test_slab_bounds_and_halos():
    assert [shard.slab_bounds(10, 3, r) for r in range(3)] == [(0, 3), (3, 6), (6, 10)]
    assert shard.halo_bounds(10, 0, 3) == (0, 4)
    assert shard.halo_bounds(10, 3, 6) == (2, 7)
    assert shard.halo_bounds(10, 6, 10) == (5, 10)
    assert shard.halo_bounds(4, 0, 4) == (0, 4)
    with pytest.raises(ValueError):
        shard.slab_bounds(2, 3, 0)


def test_published_planes():
    def planes(nz, z0, z1):
        return shard.SlabJob(None, None, (4, 4, nz), 0, z0, z1).published_planes()

    assert planes(10, 0, 3) == [2]
    assert planes(10, 3, 6) == [3, 5]
    assert planes(10, 6, 10) == [6]
    assert planes(10, 4, 5) == [4]  # one plane: published once
    assert planes(10, 0, 10) == []


def test_one_process_runs_the_phases_by_hand():
    """The phases driven slab by slab in one process (no process group), as
    a single-GPU driver holding several slabs does."""
    dims = (10, 9, 15)
    f = make_field("ramp", dims)
    jobs = []
    for r in range(4):
        z0, z1 = shard.slab_bounds(dims[2], 4, r)
        h0, h1 = shard.halo_bounds(dims[2], z0, z1)
        jobs.append(shard.SlabJob(HostSlabOps(), f[h0:h1], dims, 0, z0, z1))
    pub = [j.publish() for j in jobs]
    rows = torch.cat([p[0] for p in pub])
    zs = torch.cat([p[1] for p in pub])
    keys = torch.cat([j.resolve(rows.clone(), zs) for j in jobs])
    outs = [j.finish(keys) for j in jobs]
    ref = oracle.segment(f)
    for i, name in enumerate(("asc", "desc", "ms")):
        assert np.array_equal(np.concatenate([o[i].numpy() for o in outs]), ref[name]), name
    assert all(o[3] == ref["K"] for o in outs)
