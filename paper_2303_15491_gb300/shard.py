"""One field segmented by several processes, each holding one z-slab -- the
distributed computation the paper leaves to future work (Sec. 8) -- on top
of the library's slab calls (``ms_slab_local``, ``ms_slab_resolve``,
``ms_slab_pairs``, ``ms_slab_rank``).

A slab owns planes [z0, z1) and holds one halo plane on each side that
exists.  Three phases, with one all-gather between consecutive ones:

1. ``publish``: steepest steps and pointer jumping inside the slab; a line
   that leaves the slab keeps an exit code.  The slab publishes the labels of
   its first and last owned planes -- the only planes through which another
   slab's lines enter it.
2. ``resolve``: with every slab's rows, each exit is followed to the
   extremum its line reaches; the slab then lists its distinct (asc, desc)
   pairs.
3. ``finish``: with every slab's pairs, each vertex's MS id is the rank of
   its pair among all of them.

The slab outputs equal the whole-field segmentation's, vertex for vertex.
Gathered data lands in the receiving process's own memory before any call
reads it.  ``segment_sharded`` runs the phases over a ``torch.distributed``
group (NCCL for device tensors); a driver holding several slabs in one
process can call the phases of each slab itself.
"""
from __future__ import annotations

from . import ms_slab_local, ms_slab_pairs, ms_slab_rank, ms_slab_resolve, MSError

__all__ = ["slab_bounds", "halo_bounds", "CudaSlabOps", "SlabJob", "all_gather_cat",
           "segment_sharded"]


def slab_bounds(nz: int, world: int, rank: int):
    """Owned planes [z0, z1) of ``rank`` when nz planes are split as evenly
    as they go over ``world`` slabs."""
    if not 0 <= rank < world or world > nz:
        raise ValueError(f"cannot give slab {rank} of {world} planes out of {nz}")
    return rank * nz // world, (rank + 1) * nz // world


def halo_bounds(nz: int, z0: int, z1: int):
    """Planes [h0, h1) a slab must hold: its own and one halo plane per side
    that exists."""
    return z0 - (1 if z0 > 0 else 0), z1 + (1 if z1 < nz else 0)


class CudaSlabOps:
    """The slab steps on this process's GPU, through the C ABI."""

    def __init__(self, ctx):
        self.ctx = ctx

    def local(self, field_ext, dims, dtype, z0, z1):
        import torch
        n_owned = (z1 - z0) * dims[0] * dims[1]
        asc = torch.empty(n_owned, dtype=torch.int32, device=field_ext.device)
        desc = torch.empty_like(asc)
        ms_slab_local(self.ctx, field_ext, dims, dtype, z0, z1, asc, desc)
        return asc, desc

    def resolve(self, dims, rows, plane_z, asc, desc):
        ms_slab_resolve(self.ctx, dims, rows, plane_z, asc, desc, asc.numel())

    def pairs(self, asc, desc, n_labels):
        import torch
        cap = max(1024, asc.numel() // 64)
        for _ in range(2):
            keys = torch.empty(max(cap, 1), dtype=torch.int64, device=asc.device)
            try:
                m = ms_slab_pairs(self.ctx, asc, desc, asc.numel(), n_labels, keys, cap)
            except MSError as e:
                if e.name != "MS_ERR_TOO_LARGE" or e.count <= cap:
                    raise
                cap = e.count
                continue
            return keys[:m]
        raise RuntimeError("ms_slab_pairs: pair count changed between calls")

    def rank(self, asc, desc, n_labels, keys):
        import torch
        ms = torch.empty_like(asc)
        k = ms_slab_rank(self.ctx, asc, desc, asc.numel(), n_labels, keys.contiguous(), keys.numel(),
                         ms)
        return ms, k


class SlabJob:
    """The three phases of one slab.  ``field_ext``: the planes
    ``halo_bounds(nz, z0, z1)`` of the field; ``dims``: the whole field's
    (nx, ny, nz)."""

    def __init__(self, ops, field_ext, dims, dtype, z0, z1):
        self.ops, self.field_ext, self.dims, self.dtype = ops, field_ext, tuple(dims), dtype
        self.z0, self.z1 = int(z0), int(z1)
        self.nxy = self.dims[0] * self.dims[1]
        self.n_labels = self.nxy * self.dims[2]
        self.asc = self.desc = None

    def published_planes(self):
        nz = self.dims[2]
        planes = []
        if self.z0 > 0:
            planes.append(self.z0)
        if self.z1 < nz and self.z1 - 1 not in planes:
            planes.append(self.z1 - 1)
        return planes

    def publish(self):
        """Phase 1: (rows [p, 2, nx ny] int32, their z as int64 [p])."""
        import torch
        self.asc, self.desc = self.ops.local(self.field_ext, self.dims, self.dtype, self.z0, self.z1)
        planes = self.published_planes()
        nxy = self.nxy
        rows = [torch.stack([self.asc[(z - self.z0) * nxy:(z - self.z0 + 1) * nxy],
                             self.desc[(z - self.z0) * nxy:(z - self.z0 + 1) * nxy]]) for z in planes]
        if rows:
            rows = torch.stack(rows)
        else:
            rows = torch.empty((0, 2, nxy), dtype=torch.int32, device=self.asc.device)
        return rows.contiguous(), torch.tensor(planes, dtype=torch.int64, device=self.asc.device)

    def resolve(self, rows_all, plane_z_all):
        """Phase 2: this slab's distinct pairs (int64 keys asc << 32 | desc)."""
        self.ops.resolve(self.dims, rows_all.contiguous(), [int(z) for z in plane_z_all.tolist()],
                         self.asc, self.desc)
        return self.ops.pairs(self.asc, self.desc, self.n_labels)

    def finish(self, keys_all):
        """Phase 3: (asc, desc, ms, K) of the owned vertices."""
        ms, k = self.ops.rank(self.asc, self.desc, self.n_labels, keys_all)
        return self.asc, self.desc, ms, k


def all_gather_cat(t, group=None):
    """Every rank's tensor (first dimensions may differ), concatenated in
    rank order, on every rank."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    n = torch.tensor([t.shape[0]], dtype=torch.int64, device=t.device)
    sizes = [torch.empty_like(n) for _ in range(world)]
    dist.all_gather(sizes, n, group=group)
    sizes = [int(s.item()) for s in sizes]
    top = max(sizes)
    if top == 0:
        return t[:0].clone()
    pad = torch.zeros((top,) + tuple(t.shape[1:]), dtype=t.dtype, device=t.device)
    pad[:t.shape[0]] = t
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad, group=group)
    return torch.cat([p[:s] for p, s in zip(parts, sizes)])


def segment_sharded(ops, field_ext, dims, dtype, z0, z1, group=None, gather=None):
    """(asc, desc, ms, K) of this process's slab; the other ranks of the
    group hold the other slabs and call this at the same time."""
    gather = gather or (lambda t: all_gather_cat(t, group))
    job = SlabJob(ops, field_ext, dims, dtype, z0, z1)
    rows, zs = job.publish()
    keys = job.resolve(gather(rows), gather(zs))
    return job.finish(gather(keys))
