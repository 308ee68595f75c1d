"""Z-slab partition of one grid over ranks (one GPU each).

The truncated field at a voxel depends only on obstacles closer than dmax (Eq. 1 with the
truncation), so a voxel's value needs the occupancy of at most dmax - 1 planes above and below it.
Rank r owns a brick-aligned range of z-planes [z0, z1); it receives once, from its two neighbours,
the occupancy of H = 8R planes beyond each end (R = floor((dmax + 6) / 8), so H >= dmax - 1),
transforms its extended slab with the single-GPU library and keeps the owned planes.  After that
one exchange no rank needs anything from another: there is no exchange of distances.

Only a neighbour's own planes are exchanged, so every owned slab must be at least H planes thick
(slab_bounds checks this).
"""
from __future__ import annotations


def halo_planes(dmax: int) -> int:
    """Planes of occupancy needed beyond each end of a slab: 8R, R = floor((dmax + 6) / 8)."""
    return 8 * ((dmax + 6) // 8)


def slab_bounds(nz: int, world: int, dmax: int) -> list:
    """Owned z ranges [(z0, z1), ...] for ranks 0 .. world - 1: contiguous, starting on brick
    boundaries, the bricks split as evenly as possible (lower ranks take the extra ones)."""
    if world < 1 or nz < 1:
        raise ValueError("need world >= 1 and nz >= 1")
    nbz = (nz + 7) // 8
    if world > nbz:
        raise ValueError(f"{world} slabs but only {nbz} brick layers")
    base, extra = divmod(nbz, world)
    bounds, b = [], 0
    for r in range(world):
        nb = base + (1 if r < extra else 0)
        bounds.append((8 * b, min(nz, 8 * (b + nb))))
        b += nb
    h = halo_planes(dmax)
    if world > 1 and min(z1 - z0 for z0, z1 in bounds) < h:
        raise ValueError(f"slabs of {min(z1 - z0 for z0, z1 in bounds)} planes are thinner than the "
                         f"{h}-plane halo of dmax {dmax}: use fewer ranks")
    return bounds


def extended_range(bounds: list, rank: int, dmax: int) -> tuple:
    """The planes [h0, h1) a rank transforms: its own plus up to H on each side."""
    h = halo_planes(dmax)
    z0, z1 = bounds[rank]
    return max(bounds[0][0], z0 - h), min(bounds[-1][1], z1 + h)


def exchange_halos(owned, rank: int, world: int, bounds: list, dmax: int, group=None):
    """Extended occupancy slab of this rank from its owned planes `owned` ([z1 - z0, ny, nx] uint8,
    on the device the process group communicates from): the lower neighbour's top planes, the
    owned planes, the upper neighbour's bottom planes.  Point-to-point sends, one per neighbour."""
    import torch
    import torch.distributed as dist
    z0, z1 = bounds[rank]
    h0, h1 = extended_range(bounds, rank, dmax)
    if owned.shape[0] != z1 - z0:
        raise ValueError(f"rank {rank} owns {z1 - z0} planes, got {owned.shape[0]}")
    owned = owned.contiguous()
    ny, nx = owned.shape[1], owned.shape[2]
    below = torch.empty((z0 - h0, ny, nx), dtype=owned.dtype, device=owned.device)
    above = torch.empty((h1 - z1, ny, nx), dtype=owned.dtype, device=owned.device)
    ops = []
    if rank > 0:
        lo_h0, lo_h1 = extended_range(bounds, rank - 1, dmax)
        ops.append(dist.P2POp(dist.isend, owned[: lo_h1 - z0].contiguous(), rank - 1, group))
        ops.append(dist.P2POp(dist.irecv, below, rank - 1, group))
    if rank < world - 1:
        up_h0, _ = extended_range(bounds, rank + 1, dmax)
        ops.append(dist.P2POp(dist.isend, owned[up_h0 - z0:].contiguous(), rank + 1, group))
        ops.append(dist.P2POp(dist.irecv, above, rank + 1, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    return torch.cat([below, owned, above], 0)


def owned_part(field_ext, bounds: list, rank: int, dmax: int):
    """The owned planes of a field computed on the extended slab."""
    z0, z1 = bounds[rank]
    h0, _ = extended_range(bounds, rank, dmax)
    return field_ext[z0 - h0: z1 - h0]


def sharded_global(owned, rank: int, world: int, nz: int, dmax: int, group=None, stream=None):
    """One rank's share of the global transform of a grid split into z-slabs: exchange the halos,
    transform the extended slab on this rank's GPU, return the owned planes of D
    ([z1 - z0, ny, nx] int32 CUDA tensor).  `owned` is this rank's occupancy planes on its GPU."""
    from .lib import Map
    bounds = slab_bounds(nz, world, dmax)
    ext = exchange_halos(owned, rank, world, bounds, dmax, group)
    m = Map(ext.shape[2], ext.shape[1], ext.shape[0], dmax, device=ext.device.index or 0, stream=stream)
    try:
        m.set_occupancy_dense(ext)
        m.global_()
        return owned_part(m.export_dense(on_device=True), bounds, rank, dmax).clone()
    finally:
        m.close()
