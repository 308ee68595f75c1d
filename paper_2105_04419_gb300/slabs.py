"""Z-slab partition of one grid over ranks (one GPU each).

The truncated field at a voxel depends only on obstacles closer than dmax (Eq. 1 with the
truncation), so a voxel's value needs the occupancy of at most dmax - 1 planes above and below it.
Rank r owns a brick-aligned range of z-planes [z0, z1); it receives once, from its two neighbours,
the occupancy of H = 8R planes beyond each end (R = floor((dmax + 6) / 8), so H >= dmax - 1),
transforms its extended slab with the single-GPU library and keeps the owned planes.  After that
one exchange no rank needs anything from another: there is no exchange of distances.

Only a neighbour's own planes are exchanged, so every owned slab must be at least H planes thick
(slab_bounds checks this).

Two forms of the exchange:
  * dense (exchange_halos, sharded_global): uint8 planes, then a dense transform of the slab;
  * sparse (SlabMap): each rank's map covers its extended slab; only records cross between ranks --
    the occupied voxels of the H planes a neighbour holds as halo (global form: the rank transforms
    its own obstacles, exports that band with vdbedt_export_occupancy, receives its neighbours'
    bands and applies them with an incremental update), or every voxel of the bricks its last update
    changed inside that band (incremental form: own edits -> update -> exchange -> a second, small
    update).  The bytes exchanged follow the obstacles (or the changes) near the slab ends, not the
    slab's volume, and the grid stays sparse on every rank.
"""
from __future__ import annotations


def halo_planes(dmax: int) -> int:
    """Planes of occupancy needed beyond each end of a slab: 8R, R = floor((dmax + 6) / 8).  An
    untruncated grid (dmax None) has no finite halo -- any obstacle can be a voxel's nearest -- so
    it cannot be split into slabs."""
    if dmax is None or isinstance(dmax, float) or int(dmax) < 1:
        raise ValueError("z-slabs need a finite truncation dmax >= 1 (an untruncated grid has no finite halo)")
    return 8 * ((int(dmax) + 6) // 8)


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


def band_ranges(bounds: list, rank: int, dmax: int) -> dict:
    """The planes of this rank's own range that each neighbour holds in its halo: {peer: (z_lo,
    z_hi)} in grid z."""
    h = halo_planes(dmax)
    z0, z1 = bounds[rank]
    out = {}
    if rank > 0:
        out[rank - 1] = (z0, min(z1, z0 + h))
    if rank < len(bounds) - 1:
        out[rank + 1] = (max(z0, z1 - h), z1)
    return out


def exchange_records(send: dict, rank: int, world: int, group=None) -> dict:
    """Variable-length point-to-point exchange with the neighbours: send[peer] is a 1-D int64 tensor
    (packed records) for each neighbour; returns {peer: received tensor}.  Counts go first, then the
    payloads that are not empty.  CPU tensors for gloo, CUDA tensors for NCCL."""
    import torch
    import torch.distributed as dist
    peers = [p for p in (rank - 1, rank + 1) if 0 <= p < world]
    if not peers:
        return {}
    dev = next(iter(send.values())).device if send else torch.device("cpu")
    n_out = {p: torch.tensor([int(send[p].numel())], dtype=torch.int64, device=dev) for p in peers}
    n_in = {p: torch.zeros(1, dtype=torch.int64, device=dev) for p in peers}
    ops = []
    for p in peers:
        ops.append(dist.P2POp(dist.isend, n_out[p], p, group))
        ops.append(dist.P2POp(dist.irecv, n_in[p], p, group))
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    recv = {p: torch.empty(int(n_in[p].item()), dtype=torch.int64, device=dev) for p in peers}
    ops = []
    for p in peers:
        if send[p].numel():
            ops.append(dist.P2POp(dist.isend, send[p].contiguous(), p, group))
        if recv[p].numel():
            ops.append(dist.P2POp(dist.irecv, recv[p], p, group))
    if ops:
        for req in dist.batch_isend_irecv(ops):
            req.wait()
    return recv


class SlabMap:
    """One rank's share of a grid split into z-slabs, kept sparse: a Map of the rank's extended slab
    (its own planes and H planes of halo each side; local z = grid z - h0).  The exchange is split
    into begin_* (returns the records to send to each neighbour) and finish (applies the records
    received), so that ranks can be emulated in one process; global_() / update() do both around a
    torch.distributed exchange.  Records passed in are in local coordinates and must lie in the
    rank's own planes; bytes_sent / bytes_received count the records exchanged."""

    def __init__(self, nx: int, ny: int, nz: int, dmax: int, rank: int, world: int, device: int = 0, stream=None,
                 max_bricks: int = 0, max_nodes: int = 0):
        from .lib import Map
        self.nz, self.dmax, self.rank, self.world = nz, dmax, rank, world
        self.bounds = slab_bounds(nz, world, dmax)
        self.h0, self.h1 = extended_range(self.bounds, rank, dmax)
        self.z0, self.z1 = self.bounds[rank]
        self.map = Map(nx, ny, self.h1 - self.h0, dmax, device=device, stream=stream, max_bricks=max_bricks,
                       max_nodes=max_nodes)
        self.bytes_sent = 0
        self.bytes_received = 0

    def close(self):
        self.map.close()

    def _stage(self, xyz=None, occ=None, packed=None):
        if packed is not None:
            self.map.set_occupancy_packed(packed)
        if xyz is not None and len(xyz):
            self.map.set_occupancy(xyz, occ)

    def _sends(self, changed_only: bool) -> dict:
        out = {}
        for peer, (z_lo, z_hi) in band_ranges(self.bounds, self.rank, self.dmax).items():
            peer_h0, _ = extended_range(self.bounds, peer, self.dmax)
            out[peer] = self.map.export_occupancy(z_lo - self.h0, z_hi - self.h0, dz=self.h0 - peer_h0,
                                                  changed_only=changed_only)
            self.bytes_sent += 8 * out[peer].numel()
        return out

    def begin_global(self, xyz=None, occ=None, packed=None) -> dict:
        """The rank's own occupancy (records in local coordinates) -> its own global transform; returns
        the occupied voxels of each neighbour's halo band, in that neighbour's local coordinates."""
        self.map.reset()
        self._stage(xyz, occ, packed)
        self.map.global_()
        return self._sends(False)

    def begin_update(self, xyz=None, occ=None, packed=None) -> dict:
        """The rank's own edits (local coordinates) -> incremental update; returns every voxel of the
        bricks that update changed inside each neighbour's halo band."""
        self._stage(xyz, occ, packed)
        self.map.update()
        return self._sends(True)

    def finish(self, received: dict):
        """Apply the neighbours' records (halo planes) with an incremental update."""
        for rec in received.values():
            self.bytes_received += 8 * rec.numel()
            if rec.numel():
                self.map.set_occupancy_packed(rec)
        self.map.update()

    def global_(self, xyz=None, occ=None, packed=None, group=None):
        self.finish(exchange_records(self.begin_global(xyz, occ, packed), self.rank, self.world, group))

    def update(self, xyz=None, occ=None, packed=None, group=None):
        self.finish(exchange_records(self.begin_update(xyz, occ, packed), self.rank, self.world, group))

    def owned_field(self):
        """D of the rank's own planes ([z1 - z0, ny, nx] int32 CUDA tensor)."""
        d = self.map.export_dense(on_device=True)
        return d[self.z0 - self.h0: self.z1 - self.h0]
