"""Z-slab partition of one grid (paper_2105_04419_gb300.slabs), on CPU: the oracle's field of every
rank's extended slab, cut to the owned planes and stacked, equals the oracle's field of the whole
grid (Eq. 1 with the truncation: a voxel's value depends only on obstacles closer than dmax); the
halo exchange over gloo ranks delivers exactly the neighbours' planes."""
import os
import socket
import sys

import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_2105_04419_gb300 import slabs as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def scene(seed, shape):
    occ = W.bernoulli_grid(seed, shape, 0.004)
    occ[shape[0] // 2, :, 3] = 1  # a wall line crossing every slab boundary's neighbourhood
    return occ


@pytest.mark.parametrize("nz,world,dmax", [(70, 1, 9), (70, 2, 9), (70, 4, 9), (64, 2, 16), (131, 3, 24), (72, 9, 5)])
def test_bounds_cover_and_align(nz, world, dmax):
    b = S.slab_bounds(nz, world, dmax)
    assert len(b) == world and b[0][0] == 0 and b[-1][1] == nz
    for (a0, a1), (c0, c1) in zip(b, b[1:]):
        assert a1 == c0 and a0 % 8 == 0 and c0 % 8 == 0 and a1 > a0
    assert S.halo_planes(dmax) >= dmax - 1
    if world > 1:
        assert min(z1 - z0 for z0, z1 in b) >= S.halo_planes(dmax)


def test_bounds_reject_thin_slabs():
    assert len(S.slab_bounds(64, 4, 16)) == 4  # 16-plane slabs carry the 16-plane halo of dmax 16
    with pytest.raises(ValueError):
        S.slab_bounds(64, 5, 16)  # some slabs of 8 planes
    with pytest.raises(ValueError):
        S.slab_bounds(16, 3, 4)  # more ranks than brick layers


@pytest.mark.parametrize("shape,world,dmax", [((70, 33, 41), 2, 9), ((70, 33, 41), 4, 9), ((131, 20, 27), 3, 24),
                                              ((72, 17, 19), 9, 5), ((64, 30, 30), 2, 16)])
def test_slabs_equal_whole(shape, world, dmax):
    occ = scene(world * 100 + dmax, shape)
    whole = O.edt_factorised(occ, dmax)
    b = S.slab_bounds(shape[0], world, dmax)
    parts = []
    for r in range(world):
        h0, h1 = S.extended_range(b, r, dmax)
        parts.append(S.owned_part(O.edt_factorised(np.ascontiguousarray(occ[h0:h1]), dmax), b, r, dmax))
    assert np.array_equal(np.concatenate(parts, 0), whole)


def test_halo_is_needed():
    """An obstacle dmax - 1 planes past a slab's end lowers the slab's last plane below dmax^2; a
    halo one plane shorter would miss it."""
    shape, dmax = (48, 9, 9), 9
    b = S.slab_bounds(shape[0], 2, dmax)
    assert b[0] == (0, 24)
    occ = np.zeros(shape, np.uint8)
    occ[23 + dmax - 1, 4, 4] = 1
    h0, h1 = S.extended_range(b, 0, dmax)
    assert h1 == 23 + dmax
    assert O.edt_factorised(occ, dmax)[23, 4, 4] == (dmax - 1) ** 2
    short = O.edt_factorised(np.ascontiguousarray(occ[h0:h1 - 1]), dmax)
    assert short[23 - h0, 4, 4] == dmax * dmax
    full = O.edt_factorised(np.ascontiguousarray(occ[h0:h1]), dmax)
    assert full[23 - h0, 4, 4] == (dmax - 1) ** 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, shape, dmax, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import oracle as O_
    from paper_2105_04419_gb300 import slabs as S_
    from test_slabs import scene as scene_
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        occ = scene_(world * 100 + dmax, shape)  # every rank derives the grid from the seed, keeps its planes
        b = S_.slab_bounds(shape[0], world, dmax)
        z0, z1 = b[rank]
        ext = S_.exchange_halos(torch.from_numpy(np.ascontiguousarray(occ[z0:z1])), rank, world, b, dmax)
        h0, h1 = S_.extended_range(b, rank, dmax)
        exact = bool(np.array_equal(ext.numpy(), occ[h0:h1]))
        part = S_.owned_part(O_.edt_factorised(np.ascontiguousarray(ext.numpy()), dmax), b, rank, dmax)
        q.put((rank, exact, part))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,shape,dmax", [(2, (70, 21, 23), 9), (3, (131, 14, 17), 24)])
def test_exchange_halos_gloo(world, shape, dmax):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, shape, dmax, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted((q.get(timeout=180) for _ in range(world)), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert all(exact for _, exact, _ in got)
    occ = scene(world * 100 + dmax, shape)
    assert np.array_equal(np.concatenate([part for _, _, part in got], 0), O.edt_factorised(occ, dmax))


def test_band_ranges_match_neighbour_halos():
    for nz, world, dmax in ((256, 4, 32), (131, 3, 24), (72, 9, 5)):
        b = S.slab_bounds(nz, world, dmax)
        for r in range(world):
            for peer, (z_lo, z_hi) in S.band_ranges(b, r, dmax).items():
                h0, h1 = S.extended_range(b, peer, dmax)
                z0, z1 = b[r]
                # exactly the planes of this rank's own range that lie in the peer's extended slab
                assert (z_lo, z_hi) == (max(z0, h0), min(z1, h1))


def _exchange_main(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    from paper_2105_04419_gb300 import slabs as S_
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        def payload(src, dst):  # deterministic, of a size that may be 0
            n = (7 * src + 3 * dst) % 5 * 1000
            return torch.arange(n, dtype=torch.int64) * (src + 1) + dst
        send = {p: payload(rank, p) for p in (rank - 1, rank + 1) if 0 <= p < world}
        got = S_.exchange_records(send, rank, world)
        ok = all(torch.equal(got[p], payload(p, rank)) for p in got) and set(got) == set(send)
        q.put((rank, ok))
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3, 4])
def test_exchange_records_gloo(world):
    """Variable-length record exchange between neighbours (some payloads empty) over gloo ranks."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_exchange_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = sorted(q.get(timeout=180) for _ in range(world))
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert all(ok for _, ok in got)


def test_sparse_protocol_oracle_emulation():
    """The sparse slab protocol's arithmetic on CPU with the oracle: each rank holds its own obstacles
    plus the neighbours' band obstacles (as the record exchange delivers them) in its extended slab;
    after edits, each rank replays the neighbours' changed band voxels.  The owned parts, stacked,
    equal the oracle on the whole grid, before and after the edits."""
    rs = np.random.default_rng(5)
    nz, ny, nx, world, dmax = 96, 20, 24, 3, 12
    b = S.slab_bounds(nz, world, dmax)
    occ = scene(77, (nz, ny, nx))
    for frame in range(3):
        if frame:
            k = 400
            pts = np.stack([rs.integers(0, nz, k), rs.integers(0, ny, k), rs.integers(0, nx, k)], 1)
            occ[pts[:, 0], pts[:, 1], pts[:, 2]] = rs.integers(0, 2, k)
        parts = []
        for r in range(world):
            h0, h1 = S.extended_range(b, r, dmax)
            ext = np.zeros((h1 - h0, ny, nx), np.uint8)
            z0, z1 = b[r]
            ext[z0 - h0: z1 - h0] = occ[z0:z1]  # own planes
            for peer in (r - 1, r + 1):
                if 0 <= peer < world:
                    lo, hi = S.band_ranges(b, peer, dmax)[r]  # what the peer sends to r
                    ext[lo - h0: hi - h0] = occ[lo:hi]
            parts.append(S.owned_part(O.edt_factorised(ext, dmax), b, r, dmax))
        assert np.array_equal(np.concatenate(parts, 0), O.edt_factorised(occ, dmax)), frame


def test_untruncated_grid_has_no_slabs():
    """Without a truncation every obstacle can be a voxel's nearest: no finite halo, so the slab
    split is refused with a clear error."""
    import paper_2105_04419_gb300.slabs as S
    with pytest.raises(ValueError):
        S.slab_bounds(256, 2, None)
    with pytest.raises(ValueError):
        S.halo_planes(0)
    assert S.halo_planes(32) == 32 and S.halo_planes(2) == 8 and S.halo_planes(1) == 0
