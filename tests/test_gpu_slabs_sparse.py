"""GPU parity of the sparse z-slab protocol (paper_2105_04419_gb300.slabs.SlabMap) and of the
occupancy export it is built on, against the CPU oracle, bit-exact.

Ranks are emulated in one process on one GPU: each
rank's SlabMap returns the records for its neighbours, which are handed over directly, so the
library side of the protocol -- own transform, band export, staging of the neighbours' records,
the incremental updates -- runs exactly as on separate GPUs.  The owned fields, stacked, equal the
oracle's field of the whole grid after the global transform and after every edit frame.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import coords_of, first_mismatch
from paper_2105_04419_gb300 import slabs as S

pytestmark = pytest.mark.gpu


def run_ranks(maps, begin):
    sends = [begin(r, m) for r, m in enumerate(maps)]
    for r, m in enumerate(maps):
        m.finish({p: sends[p][r] for p in sends[r]})


def stacked(maps):
    return np.concatenate([m.owned_field().cpu().numpy() for m in maps], 0)


@pytest.mark.parametrize("shape,world,dmax", [((96, 40, 48), 2, 12), ((131, 33, 41), 3, 24), ((256, 48, 64), 4, 32)])
def test_sparse_slabs_global_and_frames(shape, world, dmax):
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(world * 10 + dmax)
    nz, ny, nx = shape
    occ = W.bernoulli_grid(world + dmax, shape, 0.002)
    occ[:, ny // 2, 3] = 1  # a wall crossing every slab boundary
    maps = [S.SlabMap(nx, ny, nz, dmax, r, world) for r in range(world)]

    def own_records(r, pts, val):
        z0, z1 = maps[r].z0, maps[r].z1
        sel = (pts[:, 2] >= z0) & (pts[:, 2] < z1)
        loc = pts[sel].copy()
        loc[:, 2] -= maps[r].h0
        return loc.astype(np.int32), val[sel]

    xyz = coords_of(occ)
    ones = np.ones(len(xyz), np.uint8)
    run_ranks(maps, lambda r, m: m.begin_global(*own_records(r, xyz, ones)))
    assert first_mismatch(stacked(maps), O.edt_factorised(occ, dmax)) is None
    for frame in range(3):
        k = 600
        pts = np.stack([rs.integers(0, nx, k), rs.integers(0, ny, k), rs.integers(0, nz, k)], 1).astype(np.int32)
        # edits crowd the slab boundaries, where the halos matter
        for (z0, z1) in maps[0].bounds[1:]:
            pts[: k // 4, 2] = rs.integers(max(0, z0 - dmax), min(nz, z0 + dmax), k // 4)
        val = rs.integers(0, 2, k).astype(np.uint8)
        for (x, y, z), v in zip(pts, val):
            occ[z, y, x] = v
        run_ranks(maps, lambda r, m: m.begin_update(*own_records(r, pts, val)))
        got = stacked(maps)
        assert first_mismatch(got, O.edt_factorised(occ, dmax)) is None, (frame, first_mismatch(got, O.edt_factorised(occ, dmax)))
    assert all(m.bytes_sent > 0 for m in maps)
    for m in maps:
        m.close()


def test_export_occupancy_modes():
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(8)
    occ = W.bernoulli_grid(8, (40, 30, 50), 0.01)
    nz, ny, nx = occ.shape
    m = V.Map(nx, ny, nz, 10)
    xyz = coords_of(occ)
    m.set_occupancy(xyz, np.ones(len(xyz), np.uint8))
    m.global_()

    def unpack(t):
        u = t.cpu().numpy().view(np.uint64)
        return np.stack([u & 0x1FFFFF, (u >> 21) & 0x1FFFFF, (u >> 42) & 0x1FFFFF, u >> 63], 1).astype(np.int64)

    r = unpack(m.export_occupancy(5, 23, dz=100, max_n=10))  # too small a buffer: grown and retried
    want = {(x, y, z + 100) for z, y, x in np.argwhere(occ[5:23]) + [5, 0, 0]}
    assert {tuple(v[:3]) for v in r} == want and (r[:, 3] == 1).all() and len(r) == len(want)
    pts = np.stack([rs.integers(0, nx, 50), rs.integers(0, ny, 50), rs.integers(0, nz, 50)], 1).astype(np.int32)
    val = rs.integers(0, 2, 50).astype(np.uint8)
    before = occ.copy()
    for (x, y, z), v in zip(pts, val):
        occ[z, y, x] = v
    m.set_occupancy(pts, val)
    m.update()
    r = unpack(m.export_occupancy(0, nz, changed_only=True))
    changed = {(z // 8, y // 8, x // 8) for z, y, x in np.argwhere(before != occ)}
    want = {(x, y, z, int(occ[z, y, x])) for bz, by, bx in changed for z in range(8 * bz, min(nz, 8 * bz + 8))
            for y in range(8 * by, min(ny, 8 * by + 8)) for x in range(8 * bx, min(nx, 8 * bx + 8))}
    assert {tuple(v) for v in r} == want
