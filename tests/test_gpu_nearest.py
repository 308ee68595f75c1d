"""GPU parity of the nearest-obstacle query against the oracle's brute force: every voxel of
ragged random grids, ties along and across axes, voxels outside the grid, after incremental
updates, and sampled voxels of the full 1024 x 1024 x 256 tunnel scene (checked against the
oracle's field and the occupancy: on the sphere |o - v|^2 = D, occupied, and no occupied point of
that sphere earlier in (z, y, x) order)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import coords_of

pytestmark = pytest.mark.gpu


def all_voxels(shape):
    nz, ny, nx = shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1).astype(np.int32)


@pytest.mark.parametrize("dmax", [3, 9, 20, 33])
def test_every_voxel_matches_oracle(dmax):
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(dmax)
    shape = (21, 26, 35)
    occ = (rs.random(shape) < 0.004).astype(np.uint8)
    nz, ny, nx = shape
    m = V.Map(nx, ny, nz, dmax)
    m.set_occupancy_dense(occ)
    m.global_()
    q = all_voxels(shape)
    q = np.concatenate([q, np.array([[-1, 0, 0], [nx, 0, 0], [0, ny, 0], [0, 0, nz]], np.int32)])
    got = m.query_nearest(q)
    ref = O.nearest_obstacle(occ, dmax, q)
    assert np.array_equal(got, ref), np.argwhere((got != ref).any(axis=1))[:5]
    m.synchronize()


def test_ties():
    import paper_2105_04419_gb300 as V
    occ = np.zeros((11, 11, 11), np.uint8)
    occ[5, 5, 8] = occ[5, 8, 5] = occ[8, 5, 5] = 1
    occ[2, 9, 5] = occ[5, 2, 9] = 1
    m = V.Map(11, 11, 11, 10)
    m.set_occupancy_dense(occ)
    m.global_()
    q = all_voxels(occ.shape)
    assert np.array_equal(m.query_nearest(q), O.nearest_obstacle(occ, 10, q))


def test_after_updates_and_device_queries():
    import torch
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(8)
    shape = (30, 40, 50)
    nz, ny, nx = shape
    occ = (rs.random(shape) < 0.003).astype(np.uint8)
    m = V.Map(nx, ny, nz, 12)
    m.set_occupancy_dense(occ)
    m.global_()
    for f in range(3):
        k = 150
        xyz = np.stack([rs.integers(0, nx, k), rs.integers(0, ny, k), rs.integers(0, nz, k)], 1).astype(np.int32)
        val = rs.integers(0, 2, k).astype(np.uint8)
        for r in range(k):
            occ[xyz[r, 2], xyz[r, 1], xyz[r, 0]] = val[r]
        m.set_occupancy(xyz, val)
        m.update()
        q = np.stack([rs.integers(-2, nx + 2, 4000), rs.integers(-2, ny + 2, 4000),
                      rs.integers(-2, nz + 2, 4000)], 1).astype(np.int32)
        got = m.query_nearest(torch.from_numpy(q).cuda()).cpu().numpy()
        assert np.array_equal(got, O.nearest_obstacle(occ, 12, q)), f


def test_tunnel_sampled_against_oracle_field():
    import torch
    import paper_2105_04419_gb300 as V
    dims, dmax = (1024, 1024, 256), 32
    occ = W.tunnel_scene(1, dims)
    ref = O.edt_factorised(occ, dmax)
    xyz = torch.from_numpy(W.occupied_coords(occ)).cuda()
    m = V.Map(*dims, dmax)
    m.set_occupancy(xyz, torch.ones(xyz.shape[0], dtype=torch.uint8, device="cuda"))
    m.global_()
    rs = np.random.default_rng(2)
    q = np.stack([rs.integers(0, 1024, 3000), rs.integers(0, 1024, 3000), rs.integers(0, 256, 3000)], 1).astype(np.int32)
    got = m.query_nearest(q)
    D = ref[q[:, 2], q[:, 1], q[:, 0]].astype(np.int64)
    none = (got == -1).all(axis=1)
    assert np.array_equal(none, D >= dmax * dmax)
    g = got[~none].astype(np.int64)
    v = q[~none].astype(np.int64)
    assert np.array_equal(((g - v) ** 2).sum(axis=1), D[~none])
    assert occ[g[:, 2], g[:, 1], g[:, 0]].all()
    # no occupied point of the same sphere comes earlier in (z, y, x) order
    for (x, y, z), (ox, oy, oz), d2 in zip(v[:400], g[:400], D[~none][:400]):
        r = int(np.sqrt(d2))
        for dz in range(-r, r + 1):
            for dy in range(-r, r + 1):
                rem = d2 - dz * dz - dy * dy
                if rem < 0:
                    continue
                dx = int(round(np.sqrt(rem)))
                if dx * dx != rem:
                    continue
                for sx in ((-dx, dx) if dx else (0,)):
                    px, py, pz = x + sx, y + dy, z + dz
                    if not (0 <= px < 1024 and 0 <= py < 1024 and 0 <= pz < 256) or not occ[pz, py, px]:
                        continue
                    assert (pz, py, px) >= (oz, oy, ox)
    m.close()
