"""Untruncated grids (VDBEDT_FLAG_UNTRUNCATED; the paper's dmax = infinity runs, Table II): D is Eq.
1's exact squared distance to the nearest obstacle anywhere in the grid.  Bit-exact against the
oracle's untruncated transform on ragged grids, record and dense ingest, empty grids (D_NONE),
updates that set and clear voxels, queries inside and outside the grid, and sampled voxels of the
full-size tunnel scene; the calls that have no meaning without a truncation are rejected."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import first_mismatch

pytestmark = pytest.mark.gpu


def untrunc_map(nx, ny, nz, **kw):
    import paper_2105_04419_gb300 as V
    return V.Map(nx, ny, nz, None, **kw)


@pytest.mark.parametrize("shape_xyz,p,seed", [((37, 29, 23), 0.002, 1), ((64, 64, 64), 0.0004, 2),
                                               ((100, 20, 9), 0.01, 3), ((9, 130, 17), 0.001, 4),
                                               ((1, 1, 70), 0.05, 5), ((200, 3, 1), 0.02, 6)])
def test_records_against_oracle(shape_xyz, p, seed):
    nx, ny, nz = shape_xyz
    occ = W.bernoulli_grid(seed, (nz, ny, nx), p)
    occ.flat[(seed * 7919) % occ.size] = 1
    m = untrunc_map(nx, ny, nz)
    xyz = W.occupied_coords(occ)
    m.set_occupancy(xyz, np.ones(len(xyz), np.uint8))
    m.global_()
    D = m.export_dense()
    ref = O.edt_untruncated(occ)
    assert first_mismatch(D, ref) is None, first_mismatch(D, ref)
    info = m.info()
    assert info["allocated_bricks"] == info["capacity_bricks"] == -(-nx // 8) * -(-ny // 8) * -(-nz // 8)
    assert info["finite_bricks"] == info["allocated_bricks"]
    m.close()


def test_dense_tunnel_scene_and_far_empty_box():
    occ = W.tunnel_scene(9, (200, 160, 96), ntunnels=4, rmin=6, rmax=14)
    occ[:, 40:130, 30:170] = 0  # distances of tens of voxels, beyond any windowed truncation
    nz, ny, nx = occ.shape
    m = untrunc_map(nx, ny, nz)
    m.set_occupancy_dense(occ)
    m.global_()
    D = m.export_dense()
    ref = O.edt_untruncated(occ)
    assert ref.max() > 45 * 45
    assert first_mismatch(D, ref) is None, first_mismatch(D, ref)
    m.close()


def test_empty_grid_single_obstacle_and_reset():
    import paper_2105_04419_gb300 as V
    nx, ny, nz = 45, 33, 27
    m = untrunc_map(nx, ny, nz)
    m.global_()
    assert (m.export_dense() == V.D_NONE).all()
    m.set_occupancy(np.array([[44, 0, 13]], np.int32), np.ones(1, np.uint8))
    m.global_()
    z, y, x = np.indices((nz, ny, nx))
    assert np.array_equal(m.export_dense(), (x - 44) ** 2 + y ** 2 + (z - 13) ** 2)
    m.reset()
    m.global_()
    assert (m.export_dense() == V.D_NONE).all()
    assert m.info()["finite_bricks"] == 0
    m.close()


def test_updates_set_and_clear():
    """Frames of records that set and clear voxels (repeats, last record wins); after every update
    the field equals the oracle's on the current occupancy."""
    rs = np.random.default_rng(12)
    nx, ny, nz = 70, 52, 41
    occ = W.bernoulli_grid(12, (nz, ny, nx), 0.001)
    m = untrunc_map(nx, ny, nz)
    m.set_occupancy_dense(occ)
    m.global_()
    for f in range(5):
        k = int(rs.integers(1, 60))
        xyz = np.stack([rs.integers(0, nx, k), rs.integers(0, ny, k), rs.integers(0, nz, k)], 1).astype(np.int32)
        val = rs.integers(0, 2, k).astype(np.uint8)
        if f == 3:  # clear everything: D_NONE everywhere
            xyz = W.occupied_coords(occ)
            val = np.zeros(len(xyz), np.uint8)
        for (x, y, z), v in zip(xyz, val):
            occ[z, y, x] = v
        m.set_occupancy(xyz, val)
        st = m.update(stats=True)
        assert st["global_form"] == 1
        ref = O.edt_untruncated(occ)
        assert first_mismatch(m.export_dense(), ref) is None, (f, first_mismatch(m.export_dense(), ref))
    m.close()


def test_queries_and_distance():
    import torch

    import paper_2105_04419_gb300 as V
    nx, ny, nz = 50, 40, 30
    occ = W.bernoulli_grid(21, (nz, ny, nx), 0.0005)
    occ[5, 6, 7] = 1
    m = untrunc_map(nx, ny, nz, voxel_size=0.1)
    m.set_occupancy_dense(occ)
    m.global_()
    ref = O.edt_untruncated(occ)
    rs = np.random.default_rng(5)
    q = np.stack([rs.integers(-5, nx + 5, 500), rs.integers(-5, ny + 5, 500), rs.integers(-5, nz + 5, 500)], 1)
    q = q.astype(np.int32)
    got = m.query(q)
    inside = (q[:, 0] >= 0) & (q[:, 0] < nx) & (q[:, 1] >= 0) & (q[:, 1] < ny) & (q[:, 2] >= 0) & (q[:, 2] < nz)
    assert (got[~inside] == V.D_NONE).all()
    assert np.array_equal(got[inside], ref[q[inside, 2], q[inside, 1], q[inside, 0]])
    # the trilinear distance at voxel centres is the square root of D, in metres
    pts = torch.tensor(q[inside][:50].astype(np.float32) * 0.1, device="cuda")
    d = m.distance_at(pts, with_grad=False).cpu().numpy()
    expect = 0.1 * np.sqrt(ref[q[inside][:50, 2], q[inside][:50, 1], q[inside][:50, 0]].astype(np.float64))
    assert np.allclose(d, expect, rtol=1e-5, atol=1e-5)
    m.close()


def test_rejected_calls():
    import ctypes

    import paper_2105_04419_gb300 as V
    from paper_2105_04419_gb300 import lib as L
    m = untrunc_map(16, 16, 16)
    m.set_occupancy(np.array([[1, 2, 3]], np.int32), np.ones(1, np.uint8))
    m.global_()
    with pytest.raises(V.VdbedtError):
        m.set_tuning(8, 8, 8, 3)
    with pytest.raises(V.VdbedtError):
        m.query_nearest(np.array([[0, 0, 0]], np.int32))
    with pytest.raises(V.VdbedtError):
        m.export_occupancy(0, 16, changed_only=True)
    assert len(m.export_occupancy(0, 16)) == 1  # every occupied voxel: still available
    m.close()
    lb = L.load()
    h = ctypes.c_void_p()
    for cfg in (L.Config(16, 16, 16, 8, 0.1, 0, None, L.FLAG_UNTRUNCATED, 0, 0),  # dmax must be 0
                L.Config(16, 16, 16, 0, 0.1, 0, None, L.FLAG_UNTRUNCATED, 3, 0),  # every brick stored
                L.Config(0, 0, 0, 0, 0.1, 0, None, L.FLAG_UNTRUNCATED | L.FLAG_UNBOUNDED, 100, 10),
                L.Config(30000, 30000, 30000, 0, 0.1, 0, None, L.FLAG_UNTRUNCATED, 0, 0),  # D beyond int32
                L.Config(16, 16, 16, 0, 0.1, 0, None, 0, 0, 0)):  # dmax 0 without the flag
        assert lb.vdbedt_create(ctypes.byref(cfg), ctypes.byref(h)) == 1


def test_full_size_tunnel_scene_sampled():
    """The 1024 x 1024 x 256 tunnel scene untruncated: voxels sampled uniformly and near the walls,
    each against the oracle's brute force over every occupied voxel."""
    import bench
    wl = bench.WORKLOADS["tunnel"]
    nx, ny, nz = wl["dims"]
    occ = bench.make_occupancy(wl)
    m = untrunc_map(nx, ny, nz)
    xyz = W.occupied_coords(occ)
    m.set_occupancy(xyz, np.ones(len(xyz), np.uint8))
    m.global_()
    rs = np.random.default_rng(77)
    q = np.stack([rs.integers(0, nx, 40), rs.integers(0, ny, 40), rs.integers(0, nz, 40)], 1)
    q = np.concatenate([q, xyz[rs.integers(0, len(xyz), 20)] + rs.integers(-3, 4, (20, 3))]).astype(np.int32)
    q = np.clip(q, 0, [nx - 1, ny - 1, nz - 1]).astype(np.int32)
    got = m.query(q)
    ref = O.edt_untruncated_at(occ, q)
    assert ref.max() > 32 * 32  # samples beyond the headline truncation
    assert np.array_equal(got, ref), np.nonzero(got != ref)[0][:5]
    m.close()


def test_captured_update():
    """An untruncated map's update captured once (UpdateGraph) and replayed per frame: the transform
    allocates nothing, so it captures; every replay equals the oracle."""
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(31)
    nx, ny, nz = 48, 40, 36
    occ = W.bernoulli_grid(31, (nz, ny, nx), 0.001)
    occ[1, 2, 3] = 1
    m = untrunc_map(nx, ny, nz)
    m.set_occupancy_dense(occ)
    m.global_()
    g = V.UpdateGraph(m, 256)
    for f in range(3):
        k = 120
        xyz = np.stack([rs.integers(0, nx, k), rs.integers(0, ny, k), rs.integers(0, nz, k)], 1).astype(np.int32)
        val = rs.integers(0, 2, k).astype(np.uint8)
        for (x, y, z), v in zip(xyz, val):
            occ[z, y, x] = v
        g.run(xyz, val)
        assert first_mismatch(m.export_dense(), O.edt_untruncated(occ)) is None, f
    m.close()
