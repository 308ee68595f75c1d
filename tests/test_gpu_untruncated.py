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
    the field equals the oracle's on the current occupancy.  The update recomputes only the lines
    the flips reach: the x rows holding a flipped voxel, and y / z lines where the previous pass's
    output changed (at most every line of the grid)."""
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(12)
    nx, ny, nz = 70, 52, 41
    occ = W.bernoulli_grid(12, (nz, ny, nx), 0.001)
    m = untrunc_map(nx, ny, nz)
    m.set_occupancy_dense(occ)
    m.global_()
    for f in range(9):
        k = int(rs.integers(1, 60))
        xyz = np.stack([rs.integers(0, nx, k), rs.integers(0, ny, k), rs.integers(0, nz, k)], 1).astype(np.int32)
        val = rs.integers(0, 2, k).astype(np.uint8)
        if f == 3:  # clear everything: D_NONE everywhere
            xyz = W.occupied_coords(occ)
            val = np.zeros(len(xyz), np.uint8)
        if f == 4:  # one obstacle into the empty grid
            xyz, val = np.array([[nx - 1, 0, nz // 2]], np.int32), np.ones(1, np.uint8)
        if f == 5:  # records that flip nothing (the voxel's current state): no line recomputed
            xyz = np.array([[nx - 1, 0, nz // 2], [0, 0, 0]], np.int32)
            val = np.array([1, 0], np.uint8)
        prev = occ.copy()
        for (x, y, z), v in zip(xyz, val):
            occ[z, y, x] = v
        m.set_occupancy(xyz, val)
        st = m.update(stats=True)
        assert st["global_form"] == 0
        flips = np.argwhere(prev != occ)
        assert st["net_flips"] == len(flips)
        assert st["changed_bricks"] == len({(z // 8, y // 8, x // 8) for z, y, x in flips})
        assert st["x_items"] == len({(y, z) for z, y, _ in flips})
        assert st["y_items"] <= nx * nz and st["z_items"] <= nx * ny
        if f == 5:
            assert st["x_items"] == st["y_items"] == st["z_items"] == 0
        ref = O.edt_untruncated(occ)
        got = m.export_dense()
        assert first_mismatch(got, ref) is None, (f, first_mismatch(got, ref))
        if f == 3:
            assert (got == V.D_NONE).all()
    m.close()


@pytest.mark.parametrize("shape_xyz,seed", [((200, 160, 96), 41), ((75, 131, 58), 42)])
def test_local_edits_against_oracle(shape_xyz, seed):
    """Edits clustered in a small box of a larger scene, as a sensor's frame is: obstacles added and
    removed there change distances far away only where the edited voxels were, or become, the
    nearest obstacle.  Every frame's field equals the oracle's; the lines recomputed stay a fraction
    of the grid's."""
    rs = np.random.default_rng(seed)
    nx, ny, nz = shape_xyz
    occ = W.tunnel_scene(seed, (nx, ny, nz), ntunnels=3, rmin=5, rmax=12) if nx >= 100 else \
        W.bernoulli_grid(seed, (nz, ny, nx), 0.0008)
    m = untrunc_map(nx, ny, nz)
    xyz0 = W.occupied_coords(occ)
    m.set_occupancy(xyz0, np.ones(len(xyz0), np.uint8))
    m.global_()
    for f in range(6):
        c = np.array([rs.integers(8, nx - 8), rs.integers(8, ny - 8), rs.integers(8, nz - 8)])
        k = int(rs.integers(20, 400))
        xyz = np.clip(c + rs.integers(-6, 7, (k, 3)), 0, [nx - 1, ny - 1, nz - 1]).astype(np.int32)
        val = (rs.random(k) < 0.6).astype(np.uint8)
        # and some of the box's existing obstacles removed
        box = W.occupied_coords(occ)
        near = box[(np.abs(box - c) <= 6).all(1)]
        if len(near):
            pick = near[rs.integers(0, len(near), min(50, len(near)))]
            xyz = np.concatenate([xyz, pick]).astype(np.int32)
            val = np.concatenate([val, np.zeros(len(pick), np.uint8)])
        for (x, y, z), v in zip(xyz, val):
            occ[z, y, x] = v
        m.set_occupancy(xyz, val)
        st = m.update(stats=True)
        assert st["global_form"] == 0
        got = m.export_dense()
        ref = O.edt_untruncated(occ)
        assert first_mismatch(got, ref) is None, (f, first_mismatch(got, ref))
        assert st["x_items"] <= 13 * 13 and st["y_items"] <= nx * nz and st["z_items"] <= nx * ny
    m.close()


def test_changed_bricks_export_after_update():
    """The changed-brick export (mode 1) after an untruncated update: every voxel of each brick that
    holds a flipped voxel, with its current occupancy."""
    nx, ny, nz = 40, 36, 30
    occ = W.bernoulli_grid(5, (nz, ny, nx), 0.002)
    m = untrunc_map(nx, ny, nz)
    m.set_occupancy_dense(occ)
    m.global_()
    xyz = np.array([[3, 4, 5], [33, 20, 17], [34, 21, 17]], np.int32)
    val = np.array([1, 1, 1], np.uint8)
    val[occ[xyz[:, 2], xyz[:, 1], xyz[:, 0]] == 1] = 0  # each record flips its voxel
    for (x, y, z), v in zip(xyz, val):
        occ[z, y, x] = v
    m.set_occupancy(xyz, val)
    m.update()
    # after a reset the update epochs start over: an update from the empty grid lists every brick
    # that holds an obstacle, those of the update before the reset included
    m.reset()
    m.global_()
    occ_xyz = W.occupied_coords(occ)
    m.set_occupancy(occ_xyz, np.ones(len(occ_xyz), np.uint8))
    st = m.update(stats=True)
    assert st["changed_bricks"] == len({tuple(b) for b in (occ_xyz // 8).tolist()})
    assert first_mismatch(m.export_dense(), O.edt_untruncated(occ)) is None
    m.set_occupancy(xyz, 1 - val)
    m.update()
    m.set_occupancy(xyz, val)
    st = m.update(stats=True)
    assert st["changed_bricks"] == len({tuple(b) for b in (xyz // 8).tolist()})
    assert first_mismatch(m.export_dense(), O.edt_untruncated(occ)) is None
    u = m.export_occupancy(0, nz, changed_only=True).cpu().numpy().view(np.uint64)
    mask = np.uint64((1 << 21) - 1)
    got = np.stack([u & mask, (u >> np.uint64(21)) & mask, (u >> np.uint64(42)) & mask], 1).astype(np.int64)
    got_occ = (u >> np.uint64(63)).astype(np.uint8)
    bricks = {tuple(b) for b in (xyz // 8).tolist()}
    assert {tuple(b) for b in (got // 8).tolist()} == bricks
    inside = [(x, y, z) for bx, by, bz in bricks for z in range(8 * bz, min(8 * bz + 8, nz))
              for y in range(8 * by, min(8 * by + 8, ny)) for x in range(8 * bx, min(8 * bx + 8, nx))]
    assert len(got) == len(inside)
    assert np.array_equal(got_occ, occ[got[:, 2], got[:, 1], got[:, 0]])
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
    assert len(m.export_occupancy(0, 16)) == 1  # every occupied voxel
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
    # an update at full size: three boxes of wall lose most of their voxels and gain a few new ones;
    # voxels sampled around the boxes (where distances change) and uniformly
    cs = xyz[rs.integers(0, len(xyz), 3)]
    recs, vals = [], []
    for c in cs:
        near = xyz[(np.abs(xyz - c) <= 8).all(1)]
        gone = near[rs.random(len(near)) < 0.7]
        new = np.clip(c + rs.integers(-8, 9, (40, 3)), 0, [nx - 1, ny - 1, nz - 1])
        recs += [gone, new]
        vals += [np.zeros(len(gone), np.uint8), np.ones(len(new), np.uint8)]
    rec = np.concatenate(recs).astype(np.int32)
    val = np.concatenate(vals)
    for (x, y, z), v in zip(rec, val):
        occ[z, y, x] = v
    m.set_occupancy(rec, val)
    st = m.update(stats=True)
    assert st["global_form"] == 0 and st["net_flips"] > 0
    assert 0 < st["z_items"] < nx * ny
    q = np.concatenate([np.repeat(cs, 30, 0) + rs.integers(-40, 41, (90, 3)),
                        np.stack([rs.integers(0, nx, 30), rs.integers(0, ny, 30), rs.integers(0, nz, 30)], 1)])
    q = np.clip(q, 0, [nx - 1, ny - 1, nz - 1]).astype(np.int32)
    got = m.query(q)
    ref = O.edt_untruncated_at(occ, q)
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
