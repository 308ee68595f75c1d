"""GPU parity of the incremental transform: after every frame of edits, vdbedt_update equals the
oracle's exact transform of the resulting occupancy (and vdbedt_global on it), bit for bit.

Edit streams: random records (sets, clears, duplicates) on ragged grids; the paper's ablation
shape (half of the obstacles removed, as many added; Sec. V-A); and the lidar sequence on a small
tunnel scene, starting from an empty map.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import coords_of, first_mismatch

pytestmark = pytest.mark.gpu


def apply_records(occ, xyz, val):
    for k in range(len(val)):
        occ[xyz[k, 2], xyz[k, 1], xyz[k, 0]] = val[k]


@pytest.mark.parametrize("dmax", [3, 9, 16, 32, 47])
def test_random_edit_frames(dmax):
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(dmax)
    shape = (29, 54, 61)
    occ = (rs.random(shape) < 0.004).astype(np.uint8)
    nz, ny, nx = shape
    m = V.Map(nx, ny, nz, dmax)
    xyz0 = coords_of(occ)
    m.set_occupancy(xyz0, np.ones(len(xyz0), np.uint8))
    m.global_()
    for f in range(6):
        k = int(rs.integers(1, 300))
        xyz = np.stack([rs.integers(0, nx, k), rs.integers(0, ny, k), rs.integers(0, nz, k)], 1).astype(np.int32)
        # also clear some existing obstacles
        occ_xyz = coords_of(occ)
        if len(occ_xyz):
            pick = occ_xyz[rs.integers(0, len(occ_xyz), min(50, len(occ_xyz)))]
            xyz = np.concatenate([xyz, pick])
        val = rs.integers(0, 2, len(xyz)).astype(np.uint8)
        val[-min(50, len(occ_xyz)):] = 0 if len(occ_xyz) else val[-1:]
        apply_records(occ, xyz, val)
        m.set_occupancy(xyz, val)
        st = m.update(stats=True)
        ref = O.edt_factorised(occ, dmax)
        got = m.export_dense()
        assert first_mismatch(got, ref) is None, (f, st, first_mismatch(got, ref))
        assert st["records"] == len(val)


def test_ablation_shape_remove_half_add_half():
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(11)
    side, dmax = 100, 10
    idx = rs.choice(side ** 3, 500, replace=False)
    occ = np.zeros(side ** 3, np.uint8)
    occ[idx] = 1
    occ = occ.reshape(side, side, side)
    m = V.Map(side, side, side, dmax)
    xyz0 = coords_of(occ)
    m.set_occupancy(xyz0, np.ones(len(xyz0), np.uint8))
    m.global_()
    removed = rs.choice(idx, 250, replace=False)
    free = np.flatnonzero(occ.ravel() == 0)
    added = rs.choice(free, 250, replace=False)
    lin = np.concatenate([removed, added])
    val = np.concatenate([np.zeros(250, np.uint8), np.ones(250, np.uint8)])
    z, r = np.divmod(lin, side * side)
    y, x = np.divmod(r, side)
    xyz = np.stack([x, y, z], 1).astype(np.int32)
    apply_records(occ, xyz, val)
    m.set_occupancy(xyz, val)
    st = m.update(stats=True)
    assert st["net_flips"] == 500
    ref = O.edt_factorised(occ, dmax)
    assert first_mismatch(m.export_dense(), ref) is None


def test_update_equals_global_on_lidar_frames():
    import paper_2105_04419_gb300 as V
    dims = (160, 144, 64)
    truth = W.tunnel_scene(4, dims, ntunnels=4, rmin=6, rmax=10)
    _, lines = W.tunnel_lines(4, dims, ntunnels=4, rmin=6, rmax=10)
    seq = W.LidarSequence(truth, 4, lines[0], nframes=12, nbeams=16, nazim=256, maxrange=120)
    dmax = 16
    inc = V.Map(*dims, dmax)
    inc.global_()
    for f in range(12):
        xyz, val = seq.next()
        inc.set_occupancy(xyz, val)
        inc.update()
        ref = O.edt_factorised(seq.map, dmax)
        got = inc.export_dense()
        assert first_mismatch(got, ref) is None, (f, first_mismatch(got, ref))
        glob = V.Map(*dims, dmax)
        glob.set_occupancy_dense(seq.map)
        glob.global_()
        assert np.array_equal(glob.export_dense(), got)


def test_update_before_any_global_and_after_dense():
    import paper_2105_04419_gb300 as V
    occ = W.bernoulli_grid(1, (24, 25, 26), 0.01)
    m = V.Map(26, 25, 24, 6)
    xyz = coords_of(occ)
    m.set_occupancy(xyz, np.ones(len(xyz), np.uint8))
    m.update()  # first call computes globally
    assert np.array_equal(m.export_dense(), O.edt_factorised(occ, 6))
    occ2 = W.bernoulli_grid(2, (24, 25, 26), 0.02)
    m.set_occupancy_dense(occ2)
    m.update()  # a replaced grid is recomputed globally
    assert np.array_equal(m.export_dense(), O.edt_factorised(occ2, 6))
    # an empty update changes nothing
    st = m.update(stats=True)
    assert st["net_flips"] == 0 and st["z_items"] == 0
    assert np.array_equal(m.export_dense(), O.edt_factorised(occ2, 6))


def test_small_frames_in_large_grid():
    """Frames of a few hundred records in a 320 x 300 x 96 grid: the incremental ingest takes the
    radix-sort path and touches few bricks."""
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(3)
    nx, ny, nz = 320, 300, 96
    dmax = 24
    occ = (rs.random((nz, ny, nx)) < 0.0005).astype(np.uint8)
    m = V.Map(nx, ny, nz, dmax)
    m.set_occupancy_dense(occ)
    m.global_()
    for f in range(5):
        k = 200
        xyz = np.stack([rs.integers(0, nx, k), rs.integers(0, ny, k), rs.integers(0, nz, k)], 1).astype(np.int32)
        occ_xyz = coords_of(occ)
        pick = occ_xyz[rs.integers(0, len(occ_xyz), 100)]
        xyz = np.concatenate([xyz, pick])
        val = np.concatenate([np.ones(k, np.uint8), np.zeros(100, np.uint8)])
        apply_records(occ, xyz, val)
        m.set_occupancy(xyz, val)
        st = m.update(stats=True)
        ref = O.edt_factorised(occ, dmax)
        assert first_mismatch(m.export_dense(), ref) is None, (f, st)


def _edit_fraction(rs, occ, f):
    """The paper's ablation shape (Sec. V-A): remove a fraction f of the obstacles at random and add
    as many new ones uniformly in the grid."""
    nz, ny, nx = occ.shape
    obs = np.argwhere(occ)
    k = max(1, int(round(f * len(obs))))
    rm = obs[rs.choice(len(obs), k, replace=False)][:, ::-1].astype(np.int32)
    add = np.stack([rs.integers(0, nx, k), rs.integers(0, ny, k), rs.integers(0, nz, k)], 1).astype(np.int32)
    xyz = np.concatenate([rm, add])
    val = np.concatenate([np.zeros(k, np.uint8), np.ones(k, np.uint8)])
    return xyz, val


def test_switch_to_global_form_on_each_side():
    """Small edits stay incremental, large ones switch to the global form on the device; both, and an
    incremental frame after a switched one, equal Eq. 1."""
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(41)
    occ = W.tunnel_scene(6, (200, 160, 96), ntunnels=6, rmin=5, rmax=12)
    nz, ny, nx = occ.shape
    m = V.Map(nx, ny, nz, 16)
    m.set_occupancy_dense(occ)
    m.global_()
    for f, expect in ((0.0005, 0), (0.3, 1), (0.0005, 0), (0.05, 1)):
        xyz, val = _edit_fraction(rs, occ, f)
        for (x, y, z), v in zip(xyz, val):
            occ[z, y, x] = v
        m.set_occupancy(xyz, val)
        st = m.update(stats=True)
        assert st["global_form"] == expect, (f, st)
        # recomputed bricks: the global form's runs hold every stored brick once per axis; an
        # incremental update's z runs hold at least its changed bricks
        nb = m.info()["allocated_bricks"]
        if expect:
            assert st["x_bricks"] == st["y_bricks"] == st["z_bricks"] == nb, (st, nb)
        else:
            assert st["changed_bricks"] <= st["z_bricks"] <= nb and 0 < st["x_bricks"] <= nb, (st, nb)
            assert 0 < st["y_bricks"] <= nb, (st, nb)
        ref = O.edt_factorised(occ, 16)
        assert first_mismatch(m.export_dense(), ref) is None, (f, first_mismatch(m.export_dense(), ref))


def test_switch_inside_a_captured_update():
    """One captured update replayed with a large frame (the device switches to the global form) and
    then small frames (incremental): every replay equals Eq. 1."""
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(42)
    occ = W.bernoulli_grid(42, (64, 96, 120), 0.01)
    nz, ny, nx = occ.shape
    m = V.Map(nx, ny, nz, 12)
    m.set_occupancy_dense(occ)
    m.global_()
    g = V.UpdateGraph(m, 40000)
    for f in (0.4, 0.001, 0.2, 0.0005):
        xyz, val = _edit_fraction(rs, occ, f)
        for (x, y, z), v in zip(xyz, val):
            occ[z, y, x] = v
        g.run(xyz, val)
        ref = O.edt_factorised(occ, 12)
        assert first_mismatch(m.export_dense(), ref) is None, (f, first_mismatch(m.export_dense(), ref))


def test_profiled_transforms_equal_the_oracle():
    """With phase events recorded between the kernels of a transform (profiling on), global and
    incremental fields still equal Eq. 1: the events do not reorder the kernels that start early."""
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(77)
    occ = W.tunnel_scene(5, (160, 128, 64), ntunnels=5, rmin=5, rmax=10)
    nz, ny, nx = occ.shape
    m = V.Map(nx, ny, nz, 16)
    m.set_profiling(True)
    xyz = W.occupied_coords(occ)
    m.set_occupancy(xyz, np.ones(len(xyz), np.uint8))
    m.global_()
    assert first_mismatch(m.export_dense(), O.edt_factorised(occ, 16)) is None
    assert m.phase_times()["z_ms"] > 0
    for f in range(4):
        xyz, val = _edit_fraction(rs, occ, 0.002)
        for (x, y, z), v in zip(xyz, val):
            occ[z, y, x] = v
        m.set_occupancy(xyz, val)
        m.update()
        assert first_mismatch(m.export_dense(), O.edt_factorised(occ, 16)) is None, f
        m.phase_times()
    m.close()


def test_clears_in_bricks_added_by_the_same_frame():
    """A frame that sets voxels in bricks not stored yet and clears some of them again (the clear
    last): the bricks are added by the frame's own set records, and the later clears must still win
    (last record of a voxel), with or without a capture."""
    import paper_2105_04419_gb300 as V
    nx, ny, nz = 96, 80, 64
    occ = np.zeros((nz, ny, nx), np.uint8)
    occ[5:9, 5:9, 5:9] = 1  # something stored far from the edits
    for captured in (False, True):
        m = V.Map(nx, ny, nz, 12)
        m.set_occupancy_dense(occ)
        m.global_()
        cur = occ.copy()
        g = V.UpdateGraph(m, 64) if captured else None
        rs = np.random.default_rng(3 + captured)
        for f in range(3):
            base = np.array([60 + 4 * f, 50, 40], np.int32)
            pts = base + rs.integers(0, 8, (6, 3)).astype(np.int32)
            # set all six, then clear the first three again, then set the first once more and clear it
            xyz = np.concatenate([pts, pts[:3], pts[:1], pts[:1]])
            val = np.array([1] * 6 + [0] * 3 + [1, 0], np.uint8)
            apply_records(cur, xyz, val)
            if captured:
                g.run(xyz, val)
            else:
                m.set_occupancy(xyz, val)
                m.update()
            assert first_mismatch(m.export_dense(), O.edt_factorised(cur, 12)) is None, (captured, f)
        m.close()


def test_many_changed_bricks_without_the_switch():
    """An update whose changed bricks outnumber twice the marking launch's blocks (the kernel then
    takes a thread per (changed brick, row / cube offset)) while staying incremental: small dmax,
    every brick stored, random edits over the whole grid; several frames, each equal to Eq. 1."""
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(19)
    nx, ny, nz = 256, 256, 128
    occ = (rs.random((nz, ny, nx)) < 0.01).astype(np.uint8)
    m = V.Map(nx, ny, nz, 3)
    m.set_occupancy_dense(occ)
    m.global_()
    for f in range(3):
        k = 16000  # mostly sets of free voxels: about 8,000 changed bricks of the 16,384
        xyz = np.stack([rs.integers(0, nx, k), rs.integers(0, ny, k), rs.integers(0, nz, k)], 1).astype(np.int32)
        val = (rs.random(k) < 0.9).astype(np.uint8)
        apply_records(occ, xyz, val)
        m.set_occupancy(xyz, val)
        st = m.update(stats=True)
        assert st["global_form"] == 0 and st["changed_bricks"] > 2 * 2432, st
        assert first_mismatch(m.export_dense(), O.edt_factorised(occ, 3)) is None, f
    m.close()
