"""Pins for the oracle's transcription of the paper's raise/lower transform (Alg. 1, Sec. IV-B).

The paper does not claim that Alg. 1 reaches Eq. 1 exactly, so its disagreements with the exact
transform are counted, not assumed away.  What must hold regardless:
  * occupancy after a frame is the records applied in order (last write wins);
  * an incremental result that differs from the global result at a voxel must also differ from
    the exact transform there (otherwise the incremental transcription is wrong);
  * on these seeded workloads the counts are recorded and are zero.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


def random_frames(rs, shape, nframes, max_edits):
    for _ in range(nframes):
        m = int(rs.integers(0, max_edits + 1))
        xyz = np.stack([rs.integers(0, shape[2], m), rs.integers(0, shape[1], m), rs.integers(0, shape[0], m)],
                       1).astype(np.int32)
        val = rs.integers(0, 2, m).astype(np.uint8)
        yield xyz, val


def apply_records(occ, xyz, val):
    for k in range(len(val)):
        occ[xyz[k, 2], xyz[k, 1], xyz[k, 0]] = val[k]


@pytest.mark.parametrize("seed", range(5))
def test_alg1_global_vs_exact(seed):
    rs = np.random.default_rng(seed)
    shape = tuple(int(v) for v in rs.integers(6, 22, 3))
    dmax = int(rs.integers(1, 10))
    occ = (rs.random(shape) < rs.uniform(0.003, 0.08)).astype(np.uint8)
    a = O.Alg1(shape, dmax)
    a.global_(occ)
    exact = O.edt_naive(occ, dmax)
    mism = int((a.dist() != exact).sum())
    assert mism == 0, f"Alg. 1 global disagrees with Eq. 1 at {mism} voxels"
    c = a.counters()
    assert c["raised"] == 0  # a global transform only lowers (Sec. V-A)
    assert c["lowered"] >= int(occ.sum())


@pytest.mark.parametrize("seed", range(6))
def test_alg1_incremental(seed):
    rs = np.random.default_rng(50 + seed)
    shape = tuple(int(v) for v in rs.integers(5, 18, 3))
    dmax = int(rs.integers(1, 9))
    occ = (rs.random(shape) < rs.uniform(0.005, 0.1)).astype(np.uint8)
    inc = O.Alg1(shape, dmax)
    inc.global_(occ)
    total_bad = 0
    for xyz, val in random_frames(rs, shape, 6, 80):
        inc.update(xyz, val)
        apply_records(occ, xyz, val)
        assert np.array_equal(inc.occupancy(), occ)
        glob = O.Alg1(shape, dmax)
        glob.global_(occ)
        exact = O.edt_naive(occ, dmax)
        di, dg = inc.dist(), glob.dist()
        # a voxel where incremental and global differ must be an Alg. 1 error, visible against Eq. 1
        assert ((di == dg) | (di != exact) | (dg != exact)).all()
        assert (di >= exact).all()
        total_bad += int((di != exact).sum())
    assert total_bad == 0


def test_alg1_paper_ablation_shape():
    """The ablation workload shape of Sec. V-A: a cube with 500 random obstacles, then half of them
    removed and the same number added; dmax 10 cells (side reduced from 100 to 40 for speed)."""
    rs = np.random.default_rng(11)
    side, dmax = 40, 10
    shape = (side, side, side)
    idx = rs.choice(side ** 3, 500, replace=False)
    occ = np.zeros(side ** 3, np.uint8)
    occ[idx] = 1
    occ = occ.reshape(shape)
    a = O.Alg1(shape, dmax)
    a.global_(occ)
    removed = rs.choice(idx, 250, replace=False)
    free = np.flatnonzero(occ.ravel() == 0)
    added = rs.choice(free, 250, replace=False)
    lin = np.concatenate([removed, added])
    val = np.concatenate([np.zeros(250, np.uint8), np.ones(250, np.uint8)])
    z, r = np.divmod(lin, side * side)
    y, x = np.divmod(r, side)
    xyz = np.stack([x, y, z], 1).astype(np.int32)
    a.reset_counters()
    a.update(xyz, val)
    apply_records(occ, xyz, val)
    exact = O.edt_factorised(occ, dmax)
    glob = O.Alg1(shape, dmax)
    glob.global_(occ)
    di, dg = a.dist(), glob.dist()
    # Alg. 1 only ever stores a true squared distance to some obstacle, so it can overshoot the
    # exact minimum but never undershoot it.
    assert (di >= exact).all() and (dg >= exact).all()
    assert ((di == dg) | (di != exact) | (dg != exact)).all()
    mism_inc, mism_glob = int((di != exact).sum()), int((dg != exact).sum())
    # Observed on this seed: one voxel (value 50 where Eq. 1 gives 49) in both forms: the 26-
    # neighbour propagation of nearest-obstacle indices does not always reach the true minimiser.
    assert mism_inc <= 4 and mism_glob <= 4, (mism_inc, mism_glob)
    c = a.counters()
    assert c["raised"] > 0 and c["lowered"] > 0


def test_alg1_duplicate_records_last_wins():
    shape = (6, 7, 8)
    a = O.Alg1(shape, 4)
    occ = np.zeros(shape, np.uint8)
    a.global_(occ)
    xyz = np.array([[1, 2, 3], [1, 2, 3], [4, 4, 4], [4, 4, 4], [4, 4, 4]], np.int32)
    val = np.array([1, 0, 0, 1, 1], np.uint8)
    a.update(xyz, val)
    apply_records(occ, xyz, val)
    assert occ[3, 2, 1] == 0 and occ[4, 4, 4] == 1
    assert np.array_equal(a.occupancy(), occ)
    assert np.array_equal(a.dist(), O.edt_naive(occ, 4))


def test_alg1_lidar_frames():
    """Incremental transform fed by the lidar edit stream on a small tunnel scene."""
    dims = (96, 96, 48)
    truth = W.tunnel_scene(4, dims, ntunnels=3, rmin=5, rmax=8)
    radii, lines = W.tunnel_lines(4, dims, ntunnels=3, rmin=5, rmax=8)
    seq = W.LidarSequence(truth, 4, lines[0], nframes=6, nbeams=8, nazim=64, maxrange=60)
    shape = truth.shape
    dmax = 6
    a = O.Alg1(shape, dmax)
    a.global_(np.zeros(shape, np.uint8))
    for f in range(6):
        xyz, val = seq.next()
        a.update(xyz, val)
        assert np.array_equal(a.occupancy(), seq.map)
        assert np.array_equal(a.dist(), O.edt_factorised(seq.map, dmax))
