"""Unbounded grids (VDBEDT_FLAG_UNBOUNDED): signed coordinates anywhere in [-2^20, 2^20 - 128) on
each axis, nodes created only where obstacles and their dilation fall (the paper's VDB motivation,
Sec. I and Sec. IV-A), bit-exact against the CPU oracle.

Clusters of obstacles sit at the corners of the range, across the origin and far out; they are
further apart than dmax, so the field around each equals the oracle's field of the cluster's box
padded by dmax.  Checked after the global transform and after an update that edits the clusters and
adds a new one (creating nodes); queries far from every cluster and outside the range give dmax^2;
the nearest-obstacle query, packed records and the clearance cost work in signed coordinates.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import first_mismatch

pytestmark = pytest.mark.gpu

LO, HI = -(1 << 20), (1 << 20) - 128
S = 40     # cluster box side
DMAX = 12


def cluster(seed, p=0.01):
    occ = W.bernoulli_grid(seed, (S, S, S), p)
    occ[S // 2, S // 2, S // 2] = 1
    return occ


ORIGINS = [(LO, LO, LO), (HI - S, 5000, -70000), (-3, -3, -3), (700000, -900000, HI - S)]


def box_query(m, origin, occ):
    """The map's field on the cluster's box padded by DMAX (clipped to the range) against the
    oracle's field of the padded box."""
    ox, oy, oz = origin
    lo = [max(LO, o - DMAX) for o in (ox, oy, oz)]
    hi = [min(HI, o + S + DMAX) for o in (ox, oy, oz)]
    pad = np.zeros((hi[2] - lo[2], hi[1] - lo[1], hi[0] - lo[0]), np.uint8)
    pad[oz - lo[2]: oz - lo[2] + S, oy - lo[1]: oy - lo[1] + S, ox - lo[0]: ox - lo[0] + S] = occ
    ref = O.edt_factorised(pad, DMAX)
    zz, yy, xx = np.meshgrid(np.arange(lo[2], hi[2]), np.arange(lo[1], hi[1]), np.arange(lo[0], hi[0]), indexing="ij")
    q = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1).astype(np.int32)
    got = m.query(q).reshape(pad.shape)
    return got, ref, pad, lo


def records(origin, occ):
    z, y, x = np.nonzero(occ)
    xyz = np.stack([x + origin[0], y + origin[1], z + origin[2]], 1).astype(np.int32)
    return xyz


def test_unbounded_clusters_global_and_update():
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(3)
    m = V.Map(0, 0, 0, DMAX, unbounded=True, max_bricks=60000, max_nodes=400)
    occs = [cluster(10 + i) for i in range(len(ORIGINS))]
    for o, occ in zip(ORIGINS, occs):
        xyz = records(o, occ)
        m.set_occupancy(xyz, np.ones(len(xyz), np.uint8))
    m.global_()
    for i, (o, occ) in enumerate(zip(ORIGINS, occs)):
        got, ref, _, _ = box_query(m, o, occ)
        assert first_mismatch(got, ref) is None, (i, first_mismatch(got, ref))
    # far from every cluster, and outside the range
    far = np.array([[0, 400000, 0], [-500000, 0, 300000], [LO - 5, 0, 0], [HI, HI, HI], [2**30, -2**30, 7]], np.int32)
    assert (m.query(far) == DMAX * DMAX).all()
    n_before = m.info()["nodes"]
    # update: edits inside every cluster, and a new cluster far away (new nodes)
    new_origin = (-600000, 123456, 333333)
    new = cluster(99)
    xyz_all, val_all = [records(new_origin, new)], [np.ones(int(new.sum()), np.uint8)]
    for i, (o, occ) in enumerate(zip(ORIGINS, occs)):
        k = 200
        p = rs.integers(0, S, (k, 3))
        v = rs.integers(0, 2, k).astype(np.uint8)
        for (x, y, z), vv in zip(p, v):  # applied in record order: the last record of a voxel wins
            occ[z, y, x] = vv
        xyz_all.append((p + np.array(o)).astype(np.int32))
        val_all.append(v)
    m.set_occupancy(np.concatenate(xyz_all), np.concatenate(val_all))
    st = m.update(stats=True)
    assert m.info()["nodes"] > n_before and st["new_bricks"] > 0
    for i, (o, occ) in enumerate(zip(ORIGINS + [new_origin], occs + [new])):
        got, ref, _, _ = box_query(m, o, occ)
        assert first_mismatch(got, ref) is None, (i, first_mismatch(got, ref))
    m.close()


def test_unbounded_nearest_packed_and_clearance():
    import torch
    import paper_2105_04419_gb300 as V
    origin = (-20, -17, -25)  # a box across the origin: negative and positive coordinates
    occ = cluster(7, 0.004)
    xyz = records(origin, occ)
    ones = np.ones(len(xyz), np.uint8)
    a = V.Map(0, 0, 0, DMAX, unbounded=True, max_bricks=4000, max_nodes=64)
    a.set_occupancy(xyz, ones)
    a.global_()
    b = V.Map(0, 0, 0, DMAX, unbounded=True, max_bricks=4000, max_nodes=64)
    b.set_occupancy_packed(V.pack_records(xyz, ones, offset=V.UNBOUNDED_OFFSET))
    b.global_()
    got_a, ref, pad, lo = box_query(a, origin, occ)
    got_b, _, _, _ = box_query(b, origin, occ)
    assert first_mismatch(got_a, ref) is None and np.array_equal(got_a, got_b)
    # nearest obstacle, in signed coordinates
    rs = np.random.default_rng(1)
    qloc = np.stack([rs.integers(0, pad.shape[2], 500), rs.integers(0, pad.shape[1], 500),
                     rs.integers(0, pad.shape[0], 500)], 1).astype(np.int32)
    ref_n = O.nearest_obstacle(pad, DMAX, qloc)
    got_n = a.query_nearest(qloc + np.array(lo, np.int32))
    want = np.where(ref_n[:, :1] >= 0, ref_n + np.array(lo), -1)
    assert np.array_equal(got_n, want)
    # clearance cost of points in metres around the box (signed), against the float64 oracle on the
    # padded box (the same points shifted into the box: cells and weights agree within rounding)
    vs, tau = 0.1, 0.5
    D = O.edt_factorised(pad, DMAX)
    ploc = W.free_points(4, pad, vs, 2 * 64).reshape(2, 64, 3)
    pglob = (ploc.astype(np.float64) + np.array(lo) * vs).astype(np.float32)
    cost_o, _, _ = O.clearance(D, DMAX, vs, tau, ploc)
    pt = torch.from_numpy(pglob).cuda()
    cost = V.clearance_cost(a, pt, tau).cpu().numpy()
    np.testing.assert_allclose(cost, cost_o, rtol=2e-3, atol=1e-4)
    a.close()
    b.close()


def test_unbounded_rejections():
    import paper_2105_04419_gb300 as V
    with pytest.raises(V.VdbedtError) as e:
        V.Map(0, 0, 0, 8, unbounded=True)  # capacities are required
    assert e.value.code == "EINVAL"
    m = V.Map(0, 0, 0, 8, unbounded=True, max_bricks=100, max_nodes=8)
    with pytest.raises(V.VdbedtError) as e:
        m.set_occupancy(np.array([[HI, 0, 0]], np.int32), np.array([1], np.uint8))  # outside the range
    assert e.value.code == "EINVAL"
    with pytest.raises(V.VdbedtError) as e:
        m.set_occupancy_dense(np.zeros((2, 2, 2), np.uint8))
    assert e.value.code == "EINVAL"
    m.close()
