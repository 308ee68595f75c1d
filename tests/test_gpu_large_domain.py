"""GPU parity on a grid far larger than its mapped part: 16384 x 16384 x 8184 voxels (2^32 - 2^22
bricks) with a node capacity of 48 and a brick capacity of 20,000, obstacles in a few clusters far
apart.  The handle's memory follows the capacities, and around every cluster the field equals the
oracle's transform of a box that holds every obstacle within dmax, bit for bit; far from every
obstacle it is dmax^2.  An update then adds a cluster in nodes that do not exist yet (the deferred
listing of the tracked ingest), removes and adds obstacles in an existing one, and the same checks
hold.  A capacity that is too small is reported as EOVERFLOW."""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

DIMS = (16384, 16384, 8184)  # x, y, z
DMAX = 16


def cluster(rs, lo, size, p=0.01):
    """Sparse random obstacles plus a wall in the box [lo, lo + size) (x, y, z)."""
    occ = (rs.random((size, size, size)) < p)
    occ[size // 2, :, 3:size - 3] = True  # a wall at one z
    z, y, x = np.nonzero(occ)
    return np.stack([x + lo[0], y + lo[1], z + lo[2]], 1).astype(np.int32)


def box_field(m, pts, lo, size):
    """GPU field on the box [lo, lo + size) against the oracle on the box grown by dmax on every
    side (which holds every obstacle closer than dmax to the inner box)."""
    lo = np.asarray(lo)
    hi = np.minimum(lo + size, DIMS)
    lo = np.maximum(lo, 0)
    elo = np.maximum(lo - DMAX, 0)
    ehi = np.minimum(hi + DMAX, DIMS)
    ext = np.zeros((ehi[2] - elo[2], ehi[1] - elo[1], ehi[0] - elo[0]), np.uint8)
    inside = np.all((pts >= elo) & (pts < ehi), 1)
    q = pts[inside] - elo
    ext[q[:, 2], q[:, 1], q[:, 0]] = 1
    ref = O.edt_factorised(ext, DMAX)[lo[2] - elo[2]:hi[2] - elo[2], lo[1] - elo[1]:hi[1] - elo[1],
                                      lo[0] - elo[0]:hi[0] - elo[0]]
    z, y, x = np.meshgrid(np.arange(lo[2], hi[2]), np.arange(lo[1], hi[1]), np.arange(lo[0], hi[0]), indexing="ij")
    xyz = np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.int32)
    got = m.query(xyz).reshape(ref.shape)
    return got, ref


def check_all(m, occupied, boxes):
    pts = np.array(sorted(occupied), np.int32).reshape(-1, 3)
    for lo, size in boxes:
        got, ref = box_field(m, pts, lo, size)
        assert np.array_equal(got, ref), (lo, size, int(np.sum(got != ref)))


def test_sparse_huge_grid_global_and_update():
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(2105)
    A = ((0, 0, 0), 72)                    # the grid's low corner
    B = ((16300, 16310, 8110), 74)         # the high corner (ragged last bricks)
    C = ((8000, 4100, 4000), 64)           # the middle
    pts = np.concatenate([cluster(rs, lo, size) for lo, size in (A, B, C)])
    m = V.Map(*DIMS, DMAX, max_bricks=20000, max_nodes=48)
    info0 = m.info()
    assert info0["device_bytes"] < (1 << 30)
    m.set_occupancy(pts, np.ones(len(pts), np.uint8))
    m.global_()
    occupied = set(map(tuple, pts.tolist()))
    boxes = [((A[0][0] - DMAX, A[0][1] - DMAX, A[0][2] - DMAX), A[1] + 2 * DMAX),
             ((B[0][0] - DMAX, B[0][1] - DMAX, B[0][2] - DMAX), B[1] + 2 * DMAX),
             ((C[0][0] - DMAX, C[0][1] - DMAX, C[0][2] - DMAX), C[1] + 2 * DMAX)]
    check_all(m, occupied, boxes)
    far = np.array([[4000, 12000, 2000], [12000, 300, 7000], [16383, 0, 8183], [0, 16383, 0]], np.int32)
    assert np.all(m.query(far) == DMAX * DMAX)
    info = m.info()
    assert 0 < info["nodes"] <= 48 and info["allocated_bricks"] <= 20000

    # update: a new cluster in nodes that do not exist yet, removals and additions in cluster C
    D = ((12000, 9000, 1000), 48)
    add_d = cluster(rs, D[0], D[1])
    c_pts = pts[np.all((pts >= C[0]) & (pts < np.asarray(C[0]) + C[1]), 1)]
    rm = c_pts[rs.choice(len(c_pts), len(c_pts) // 3, replace=False)]
    add_c = (np.asarray(C[0]) + rs.integers(0, C[1], (300, 3))).astype(np.int32)
    rec = np.concatenate([rm, add_c, add_d])
    val = np.concatenate([np.zeros(len(rm)), np.ones(len(add_c)), np.ones(len(add_d))]).astype(np.uint8)
    for p_, v_ in zip(map(tuple, rec.tolist()), val):
        if v_:
            occupied.add(p_)
        else:
            occupied.discard(p_)
    m.set_occupancy(rec, val)
    st = m.update(stats=True)
    assert st["new_bricks"] > 0
    boxes.append(((D[0][0] - DMAX, D[0][1] - DMAX, D[0][2] - DMAX), D[1] + 2 * DMAX))
    check_all(m, occupied, boxes)
    assert np.all(m.query(far) == DMAX * DMAX)

    # the same occupancy from scratch gives the same field (global == incremental)
    g = V.Map(*DIMS, DMAX, max_bricks=20000, max_nodes=48)
    allp = np.array(sorted(occupied), np.int32)
    g.set_occupancy(allp, np.ones(len(allp), np.uint8))
    g.global_()
    for lo, size in boxes:
        lo = np.maximum(np.asarray(lo), 0)
        hi = np.minimum(lo + size, DIMS)
        z, y, x = np.meshgrid(np.arange(lo[2], hi[2]), np.arange(lo[1], hi[1]), np.arange(lo[0], hi[0]), indexing="ij")
        xyz = np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.int32)
        assert np.array_equal(m.query(xyz), g.query(xyz))
    g.close()
    m.close()


def test_node_capacity_overflow_reported():
    import paper_2105_04419_gb300 as V
    m = V.Map(1024, 1024, 256, 8, max_nodes=2)
    pts = np.array([[5, 5, 5], [600, 600, 5], [1000, 20, 200]], np.int32)  # three nodes far apart
    m.set_occupancy(pts, np.ones(3, np.uint8))
    m.global_()
    with pytest.raises(V.VdbedtError) as e:
        m.synchronize()
    assert e.value.code == "EOVERFLOW"
    m.close()


def test_node_capacity_enough_matches_dense_grid():
    """With max_nodes set to what the occupancy needs (the obstacles' nodes and their halo), the
    whole field equals the oracle's."""
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(5)
    dims = (300, 260, 140)
    occ = np.zeros(dims[::-1], np.uint8)
    occ[10:30, 10:30, 10:30] = rs.random((20, 20, 20)) < 0.02
    occ[100:120, 200:230, 260:290] = rs.random((20, 30, 30)) < 0.02
    m = V.Map(*dims, 12, max_nodes=16)
    z, y, x = np.nonzero(occ)
    m.set_occupancy(np.stack([x, y, z], 1).astype(np.int32), np.ones(len(x), np.uint8))
    m.global_()
    assert m.info()["nodes"] <= 16
    assert np.array_equal(m.export_dense(), O.edt_factorised(occ, 12))
    m.close()


def test_graph_replay_on_huge_grid():
    """The captured update (UpdateGraph) on the 16384 x 16384 x 8184 grid with capacities: its
    reserved scratch does not scale with the grid, and after each frame it equals the eager
    update of a twin handle, including frames that create nodes."""
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(77)
    base = cluster(rs, (4000, 4000, 4000), 40)
    a = V.Map(*DIMS, DMAX, max_bricks=8000, max_nodes=32)
    b = V.Map(*DIMS, DMAX, max_bricks=8000, max_nodes=32)
    for m in (a, b):
        m.set_occupancy(base, np.ones(len(base), np.uint8))
        m.global_()
    g = V.UpdateGraph(a, 20000)
    boxes = [((4000 - DMAX, 4000 - DMAX, 4000 - DMAX), 40 + 2 * DMAX)]
    for f, lo in enumerate([(4030, 3990, 4010), (9000, 12000, 600), (9010, 12010, 610)]):
        add = cluster(rs, lo, 24)
        rm = base[rs.choice(len(base), 50, replace=False)]
        rec = np.concatenate([add, rm])
        val = np.concatenate([np.ones(len(add)), np.zeros(len(rm))]).astype(np.uint8)
        g.run(rec, val)
        b.set_occupancy(rec, val)
        b.update()
        boxes.append(((lo[0] - DMAX, lo[1] - DMAX, lo[2] - DMAX), 24 + 2 * DMAX))
        for blo, size in boxes:
            blo = np.maximum(np.asarray(blo), 0)
            bhi = np.minimum(blo + size, DIMS)
            z, y, x = np.meshgrid(np.arange(blo[2], bhi[2]), np.arange(blo[1], bhi[1]), np.arange(blo[0], bhi[0]),
                                  indexing="ij")
            xyz = np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.int32)
            assert np.array_equal(a.query(xyz), b.query(xyz)), (f, blo)
    assert a.info()["device_bytes"] < (1 << 30)
    a.synchronize()
    a.close()
    b.close()


def test_brick_capacity_overflow_in_update_reported():
    """An update whose new obstacle bricks exceed the brick capacity: the bricks that fit are
    stored, the rest are refused, and the next synchronising call reports EOVERFLOW."""
    import paper_2105_04419_gb300 as V
    m = V.Map(256, 256, 64, 2, max_bricks=30)  # R = 1: an obstacle brick's cube is 27 bricks
    m.set_occupancy(np.array([[100, 100, 30]], np.int32), np.ones(1, np.uint8))
    m.global_()
    m.synchronize()
    assert m.info()["allocated_bricks"] == 27
    far = np.array([[8 + 40 * k, 8, 8] for k in range(5)], np.int32)  # five new bricks, far apart
    m.set_occupancy(far, np.ones(len(far), np.uint8))
    m.update()
    with pytest.raises(V.VdbedtError) as e:
        m.synchronize()
    assert e.value.code == "EOVERFLOW"
    m.close()
