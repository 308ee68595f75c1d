"""Occupancy staged brick by brick (vdbedt_set_occupancy_bricks): the same field as the same voxels
staged as records, bit-exact against the oracle, on ragged grids, mixed with records (order of the
calls decides), before an incremental update, on unbounded and untruncated grids; bricks or bits
outside the grid reject the call."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import first_mismatch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape_zyx,p,seed", [((23, 29, 37), 0.02, 1), ((64, 64, 64), 0.01, 2), ((9, 20, 100), 0.3, 3)])
@pytest.mark.parametrize("on_device", [False, True])
def test_bricks_equal_records(shape_zyx, p, seed, on_device):
    import torch

    import paper_2105_04419_gb300 as V
    occ = W.bernoulli_grid(seed, shape_zyx, p)
    nz, ny, nx = occ.shape
    bxyz, masks = V.brick_masks(occ)
    m = V.Map(nx, ny, nz, 12)
    if on_device:
        m.set_occupancy_bricks(torch.from_numpy(bxyz).cuda(), torch.from_numpy(masks.view(np.int64)).cuda())
    else:
        m.set_occupancy_bricks(bxyz, masks)
    m.global_()
    ref = O.edt_factorised(occ, 12)
    assert first_mismatch(m.export_dense(), ref) is None
    m.close()


def test_bricks_then_records_and_update():
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(9)
    occ = W.bernoulli_grid(9, (40, 48, 56), 0.01)
    nz, ny, nx = occ.shape
    m = V.Map(nx, ny, nz, 10)
    bxyz, masks = V.brick_masks(occ)
    # clear records staged before the bricks lose to them; records staged after win
    pre = W.occupied_coords(occ)[:50]
    m.set_occupancy(pre, np.zeros(len(pre), np.uint8))
    m.set_occupancy_bricks(bxyz, masks)
    post = W.occupied_coords(occ)[50:80]
    m.set_occupancy(post, np.zeros(len(post), np.uint8))
    for x, y, z in post:
        occ[z, y, x] = 0
    m.global_()
    assert first_mismatch(m.export_dense(), O.edt_factorised(occ, 10)) is None
    # an incremental update from bricks: a new cluster
    add = np.zeros_like(occ)
    add[10:14, 20:22, 30:37] = 1
    bk, mk = V.brick_masks(add)
    m.set_occupancy_bricks(bk, mk)
    occ |= add
    st = m.update(stats=True)
    assert st["records"] == int(add.sum())
    assert first_mismatch(m.export_dense(), O.edt_factorised(occ, 10)) is None
    m.close()


def test_unbounded_and_untruncated():
    import paper_2105_04419_gb300 as V
    occ = W.bernoulli_grid(11, (24, 24, 24), 0.02)
    # unbounded: the block's voxel (0, 0, 0) at (-40, 800, -8)
    u = V.Map(0, 0, 0, 8, unbounded=True, max_bricks=5000, max_nodes=64)
    bxyz, masks = V.brick_masks(occ, origin_xyz=(-40, 800, -8))
    u.set_occupancy_bricks(bxyz, masks)
    u.global_()
    pad = np.zeros((40, 40, 40), np.uint8)
    pad[8:32, 8:32, 8:32] = occ
    ref = O.edt_factorised(pad, 8)[8:32, 8:32, 8:32]
    z, y, x = np.indices(occ.shape)
    q = np.stack([x.ravel() - 40, y.ravel() + 800, z.ravel() - 8], 1).astype(np.int32)
    assert np.array_equal(u.query(q), ref.ravel())
    u.close()
    t = V.Map(24, 24, 24, None)
    b2, m2 = V.brick_masks(occ)
    t.set_occupancy_bricks(b2, m2)
    t.global_()
    assert first_mismatch(t.export_dense(), O.edt_untruncated(occ)) is None
    t.close()


def test_outside_the_grid_rejected():
    import paper_2105_04419_gb300 as V
    m = V.Map(20, 16, 16, 6)  # ragged along x: bricks 0..2, voxels 0..19
    ok = np.zeros((1, 8), np.uint64)
    ok[0, 0] = np.uint64(1 << 3)  # voxel (19, 0, 0)
    m.set_occupancy_bricks(np.array([[2, 0, 0]], np.int32), ok)
    bad_bit = np.zeros((1, 8), np.uint64)
    bad_bit[0, 0] = np.uint64(1 << 4)  # voxel (20, 0, 0): outside
    with pytest.raises(V.VdbedtError):
        m.set_occupancy_bricks(np.array([[2, 0, 0]], np.int32), bad_bit)
    with pytest.raises(V.VdbedtError):
        m.set_occupancy_bricks(np.array([[3, 0, 0]], np.int32), ok)
    with pytest.raises(V.VdbedtError):
        m.set_occupancy_bricks(np.array([[0, -1, 0]], np.int32), ok)
    m.global_()
    D = m.export_dense()
    assert D[0, 0, 19] == 0 and D[0, 0, 18] == 1  # only the accepted call was staged
    m.close()
