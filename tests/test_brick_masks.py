"""brick_masks (host helper of vdbedt_set_occupancy_bricks): each occupied voxel appears as exactly
one bit of its brick's mask, at plane z, bit x + 8 y; empty bricks are left out (no GPU needed)."""
import numpy as np

from paper_2105_04419_gb300.lib import brick_masks


def decode(bxyz, masks):
    out = set()
    for (bx, by, bz), m in zip(bxyz, masks):
        for z in range(8):
            w = int(m[z])
            for b in range(64):
                if (w >> b) & 1:
                    out.add((8 * int(bx) + (b & 7), 8 * int(by) + (b >> 3), 8 * int(bz) + z))
    return out


def test_round_trip_ragged_grids():
    rs = np.random.default_rng(4)
    for shape in [(1, 1, 1), (9, 10, 11), (16, 8, 24), (3, 17, 5), (20, 20, 20)]:
        occ = (rs.random(shape) < 0.05).astype(np.uint8)
        bxyz, masks = brick_masks(occ)
        z, y, x = np.nonzero(occ)
        assert decode(bxyz, masks) == set(zip(x.tolist(), y.tolist(), z.tolist()))
        assert all(m.any() for m in masks)
        assert len(np.unique(bxyz, axis=0)) == len(bxyz)


def test_origin_shifts_brick_coordinates():
    occ = np.zeros((8, 8, 16), np.uint8)
    occ[2, 3, 12] = 1
    bxyz, masks = brick_masks(occ, origin_xyz=(-16, 8, 0))
    assert bxyz.tolist() == [[-1, 1, 0]]
    assert int(masks[0, 2]) == 1 << (4 + 8 * 3)
