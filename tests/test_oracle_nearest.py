"""Pins of the oracle's nearest-obstacle query: closed forms on one and two obstacles (including
ties along each axis), the truncation boundary, agreement with Eq. 1 (the squared distance to the
returned obstacle is D wherever D < dmax^2), and with scipy's exact feature transform (same
distance as scipy's nearest feature)."""
import numpy as np
import pytest

import oracle as O


def test_single_obstacle_and_truncation():
    occ = np.zeros((9, 10, 11), np.uint8)
    occ[4, 5, 6] = 1  # (x, y, z) = (6, 5, 4)
    q = np.array([[6, 5, 4], [0, 5, 4], [6, 0, 4], [6, 5, 8], [1, 5, 4], [30, 0, 0]], np.int32)
    got = O.nearest_obstacle(occ, 6, q)
    assert got[0].tolist() == [6, 5, 4]          # an obstacle is its own nearest
    assert got[1].tolist() == [-1, -1, -1]       # distance 6 = dmax: not closer than dmax
    assert got[2].tolist() == [6, 5, 4]          # distance 5
    assert got[3].tolist() == [6, 5, 4]          # distance 4
    assert got[4].tolist() == [6, 5, 4]          # distance 5
    assert got[5].tolist() == [-1, -1, -1]       # outside the grid


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_ties_go_to_the_smallest_zyx(axis):
    occ = np.zeros((11, 11, 11), np.uint8)
    a = [5, 5, 5]
    b = [5, 5, 5]
    a[axis] -= 3
    b[axis] += 3
    occ[tuple(a)] = 1  # index order (z, y, x)
    occ[tuple(b)] = 1
    q = np.array([[5, 5, 5]], np.int32)
    got = O.nearest_obstacle(occ, 10, q)[0]
    assert got.tolist() == [a[2], a[1], a[0]]  # the smaller coordinate along that axis
    # the tie between different axes: smaller z wins before smaller y before smaller x
    occ2 = np.zeros((11, 11, 11), np.uint8)
    occ2[5, 5, 8] = 1  # (x 8, y 5, z 5)
    occ2[5, 8, 5] = 1  # (x 5, y 8, z 5)
    occ2[8, 5, 5] = 1  # (x 5, y 5, z 8)
    assert O.nearest_obstacle(occ2, 10, q)[0].tolist() == [8, 5, 5]  # z 5, then y 5 < 8
    occ2[5, 2, 5] = 1  # (x 5, y 2, z 5): smaller y at the same z
    assert O.nearest_obstacle(occ2, 10, q)[0].tolist() == [5, 2, 5]
    occ2[2, 5, 5] = 1  # (x 5, y 5, z 2): smaller z wins
    assert O.nearest_obstacle(occ2, 10, q)[0].tolist() == [5, 5, 2]


def test_consistent_with_eq1_and_scipy():
    from scipy import ndimage
    rs = np.random.default_rng(4)
    occ = (rs.random((14, 17, 19)) < 0.01).astype(np.uint8)
    dmax = 7
    D = O.edt_naive(occ, dmax)
    nz, ny, nx = occ.shape
    zz, yy, xx = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    q = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1).astype(np.int32)
    got = O.nearest_obstacle(occ, dmax, q)
    Dq = D.ravel()
    none = (got == -1).all(axis=1)
    assert np.array_equal(none, Dq >= dmax * dmax)
    d2 = ((got[~none] - q[~none]).astype(np.int64) ** 2).sum(axis=1)
    assert np.array_equal(d2, Dq[~none])
    assert occ[got[~none, 2], got[~none, 1], got[~none, 0]].all()
    _, ind = ndimage.distance_transform_edt(occ == 0, return_indices=True)
    fz, fy, fx = (ind[k].ravel() for k in range(3))
    d2s = (fx - q[:, 0]) ** 2 + (fy - q[:, 1]) ** 2 + (fz - q[:, 2]) ** 2
    assert np.array_equal(d2s[~none], d2)
