"""Pins of the untruncated oracle (Eq. 1 with no truncation, the paper's dmax = infinity runs of
Table II): scipy's exact Euclidean feature transform (Maurer et al.), the single-obstacle closed
form, empty and full grids, and the truncated oracle agreeing wherever it stays below its cap."""
import numpy as np
import pytest
import scipy.ndimage as nd

import oracle as O
import workloads as W


def scipy_sq_untruncated(occ):
    _, idx = nd.distance_transform_edt(occ == 0, return_indices=True)
    grid = np.indices(occ.shape)
    return ((idx - grid) ** 2).sum(axis=0)


@pytest.mark.parametrize("shape", [(1, 1, 1), (1, 1, 9), (3, 1, 7), (9, 4, 13), (11, 23, 6), (20, 17, 33)])
def test_empty_and_full(shape):
    assert (O.edt_untruncated(np.zeros(shape, np.uint8)) == O.NONE).all()
    assert (O.edt_untruncated(np.ones(shape, np.uint8)) == 0).all()


def test_single_obstacle_closed_form():
    rs = np.random.default_rng(3)
    for _ in range(20):
        shape = tuple(int(v) for v in rs.integers(1, 40, 3))
        o = [int(rs.integers(0, n)) for n in shape]  # (z, y, x)
        occ = np.zeros(shape, np.uint8)
        occ[o[0], o[1], o[2]] = 1
        z, y, x = np.indices(shape)
        assert np.array_equal(O.edt_untruncated(occ), (x - o[2]) ** 2 + (y - o[1]) ** 2 + (z - o[0]) ** 2)


@pytest.mark.parametrize("seed", range(5))
def test_against_scipy_exact_edt(seed):
    rs = np.random.default_rng(500 + seed)
    shape = tuple(int(v) for v in rs.integers(5, 48, 3))
    occ = (rs.random(shape) < rs.choice([0.0005, 0.003, 0.02])).astype(np.uint8)
    occ.flat[int(rs.integers(0, occ.size))] = 1
    assert np.array_equal(O.edt_untruncated(occ), scipy_sq_untruncated(occ))


def test_sparse_scene_far_from_walls():
    """A tunnel slab whose empty regions reach tens of voxels: values far above any windowed
    truncation, against scipy."""
    occ = W.tunnel_scene(9, (96, 80, 48), ntunnels=3, rmin=6, rmax=14)
    occ[:, 30:70, 20:80] = 0  # a large empty box
    ref = scipy_sq_untruncated(occ)
    assert ref.max() > 45 * 45 // 4
    assert np.array_equal(O.edt_untruncated(occ), ref)


def test_truncated_oracle_agrees_below_its_cap():
    rs = np.random.default_rng(8)
    occ = (rs.random((30, 31, 29)) < 0.002).astype(np.uint8)
    occ[3, 4, 5] = 1
    U = O.edt_untruncated(occ)
    for dmax in (3, 9, 20):
        T = O.edt_factorised(occ, dmax)
        assert np.array_equal(T, np.minimum(U, dmax * dmax))


def test_sampled_brute_force_equals_field():
    rs = np.random.default_rng(11)
    occ = (rs.random((25, 31, 40)) < 0.003).astype(np.uint8)
    occ[0, 0, 0] = 1
    U = O.edt_untruncated(occ)
    q = np.stack([rs.integers(0, 40, 300), rs.integers(0, 31, 300), rs.integers(0, 25, 300)], 1)
    assert np.array_equal(O.edt_untruncated_at(occ, q), U[q[:, 2], q[:, 1], q[:, 0]])
    assert (O.edt_untruncated_at(np.zeros((3, 4, 5), np.uint8), q[:4] % 3) == O.NONE).all()
