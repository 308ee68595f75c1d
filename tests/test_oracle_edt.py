"""Pins for the CPU oracle's exact transform (Eq. 1 with truncation at dmax^2, Sec. III).

Every function of ``oracle`` is checked against something other than itself:
closed forms (empty grid, full grid, a single obstacle), an independent library routine
(scipy's exact Euclidean transform, Maurer et al.), brute force on tiny inputs, and invariants
that any exact truncated squared transform satisfies (zero exactly on obstacles, saturation,
sums of three squares, the integer form of 1-Lipschitz, reflection and axis-permutation symmetry).
"""
import numpy as np
import pytest
import scipy.ndimage as nd

import oracle as O
import workloads as W


def scipy_sq_edt(occ, dmax):
    """Squared distance to the nearest occupied voxel from scipy's exact EDT feature transform."""
    if not occ.any():
        return np.full(occ.shape, dmax * dmax, dtype=np.int64)
    _, idx = nd.distance_transform_edt(occ == 0, return_indices=True)
    grid = np.indices(occ.shape)
    sq = ((idx - grid) ** 2).sum(axis=0)
    return np.minimum(sq, dmax * dmax)


def rand_grid(rs, shape, p):
    return (rs.random(shape) < p).astype(np.uint8)


SHAPES = [(1, 1, 1), (1, 1, 9), (3, 1, 7), (5, 6, 7), (9, 4, 13), (16, 16, 16), (11, 23, 6)]


@pytest.mark.parametrize("fn", [O.edt_naive, O.edt_factorised])
@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("dmax", [1, 2, 3, 7, 40])
def test_empty_and_full(fn, shape, dmax):
    empty = np.zeros(shape, np.uint8)
    assert (fn(empty, dmax) == dmax * dmax).all()
    full = np.ones(shape, np.uint8)
    assert (fn(full, dmax) == 0).all()


@pytest.mark.parametrize("fn", [O.edt_naive, O.edt_factorised])
def test_single_obstacle_closed_form(fn):
    rs = np.random.default_rng(1)
    for _ in range(25):
        shape = tuple(int(v) for v in rs.integers(1, 14, 3))
        dmax = int(rs.integers(1, 12))
        o = [int(rs.integers(0, n)) for n in shape]  # (z, y, x)
        occ = np.zeros(shape, np.uint8)
        occ[o[0], o[1], o[2]] = 1
        z, y, x = np.indices(shape)
        expect = np.minimum((x - o[2]) ** 2 + (y - o[1]) ** 2 + (z - o[0]) ** 2, dmax * dmax)
        assert np.array_equal(fn(occ, dmax), expect)


@pytest.mark.parametrize("seed", range(6))
def test_against_scipy_exact_edt(seed):
    rs = np.random.default_rng(100 + seed)
    shape = tuple(int(v) for v in rs.integers(5, 30, 3))
    occ = rand_grid(rs, shape, rs.uniform(0.002, 0.05))
    for dmax in (1, 2, 5, 9, 17, 64):
        ref = scipy_sq_edt(occ, dmax)
        assert np.array_equal(O.edt_factorised(occ, dmax), ref)
        assert np.array_equal(O.edt_naive(occ, dmax), ref)


def test_naive_equals_factorised_many():
    rs = np.random.default_rng(7)
    for _ in range(40):
        shape = tuple(int(v) for v in rs.integers(1, 18, 3))
        dmax = int(rs.integers(1, 20))
        occ = rand_grid(rs, shape, rs.uniform(0.0, 0.2))
        assert np.array_equal(O.edt_naive(occ, dmax), O.edt_factorised(occ, dmax))


def test_exhaustive_tiny_2x2x2():
    """Every one of the 256 occupancy patterns of a 2x2x2 grid, against brute enumeration
    of the (at most 8) obstacles done here with Python integers."""
    pts = [(z, y, x) for z in range(2) for y in range(2) for x in range(2)]
    for mask in range(256):
        occ = np.array([(mask >> i) & 1 for i in range(8)], np.uint8).reshape(2, 2, 2)
        for dmax in (1, 2):
            got = O.edt_factorised(occ, dmax)
            for i, (z, y, x) in enumerate(pts):
                best = dmax * dmax
                for j, (c, b, a) in enumerate(pts):
                    if (mask >> j) & 1:
                        best = min(best, (x - a) ** 2 + (y - b) ** 2 + (z - c) ** 2)
                assert got[z, y, x] == best


def test_edt_at_matches_full():
    rs = np.random.default_rng(3)
    occ = rand_grid(rs, (20, 31, 26), 0.01)
    for dmax in (1, 4, 13):
        full = O.edt_factorised(occ, dmax)
        z, y, x = np.indices(occ.shape)
        xyz = np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.int32)[::7]
        got = O.edt_at(occ, dmax, xyz)
        assert np.array_equal(got, full[xyz[:, 2], xyz[:, 1], xyz[:, 0]])


def three_square_sums(limit):
    ok = np.zeros(limit + 1, bool)
    r = int(np.sqrt(limit)) + 1
    for a in range(r):
        for b in range(a, r):
            for c in range(b, r):
                s = a * a + b * b + c * c
                if s <= limit:
                    ok[s] = True
    return ok


def check_invariants(occ, D, dmax):
    cap = dmax * dmax
    assert D.dtype == np.int32
    # zero exactly on obstacles; saturation
    assert np.array_equal(D == 0, occ != 0)
    assert D.min() >= 0 and D.max() <= cap
    # every unsaturated value is a sum of three squares
    ok = three_square_sums(cap)
    assert ok[D[D < cap]].all()
    # 1-Lipschitz of sqrt(D) between neighbours at squared offset k in {1, 2, 3}, without
    # square roots: for a >= b, sqrt(a) <= sqrt(b) + sqrt(k)  <=>  a - b - k <= 0 or
    # (a - b - k)^2 <= 4 k b.  Saturated values are excluded (truncation caps them).
    Di = D.astype(np.int64)
    for dz in (0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dz, dy, dx) <= (0, 0, 0):
                    continue
                k = dz * dz + dy * dy + dx * dx
                a = Di[max(dz, 0):, max(dy, 0):Di.shape[1] + min(dy, 0), max(dx, 0):Di.shape[2] + min(dx, 0)]
                b = Di[:Di.shape[0] - dz, max(-dy, 0):Di.shape[1] - max(dy, 0), max(-dx, 0):Di.shape[2] - max(dx, 0)]
                hi, lo = np.maximum(a, b), np.minimum(a, b)
                m = hi < cap
                t = hi - lo - k
                assert ((t <= 0) | (t * t <= 4 * k * lo))[m].all()


@pytest.mark.parametrize("seed", range(4))
def test_invariants_and_symmetry(seed):
    rs = np.random.default_rng(200 + seed)
    shape = tuple(int(v) for v in rs.integers(8, 40, 3))
    occ = rand_grid(rs, shape, rs.uniform(0.001, 0.03))
    for dmax in (3, 8, 16):
        D = O.edt_factorised(occ, dmax)
        check_invariants(occ, D, dmax)
        for ax in range(3):
            assert np.array_equal(O.edt_factorised(np.flip(occ, ax).copy(), dmax), np.flip(D, ax))
        for perm in ((1, 0, 2), (2, 1, 0), (0, 2, 1), (1, 2, 0)):
            assert np.array_equal(O.edt_factorised(occ.transpose(perm).copy(), dmax), D.transpose(perm))


def test_bernoulli_64_cube_invariants():
    occ = W.bernoulli_grid(0, (64, 64, 64), 0.02)
    D = O.edt_factorised(occ, 16)
    check_invariants(occ, D, 16)
    assert np.array_equal(D, scipy_sq_edt(occ, 16))


def test_tunnel_slab_against_scipy():
    """A 256 x 256 x 64 corner of the tunnel scene (walls are shells, not random points)."""
    occ = W.tunnel_scene(1, (256, 256, 64), ntunnels=6)
    assert occ.any()
    for dmax in (16, 32):
        assert np.array_equal(O.edt_factorised(occ, dmax), scipy_sq_edt(occ, dmax))
