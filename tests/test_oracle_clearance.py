"""Pins for the float64 clearance-cost oracle (Eq. 2's clearance term as a squared hinge).

* closed form: obstacles on the plane x = 0 give D = x^2, so d = vs * x is linear and trilinear
  interpolation reproduces it exactly; cost and gradient then have closed forms in p_x;
* the same along y and z (catches transposed axes);
* at a voxel centre d = vs * sqrt(D) of that voxel;
* the analytic gradient against central finite differences (h = 1e-3 m) of the oracle's value
  on a real transform, away from cell faces and hinge kinks.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W


def plane_field(axis, shape=(12, 13, 14), dmax=8):
    occ = np.zeros(shape, np.uint8)
    sl = [slice(None)] * 3
    sl[2 - axis] = 0  # axis 0 = x is array axis 2
    occ[tuple(sl)] = 1
    return occ, O.edt_factorised(occ, dmax)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_plane_closed_form(axis):
    vs, tau, dmax = 0.1, 0.45, 8
    occ, D = plane_field(axis, dmax=dmax)
    rs = np.random.default_rng(axis)
    nz, ny, nx = D.shape
    hi = np.array([nx - 1, ny - 1, nz - 1]) * vs
    pts = (rs.random((5, 40, 3)) * hi).astype(np.float32)
    pts[..., axis] = np.minimum(pts[..., axis], np.float32((dmax - 1) * vs))  # stay below truncation
    cost, grad, d = O.clearance(D, dmax, vs, tau, pts)
    q = pts[..., axis].astype(np.float64)
    np.testing.assert_allclose(d, q, rtol=0, atol=1e-6)
    h = np.maximum(0.0, tau - q)
    np.testing.assert_allclose(cost, (h * h).sum(-1), rtol=1e-6, atol=1e-7)  # u is taken in float32
    expect = np.zeros_like(grad)
    expect[..., axis] = -2.0 * h
    np.testing.assert_allclose(grad, expect, rtol=1e-6, atol=1e-6)


def test_voxel_centres():
    occ = W.bernoulli_grid(5, (10, 11, 12), 0.03)
    dmax, vs = 5, 0.2
    D = O.edt_factorised(occ, dmax)
    rs = np.random.default_rng(0)
    ijk = np.stack([rs.integers(0, 11, 50), rs.integers(0, 10, 50), rs.integers(0, 9, 50)], 1)
    pts = (ijk * vs).astype(np.float32)[None]
    _, _, d = O.clearance(D, dmax, vs, 1.0, pts)
    ref = vs * np.sqrt(D[ijk[:, 2], ijk[:, 1], ijk[:, 0]].astype(np.float64))
    np.testing.assert_allclose(d[0], ref, rtol=1e-6, atol=1e-6)


def test_gradient_vs_central_differences():
    occ = W.bernoulli_grid(9, (24, 24, 24), 0.01)
    dmax, vs, tau, h = 8, 0.1, 0.5, 1e-3
    D = O.edt_factorised(occ, dmax)
    pts = W.free_points(3, occ, vs, 400).reshape(1, 400, 3)
    _, grad, d = O.clearance(D, dmax, vs, tau, pts)
    u = pts[0].astype(np.float64) / vs
    frac = u - np.floor(u)
    keep = ((frac > 2 * h / vs) & (frac < 1 - 2 * h / vs)).all(1) & (np.abs(tau - d[0]) > 2 * h)
    assert keep.sum() > 100
    vs32 = np.float32(vs)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        # central differences in float64 on the oracle's own value, point by point; the points are
        # float32 and u = p / vs is taken in float32, so the quotient divides by the step actually
        # taken in u (the squared hinge of a trilinear distance is exactly quadratic along one axis
        # inside a cell, so that quotient is the derivative at the step's midpoint)
        idx = np.flatnonzero(keep)
        pp = [(pts[0, i] + e).astype(np.float32) for i in idx]
        pm = [(pts[0, i] - e).astype(np.float32) for i in idx]
        cp = np.array([O.clearance(D, dmax, vs, tau, q[None, None])[0][0] for q in pp])
        cm = np.array([O.clearance(D, dmax, vs, tau, q[None, None])[0][0] for q in pm])
        step = np.array([(float(q[a] / vs32) - float(r[a] / vs32)) * vs for q, r in zip(pp, pm)])
        fd = (cp - cm) / step
        an = grad[0, keep, a]
        np.testing.assert_allclose(an, fd, rtol=1e-3, atol=1e-5)


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_distance_at_plane_closed_form(axis):
    """Obstacles on the plane (axis) = 0: d = vs * coordinate along the axis (linear, so trilinear
    interpolation reproduces it exactly) and its gradient is the axis' unit vector."""
    vs, dmax = 0.1, 8
    occ, D = plane_field(axis, dmax=dmax)
    rs = np.random.default_rng(10 + axis)
    nz, ny, nx = D.shape
    hi = np.array([nx - 1, ny - 1, nz - 1]) * vs
    pts = (rs.random((300, 3)) * hi).astype(np.float32)
    pts[:, axis] = np.minimum(pts[:, axis], np.float32((dmax - 1) * vs))
    d, g = O.distance_at(D, dmax, vs, pts)
    np.testing.assert_allclose(d, pts[:, axis].astype(np.float64), rtol=0, atol=1e-6)
    expect = np.zeros_like(g)
    expect[:, axis] = 1.0
    np.testing.assert_allclose(g, expect, rtol=0, atol=1e-9)


def test_distance_at_matches_clearance_and_differences():
    """distance_at's d is the clearance's d; its gradient matches central differences divided by
    the step taken in the float32 cell coordinate (exact for a trilinear function inside a cell)."""
    occ = W.bernoulli_grid(21, (20, 22, 24), 0.01)
    dmax, vs, h = 8, 0.1, 1e-3
    D = O.edt_factorised(occ, dmax)
    pts = W.free_points(5, occ, vs, 300)
    d, g = O.distance_at(D, dmax, vs, pts)
    _, _, dc = O.clearance(D, dmax, vs, 10.0, pts[None])
    np.testing.assert_allclose(d, dc[0], rtol=0, atol=1e-12)
    u = pts.astype(np.float64) / vs
    frac = u - np.floor(u)
    keep = ((frac > 2 * h / vs) & (frac < 1 - 2 * h / vs)).all(1)
    vs32 = np.float32(vs)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        for i in np.flatnonzero(keep):
            pp = (pts[i] + e).astype(np.float32)
            pm = (pts[i] - e).astype(np.float32)
            step = (float(pp[a] / vs32) - float(pm[a] / vs32)) * vs
            fd = (O.distance_at(D, dmax, vs, pp[None])[0][0] - O.distance_at(D, dmax, vs, pm[None])[0][0]) / step
            assert abs(fd - g[i, a]) <= 1e-6 * max(1.0, abs(g[i, a])), (i, a, fd, g[i, a])
