"""GPU clearance cost (Eq. 2's clearance term as a squared hinge) against the float64 oracle.

Tolerances (stated): value |gpu - oracle| <= 1e-4 |oracle| + 1e-6; gradient <= 1e-3 |oracle| + 1e-5.
The gradient of the autograd path is also checked against central finite differences (h = 1e-3 m)
of the oracle in float64, away from cell faces and the hinge.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import gpu_global

pytestmark = pytest.mark.gpu

VAL_RTOL, VAL_ATOL = 1e-4, 1e-6
GRAD_RTOL, GRAD_ATOL = 1e-3, 1e-5


def setup_field(seed=3, shape=(40, 48, 56), p=0.004, dmax=12, vs=0.1):
    occ = W.bernoulli_grid(seed, shape, p)
    m = gpu_global(occ, dmax, vs=vs)
    D = O.edt_factorised(occ, dmax)
    return occ, m, D


def test_forward_backward_vs_oracle():
    import torch
    import paper_2105_04419_gb300 as V
    occ, m, D = setup_field()
    vs, tau, T, P = 0.1, 1.0, 64, 128
    pts = W.free_points(7, occ, vs, T * P).reshape(T, P, 3)
    cost_o, grad_o, _ = O.clearance(D, 12, vs, tau, pts)
    pt = torch.from_numpy(pts).cuda().requires_grad_(True)
    cost = V.clearance_cost(m, pt, tau)
    np.testing.assert_allclose(cost.detach().cpu().numpy(), cost_o, rtol=VAL_RTOL, atol=VAL_ATOL)
    w = torch.linspace(0.5, 2.0, T, device="cuda")
    (cost * w).sum().backward()
    grad = pt.grad.cpu().numpy()
    np.testing.assert_allclose(grad, grad_o * w.cpu().numpy()[:, None, None], rtol=GRAD_RTOL, atol=GRAD_ATOL)
    assert (np.abs(grad_o) > 0).any()


def test_boundary_points_and_clamping():
    """Points on the last voxel face and on cell faces (one-sided cell choice, clamped at n-2)."""
    import torch
    import paper_2105_04419_gb300 as V
    occ, m, D = setup_field(seed=4, shape=(16, 17, 18), p=0.02, dmax=6)
    vs, tau = 0.1, 0.35
    nz, ny, nx = occ.shape
    pts = np.array([[0, 0, 0], [(nx - 1) * vs, (ny - 1) * vs, (nz - 1) * vs], [0.5, 0.5, 0.5], [1.0, 0.3, 0.7],
                    [0.25, 1.15, (nz - 1) * vs]], np.float32).reshape(1, -1, 3)
    cost_o, grad_o, _ = O.clearance(D, 6, vs, tau, pts)
    pt = torch.from_numpy(pts).cuda().requires_grad_(True)
    cost = V.clearance_cost(m, pt, tau)
    cost.sum().backward()
    np.testing.assert_allclose(cost.detach().cpu().numpy(), cost_o, rtol=VAL_RTOL, atol=VAL_ATOL)
    np.testing.assert_allclose(pt.grad.cpu().numpy(), grad_o, rtol=GRAD_RTOL, atol=GRAD_ATOL)


def test_gradient_vs_finite_differences():
    """Central differences of the float64 oracle at h = 1e-3 m against the GPU gradient, held to the
    stated gradient tolerance (1e-3 relative, 1e-5 absolute floor where the hinge is inactive).

    The perturbed points are float32 and the cell coordinate u = p / vs is taken in float32 (the
    precision both sides pick the cell in), so the step actually taken in u differs from 2 h / vs by
    up to an ulp of u on each side.  Inside a cell the squared hinge of a trilinear distance is
    exactly quadratic along one axis, so the divided difference over the step actually taken is the
    derivative at its midpoint; dividing by that step (not by 2 h) removes the rounding of the
    perturbation from the comparison."""
    import torch
    import paper_2105_04419_gb300 as V
    occ, m, D = setup_field(seed=5)
    vs, tau, h = 0.1, 1.0, 1e-3
    pts = W.free_points(8, occ, vs, 256).reshape(1, 256, 3)
    pt = torch.from_numpy(pts).cuda().requires_grad_(True)
    V.clearance_cost(m, pt, tau).sum().backward()
    grad = pt.grad.cpu().numpy()[0]
    _, _, d = O.clearance(D, 12, vs, tau, pts)
    u = pts[0].astype(np.float64) / vs
    frac = u - np.floor(u)
    keep = ((frac > 2 * h / vs) & (frac < 1 - 2 * h / vs)).all(1) & (np.abs(tau - d[0]) > 2 * h)
    assert keep.sum() > 100
    fd = np.zeros((keep.sum(), 3))
    vs32 = np.float32(vs)
    for a in range(3):
        e = np.zeros(3)
        e[a] = h
        for j, i in enumerate(np.flatnonzero(keep)):
            pp = (pts[0, i] + e).astype(np.float32)
            pm = (pts[0, i] - e).astype(np.float32)
            cp = O.clearance(D, 12, vs, tau, pp[None, None])[0][0]
            cm = O.clearance(D, 12, vs, tau, pm[None, None])[0][0]
            step = (float(pp[a] / vs32) - float(pm[a] / vs32)) * vs  # metres, as the oracle sees it
            fd[j, a] = (cp - cm) / step
    np.testing.assert_allclose(grad[keep], fd, rtol=GRAD_RTOL, atol=GRAD_ATOL)


def test_distance_and_gradient_at_points():
    """vdbedt_distance_at against the float64 oracle: the trilinear distance within 1e-4 relative
    and its gradient within 1e-3 relative (the stated tolerances), on points in free space, on cell
    faces and at the grid's last face."""
    import torch
    occ, m, D = setup_field(seed=6)
    vs = 0.1
    nz, ny, nx = occ.shape
    pts = W.free_points(9, occ, vs, 2000).reshape(-1, 3)
    extra = np.array([[0, 0, 0], [(nx - 1) * vs, (ny - 1) * vs, (nz - 1) * vs], [1.0, 1.2, 0.5]], np.float32)
    pts = np.concatenate([pts, extra]).astype(np.float32)
    d_o, g_o = O.distance_at(D, 12, vs, pts)
    d, g = m.distance_at(torch.from_numpy(pts).cuda())
    np.testing.assert_allclose(d.cpu().numpy(), d_o, rtol=VAL_RTOL, atol=VAL_ATOL)
    np.testing.assert_allclose(g.cpu().numpy(), g_o, rtol=GRAD_RTOL, atol=GRAD_ATOL)
    assert np.abs(g_o).max() > 0.5
