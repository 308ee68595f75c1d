"""GPU parity at the full workload sizes, in the launch configurations the benchmark times.

* The tunnel scene, 1024 x 1024 x 256 voxels, dmax 32: the global transform from device records
  (default tuning) equals the oracle's factorised transform on all 268 million voxels.
* The clearance cost of 8192 trajectories x 128 points in free space on that field: every
  trajectory's cost and gradient within the stated tolerances of the float64 oracle (fed the
  oracle's own field).
* 300 lidar frames on the tunnel scene through the captured update (CUDA graph replay): the whole
  field equals the oracle's transform of the map after frames 100, 200 and 300.
* 96 maps of uneven size (cubes of side 40..504, dmax 24) in one batch: every map equals the
  oracle's transform.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import first_mismatch

pytestmark = pytest.mark.gpu

DIMS = (1024, 1024, 256)
DMAX = 32


@pytest.fixture(scope="module")
def tunnel():
    occ = W.tunnel_scene(1, DIMS)
    ref = O.edt_factorised(occ, DMAX)
    return occ, ref


@pytest.fixture(scope="module")
def tunnel_map(tunnel):
    import torch
    import paper_2105_04419_gb300 as V
    occ, _ = tunnel
    xyz = torch.from_numpy(W.occupied_coords(occ)).cuda()
    m = V.Map(*DIMS, DMAX, voxel_size=0.1)
    m.set_occupancy(xyz, torch.ones(xyz.shape[0], dtype=torch.uint8, device="cuda"))
    m.global_()
    m.synchronize()
    yield m
    m.close()


def test_tunnel_global_whole_field(tunnel, tunnel_map):
    _, ref = tunnel
    got = tunnel_map.export_dense()
    assert first_mismatch(got, ref) is None, first_mismatch(got, ref)


def test_tunnel_clearance_all_trajectories(tunnel, tunnel_map):
    import torch
    import paper_2105_04419_gb300 as V
    occ, ref = tunnel
    T, P, tau, vs = 8192, 128, 1.0, 0.1
    pts_h = W.free_points(11, occ, vs, T * P).reshape(T, P, 3)
    pts = torch.from_numpy(pts_h).cuda().requires_grad_(True)
    cost = V.clearance_cost(tunnel_map, pts, tau)
    cost.sum().backward()
    c_ref, g_ref, d_ref = O.clearance(ref, DMAX, vs, tau, pts_h)
    c = cost.detach().cpu().numpy().astype(np.float64)
    g = pts.grad.cpu().numpy().astype(np.float64)
    assert np.all(np.abs(c - c_ref) <= 1e-4 * np.abs(c_ref) + 1e-6)
    assert np.all(np.abs(g - g_ref) <= 1e-3 * np.abs(g_ref) + 1e-5)
    active = float((d_ref < tau).mean())
    assert 0.05 < active < 0.95  # the hinge is exercised on both sides


def test_lidar_300_frames_graph_replay(tunnel):
    import torch
    import paper_2105_04419_gb300 as V
    occ, _ = tunnel
    _, lines = W.tunnel_lines(1, DIMS)
    seq = W.LidarSequence(occ, 1, lines[0], nframes=300)
    frames = [seq.next() for _ in range(100)]
    m = V.Map(*DIMS, DMAX)
    m.global_()
    g = V.UpdateGraph(m, 262144)
    for block in range(3):
        if block:
            frames = [seq.next() for _ in range(100)]
        for xyz, val in frames:
            g.run(torch.from_numpy(xyz).cuda(), torch.from_numpy(val).cuda())
        ref = O.edt_factorised(seq.map, DMAX)
        got = m.export_dense()
        assert first_mismatch(got, ref) is None, (block, first_mismatch(got, ref))
    m.close()


def test_batched_96_maps():
    import torch
    import paper_2105_04419_gb300 as V
    k, dmax = 96, 24
    grids = [W.batched_map(7, i) for i in range(k)]
    b = V.Batch([(gr.shape[2], gr.shape[1], gr.shape[0]) for gr in grids], dmax)
    b.set_occupancy_dense([torch.from_numpy(gr).cuda() for gr in grids])
    b.global_()
    b.synchronize()
    for i, gr in enumerate(grids):
        got = b.maps[i].export_dense()
        ref = O.edt_factorised(gr, dmax)
        assert first_mismatch(got, ref) is None, (i, gr.shape, first_mismatch(got, ref))
    b.close()
