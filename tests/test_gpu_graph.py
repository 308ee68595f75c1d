"""GPU parity of the incremental transform in its captured form: records staged with a device-side
count (vdbedt_set_occupancy_counted) and the update replayed from a CUDA graph give, after every
frame, the oracle's exact transform of the resulting occupancy, bit for bit -- the same as the
plain staging call followed by vdbedt_update.

Frames: the lidar sequence on a small tunnel scene (starting from an empty map, frames of
different sizes, an empty frame), and random set / clear records on a ragged grid.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import coords_of, first_mismatch

pytestmark = pytest.mark.gpu


def lidar_frames(nframes=10):
    dims = (160, 144, 64)
    truth = W.tunnel_scene(4, dims, ntunnels=4, rmin=6, rmax=10)
    _, lines = W.tunnel_lines(4, dims, ntunnels=4, rmin=6, rmax=10)
    seq = W.LidarSequence(truth, 4, lines[0], nframes=nframes, nbeams=16, nazim=256, maxrange=120)
    frames = []
    for _ in range(nframes):
        xyz, val = seq.next()
        frames.append((xyz, val, seq.map.copy()))
    return dims, frames


def test_counted_staging_equals_plain_staging():
    import torch
    import paper_2105_04419_gb300 as V
    dims, frames = lidar_frames(8)
    dmax = 16
    plain = V.Map(*dims, dmax)
    counted = V.Map(*dims, dmax)
    plain.global_()
    counted.global_()
    n_max = max(len(v) for _, v, _ in frames) + 77
    xyz_buf = torch.zeros((n_max, 3), dtype=torch.int32, device="cuda")
    occ_buf = torch.zeros(n_max, dtype=torch.uint8, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int32, device="cuda")
    for f, (xyz, val, occ) in enumerate(frames):
        plain.set_occupancy(xyz, val)
        sp = plain.update(stats=True)
        n = len(val)
        # stale data past the count must be ignored: fill the tail with obstacles
        xyz_buf.zero_()
        occ_buf.fill_(1)
        xyz_buf[:n] = torch.from_numpy(xyz).cuda()
        occ_buf[:n] = torch.from_numpy(val).cuda()
        cnt.fill_(n)
        counted.set_occupancy_counted(xyz_buf, occ_buf, cnt, n_max)
        sc = counted.update(stats=True)
        assert sc["records"] == n and sc["net_flips"] == sp["net_flips"], (f, sc, sp)
        got = counted.export_dense()
        assert np.array_equal(got, plain.export_dense()), f
        assert first_mismatch(got, O.edt_factorised(occ, dmax)) is None, f


@pytest.mark.parametrize("dmax", [16, 32])
def test_graph_replay_lidar_frames(dmax):
    import paper_2105_04419_gb300 as V
    dims, frames = lidar_frames(10)
    m = V.Map(*dims, dmax)
    m.global_()
    n_max = max(len(v) for _, v, _ in frames)
    g = V.UpdateGraph(m, n_max)
    empty = (np.zeros((0, 3), np.int32), np.zeros(0, np.uint8))
    for f, (xyz, val, occ) in enumerate(frames):
        g.run(xyz, val)
        got = m.export_dense()
        assert first_mismatch(got, O.edt_factorised(occ, dmax)) is None, (f, first_mismatch(got, O.edt_factorised(occ, dmax)))
        if f == 4:
            g.run(*empty)  # an empty frame changes nothing
            assert np.array_equal(m.export_dense(), got)
    m.synchronize()


def test_graph_replay_random_records_device_inputs():
    import torch
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(7)
    shape = (29, 54, 61)
    nz, ny, nx = shape
    dmax = 12
    occ = (rs.random(shape) < 0.004).astype(np.uint8)
    m = V.Map(nx, ny, nz, dmax)
    m.set_occupancy_dense(occ)
    m.global_()
    g = V.UpdateGraph(m, 700)
    for f in range(8):
        k = int(rs.integers(1, 400))
        xyz = np.stack([rs.integers(0, nx, k), rs.integers(0, ny, k), rs.integers(0, nz, k)], 1).astype(np.int32)
        occ_xyz = coords_of(occ)
        pick = occ_xyz[rs.integers(0, len(occ_xyz), min(200, len(occ_xyz)))]
        xyz = np.concatenate([xyz, pick])
        val = np.concatenate([rs.integers(0, 2, k), np.zeros(len(pick), np.int64)]).astype(np.uint8)
        for r in range(len(val)):
            occ[xyz[r, 2], xyz[r, 1], xyz[r, 0]] = val[r]
        if f % 3 == 1:
            g.run(torch.from_numpy(xyz).cuda(), torch.from_numpy(val).cuda())
        elif f % 3 == 2:  # the records loaded ahead, then a bare replay
            g.load(xyz, val)
            g.replay()
        else:  # a producer writing the input buffers itself, then a bare replay
            n = len(val)
            with torch.cuda.stream(m.stream):
                g.xyz[:n].copy_(torch.from_numpy(xyz).cuda())
                g.occ[:n].copy_(torch.from_numpy(val).cuda())
                g.count.fill_(n)
            g.replay()
        assert first_mismatch(m.export_dense(), O.edt_factorised(occ, dmax)) is None, f


def test_counted_count_out_of_range_reported():
    import torch
    import paper_2105_04419_gb300 as V
    m = V.Map(16, 16, 16, 4)
    m.global_()
    xyz = torch.tensor([[1, 2, 3], [4, 5, 6], [7, 8, 9]], dtype=torch.int32, device="cuda")
    occ = torch.ones(3, dtype=torch.uint8, device="cuda")
    cnt = torch.tensor([5], dtype=torch.int32, device="cuda")  # above n_max = 3: clamped to 3
    m.set_occupancy_counted(xyz, occ, cnt, 3)
    m.update()
    with pytest.raises(V.VdbedtError) as e:
        m.synchronize()
    assert e.value.code == "EINVAL"
    ref = np.zeros((16, 16, 16), np.uint8)
    ref[3, 2, 1] = ref[6, 5, 4] = ref[9, 8, 7] = 1
    assert np.array_equal(m.export_dense(), O.edt_factorised(ref, 4))
    cnt.fill_(-2)  # below 0: nothing applied
    m.set_occupancy_counted(xyz, torch.zeros(3, dtype=torch.uint8, device="cuda"), cnt, 3)
    m.update()
    with pytest.raises(V.VdbedtError):
        m.synchronize()
    assert np.array_equal(m.export_dense(), O.edt_factorised(ref, 4))


def test_counted_stage_must_be_alone():
    import torch
    import paper_2105_04419_gb300 as V
    m = V.Map(16, 16, 16, 4)
    xyz = torch.tensor([[1, 2, 3]], dtype=torch.int32, device="cuda")
    occ = torch.ones(1, dtype=torch.uint8, device="cuda")
    cnt = torch.ones(1, dtype=torch.int32, device="cuda")
    m.set_occupancy(xyz, occ)
    with pytest.raises(V.VdbedtError) as e:
        m.set_occupancy_counted(xyz, occ, cnt, 1)
    assert e.value.code == "EINVAL"
    m.global_()
    m.set_occupancy_counted(xyz, occ, cnt, 1)
    with pytest.raises(V.VdbedtError):
        m.set_occupancy(xyz, occ)
    m.update()
    ref = np.zeros((16, 16, 16), np.uint8)
    ref[3, 2, 1] = 1
    assert np.array_equal(m.export_dense(), O.edt_factorised(ref, 4))


def test_global_graph_replay():
    import torch
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(12)
    shape = (40, 50, 60)
    nz, ny, nx = shape
    m = V.Map(nx, ny, nz, 14)
    g = V.GlobalGraph(m, 20000)
    for f in range(3):
        occ = (rs.random(shape) < 0.003 * (f + 1)).astype(np.uint8)
        xyz = coords_of(occ)
        g.run(torch.from_numpy(xyz).cuda(), torch.ones(len(xyz), dtype=torch.uint8, device="cuda"))
        assert first_mismatch(m.export_dense(), O.edt_factorised(occ, 14)) is None, f
    # replay with the buffers as they are gives the same field again
    g.replay()
    assert first_mismatch(m.export_dense(), O.edt_factorised(occ, 14)) is None
