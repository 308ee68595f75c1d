"""GPU parity of the global transform against the CPU oracle (bit-exact int32), through the C ABI.

Covers: the dense 64^3 Bernoulli(0.02) workload at dmax 16 (five seeds); ragged grids that are not
multiples of the 8^3 brick and span several 16^3-brick interior nodes; every dmax class (the half
kernels for dmax <= 45 with brick radius R = 1..6, the lower-envelope kernels above); empty, full,
single-obstacle and corner cases; the dense and the record ingest; every tuning of the work-item
runs; duplicate and clearing records (last record wins); and the counters of the grid.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import coords_of, first_mismatch, gpu_global

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("seed", range(5))
def test_bernoulli64_dmax16(seed):
    occ = W.bernoulli_grid(seed, (64, 64, 64), 0.02)
    ref = O.edt_factorised(occ, 16)
    got = gpu_global(occ, 16).export_dense()
    assert first_mismatch(got, ref) is None, first_mismatch(got, ref)


@pytest.mark.parametrize("dmax", [1, 2, 3, 5, 8, 9, 15, 16, 17, 24, 25, 31, 32, 33, 40, 45])
def test_ragged_half_path(dmax):
    rs = np.random.default_rng(dmax)
    shape = (37, 45, 70)  # nz, ny, nx: none a multiple of 8
    occ = (rs.random(shape) < 0.003).astype(np.uint8)
    ref = O.edt_factorised(occ, dmax)
    got = gpu_global(occ, dmax).export_dense()
    assert first_mismatch(got, ref) is None, first_mismatch(got, ref)


@pytest.mark.parametrize("dmax", [46, 60, 100])
def test_generic_path(dmax):
    rs = np.random.default_rng(dmax)
    shape = (23, 30, 41)
    occ = (rs.random(shape) < 0.0015).astype(np.uint8)
    ref = O.edt_factorised(occ, dmax)
    got = gpu_global(occ, dmax).export_dense()
    assert first_mismatch(got, ref) is None, first_mismatch(got, ref)


def test_generic_path_max_dmax():
    shape = (20, 17, 29)
    occ = np.zeros(shape, np.uint8)
    occ[3, 4, 5] = 1
    occ[19, 16, 28] = 1
    ref = O.edt_factorised(occ, 181)
    got = gpu_global(occ, 181).export_dense()
    assert first_mismatch(got, ref) is None, first_mismatch(got, ref)


def test_multi_node_grid():
    """300 x 140 x 20 voxels: 38 x 18 x 3 bricks, 3 x 2 x 1 interior nodes; sparse shells."""
    occ = W.tunnel_scene(9, (300, 140, 20), ntunnels=5, rmin=3, rmax=6)
    if occ.sum() == 0:
        occ[10, 70, 150] = 1
    for dmax in (6, 20, 32):
        ref = O.edt_factorised(occ, dmax)
        got = gpu_global(occ, dmax).export_dense()
        assert first_mismatch(got, ref) is None, (dmax, first_mismatch(got, ref))


@pytest.mark.parametrize("dense", [False, True])
def test_empty_full_single_corner(dense):
    shape = (19, 26, 33)
    for dmax in (1, 7, 32, 50):
        empty = np.zeros(shape, np.uint8)
        got = gpu_global(empty, dmax, dense=dense).export_dense()
        assert (got == dmax * dmax).all()
    full = np.ones(shape, np.uint8)
    assert (gpu_global(full, 9, dense=dense).export_dense() == 0).all()
    for corner in ((0, 0, 0), (18, 25, 32), (0, 25, 0), (18, 0, 32)):
        occ = np.zeros(shape, np.uint8)
        occ[corner] = 1
        for dmax in (4, 16, 45):
            ref = O.edt_factorised(occ, dmax)
            got = gpu_global(occ, dmax, dense=dense).export_dense()
            assert first_mismatch(got, ref) is None, (corner, dmax, first_mismatch(got, ref))


@pytest.mark.parametrize("runs", [(4, 4, 4), (16, 4, 16), (8, 8, 8), (4, 16, 4), (16, 16, 16)])
@pytest.mark.parametrize("variant", [1, 3, 5, 7])
def test_tunings(runs, variant):
    """Work-item runs and pass variants: 1 full window, 3 window with early exit and skips; 5 and 7
    the same with the x pass on plain loads."""
    x_run, y_run, z_run = runs
    occ = W.bernoulli_grid(3, (48, 80, 72), 0.002)
    ref = O.edt_factorised(occ, 24)
    got = gpu_global(occ, 24, tuning=dict(x_run=x_run, y_run=y_run, z_run=z_run, variant=variant)).export_dense()
    assert first_mismatch(got, ref) is None, first_mismatch(got, ref)


@pytest.mark.parametrize("variant", [1, 3, 7, 8])
@pytest.mark.parametrize("dmax", [2, 12, 20, 28, 36, 44])
def test_variants_every_radius(variant, dmax):
    """Brick radius R = 1..6 for both window variants and the lower-envelope form (8)."""
    rs = np.random.default_rng(100 + dmax)
    occ = (rs.random((44, 57, 66)) < 0.002).astype(np.uint8)
    ref = O.edt_factorised(occ, dmax)
    got = gpu_global(occ, dmax, tuning=dict(variant=variant)).export_dense()
    assert first_mismatch(got, ref) is None, first_mismatch(got, ref)


def test_dense_ingest_matches_records():
    occ = W.bernoulli_grid(4, (40, 50, 60), 0.01)
    a = gpu_global(occ, 12, dense=True).export_dense()
    b = gpu_global(occ, 12, dense=False).export_dense()
    assert np.array_equal(a, b)
    assert np.array_equal(a, O.edt_factorised(occ, 12))


@pytest.mark.parametrize("nx", [200, 520, 1040, 1037])
def test_dense_ingest_row_widths(nx):
    """Row widths for each load form of the dense ingest: 16-byte loads (1040, several chunks of
    64 bricks with a ragged last one), 8-byte loads (200; 520 ends in a lone brick) and byte loads
    (1037); ny and nz ragged."""
    occ = W.bernoulli_grid(nx, (21, 19, nx), 0.01)
    occ[3:9, 0, nx - 5:] = 1
    a = gpu_global(occ, 9, dense=True).export_dense()
    assert np.array_equal(a, gpu_global(occ, 9, dense=False).export_dense())
    assert first_mismatch(a, O.edt_factorised(occ, 9)) is None


def test_duplicates_and_clears_last_record_wins():
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(5)
    shape = (24, 24, 24)
    n = 4000
    xyz = np.stack([rs.integers(0, 24, n)] * 1 + [rs.integers(0, 24, n), rs.integers(0, 24, n)], 1).astype(np.int32)
    xyz = np.concatenate([xyz, xyz[:1500]])  # every one of the first 1500 voxels appears again
    val = rs.integers(0, 2, len(xyz)).astype(np.uint8)
    occ = np.zeros(shape, np.uint8)
    for k in range(len(val)):
        occ[xyz[k, 2], xyz[k, 1], xyz[k, 0]] = val[k]
    m = V.Map(24, 24, 24, 7)
    # stage in three calls: order across calls is record order
    m.set_occupancy(xyz[:1000], val[:1000])
    m.set_occupancy(xyz[1000:3000], val[1000:3000])
    m.set_occupancy(xyz[3000:], val[3000:])
    m.global_()
    got = m.export_dense()
    ref = O.edt_factorised(occ, 7)
    assert first_mismatch(got, ref) is None, first_mismatch(got, ref)


def test_device_records_and_query():
    import torch
    import paper_2105_04419_gb300 as V
    occ = W.bernoulli_grid(6, (33, 34, 35), 0.01)
    xyz = coords_of(occ)
    m = V.Map(35, 34, 33, 10)
    m.set_occupancy(torch.from_numpy(xyz).cuda(), torch.ones(len(xyz), dtype=torch.uint8, device="cuda"))
    m.global_()
    ref = O.edt_factorised(occ, 10)
    rs = np.random.default_rng(0)
    q = np.stack([rs.integers(-3, 38, 5000), rs.integers(-3, 37, 5000), rs.integers(-3, 36, 5000)], 1).astype(np.int32)
    inside = (q[:, 0] < 35) & (q[:, 1] < 34) & (q[:, 2] < 33) & (q >= 0).all(1)
    expect = np.full(len(q), 100, np.int32)
    expect[inside] = ref[q[inside, 2], q[inside, 1], q[inside, 0]]
    assert np.array_equal(m.query(q), expect)
    qd = m.query(torch.from_numpy(q).cuda()).cpu().numpy()
    assert np.array_equal(qd, expect)
    assert np.array_equal(m.export_dense(on_device=True).cpu().numpy(), ref)


def test_invalid_host_records_rejected():
    import paper_2105_04419_gb300 as V
    m = V.Map(16, 16, 16, 4)
    with pytest.raises(V.VdbedtError) as e:
        m.set_occupancy(np.array([[1, 2, 3], [16, 0, 0]], np.int32), np.array([1, 1], np.uint8))
    assert e.value.code == "EINVAL"
    with pytest.raises(V.VdbedtError):
        m.set_occupancy(np.array([[1, 2, 3]], np.int32), np.array([2], np.uint8))
    # the rejected calls staged nothing
    m.global_()
    assert (m.export_dense() == 16).all()


def test_invalid_device_records_reported():
    import torch
    import paper_2105_04419_gb300 as V
    m = V.Map(16, 16, 16, 4)
    xyz = torch.tensor([[1, 2, 3], [99, 0, 0]], dtype=torch.int32, device="cuda")
    m.set_occupancy(xyz, torch.ones(2, dtype=torch.uint8, device="cuda"))
    m.global_()
    with pytest.raises(V.VdbedtError) as e:
        m.synchronize()
    assert e.value.code == "EINVAL"
    m.synchronize()  # reported once
    ref = np.zeros((16, 16, 16), np.uint8)
    ref[3, 2, 1] = 1
    assert np.array_equal(m.export_dense(), O.edt_factorised(ref, 4))


def test_capacity_overflow_reported():
    import paper_2105_04419_gb300 as V
    occ = W.bernoulli_grid(2, (32, 32, 32), 0.05)
    m = V.Map(32, 32, 32, 8, max_bricks=10)
    m.set_occupancy(coords_of(occ), np.ones(int(occ.sum()), np.uint8))
    m.global_()
    with pytest.raises(V.VdbedtError) as e:
        m.synchronize()
    assert e.value.code == "EOVERFLOW"


def test_info_counts():
    occ = W.bernoulli_grid(8, (64, 64, 64), 0.001)
    m = gpu_global(occ, 16)
    info = m.info()
    ob = occ.reshape(8, 8, 8, 8, 8, 8).any(axis=(1, 3, 5))
    assert info["obstacle_bricks"] == int(ob.sum())
    ref = O.edt_factorised(occ, 16)
    fin = (ref < 256).reshape(8, 8, 8, 8, 8, 8).any(axis=(1, 3, 5))
    assert info["finite_bricks"] == int(fin.sum())
    assert info["error_bits"] == 0 and info["R"] == 2


def test_sparse_records_take_the_radix_path():
    """Few records in a large grid (fewer than a quarter of its bricks): brick keys go through the
    LSD radix sort / unique / compaction path; includes duplicates and clears."""
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(21)
    nx, ny, nz = 300, 260, 90  # 38 x 33 x 12 = 15048 bricks
    n = 1500
    xyz = np.stack([rs.integers(0, nx, n), rs.integers(0, ny, n), rs.integers(0, nz, n)], 1).astype(np.int32)
    xyz = np.concatenate([xyz, xyz[:300]])
    val = np.ones(len(xyz), np.uint8)
    val[1500:1400 + 300] = 0  # later clears of earlier sets
    occ = np.zeros((nz, ny, nx), np.uint8)
    for k in range(len(val)):
        occ[xyz[k, 2], xyz[k, 1], xyz[k, 0]] = val[k]
    m = V.Map(nx, ny, nz, 11)
    m.set_occupancy(xyz, val)
    m.global_()
    ref = O.edt_factorised(occ, 11)
    got = m.export_dense()
    assert first_mismatch(got, ref) is None, first_mismatch(got, ref)
    single = np.zeros((nz, ny, nx), np.uint8)
    single[45, 130, 150] = 1
    got = gpu_global(single, 40).export_dense()
    assert first_mismatch(got, O.edt_factorised(single, 40)) is None


def test_pinned_host_records_read_in_place():
    """Page-locked host records are read by the pack kernel in place; results and validation are
    those of pageable records."""
    import torch
    import paper_2105_04419_gb300 as V
    occ = W.bernoulli_grid(11, (40, 44, 52), 0.01)
    xyz = coords_of(occ)
    val = np.ones(len(xyz), np.uint8)
    xyz_p = torch.from_numpy(xyz).pin_memory().numpy()
    val_p = torch.from_numpy(val).pin_memory().numpy()
    m = V.Map(52, 44, 40, 13)
    m.set_occupancy(xyz_p, val_p)
    m.global_()
    assert first_mismatch(m.export_dense(), O.edt_factorised(occ, 13)) is None
    bad = xyz_p.copy()
    bad_p = torch.from_numpy(bad).pin_memory().numpy()
    bad_p[5] = (52, 0, 0)  # outside the grid: the whole call is rejected
    with pytest.raises(V.VdbedtError) as e:
        m.set_occupancy(bad_p, val_p)
    assert e.value.code == "EINVAL"
    m.global_()
    assert first_mismatch(m.export_dense(), O.edt_factorised(occ, 13)) is None


def test_packed_records_match_triples():
    """Records packed in 64 bits (host, pinned host and device) give the same field as the
    (x, y, z) + occ format, for the global transform and an update with clears and repeats."""
    import torch
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(17)
    occ = W.bernoulli_grid(17, (40, 64, 72), 0.01)
    nz, ny, nx = occ.shape
    xyz = coords_of(occ)
    val = np.ones(len(xyz), np.uint8)
    edits = np.stack([rs.integers(0, nx, 500), rs.integers(0, ny, 500), rs.integers(0, nz, 500)], 1).astype(np.int32)
    ev = rs.integers(0, 2, 500).astype(np.uint8)
    ref_maps = []
    for form in ("triples", "host", "pinned", "device"):
        m = V.Map(nx, ny, nz, 20)
        for k, (x, v) in enumerate(((xyz, val), (edits, ev))):
            if form == "triples":
                m.set_occupancy(x, v)
            else:
                p = V.pack_records(x, v)
                if form == "pinned":
                    p = torch.from_numpy(p.view(np.int64)).pin_memory().numpy().view(np.uint64)
                elif form == "device":
                    p = torch.from_numpy(p.view(np.int64)).cuda()
                m.set_occupancy_packed(p)
            if k == 0:
                m.global_()
            else:
                m.update()
        ref_maps.append(m.export_dense())
        m.close()
    for got in ref_maps[1:]:
        assert np.array_equal(got, ref_maps[0])
    for (x, y, z), v in zip(edits, ev):
        occ[z, y, x] = v
    assert first_mismatch(ref_maps[0], O.edt_factorised(occ, 20)) is None


def test_packed_records_outside_the_grid():
    import torch
    import paper_2105_04419_gb300 as V
    m = V.Map(16, 16, 16, 6)
    bad = V.pack_records(np.array([[1, 2, 3], [16, 0, 0]], np.int32), np.array([1, 1], np.uint8))
    with pytest.raises(V.VdbedtError) as e:
        m.set_occupancy_packed(bad)
    assert e.value.code == "EINVAL"
    m.set_occupancy_packed(torch.from_numpy(bad.view(np.int64)).cuda())  # device: skipped, reported later
    m.global_()
    with pytest.raises(V.VdbedtError) as e:
        m.synchronize()
    assert e.value.code == "EINVAL"
    d = m.export_dense()
    assert d[3, 2, 1] == 0 and (d == 0).sum() == 1
