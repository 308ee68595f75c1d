"""GPU parity of the batched global transform: k grids of uneven size whose steps run once for all
of them (vdbedt_batch_*), bit-exact against the oracle on every grid and equal to the single-grid
transform.

Covers: uneven, ragged grids (sizes that are not multiples of 8, grids spanning several interior
nodes) with random occupancy plus solid boxes; host and device dense input; vdbedt_global_batched
over a batch's grids in shuffled order and over independent handles; staged records and
incremental updates on a grid of a batch; dmax above 45 (grid-by-grid fallback); tunings; the
batch form of the paper-sized random maps (scaled down); errors.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import coords_of, first_mismatch, gpu_global

pytestmark = pytest.mark.gpu


def uneven_grids(seed, k, lo=9, hi=150, p=(0.002, 0.03), boxes=4):
    rs = np.random.default_rng(seed)
    grids = []
    for i in range(k):
        nz, ny, nx = (int(v) for v in rs.integers(lo, hi, 3))
        occ = (rs.random((nz, ny, nx)) < rs.uniform(*p)).astype(np.uint8)
        for _ in range(int(rs.integers(0, boxes + 1))):
            a = [int(rs.integers(0, d)) for d in (nz, ny, nx)]
            e = [int(rs.integers(1, max(2, d // 4))) for d in (nz, ny, nx)]
            occ[a[0]:a[0] + e[0], a[1]:a[1] + e[1], a[2]:a[2] + e[2]] = 1
        grids.append(occ)
    return grids


def dims_of(grids):
    return [(g.shape[2], g.shape[1], g.shape[0]) for g in grids]


@pytest.mark.parametrize("dmax", [5, 16, 24, 40])
def test_batch_dense_host_matches_oracle(dmax):
    import paper_2105_04419_gb300 as V
    grids = uneven_grids(dmax, 7)
    b = V.Batch(dims_of(grids), dmax)
    b.set_occupancy_dense(grids)
    b.global_()
    b.synchronize()
    for i, (occ, m) in enumerate(zip(grids, b.maps)):
        got = m.export_dense()
        assert first_mismatch(got, O.edt_factorised(occ, dmax)) is None, (i, occ.shape)
    b.close()


def test_batch_device_input_equals_single_grids():
    import torch
    import paper_2105_04419_gb300 as V
    grids = uneven_grids(3, 9, lo=20, hi=200)
    dmax = 24
    b = V.Batch(dims_of(grids), dmax)
    b.set_occupancy_dense([torch.from_numpy(g).cuda() for g in grids])
    b.global_()
    for i, occ in enumerate(grids):
        single = gpu_global(occ, dmax, dense=True).export_dense()
        got = b.maps[i].export_dense()
        assert np.array_equal(got, single), i
        assert first_mismatch(got, O.edt_factorised(occ, dmax)) is None, i
    # a second round on new occupancy reuses the batch
    grids2 = uneven_grids(4, 9, lo=20, hi=200)
    grids2 = [g[: a.shape[0], : a.shape[1], : a.shape[2]] for g, a in zip(grids2, grids)]
    grids2 = [np.pad(g, [(0, a.shape[d] - g.shape[d]) for d in range(3)]) for g, a in zip(grids2, grids)]
    b.set_occupancy_dense(grids2)
    b.global_()
    for i, occ in enumerate(grids2):
        assert first_mismatch(b.maps[i].export_dense(), O.edt_factorised(occ, dmax)) is None, i


def test_global_batched_handles():
    import paper_2105_04419_gb300 as V
    grids = uneven_grids(5, 5)
    dmax = 12
    b = V.Batch(dims_of(grids), dmax)
    b.set_occupancy_dense(grids)
    order = [3, 0, 4, 1, 2]
    V.global_batched([b.maps[i] for i in order])  # the whole batch: one launch per step
    for i, occ in enumerate(grids):
        assert first_mismatch(b.maps[i].export_dense(), O.edt_factorised(occ, dmax)) is None, i
    # independent handles: grid by grid
    maps = []
    for occ in grids:
        nz, ny, nx = occ.shape
        m = V.Map(nx, ny, nz, dmax)
        m.set_occupancy_dense(occ)
        maps.append(m)
    V.global_batched(maps)
    for i, occ in enumerate(grids):
        assert np.array_equal(maps[i].export_dense(), b.maps[i].export_dense()), i


def test_records_and_updates_on_batch_grids():
    import paper_2105_04419_gb300 as V
    grids = uneven_grids(6, 4, lo=30, hi=120, p=(0.001, 0.004), boxes=1)
    dmax = 16
    b = V.Batch(dims_of(grids), dmax)
    # grid 1 by records, the others dense; then one batched transform
    b.set_occupancy_dense(grids)
    rs = np.random.default_rng(0)
    occs = [g.copy() for g in grids]
    nz, ny, nx = occs[1].shape
    xyz = np.stack([rs.integers(0, nx, 300), rs.integers(0, ny, 300), rs.integers(0, nz, 300)], 1).astype(np.int32)
    val = rs.integers(0, 2, 300).astype(np.uint8)
    for r in range(300):
        occs[1][xyz[r, 2], xyz[r, 1], xyz[r, 0]] = val[r]
    b.maps[1].set_occupancy(xyz, val)
    b.global_()
    for i, occ in enumerate(occs):
        assert first_mismatch(b.maps[i].export_dense(), O.edt_factorised(occ, dmax)) is None, i
    # incremental updates on single grids of the batch
    for i in (0, 3, 2):
        nz, ny, nx = occs[i].shape
        xyz = np.stack([rs.integers(0, nx, 200), rs.integers(0, ny, 200), rs.integers(0, nz, 200)], 1).astype(np.int32)
        val = rs.integers(0, 2, 200).astype(np.uint8)
        for r in range(200):
            occs[i][xyz[r, 2], xyz[r, 1], xyz[r, 0]] = val[r]
        b.maps[i].set_occupancy(xyz, val)
        st = b.maps[i].update(stats=True)
        assert st["records"] == 200
        for j, occ in enumerate(occs):
            assert first_mismatch(b.maps[j].export_dense(), O.edt_factorised(occ, dmax)) is None, (i, j)
    # a single-grid global on one grid of the batch
    b.maps[2].global_()
    assert first_mismatch(b.maps[2].export_dense(), O.edt_factorised(occs[2], dmax)) is None
    # query through a batch grid
    q = coords_of(occs[3])[:50]
    assert (b.maps[3].query(q) == 0).all()


def test_batch_generic_dmax():
    import paper_2105_04419_gb300 as V
    grids = uneven_grids(8, 3, lo=15, hi=60, p=(0.0005, 0.002), boxes=0)
    dmax = 60
    b = V.Batch(dims_of(grids), dmax)
    b.set_occupancy_dense(grids)
    b.global_()
    for i, occ in enumerate(grids):
        assert first_mismatch(b.maps[i].export_dense(), O.edt_factorised(occ, dmax)) is None, i


@pytest.mark.parametrize("tuning", [dict(x_run=8, y_run=16, z_run=4, variant=1), dict(x_run=16, y_run=8, z_run=16)])
def test_batch_tunings(tuning):
    import paper_2105_04419_gb300 as V
    grids = uneven_grids(9, 6)
    dmax = 20
    b = V.Batch(dims_of(grids), dmax)
    b.set_tuning(**tuning)
    b.set_occupancy_dense(grids)
    b.set_profiling(True)
    b.global_()
    pt = b.phase_times()
    assert pt["z_ms"] > 0 and pt["x_ms"] > 0
    for i, occ in enumerate(grids):
        assert first_mismatch(b.maps[i].export_dense(), O.edt_factorised(occ, dmax)) is None, i


def test_batched_random_maps_scaled():
    """The batched workload's generator (log-uniform cube sides, Bernoulli density, solid boxes) at
    sides 32..96: every map against the oracle."""
    import paper_2105_04419_gb300 as V
    k = 12
    grids = [W.batched_map(7, i, smin=32, smax=96) for i in range(k)]
    dmax = 24
    b = V.Batch(dims_of(grids), dmax)
    b.set_occupancy_dense(grids)
    b.global_()
    for i, occ in enumerate(grids):
        assert first_mismatch(b.maps[i].export_dense(), O.edt_factorised(occ, dmax)) is None, i


def test_batch_errors():
    import paper_2105_04419_gb300 as V
    from paper_2105_04419_gb300 import lib as L
    import ctypes
    lib = L.load()
    cfgs = (L.Config * 2)(L.Config(16, 16, 16, 4, 0.1, 0, None, 0, 0), L.Config(16, 16, 16, 5, 0.1, 0, None, 0, 0))
    bh = ctypes.c_void_p()
    assert lib.vdbedt_batch_create(cfgs, 2, ctypes.byref(bh)) == 1  # dmax differs
    assert lib.vdbedt_batch_create(cfgs, 0, ctypes.byref(bh)) == 1
    b = V.Batch([(16, 16, 16), (24, 8, 40)], 4)
    assert lib.vdbedt_destroy(b.maps[0].handle) == 1  # owned by the batch
    b.close()
