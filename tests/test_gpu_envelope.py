"""GPU parity of the lower-envelope form of the separable passes (Eq. 1 line by line) against the
CPU oracle, bit-exact int32, through the C ABI.

The envelope kernels serve every grid with dmax above 45 and any grid tuned to variant 8.  Covered:
every brick radius class from R = 1 to R = 23 (dmax 181) on ragged grids of several interior
nodes, so that runs of 16 bricks and their halos cross node boundaries and the grid's faces; lines
whose envelope holds many parabolas (dense obstacles) and few (one obstacle); the incremental form
in the envelope kernels; switching a map between the windowed and envelope forms (the next update
recomputes the field); and a batch in the envelope form.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import coords_of, first_mismatch, gpu_global

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("dmax", [1, 2, 9, 17, 31, 45, 46, 53, 64, 90, 128, 150, 181])
def test_envelope_every_radius_multi_node(dmax):
    rs = np.random.default_rng(300 + dmax)
    shape = (37, 141, 150)  # nz, ny, nx: 19 x 18 x 5 bricks, 2 x 2 x 1 nodes, ragged on every axis
    occ = (rs.random(shape) < 0.0004).astype(np.uint8)
    ref = O.edt_factorised(occ, dmax)
    got = gpu_global(occ, dmax, tuning=dict(variant=8)).export_dense()
    assert first_mismatch(got, ref) is None, first_mismatch(got, ref)


@pytest.mark.parametrize("dmax", [20, 64, 181])
def test_envelope_dense_and_single_obstacle(dmax):
    # dense obstacles: many parabolas on every line's envelope; one obstacle: one parabola
    occ = W.bernoulli_grid(dmax, (24, 40, 56), 0.2)
    assert first_mismatch(gpu_global(occ, dmax, tuning=dict(variant=8)).export_dense(),
                          O.edt_factorised(occ, dmax)) is None
    one = np.zeros((30, 33, 35), np.uint8)
    one[29, 0, 17] = 1
    assert first_mismatch(gpu_global(one, dmax, tuning=dict(variant=8)).export_dense(),
                          O.edt_factorised(one, dmax)) is None


def test_envelope_tunnel_scene():
    occ = W.tunnel_scene(4, (256, 192, 64), ntunnels=8, rmin=6, rmax=14)
    for dmax in (32, 70):
        ref = O.edt_factorised(occ, dmax)
        got = gpu_global(occ, dmax, tuning=dict(variant=8), dense=True).export_dense()
        assert first_mismatch(got, ref) is None, (dmax, first_mismatch(got, ref))


@pytest.mark.parametrize("dmax", [16, 60])
def test_envelope_incremental_frames(dmax):
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(dmax)
    nz, ny, nx = 40, 72, 150
    occ = (rs.random((nz, ny, nx)) < 0.001).astype(np.uint8)
    m = V.Map(nx, ny, nz, dmax)
    m.set_tuning(variant=8)
    xyz = coords_of(occ)
    m.set_occupancy(xyz, np.ones(len(xyz), np.uint8))
    m.global_()
    for f in range(4):
        k = 300
        pts = np.stack([rs.integers(0, nx, k), rs.integers(0, ny, k), rs.integers(0, nz, k)], 1).astype(np.int32)
        val = rs.integers(0, 2, k).astype(np.uint8)
        for (x, y, z), v in zip(pts, val):
            occ[z, y, x] = v
        m.set_occupancy(pts, val)
        m.update()
        ref = O.edt_factorised(occ, dmax)
        assert first_mismatch(m.export_dense(), ref) is None, (f, first_mismatch(m.export_dense(), ref))


def test_switching_forms_recomputes():
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(5)
    nz, ny, nx = 30, 50, 60
    occ = (rs.random((nz, ny, nx)) < 0.002).astype(np.uint8)
    m = V.Map(nx, ny, nz, 24)
    xyz = coords_of(occ)
    m.set_occupancy(xyz, np.ones(len(xyz), np.uint8))
    m.global_()
    for variant in (8, 3, 8, 1):
        m.set_tuning(variant=variant)
        pts = np.stack([rs.integers(0, nx, 50), rs.integers(0, ny, 50), rs.integers(0, nz, 50)], 1).astype(np.int32)
        val = rs.integers(0, 2, 50).astype(np.uint8)
        for (x, y, z), v in zip(pts, val):
            occ[z, y, x] = v
        m.set_occupancy(pts, val)
        m.update()
        assert first_mismatch(m.export_dense(), O.edt_factorised(occ, 24)) is None, variant


def test_envelope_batch():
    import paper_2105_04419_gb300 as V
    grids = [W.batched_map(9, i, smin=24, smax=72) for i in range(4)]
    b = V.Batch([(g.shape[2], g.shape[1], g.shape[0]) for g in grids], 24)
    b.set_tuning(variant=8)
    b.set_occupancy_dense(grids)
    b.global_()
    for i, g in enumerate(grids):
        assert first_mismatch(b.maps[i].export_dense(), O.edt_factorised(g, 24)) is None, i
    b.set_tuning(variant=3)
    b.set_occupancy_dense(grids)
    b.global_()
    for i, g in enumerate(grids):
        assert first_mismatch(b.maps[i].export_dense(), O.edt_factorised(g, 24)) is None, i
