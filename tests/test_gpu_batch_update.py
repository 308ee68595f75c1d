"""Batched incremental update (vdbedt_batch_update) against the CPU oracle, bit-exact int32.

Many maps of uneven size, each with its own random edit set per frame (sets, clears, repeated
voxels with the last record winning, maps left without edits), updated together with each step
launched once for the whole batch; after every frame every map equals Eq. 1 of its occupancy
(the oracle's factorised transform).  Also: the per-grid statistics, the launch count (independent
of the number of grids), the update replayed from one CUDA graph, the lower-envelope form (grid by
grid) and a batch whose grids have no field yet.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import first_mismatch

pytestmark = pytest.mark.gpu


def make_batch(k, dmax, seed, smin=24, smax=64, variant=0):
    import paper_2105_04419_gb300 as V
    grids = [W.batched_map(seed, i, smin=smin, smax=smax) for i in range(k)]
    b = V.Batch([(g.shape[2], g.shape[1], g.shape[0]) for g in grids], dmax)
    if variant:
        b.set_tuning(variant=variant)
    b.set_occupancy_dense(grids)
    b.global_()
    return b, grids


def random_edits(rs, occ, n):
    nz, ny, nx = occ.shape
    xyz = np.stack([rs.integers(0, nx, n), rs.integers(0, ny, n), rs.integers(0, nz, n)], 1).astype(np.int32)
    # a third of the records clear an occupied voxel, the rest set or clear at random; some repeat
    occupied = np.argwhere(occ)
    if len(occupied) and n >= 3:
        pick = occupied[rs.integers(0, len(occupied), n // 3)]
        xyz[: n // 3] = pick[:, ::-1]
    val = rs.integers(0, 2, n).astype(np.uint8)
    val[: n // 3] = 0
    if n >= 4:
        xyz[-1] = xyz[0]
        val[-1] = 1 - val[0]
    return xyz, val


def apply(occ, xyz, val):
    before = occ.copy()
    for (x, y, z), v in zip(xyz, val):
        occ[z, y, x] = v
    return int((before != occ).sum())


@pytest.mark.parametrize("dmax", [16, 24])
def test_batch_update_96_maps_every_frame(dmax):
    rs = np.random.default_rng(dmax)
    b, grids = make_batch(96, dmax, seed=dmax)
    occs = [g.copy() for g in grids]
    for frame in range(3):
        flips = []
        for i, m in enumerate(b.maps):
            if i % 7 == frame:  # some maps get no edits this frame
                flips.append(0)
                continue
            xyz, val = random_edits(rs, occs[i], int(rs.integers(1, 400)))
            flips.append(apply(occs[i], xyz, val))
            m.set_occupancy(xyz, val)
        stats = b.update(stats=True)
        for i, m in enumerate(b.maps):
            got = m.export_dense()
            ref = O.edt_factorised(occs[i], dmax)
            assert first_mismatch(got, ref) is None, (frame, i, first_mismatch(got, ref))
            assert stats[i]["net_flips"] == flips[i], (frame, i)
    b.close()


def test_batch_update_launches_do_not_grow_with_grids():
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(3)
    counts = []
    for k in (4, 24):
        b, grids = make_batch(k, 12, seed=5)
        for i, m in enumerate(b.maps):
            xyz, val = random_edits(rs, grids[i], 50)
            m.set_occupancy(xyz, val)
        b.synchronize()
        l0 = V.kernel_launches()
        b.update()
        counts.append(V.kernel_launches() - l0)
        b.close()
    assert counts[0] == counts[1] and counts[0] <= 22, counts


def test_batch_update_graph_replay():
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(11)
    b, grids = make_batch(10, 20, seed=11)
    occs = [g.copy() for g in grids]
    graph = V.BatchUpdateGraph(b, 256)
    for frame in range(3):
        frames = []
        for i in range(len(b.maps)):
            n = int(rs.integers(0, 256))
            xyz, val = random_edits(rs, occs[i], n) if n else (np.zeros((0, 3), np.int32), np.zeros(0, np.uint8))
            apply(occs[i], xyz, val)
            frames.append((xyz, val))
        graph.run(frames)
        for i, m in enumerate(b.maps):
            assert first_mismatch(m.export_dense(), O.edt_factorised(occs[i], 20)) is None, (frame, i)
    del graph
    b.close()


def test_batch_update_envelope_form_and_fresh_batch():
    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(4)
    b, grids = make_batch(6, 50, seed=4)  # dmax 50: the envelope form, grid by grid
    occs = [g.copy() for g in grids]
    for i, m in enumerate(b.maps):
        xyz, val = random_edits(rs, occs[i], 100)
        apply(occs[i], xyz, val)
        m.set_occupancy(xyz, val)
    b.update()
    for i, m in enumerate(b.maps):
        assert first_mismatch(m.export_dense(), O.edt_factorised(occs[i], 50)) is None, i
    b.close()
    # grids without a field yet: the update is a global transform of the batch
    grids = [W.batched_map(8, i, smin=24, smax=48) for i in range(5)]
    b = V.Batch([(g.shape[2], g.shape[1], g.shape[0]) for g in grids], 16)
    b.set_occupancy_dense(grids)
    b.update()
    for i, m in enumerate(b.maps):
        assert first_mismatch(m.export_dense(), O.edt_factorised(grids[i], 16)) is None, i
    b.close()


def test_batch_update_mixed_global_and_incremental_grids():
    """Some grids get edits large enough to switch to the global form, others small ones: the grids
    decide on the device, in the same launches; every grid equals Eq. 1."""
    rs = np.random.default_rng(19)
    b, grids = make_batch(12, 16, seed=19)
    occs = [g.copy() for g in grids]
    for frame in range(2):
        for i, m in enumerate(b.maps):
            big = (i + frame) % 3 == 0
            obs = np.argwhere(occs[i])
            k = max(1, int((0.3 if big else 0.0005) * len(obs)))
            nz, ny, nx = occs[i].shape
            rm = obs[rs.choice(len(obs), k, replace=False)][:, ::-1].astype(np.int32)
            add = np.stack([rs.integers(0, nx, k), rs.integers(0, ny, k), rs.integers(0, nz, k)], 1).astype(np.int32)
            xyz = np.concatenate([rm, add])
            val = np.concatenate([np.zeros(k, np.uint8), np.ones(k, np.uint8)])
            apply(occs[i], xyz, val)
            m.set_occupancy(xyz, val)
        stats = b.update(stats=True)
        assert any(s["global_form"] for s in stats) and not all(s["global_form"] for s in stats)
        for i, m in enumerate(b.maps):
            assert first_mismatch(m.export_dense(), O.edt_factorised(occs[i], 16)) is None, (frame, i)
    b.close()
