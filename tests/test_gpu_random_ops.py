"""Random sequences of the map's operations -- records (set / clear, repeats), packed records,
brick masks, dense grids, reset, global, update (eager or captured), queries -- on small ragged
grids, the field checked against Eq. 1 (the oracle's factorised transform) after every transform:
the staging paths, the incremental bookkeeping and the global-form switch meet in every order
(and an untruncated grid's, against the untruncated oracle)."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import first_mismatch

pytestmark = pytest.mark.gpu


def _apply(occ, xyz, val):
    for (x, y, z), v in zip(xyz, val):
        occ[z, y, x] = v


@pytest.mark.parametrize("seed,shape_xyz,dmax", [(1, (40, 36, 28), 7), (2, (70, 20, 33), 12), (3, (17, 64, 50), 24),
                                                 (4, (33, 33, 33), 3), (5, (29, 41, 23), None),
                                                 (6, (1, 37, 9), None), (7, (45, 1, 40), None)])
def test_random_operation_sequences(seed, shape_xyz, dmax):
    import torch

    import paper_2105_04419_gb300 as V
    rs = np.random.default_rng(seed)
    nx, ny, nz = shape_xyz
    m = V.Map(nx, ny, nz, dmax)
    occ = np.zeros((nz, ny, nx), np.uint8)
    graph = None
    field = (lambda o: O.edt_untruncated(o)) if dmax is None else (lambda o: O.edt_factorised(o, dmax))
    outside = V.D_NONE if dmax is None else dmax * dmax
    for step in range(60):
        op = rs.choice(["records", "records", "packed", "bricks", "dense", "reset", "cluster"])
        if op == "records":
            k = int(rs.integers(1, 400))
            xyz = np.stack([rs.integers(0, nx, k), rs.integers(0, ny, k), rs.integers(0, nz, k)], 1).astype(np.int32)
            val = (rs.random(k) < rs.choice([0.2, 0.5, 0.9])).astype(np.uint8)
            if rs.random() < 0.5:
                m.set_occupancy(xyz, val)
            else:
                m.set_occupancy(torch.from_numpy(xyz).cuda(), torch.from_numpy(val).cuda())
            _apply(occ, xyz, val)
        elif op == "packed":
            k = int(rs.integers(1, 300))
            xyz = np.stack([rs.integers(0, nx, k), rs.integers(0, ny, k), rs.integers(0, nz, k)], 1).astype(np.int32)
            val = rs.integers(0, 2, k).astype(np.uint8)
            m.set_occupancy_packed(V.pack_records(xyz, val))
            _apply(occ, xyz, val)
        elif op == "bricks":
            add = (rs.random(occ.shape) < 0.003).astype(np.uint8)
            bk, mk = V.brick_masks(add)
            if len(bk):
                m.set_occupancy_bricks(bk, mk)
            occ |= add
        elif op == "cluster":  # a dense clump of sets: many bricks at once, sometimes the global form
            x0, y0, z0 = rs.integers(0, nx), rs.integers(0, ny), rs.integers(0, nz)
            sl = (slice(z0, min(nz, z0 + 9)), slice(y0, min(ny, y0 + 9)), slice(x0, min(nx, x0 + 9)))
            blk = (rs.random(occ[sl].shape) < 0.3).astype(np.uint8)
            zz, yy, xx = np.nonzero(blk)
            xyz = np.stack([xx + x0, yy + y0, zz + z0], 1).astype(np.int32)
            if len(xyz):
                m.set_occupancy(xyz, np.ones(len(xyz), np.uint8))
                _apply(occ, xyz, np.ones(len(xyz), np.uint8))
        elif op == "dense":
            occ = W.bernoulli_grid(int(rs.integers(0, 1 << 30)), (nz, ny, nx), float(rs.choice([0.0, 0.002, 0.02])))
            m.set_occupancy_dense(occ)
            graph = None
        else:  # reset
            m.reset()
            occ[:] = 0
            graph = None
        how = rs.choice(["update", "update", "global", "graph", "none"])
        if how == "none" and op not in ("dense", "reset"):
            continue
        if how == "global":
            m.global_()
        elif how == "graph" and op in ("records",):
            # the staged records of this step were applied through the map already: replay an
            # empty frame through a captured update (the graph's own staging)
            if graph is None:
                m.update()  # a field to capture on
                graph = V.UpdateGraph(m, 512)
            k = int(rs.integers(0, 200))
            xyz = np.stack([rs.integers(0, nx, k), rs.integers(0, ny, k), rs.integers(0, nz, k)], 1).astype(np.int32)
            val = rs.integers(0, 2, k).astype(np.uint8)
            m.update()
            graph.run(xyz, val)
            _apply(occ, xyz, val)
        else:
            m.update()
        ref = field(occ)
        got = m.export_dense()
        assert first_mismatch(got, ref) is None, (step, op, how, first_mismatch(got, ref))
        q = np.stack([rs.integers(-2, nx + 2, 64), rs.integers(-2, ny + 2, 64), rs.integers(-2, nz + 2, 64)], 1)
        q = q.astype(np.int32)
        inside = (q >= 0).all(1) & (q[:, 0] < nx) & (q[:, 1] < ny) & (q[:, 2] < nz)
        d = m.query(q)
        assert np.array_equal(d[inside], ref[q[inside, 2], q[inside, 1], q[inside, 0]])
        assert (d[~inside] == outside).all()
    m.close()
