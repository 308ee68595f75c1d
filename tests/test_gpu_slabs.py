"""GPU parity of the z-slab partition on one GPU: the library's field of every rank's extended slab
(the slabs transformed one after another, each on its own handle), cut to the owned planes and
stacked, equals the oracle's field of the whole grid bit for bit; sharded_global with a world of
one rank is the plain global transform."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from paper_2105_04419_gb300 import slabs as S

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("shape,world,dmax", [((70, 33, 41), 2, 9), ((131, 40, 37), 3, 24), ((256, 64, 64), 4, 32),
                                              ((72, 17, 19), 9, 5)])
def test_library_slabs_equal_whole(shape, world, dmax):
    import torch
    import paper_2105_04419_gb300 as V
    occ = W.bernoulli_grid(world + dmax, shape, 0.003)
    occ[shape[0] // 3: shape[0] // 3 + 2, :, 5] = 1
    b = S.slab_bounds(shape[0], world, dmax)
    parts = []
    for r in range(world):
        h0, h1 = S.extended_range(b, r, dmax)
        ext = torch.from_numpy(np.ascontiguousarray(occ[h0:h1])).cuda()
        m = V.Map(shape[2], shape[1], h1 - h0, dmax)
        m.set_occupancy_dense(ext)
        m.global_()
        parts.append(S.owned_part(m.export_dense(), b, r, dmax))
        m.close()
    got = np.concatenate(parts, 0)
    ref = O.edt_factorised(occ, dmax)
    assert np.array_equal(got, ref)


def test_sharded_global_single_rank():
    import torch
    occ = W.bernoulli_grid(3, (40, 24, 32), 0.01)
    d = S.sharded_global(torch.from_numpy(occ).cuda(), 0, 1, occ.shape[0], 12)
    assert np.array_equal(d.cpu().numpy(), O.edt_factorised(occ, 12))
