"""The allocation-free entry point (vdbedt_edt_dense_noalloc) against the handle path.

Callers that cannot allocate device memory (inside another component's stream capture, in
real-time loops, under a load-time memory budget) use vdbedt_edt_dense_noalloc, whose scratch is a
fixed array of the library.  Its output must equal what a handle computes (vdbedt_create +
vdbedt_set_occupancy_dense + vdbedt_global + vdbedt_export_dense), bit for bit (the transform is
integer), on two calls in a row that share that scratch array.  This file is collected last.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


def handle_result(occ, dmax):
    import paper_2105_04419_gb300 as V
    nz, ny, nx = occ.shape
    m = V.Map(nx, ny, nz, dmax)
    m.set_occupancy_dense(occ)
    m.global_()
    out = m.export_dense()
    m.close()
    return out


def test_noalloc_matches_handle_two_calls():
    import torch
    import paper_2105_04419_gb300 as V
    cases = [(W.bernoulli_grid(11, (64, 80, 96), 0.01), 16),
             (W.bernoulli_grid(12, (40, 70, 50), 0.003), 24)]
    for occ, dmax in cases:  # two calls in a row; the second reuses the scratch of the first
        got = V.edt_dense_noalloc(torch.from_numpy(occ).cuda(), dmax)
        torch.cuda.synchronize()
        ref = handle_result(occ, dmax)
        assert np.array_equal(got.cpu().numpy(), ref)


def test_noalloc_rejects_oversized_grid():
    import torch
    import paper_2105_04419_gb300 as V
    occ = torch.zeros((129, 128, 128), dtype=torch.uint8, device="cuda")  # one plane over the limit
    with pytest.raises(V.VdbedtError) as e:
        V.edt_dense_noalloc(occ, 8)
    assert e.value.code == "EINVAL"
