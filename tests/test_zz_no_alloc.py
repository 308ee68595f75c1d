"""The allocation-free entry point (vdbedt_edt_dense_noalloc) against the oracle and the handle path.

Callers that cannot allocate device memory (inside another component's stream capture, in
real-time loops, under a load-time memory budget) use vdbedt_edt_dense_noalloc, whose scratch is a
fixed array of the library.  Its output must equal Eq. 1 truncated at dmax (the oracle's factorised
transform, and its brute force on tiny grids) and what a handle computes (vdbedt_create +
vdbedt_set_occupancy_dense + vdbedt_global + vdbedt_export_dense), bit for bit, on calls in a row
that share that scratch array; the cases cover dmax above 45, the largest grid the array allows
(128^3 = VDBEDT_NOALLOC_MAX_VOXELS voxels), degenerate axes of one voxel, dmax 1 and dmax 181.
This file is collected last.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import first_mismatch

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


def noalloc(occ, dmax, out=None):
    import torch
    import paper_2105_04419_gb300 as V
    got = V.edt_dense_noalloc(torch.from_numpy(np.ascontiguousarray(occ)).cuda(), dmax, out=out)
    torch.cuda.synchronize()
    return got.cpu().numpy()


def test_noalloc_matches_oracle_and_handle_two_calls():
    cases = [(W.bernoulli_grid(11, (64, 80, 96), 0.01), 16),
             (W.bernoulli_grid(12, (40, 70, 50), 0.003), 24)]
    for occ, dmax in cases:  # two calls in a row; the second reuses the scratch of the first
        got = noalloc(occ, dmax)
        ref = O.edt_factorised(occ, dmax)
        assert first_mismatch(got, ref) is None, first_mismatch(got, ref)
        assert np.array_equal(got, handle_result(occ, dmax))


@pytest.mark.parametrize("shape,p,dmax", [
    ((48, 40, 56), 0.0005, 60),     # dmax above 45 (the handle path's int32 kernels)
    ((33, 29, 31), 0.0002, 181),    # the largest dmax: dmax^2 = 32761 near the 16-bit scratch range
    ((128, 128, 128), 0.00003, 20),  # exactly VDBEDT_NOALLOC_MAX_VOXELS voxels
    ((1, 37, 5), 0.05, 1),          # one z-plane, dmax 1: D is 0 or 1
    ((1, 37, 5), 0.05, 7),
    ((9, 1, 1), 0.2, 181),          # one voxel across x and y
    ((5, 1, 300), 0.01, 45),        # the last dmax of the 16-bit handle kernels
])
def test_noalloc_edge_cases(shape, p, dmax):
    occ = W.bernoulli_grid(21 + dmax, shape, p)
    occ.reshape(-1)[len(occ.reshape(-1)) // 2] = 1  # at least one obstacle
    ref = O.edt_factorised(occ, dmax)
    if occ.size <= 20000:
        assert np.array_equal(ref, O.edt_naive(occ, dmax))
    for _ in range(2):
        got = noalloc(occ, dmax)
        assert first_mismatch(got, ref) is None, first_mismatch(got, ref)


def test_noalloc_empty_grid_and_preallocated_output():
    import torch
    occ = np.zeros((7, 9, 11), np.uint8)
    out = torch.full((7, 9, 11), -5, dtype=torch.int32, device="cuda")
    got = noalloc(occ, 13, out=out)
    assert (got == 169).all()  # no obstacle: every voxel saturates at dmax^2
    assert (out.cpu().numpy() == 169).all()  # written in place


def test_noalloc_rejects_bad_arguments():
    import torch
    import paper_2105_04419_gb300 as V
    occ = torch.zeros((129, 128, 128), dtype=torch.uint8, device="cuda")  # one plane over the limit
    with pytest.raises(V.VdbedtError) as e:
        V.edt_dense_noalloc(occ, 8)
    assert e.value.code == "EINVAL"
    small = torch.zeros((4, 5, 6), dtype=torch.uint8, device="cuda")
    for d in (0, 182):
        with pytest.raises(V.VdbedtError) as e:
            V.edt_dense_noalloc(small, d)
        assert e.value.code == "EINVAL"
    with pytest.raises(TypeError):
        V.edt_dense_noalloc(small, 8, out=torch.zeros((4, 5, 6), dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        V.edt_dense_noalloc(small, 8, out=torch.zeros((4, 5, 7), dtype=torch.int32, device="cuda"))
    with pytest.raises(ValueError):
        V.edt_dense_noalloc(small, 8, out=torch.zeros((6, 5, 4), dtype=torch.int32, device="cuda").transpose(0, 2))
    with pytest.raises(TypeError):
        V.edt_dense_noalloc(small.cpu(), 8)
