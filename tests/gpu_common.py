"""Helpers for the GPU parity tests (imported by tests only)."""
import numpy as np


def coords_of(occ_zyx):
    z, y, x = np.nonzero(occ_zyx)
    return np.ascontiguousarray(np.stack([x, y, z], 1).astype(np.int32))


def gpu_global(occ_zyx, dmax, tuning=None, dense=False, vs=0.1):
    import paper_2105_04419_gb300 as V
    nz, ny, nx = occ_zyx.shape
    m = V.Map(nx, ny, nz, dmax, voxel_size=vs)
    if tuning:
        m.set_tuning(**tuning)
    if dense:
        m.set_occupancy_dense(np.ascontiguousarray(occ_zyx, dtype=np.uint8))
    else:
        xyz = coords_of(occ_zyx)
        if len(xyz):
            m.set_occupancy(xyz, np.ones(len(xyz), np.uint8))
    m.global_()
    return m


def first_mismatch(a, b):
    bad = np.argwhere(a != b)
    if len(bad) == 0:
        return None
    z, y, x = bad[0]
    return f"{len(bad)} mismatches; first at (x={x}, y={y}, z={z}): gpu {a[z, y, x]} oracle {b[z, y, x]}"
