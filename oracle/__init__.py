"""CPU oracle for the truncated Euclidean distance transform -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` import this
package.  It shares no code with the CUDA library and never imports it.

Functions (each cites the passage it follows; the exact rules are in the C header comment of
``edt_oracle.c``):

* :func:`edt_naive`       -- Eq. 1 written out (every obstacle), truncated at dmax^2 (Sec. III).
* :func:`edt_factorised`  -- Eq. 1 minimised one axis at a time (exact; min distributes over +).
* :func:`edt_at`          -- Eq. 1 at sampled voxels, offsets scanned in increasing length.
* :func:`edt_untruncated` -- Eq. 1 with no truncation (the paper's dmax = infinity runs, Table II):
                            the factorised minimum with a cap beyond every distance in the grid;
                            :func:`edt_untruncated_at` the same at sampled voxels, by brute force.
* :class:`Alg1`           -- the paper's priority-queue raise/lower transform (Alg. 1, Sec. IV-B),
                            global (Lower only, Sec. V-A) and incremental.
* :func:`clearance`       -- the clearance term of Eq. 2 as a squared hinge on a trilinear
                            distance, its sum per trajectory and its gradient, in float64.
* :func:`distance_at`     -- that trilinear distance and its gradient at points (float64).
* :func:`nearest_obstacle` -- the nearest occupied voxel of sampled voxels (the obstacle a cell
                            records with its distance, Sec. IV-B), ties to the smallest (z, y, x).

Arrays are C-ordered ``[nz, ny, nx]``; coordinates are ``(x, y, z)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``edt_oracle.c`` into ``_build/liboracle.so`` with gcc and OpenMP."""
    src = os.path.join(_HERE, "edt_oracle.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", tmp, src])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i32, i64, vp = ctypes.c_int, ctypes.c_int64, ctypes.c_void_p
            lib.oracle_num_threads.restype = i32
            lib.oracle_num_threads.argtypes = [i32]
            for f in (lib.oracle_edt_naive, lib.oracle_edt_factorised):
                f.restype = i32
                f.argtypes = [vp, i32, i32, i32, i32, vp, i32]
            lib.oracle_edt_at.restype = i32
            lib.oracle_edt_at.argtypes = [vp, i32, i32, i32, i32, vp, i64, vp, i32]
            lib.alg1_create.restype = vp
            lib.alg1_create.argtypes = [i32, i32, i32, i32]
            lib.alg1_destroy.argtypes = [vp]
            lib.alg1_global.restype = i32
            lib.alg1_global.argtypes = [vp, vp]
            lib.alg1_update.restype = i32
            lib.alg1_update.argtypes = [vp, vp, vp, i64]
            lib.alg1_read.argtypes = [vp, vp, vp]
            lib.alg1_counters.argtypes = [vp, vp]
            lib.alg1_reset_counters.argtypes = [vp]
            _lib = lib
    return _lib


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads(threads: int = 0) -> int:
    return int(_L().oracle_num_threads(threads))


def edt_naive(occ_zyx: np.ndarray, dmax: int, threads: int = 0) -> np.ndarray:
    """D(v) = min(dmax^2, min over occupied o of |v - o|^2) by direct enumeration (Eq. 1)."""
    occ = _c(occ_zyx, np.uint8)
    nz, ny, nx = occ.shape
    out = np.empty(occ.shape, dtype=np.int32)
    rc = _L().oracle_edt_naive(occ.ctypes.data, nx, ny, nz, int(dmax), out.ctypes.data, threads)
    if rc:
        raise ValueError(f"oracle_edt_naive failed ({rc})")
    return out


def edt_factorised(occ_zyx: np.ndarray, dmax: int, threads: int = 0) -> np.ndarray:
    """Eq. 1 minimised along x, then y, then z, each window |d| < dmax, saturating at dmax^2."""
    occ = _c(occ_zyx, np.uint8)
    nz, ny, nx = occ.shape
    out = np.empty(occ.shape, dtype=np.int32)
    rc = _L().oracle_edt_factorised(occ.ctypes.data, nx, ny, nz, int(dmax), out.ctypes.data, threads)
    if rc:
        raise ValueError(f"oracle_edt_factorised failed ({rc})")
    return out


NONE = 2147483647  # untruncated: no occupied voxel anywhere in the grid


def edt_untruncated(occ_zyx: np.ndarray, threads: int = 0) -> np.ndarray:
    """Eq. 1 without the truncation (the paper's dmax = infinity, Table II): at every voxel the
    squared distance to the nearest occupied voxel anywhere in the grid; NONE at every voxel of a
    grid without one.  Any two voxels lie less than nx + ny + nz apart, so the factorised minimum
    with that cap takes each whole line as its window and no value reaches the cap."""
    occ = np.asarray(occ_zyx)
    if not occ.any():
        return np.full(occ.shape, NONE, dtype=np.int32)
    nz, ny, nx = occ.shape
    return edt_factorised(occ, nx + ny + nz, threads)


def edt_untruncated_at(occ_zyx: np.ndarray, xyz: np.ndarray) -> np.ndarray:
    """Eq. 1 without truncation at the voxels ``xyz`` [m, 3] (x, y, z), written out: the least
    squared distance to every occupied voxel of the grid (brute force); NONE when it holds none."""
    occ = np.asarray(occ_zyx)
    oz, oy, ox = np.nonzero(occ)
    obs = np.stack([ox, oy, oz], 1).astype(np.int32)
    pts = np.asarray(xyz, dtype=np.int32).reshape(-1, 3)
    out = np.full(pts.shape[0], NONE, dtype=np.int64)
    if len(obs):
        for i, p in enumerate(pts):
            d = obs - p  # coordinates below 2^15: every square and sum fits int32
            out[i] = np.min(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2])
    return out.astype(np.int32)


def edt_at(occ_zyx: np.ndarray, dmax: int, xyz: np.ndarray, threads: int = 0) -> np.ndarray:
    """Eq. 1 at the voxels ``xyz`` [m, 3] (x, y, z): the first occupied voxel met when offsets are
    scanned in increasing squared length; dmax^2 when none lies closer."""
    occ = _c(occ_zyx, np.uint8)
    nz, ny, nx = occ.shape
    pts = _c(xyz, np.int32).reshape(-1, 3)
    out = np.empty(pts.shape[0], dtype=np.int32)
    rc = _L().oracle_edt_at(occ.ctypes.data, nx, ny, nz, int(dmax), pts.ctypes.data, pts.shape[0],
                            out.ctypes.data, threads)
    if rc:
        raise ValueError(f"oracle_edt_at failed ({rc})")
    return out


def nearest_obstacle(occ_zyx: np.ndarray, dmax: int, xyz: np.ndarray) -> np.ndarray:
    """The nearest occupied voxel of each query voxel ``xyz`` [m, 3] (x, y, z) -- the obstacle a
    cell keeps beside its distance in the paper's map (Sec. IV-B) -- written out by brute force over
    every occupied voxel: among the occupied o with |v - o|^2 < dmax^2, the one with the least
    |v - o|^2, ties broken by the smallest (z, y, x).  Returns [m, 3] int32 (x, y, z), or
    (-1, -1, -1) when no obstacle lies closer than dmax or v is outside the grid.  Small grids."""
    occ = np.asarray(occ_zyx)
    nz, ny, nx = occ.shape
    oz, oy, ox = np.nonzero(occ)  # C order: sorted by (z, y, x)
    obs = np.stack([ox, oy, oz], 1).astype(np.int64)
    pts = np.asarray(xyz, dtype=np.int64).reshape(-1, 3)
    out = np.full((len(pts), 3), -1, dtype=np.int32)
    if len(obs) == 0:
        return out
    lim = int(dmax) * int(dmax)
    for i, (x, y, z) in enumerate(pts):
        if not (0 <= x < nx and 0 <= y < ny and 0 <= z < nz):
            continue
        d2 = ((obs - np.array([x, y, z])) ** 2).sum(axis=1)
        j = int(np.argmin(d2))  # the first of the minima: the smallest (z, y, x)
        if d2[j] < lim:
            out[i] = obs[j]
    return out


class Alg1:
    """The paper's raise/lower priority-queue transform (Alg. 1), single-threaded like the paper.

    ``global_(occ)`` runs Initialize, SetObstacle on every occupied cell and DistanceTransform
    (Lower only).  ``update(xyz, val)`` reduces a frame's records to net flips (last write wins),
    calls SetObstacle / RemoveObstacle per flip in ascending linear index, then DistanceTransform.
    """

    def __init__(self, shape_zyx, dmax: int):
        nz, ny, nx = shape_zyx
        self.shape = (nz, ny, nx)
        self.dmax = int(dmax)
        self._h = _L().alg1_create(nx, ny, nz, self.dmax)
        if not self._h:
            raise MemoryError("alg1_create failed")

    def close(self):
        if self._h:
            _L().alg1_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def global_(self, occ_zyx: np.ndarray):
        occ = _c(occ_zyx, np.uint8)
        assert occ.shape == self.shape
        _L().alg1_global(self._h, occ.ctypes.data)

    def update(self, xyz: np.ndarray, val: np.ndarray):
        pts = _c(xyz, np.int32).reshape(-1, 3)
        v = _c(val, np.uint8)
        rc = _L().alg1_update(self._h, pts.ctypes.data, v.ctypes.data, pts.shape[0])
        if rc:
            raise ValueError("alg1_update: record out of range")

    def dist(self) -> np.ndarray:
        out = np.empty(self.shape, dtype=np.int32)
        _L().alg1_read(self._h, out.ctypes.data, None)
        return out

    def occupancy(self) -> np.ndarray:
        d = np.empty(self.shape, dtype=np.int32)
        o = np.empty(self.shape, dtype=np.uint8)
        _L().alg1_read(self._h, d.ctypes.data, o.ctypes.data)
        return o

    def counters(self):
        c = np.zeros(3, dtype=np.int64)
        _L().alg1_counters(self._h, c.ctypes.data)
        return dict(lowered=int(c[0]), raised=int(c[1]), inserts=int(c[2]))

    def reset_counters(self):
        _L().alg1_reset_counters(self._h)


def distance_at(D_zyx: np.ndarray, dmax: int, vs: float, pts: np.ndarray):
    """The trilinear distance field of Eq. 2's clearance term and its gradient, in float64: for
    points p [..., 3] (metres, float32), u = p / vs in float32 (the precision in which the GPU picks
    the cell), cell i0 = floor(u) clamped to [0, n - 2], t = u - i0; corner distance
    d_c = vs * sqrt(min(D_c, dmax^2)); d = trilinear interpolation of the eight corners at t; and
    dd/dp = (1 / vs) * grad_t(trilinear) (inside a cell; one-sided at faces by the floor).
    Returns (d [...], grad [..., 3]).  The same interpolation the clearance cost uses."""
    D = np.asarray(D_zyx)
    nz, ny, nx = D.shape
    p32 = np.asarray(pts, dtype=np.float32)
    u32 = p32 / np.float32(vs)
    dims = np.array([nx, ny, nz])
    i0 = np.clip(np.floor(u32).astype(np.int64), 0, dims - 2)
    t = u32.astype(np.float64) - i0
    dc = float(vs) * np.sqrt(np.minimum(D.astype(np.float64), float(dmax) ** 2))
    x0, y0, z0 = i0[..., 0], i0[..., 1], i0[..., 2]
    tx, ty, tz = t[..., 0], t[..., 1], t[..., 2]
    c = {}
    for a in (0, 1):
        for b in (0, 1):
            for e in (0, 1):
                c[a, b, e] = dc[z0 + e, y0 + b, x0 + a]
    wx = (1 - tx, tx)
    wy = (1 - ty, ty)
    wz = (1 - tz, tz)
    d = sum(wx[a] * wy[b] * wz[e] * c[a, b, e] for a in (0, 1) for b in (0, 1) for e in (0, 1))
    gx = sum((c[1, b, e] - c[0, b, e]) * wy[b] * wz[e] for b in (0, 1) for e in (0, 1))
    gy = sum((c[a, 1, e] - c[a, 0, e]) * wx[a] * wz[e] for a in (0, 1) for e in (0, 1))
    gz = sum((c[a, b, 1] - c[a, b, 0]) * wx[a] * wy[b] for a in (0, 1) for b in (0, 1))
    return d, np.stack([gx, gy, gz], axis=-1) / float(vs)


def clearance(D_zyx: np.ndarray, dmax: int, vs: float, tau: float, pts: np.ndarray):
    """Clearance cost of Eq. 2's second term, as a squared hinge, and its gradient (float64).

    For points p [..., P, 3] (metres, float32):
      u = p / vs in float32 (the precision in which the GPU picks the cell), cell i0 = floor(u)
      clamped to [0, n - 2], t = u - i0;
      corner distance d_c = vs * sqrt(min(D_c, dmax^2)) in metres;
      d = trilinear interpolation of the eight corners at t;
      c = max(0, tau - d)^2;  cost = sum of c over the last-but-one axis (the points of a trajectory);
      dc/dp = -2 max(0, tau - d) * (1 / vs) * grad_t(trilinear).
    Returns (cost [...], grad [..., P, 3], d [..., P]).
    """
    D = np.asarray(D_zyx)
    nz, ny, nx = D.shape
    p32 = np.asarray(pts, dtype=np.float32)
    u32 = p32 / np.float32(vs)
    dims = np.array([nx, ny, nz])
    i0 = np.clip(np.floor(u32).astype(np.int64), 0, dims - 2)
    t = u32.astype(np.float64) - i0
    dc = float(vs) * np.sqrt(np.minimum(D.astype(np.float64), float(dmax) ** 2))
    x0, y0, z0 = i0[..., 0], i0[..., 1], i0[..., 2]
    tx, ty, tz = t[..., 0], t[..., 1], t[..., 2]
    c = {}
    for a in (0, 1):
        for b in (0, 1):
            for e in (0, 1):
                c[a, b, e] = dc[z0 + e, y0 + b, x0 + a]
    wx = (1 - tx, tx)
    wy = (1 - ty, ty)
    wz = (1 - tz, tz)
    d = sum(wx[a] * wy[b] * wz[e] * c[a, b, e] for a in (0, 1) for b in (0, 1) for e in (0, 1))
    gx = sum((c[1, b, e] - c[0, b, e]) * wy[b] * wz[e] for b in (0, 1) for e in (0, 1))
    gy = sum((c[a, 1, e] - c[a, 0, e]) * wx[a] * wz[e] for a in (0, 1) for e in (0, 1))
    gz = sum((c[a, b, 1] - c[a, b, 0]) * wx[a] * wy[b] for a in (0, 1) for b in (0, 1))
    h = np.maximum(0.0, float(tau) - d)
    cost = (h * h).sum(axis=-1)
    grad = (-2.0 * h / float(vs))[..., None] * np.stack([gx, gy, gz], axis=-1)
    return cost, grad, d
