"""Seeded synthetic workloads shared by the CPU oracle, the tests and the benchmark.

This module holds no distance-transform arithmetic.  It produces inputs only:

* ``rng`` / ``bernoulli`` -- counter-based SplitMix64 (Steele, Lea, Flood, OOPSLA 2014):
  value(seed, stream, i) = mix(mix(seed * GAMMA + stream) + (i + 1) * GAMMA).
* ``bernoulli_grid``  -- i.i.d. occupancy, the dense random cube of the paper's ablations
  (Sec. V-A) and the 64^3 parity workload.
* ``tunnel_scene``    -- union of spline tunnels whose walls are occupied shells; stands in for
  the paper's subterranean (SubT) dataset, which is not available here (Sec. V-B).
* ``LidarSequence``   -- a moving range sensor that emits per-frame occupancy edits; stands in for
  the paper's online mapping module that feeds the incremental transform (Sec. V-B).
* ``batched_map``     -- random cubes of uneven size with boxes, for the batched form.
* ``free_points``     -- query points in free space for the clearance cost (Eq. 2).

The heavy generators are C (``gen.c``, OpenMP), compiled by :func:`build` with gcc.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "libworkloads.so")
_lock = threading.Lock()
_lib = None

GAMMA = np.uint64(0x9E3779B97F4A7C15)


def build(force: bool = False) -> str:
    """Compile gen.c into ``_build/libworkloads.so`` (gcc, OpenMP, no FP contraction)."""
    src = os.path.join(_HERE, "gen.c")
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fopenmp",
                               "-ffp-contract=off", "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            u64, i32, i64, dbl = ctypes.c_uint64, ctypes.c_int, ctypes.c_int64, ctypes.c_double
            vp = ctypes.c_void_p
            lib.wl_rng.restype = u64
            lib.wl_rng.argtypes = [u64, u64, u64]
            lib.wl_bernoulli.argtypes = [u64, u64, dbl, i64, vp, i32]
            lib.wl_tunnel_nsamples.restype = i32
            lib.wl_tunnel_lines.argtypes = [u64, i32, i32, i32, i32, dbl, dbl, vp, vp]
            lib.wl_tunnels.argtypes = [u64, i32, i32, i32, i32, dbl, dbl, dbl, vp, i32]
            lib.wl_polyline_pose.argtypes = [vp, i32, dbl, vp, vp]
            lib.wl_lidar_frame.restype = i64
            lib.wl_lidar_frame.argtypes = [vp, vp, i32, i32, i32, vp, dbl, i32, i32, dbl, dbl, dbl, u64, i64, dbl,
                                           vp, vp, i64, i32]
            lib.wl_batched_params.argtypes = [u64, i32, i32, i32, dbl, dbl, i32, vp, vp, vp]
            lib.wl_batched_map.argtypes = [u64, i32, i32, i32, dbl, dbl, i32, vp, i32]
            lib.wl_free_points.restype = i64
            lib.wl_free_points.argtypes = [u64, vp, i32, i32, i32, dbl, i64, vp, i32]
            _lib = lib
    return _lib


def _ptr(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


# ----------------------------------------------------------------------------------------------
# random numbers
# ----------------------------------------------------------------------------------------------

def _mix64(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def rng(seed: int, stream: int, idx) -> np.ndarray:
    """SplitMix64 value for (seed, stream, idx); numpy restatement of ``wl_rng``."""
    with np.errstate(over="ignore"):
        base = _mix64(np.asarray([(seed * int(GAMMA) + stream) % 2**64], dtype=np.uint64))[0]
        i = np.asarray(idx, dtype=np.uint64)
        return _mix64(base + (i + np.uint64(1)) * GAMMA)


def bernoulli_threshold(p: float) -> int:
    if p <= 0:
        return 0
    if p >= 1:
        return 2**64 - 1
    return int(p * 2.0**64)


def bernoulli(seed: int, stream: int, p: float, n: int, threads: int = 0) -> np.ndarray:
    out = np.empty(n, dtype=np.uint8)
    _L().wl_bernoulli(seed, stream, float(p), n, _ptr(out), threads)
    return out


def bernoulli_grid(seed: int, shape_zyx, p: float, stream: int = 0) -> np.ndarray:
    """Dense occupancy [nz, ny, nx] (uint8), voxel i occupied iff rng(seed, stream, i) < p*2^64,
    i = x + nx * (y + ny * z)."""
    n = int(np.prod(shape_zyx))
    return bernoulli(seed, stream, p, n).reshape(shape_zyx)


# ----------------------------------------------------------------------------------------------
# tunnel scene
# ----------------------------------------------------------------------------------------------

TUNNEL_DEFAULTS = dict(ntunnels=40, rmin=8.0, rmax=24.0, shell=1.5)


def tunnel_lines(seed: int, dims_xyz, ntunnels=40, rmin=8.0, rmax=24.0):
    """Radii [T] and centre-line samples [T, S, 3] (x, y, z voxel units) of the tunnel scene."""
    lib = _L()
    ns = lib.wl_tunnel_nsamples()
    radii = np.empty(ntunnels, dtype=np.float64)
    centre = np.empty((ntunnels, ns, 3), dtype=np.float64)
    nx, ny, nz = dims_xyz
    lib.wl_tunnel_lines(seed, nx, ny, nz, ntunnels, rmin, rmax, _ptr(radii), _ptr(centre))
    return radii, centre


def tunnel_scene(seed: int, dims_xyz, ntunnels=40, rmin=8.0, rmax=24.0, shell=1.5, threads: int = 0) -> np.ndarray:
    """Dense wall occupancy [nz, ny, nx] (uint8) of the tunnel scene."""
    nx, ny, nz = dims_xyz
    out = np.empty((nz, ny, nx), dtype=np.uint8)
    _L().wl_tunnels(seed, nx, ny, nz, ntunnels, rmin, rmax, shell, _ptr(out), threads)
    return out


def occupied_coords(occ_zyx: np.ndarray) -> np.ndarray:
    """[n, 3] int32 (x, y, z) coordinates of the occupied voxels, in linear-index order."""
    z, y, x = np.nonzero(occ_zyx)
    return np.ascontiguousarray(np.stack([x, y, z], axis=1).astype(np.int32))


# ----------------------------------------------------------------------------------------------
# lidar edit stream
# ----------------------------------------------------------------------------------------------

class LidarSequence:
    """Per-frame occupancy edits from a range sensor moving along tunnel 0's centre line.

    The map starts empty.  Frame f places the sensor at arc-length fraction f / nframes along the
    centre line, yawed along the local tangent, casts nbeams x nazim rays (elevations evenly over
    [elev_lo, elev_hi], azimuths over a full turn, walk limit maxrange voxels) against the
    ground-truth scene and returns the edit records (x, y, z, value) in ray order.  ``map`` tracks
    the occupancy that the records produce (last write wins)."""

    def __init__(self, truth_zyx: np.ndarray, seed: int, centre_line: np.ndarray, nframes: int = 300,
                 nbeams: int = 64, nazim: int = 1024, elev_deg=(-22.5, 22.5), maxrange: float = 400.0,
                 noise_p: float = 0.01, threads: int = 0):
        self.truth = np.ascontiguousarray(truth_zyx, dtype=np.uint8)
        self.map = np.zeros_like(self.truth)
        self.seed, self.nframes = seed, nframes
        self.line = np.ascontiguousarray(centre_line, dtype=np.float64)
        self.nbeams, self.nazim, self.maxrange, self.noise_p = nbeams, nazim, maxrange, noise_p
        self.elev = (math.radians(elev_deg[0]), math.radians(elev_deg[1]))
        self.threads = threads
        self.frame = 0
        self._cap = nbeams * nazim * 4

    def pose(self, f: int):
        pos = np.zeros(3, dtype=np.float64)
        yaw = ctypes.c_double(0.0)
        _L().wl_polyline_pose(_ptr(self.line), self.line.shape[0], f / self.nframes, _ptr(pos), ctypes.byref(yaw))
        return pos, yaw.value

    def next(self):
        """Edit records of the next frame: (xyz [n,3] int32, val [n] uint8)."""
        pos, yaw = self.pose(self.frame)
        nz, ny, nx = self.truth.shape
        while True:
            xyz = np.empty((self._cap, 3), dtype=np.int32)
            val = np.empty(self._cap, dtype=np.uint8)
            n = _L().wl_lidar_frame(_ptr(self.truth), _ptr(self.map), nx, ny, nz, _ptr(pos), yaw, self.nbeams,
                                    self.nazim, self.elev[0], self.elev[1], self.maxrange, self.seed, self.frame,
                                    self.noise_p, _ptr(xyz), _ptr(val), self._cap, self.threads)
            if n >= 0:
                break
            self._cap = int(-n) + 1024
        self.frame += 1
        return xyz[:n].copy(), val[:n].copy()


# ----------------------------------------------------------------------------------------------
# batched maps
# ----------------------------------------------------------------------------------------------

BATCH_DEFAULTS = dict(smin=32, smax=512, pmin=0.01, pmax=0.05, kmax=20)


def batched_params(seed: int, m: int, smin=32, smax=512, pmin=0.01, pmax=0.05, kmax=20):
    s, nb = ctypes.c_int(0), ctypes.c_int(0)
    p = ctypes.c_double(0.0)
    _L().wl_batched_params(seed, m, smin, smax, pmin, pmax, kmax, ctypes.byref(s), ctypes.byref(p), ctypes.byref(nb))
    return s.value, p.value, nb.value


def batched_map(seed: int, m: int, smin=32, smax=512, pmin=0.01, pmax=0.05, kmax=20, threads: int = 0) -> np.ndarray:
    s, _, _ = batched_params(seed, m, smin, smax, pmin, pmax, kmax)
    out = np.empty((s, s, s), dtype=np.uint8)
    _L().wl_batched_map(seed, m, smin, smax, pmin, pmax, kmax, _ptr(out), threads)
    return out


# ----------------------------------------------------------------------------------------------
# query points
# ----------------------------------------------------------------------------------------------

def free_points(seed: int, occ_zyx: np.ndarray, vs: float, n: int, threads: int = 0) -> np.ndarray:
    """[n, 3] float32 points (metres) uniform in the voxel-centre box, nearest voxel free."""
    occ = np.ascontiguousarray(occ_zyx, dtype=np.uint8)
    nz, ny, nx = occ.shape
    out = np.empty((n, 3), dtype=np.float32)
    _L().wl_free_points(seed, _ptr(occ), nx, ny, nz, float(vs), n, _ptr(out), threads)
    return out
