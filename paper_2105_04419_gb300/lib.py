"""ctypes binding of libvdbedt (see include/vdbedt.h for the contract of each call)."""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "libvdbedt.so")
_lock = threading.Lock()
_lib = None

VDBEDT_DMAX_LIMIT = 181

STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ETIMEOUT", 5: "EOVERFLOW", 6: "EINTERNAL"}


class VdbedtError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {STATUS.get(status, status)}: {msg}")
        self.status = status
        self.code = STATUS.get(status, str(status))


class Config(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32), ("dmax", ctypes.c_int32),
                ("voxel_size", ctypes.c_float), ("device", ctypes.c_int32), ("stream", ctypes.c_void_p),
                ("flags", ctypes.c_uint32), ("max_bricks", ctypes.c_int64), ("max_nodes", ctypes.c_int64)]


class Info(ctypes.Structure):
    _fields_ = [("allocated_bricks", ctypes.c_int64), ("obstacle_bricks", ctypes.c_int64),
                ("finite_bricks", ctypes.c_int64), ("capacity_bricks", ctypes.c_int64), ("nodes", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64), ("R", ctypes.c_int32), ("error_bits", ctypes.c_int32)]


class UpdateStats(ctypes.Structure):
    _fields_ = [("records", ctypes.c_int64), ("net_flips", ctypes.c_int64), ("changed_bricks", ctypes.c_int64),
                ("x_items", ctypes.c_int64), ("y_items", ctypes.c_int64), ("z_items", ctypes.c_int64),
                ("new_bricks", ctypes.c_int64), ("x_bricks", ctypes.c_int64), ("y_bricks", ctypes.c_int64),
                ("z_bricks", ctypes.c_int64), ("global_form", ctypes.c_int64)]


class PhaseTimes(ctypes.Structure):
    _fields_ = [("ingest_ms", ctypes.c_float), ("activation_ms", ctypes.c_float), ("items_ms", ctypes.c_float),
                ("x_ms", ctypes.c_float), ("y_ms", ctypes.c_float), ("z_ms", ctypes.c_float)]


class Tuning(ctypes.Structure):
    _fields_ = [("x_run", ctypes.c_int32), ("y_run", ctypes.c_int32), ("z_run", ctypes.c_int32),
                ("variant", ctypes.c_int32)]


# C name -> (restype, argtypes)
_H, _P, _I64, _I32, _F = ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_float
SIGNATURES = {
    "vdbedt_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.POINTER(ctypes.c_void_p)]),
    "vdbedt_destroy": (ctypes.c_int, [_H]),
    "vdbedt_set_occupancy": (ctypes.c_int, [_H, _P, _P, _I64, ctypes.c_int]),
    "vdbedt_set_occupancy_counted": (ctypes.c_int, [_H, _P, _P, _P, _I64]),
    "vdbedt_set_occupancy_packed": (ctypes.c_int, [_H, _P, _I64, ctypes.c_int]),
    "vdbedt_set_occupancy_bricks": (ctypes.c_int, [_H, _P, _P, _I64, ctypes.c_int]),
    "vdbedt_set_occupancy_dense": (ctypes.c_int, [_H, _P, ctypes.c_int]),
    "vdbedt_reset": (ctypes.c_int, [_H]),
    "vdbedt_global": (ctypes.c_int, [_H]),
    "vdbedt_update": (ctypes.c_int, [_H, ctypes.POINTER(UpdateStats)]),
    "vdbedt_query": (ctypes.c_int, [_H, _P, _I64, _P, ctypes.c_int]),
    "vdbedt_query_nearest": (ctypes.c_int, [_H, _P, _I64, _P, ctypes.c_int]),
    "vdbedt_export_dense": (ctypes.c_int, [_H, _P, ctypes.c_int]),
    "vdbedt_export_occupancy": (ctypes.c_int, [_H, _I32, _I32, _I32, _I32, _P, _I64, ctypes.POINTER(ctypes.c_int64)]),
    "vdbedt_clearance_forward": (ctypes.c_int, [_H, _P, _I64, _I64, _F, _P]),
    "vdbedt_distance_at": (ctypes.c_int, [_H, _P, _I64, _P, _P]),
    "vdbedt_clearance_backward": (ctypes.c_int, [_H, _P, _I64, _I64, _F, _P, _P]),
    "vdbedt_global_batched": (ctypes.c_int, [ctypes.POINTER(ctypes.c_void_p), _I32]),
    "vdbedt_batch_create": (ctypes.c_int, [ctypes.POINTER(Config), _I32, ctypes.POINTER(ctypes.c_void_p)]),
    "vdbedt_batch_destroy": (ctypes.c_int, [_H]),
    "vdbedt_batch_map": (ctypes.c_int, [_H, _I32, ctypes.POINTER(ctypes.c_void_p)]),
    "vdbedt_batch_set_occupancy_dense": (ctypes.c_int, [_H, ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]),
    "vdbedt_batch_global": (ctypes.c_int, [_H]),
    "vdbedt_batch_update": (ctypes.c_int, [_H, ctypes.POINTER(UpdateStats)]),
    "vdbedt_batch_set_tuning": (ctypes.c_int, [_H, ctypes.POINTER(Tuning)]),
    "vdbedt_batch_synchronize": (ctypes.c_int, [_H]),
    "vdbedt_batch_set_profiling": (ctypes.c_int, [_H, ctypes.c_int]),
    "vdbedt_batch_get_phase_times": (ctypes.c_int, [_H, ctypes.POINTER(PhaseTimes)]),
    "vdbedt_batch_last_error": (ctypes.c_char_p, [_H]),
    "vdbedt_set_tuning": (ctypes.c_int, [_H, ctypes.POINTER(Tuning)]),
    "vdbedt_synchronize": (ctypes.c_int, [_H]),
    "vdbedt_get_info": (ctypes.c_int, [_H, ctypes.POINTER(Info)]),
    "vdbedt_stream": (ctypes.c_void_p, [_H]),
    "vdbedt_set_profiling": (ctypes.c_int, [_H, ctypes.c_int]),
    "vdbedt_get_phase_times": (ctypes.c_int, [_H, ctypes.POINTER(PhaseTimes)]),
    "vdbedt_kernel_launches": (ctypes.c_int64, []),
    "vdbedt_selftest_wait_timeout": (ctypes.c_int, [_H, _I32]),
    "vdbedt_edt_dense_noalloc": (ctypes.c_int, [_P, _I32, _I32, _I32, _I32, _P, ctypes.c_void_p]),
    "vdbedt_last_error": (ctypes.c_char_p, [_H]),
}


def library_path() -> str:
    return _SO


def load():
    """Load libvdbedt.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_SO):
                raise RuntimeError(f"libvdbedt.so is not built ({_SO}); run paper_2105_04419_gb300.build.build()")
            lib = ctypes.CDLL(_SO)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(lib, name)
                f.restype = res
                f.argtypes = args
            _lib = lib
    return _lib


def _check(status, where, handle=None):
    if status != 0:
        msg = load().vdbedt_last_error(handle)
        raise VdbedtError(status, where, msg.decode() if msg else "")


def _torch():
    import torch
    return torch


def _ptr_host(a: np.ndarray) -> int:
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data


UNBOUNDED_OFFSET = 1 << 20
UNBOUNDED_MIN, UNBOUNDED_MAX = -(1 << 20), (1 << 20) - 128
FLAG_UNBOUNDED, FLAG_UNTRUNCATED = 1, 2
D_NONE = 2147483647  # untruncated grids: no obstacle anywhere (VDBEDT_D_NONE)


def pack_records(xyz, occ, offset: int = 0) -> np.ndarray:
    """Host records (x, y, z) [n, 3] and occ [n] packed as uint64 x | y << 21 | z << 42 | occ << 63
    (coordinates plus `offset`: UNBOUNDED_OFFSET for an unbounded map)."""
    x = np.ascontiguousarray(xyz, dtype=np.int64).reshape(-1, 3) + int(offset)
    o = np.ascontiguousarray(occ, dtype=np.uint64).reshape(-1)
    if x.size and (x.min() < 0 or x.max() >= 1 << 21):
        raise ValueError("coordinates must lie in [0, 2^21)")
    u = x.astype(np.uint64)
    return u[:, 0] | (u[:, 1] << np.uint64(21)) | (u[:, 2] << np.uint64(42)) | ((o & np.uint64(1)) << np.uint64(63))


def brick_masks(occ_zyx, origin_xyz=(0, 0, 0)):
    """The occupied bricks of a dense uint8 grid [nz, ny, nx] whose voxel (0, 0, 0) sits at
    `origin_xyz` (multiples of 8): brick coordinates [n, 3] int32 and their masks [n, 8] uint64
    (plane z of the brick, bit x + 8 y), for Map.set_occupancy_bricks."""
    occ = np.asarray(occ_zyx) != 0
    if any(int(o) % 8 for o in origin_xyz):
        raise ValueError("the origin must be a multiple of 8 on every axis")
    nz, ny, nx = occ.shape
    pz, py, px = -nz % 8, -ny % 8, -nx % 8
    g = np.pad(occ, ((0, pz), (0, py), (0, px)))
    bz, by, bx = g.shape[0] // 8, g.shape[1] // 8, g.shape[2] // 8
    # [bz, z, by, y, bx, x] -> [bz, by, bx, z, y, x]: per brick, plane z, row y, column x
    t = g.reshape(bz, 8, by, 8, bx, 8).transpose(0, 2, 4, 1, 3, 5)
    bits = np.packbits(t.reshape(bz, by, bx, 8, 64), axis=-1, bitorder="little")  # 8 bytes per plane
    words = bits.view(np.uint64).reshape(bz, by, bx, 8)
    keep = words.any(axis=-1)
    iz, iy, ix = np.nonzero(keep)
    o = [int(v) // 8 for v in origin_xyz]
    bxyz = np.stack([ix + o[0], iy + o[1], iz + o[2]], 1).astype(np.int32)
    return bxyz, np.ascontiguousarray(words[keep])


class Map:
    """One sparse distance field (a vdbedt handle) on a CUDA device.

    `max_bricks` and `max_nodes` (0: every brick / node of the grid) cap the storage allocated up
    front, so that a large grid mapped only in part needs memory for the mapped part alone; a
    transform that needs more reports EOVERFLOW.  With `unbounded`, nx, ny, nz are ignored and
    coordinates are signed in [UNBOUNDED_MIN, UNBOUNDED_MAX) on every axis (both capacities are
    then required; no dense entry points).  `dmax=None` (or ``math.inf``) asks for no truncation:
    D is the exact squared distance to the nearest obstacle anywhere in the grid, D_NONE while the
    grid holds none (every brick stored; no batches, tuning or nearest-obstacle query)."""

    def __init__(self, nx: int, ny: int, nz: int, dmax: int, voxel_size: float = 0.1, device: int = 0,
                 stream=None, max_bricks: int = 0, max_nodes: int = 0, unbounded: bool = False, _borrow=None):
        lib = load()
        torch = _torch()
        if _borrow is not None:
            # a grid of a Batch: the batch owns the handle and the stream
            self._h, self.stream, self._owned = _borrow, stream, False
            self.device, self.shape_xyz, self.dmax, self.voxel_size = device, (nx, ny, nz), dmax, voxel_size
            return
        self._owned = True
        untruncated = dmax is None or (isinstance(dmax, float) and math.isinf(dmax))
        if stream is None:
            # a stream of its own: the library would otherwise create one that torch cannot see
            stream = torch.cuda.Stream(device)
        self.device = device
        self.stream = stream
        flags = (FLAG_UNBOUNDED if unbounded else 0) | (FLAG_UNTRUNCATED if untruncated else 0)
        cfg = Config(nx, ny, nz, 0 if untruncated else dmax, voxel_size, device, ctypes.c_void_p(stream.cuda_stream),
                     flags, max_bricks, max_nodes)
        h = ctypes.c_void_p()
        _check(lib.vdbedt_create(ctypes.byref(cfg), ctypes.byref(h)), "vdbedt_create")
        self._h = h
        self.shape_xyz = None if unbounded else (nx, ny, nz)
        self.unbounded = unbounded
        self.untruncated = untruncated
        self.dmax = None if untruncated else dmax
        self.voxel_size = voxel_size

    # -- lifetime --
    def close(self):
        if getattr(self, "_h", None):
            if getattr(self, "_owned", True):
                load().vdbedt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # stream ordering between the caller's current torch stream and the handle's stream
    def _enter(self, *tensors):
        torch = _torch()
        for t in tensors:  # device pointers go to the library: CPU tensors or another GPU's are refused
            if not isinstance(t, torch.Tensor) or not t.is_cuda or t.device.index != self.device:
                where = t.device if isinstance(t, torch.Tensor) else type(t).__name__
                raise ValueError(f"expected a CUDA tensor on cuda:{self.device}, got {where}")
        cur = torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            self.stream.wait_stream(cur)
        for t in tensors:
            t.record_stream(self.stream)

    def _leave(self):
        torch = _torch()
        cur = torch.cuda.current_stream(self.device)
        if cur.cuda_stream != self.stream.cuda_stream:
            cur.wait_stream(self.stream)

    # -- occupancy --
    def set_occupancy(self, xyz, occ):
        """Stage records (x, y, z) -> occ; numpy arrays (host) or CUDA tensors (device)."""
        lib = load()
        if isinstance(xyz, np.ndarray):
            x = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
            o = np.ascontiguousarray(occ, dtype=np.uint8).reshape(-1)
            if x.shape[0] != o.shape[0]:
                raise ValueError(f"{x.shape[0]} coordinates but {o.shape[0]} occupancy values")
            _check(lib.vdbedt_set_occupancy(self._h, _ptr_host(x), _ptr_host(o), x.shape[0], 0),
                   "vdbedt_set_occupancy", self._h)
        else:
            torch = _torch()
            x = xyz.to(torch.int32).contiguous().view(-1, 3)
            o = occ.to(torch.uint8).contiguous().view(-1)
            if x.shape[0] != o.shape[0]:
                raise ValueError(f"{x.shape[0]} coordinates but {o.shape[0]} occupancy values")
            self._enter(x, o)
            _check(lib.vdbedt_set_occupancy(self._h, x.data_ptr(), o.data_ptr(), x.shape[0], 1),
                   "vdbedt_set_occupancy", self._h)

    def set_occupancy_packed(self, rec):
        """Stage records packed as uint64 x | y << 21 | z << 42 | occ << 63 (numpy uint64 on the
        host, or an int64 / uint64 CUDA tensor); see pack_records."""
        lib = load()
        if isinstance(rec, np.ndarray):
            r = np.ascontiguousarray(rec, dtype=np.uint64).reshape(-1)
            _check(lib.vdbedt_set_occupancy_packed(self._h, _ptr_host(r), r.shape[0], 0),
                   "vdbedt_set_occupancy_packed", self._h)
        else:
            r = rec.contiguous().view(-1)
            if r.element_size() != 8 or not r.is_cuda:
                raise TypeError("packed records are 64-bit integers")
            self._enter(r)
            _check(lib.vdbedt_set_occupancy_packed(self._h, r.data_ptr(), r.shape[0], 1),
                   "vdbedt_set_occupancy_packed", self._h)

    def set_occupancy_bricks(self, bxyz, masks):
        """Stage occupied voxels brick by brick: bxyz [n, 3] int32 brick coordinates (voxel // 8),
        masks [n, 8] uint64 (plane z, bit x + 8 y); numpy arrays (host) or CUDA tensors (device).
        One "set" record per bit; see brick_masks."""
        lib = load()
        if isinstance(bxyz, np.ndarray):
            k = np.ascontiguousarray(bxyz, dtype=np.int32).reshape(-1, 3)
            m = np.ascontiguousarray(masks, dtype=np.uint64).reshape(-1, 8)
            if k.shape[0] != m.shape[0]:
                raise ValueError("one 8-word mask per brick")
            _check(lib.vdbedt_set_occupancy_bricks(self._h, _ptr_host(k), _ptr_host(m), k.shape[0], 0),
                   "vdbedt_set_occupancy_bricks", self._h)
        else:
            torch = _torch()
            k = bxyz.to(torch.int32).contiguous().view(-1, 3)
            m = masks.contiguous().view(-1, 8)
            if m.element_size() != 8 or not m.is_cuda or k.shape[0] != m.shape[0]:
                raise TypeError("masks are 64-bit integers, one 8-word mask per brick, on the device")
            self._enter(k, m)
            _check(lib.vdbedt_set_occupancy_bricks(self._h, k.data_ptr(), m.data_ptr(), k.shape[0], 1),
                   "vdbedt_set_occupancy_bricks", self._h)

    def set_occupancy_counted(self, xyz, occ, count, n_max: int):
        """Stage up to n_max device records whose count is the int32 CUDA tensor `count` (read on
        the stream); see UpdateGraph for the captured form."""
        torch = _torch()
        if count.dtype != torch.int32 or xyz.dtype != torch.int32 or occ.dtype != torch.uint8:
            raise TypeError("xyz int32, occ uint8, count int32 (CUDA tensors)")
        if not (xyz.is_contiguous() and occ.is_contiguous()) or xyz.shape[0] < n_max or occ.shape[0] < n_max:
            raise ValueError(f"contiguous xyz [>= {n_max}, 3] and occ [>= {n_max}] needed")
        self._enter(xyz, occ, count)
        _check(load().vdbedt_set_occupancy_counted(self._h, xyz.data_ptr(), occ.data_ptr(), count.data_ptr(),
                                                   int(n_max)), "vdbedt_set_occupancy_counted", self._h)

    def set_occupancy_dense(self, grid):
        lib = load()
        if isinstance(grid, np.ndarray):
            gr = np.ascontiguousarray(grid, dtype=np.uint8)
            _check(lib.vdbedt_set_occupancy_dense(self._h, _ptr_host(gr), 0), "vdbedt_set_occupancy_dense", self._h)
        else:
            torch = _torch()
            gr = grid.to(torch.uint8).contiguous()
            self._enter(gr)
            _check(lib.vdbedt_set_occupancy_dense(self._h, gr.data_ptr(), 1), "vdbedt_set_occupancy_dense", self._h)

    def reset(self):
        _check(load().vdbedt_reset(self._h), "vdbedt_reset", self._h)

    # -- transforms --
    def global_(self):
        _check(load().vdbedt_global(self._h), "vdbedt_global", self._h)

    def update(self, stats: bool = False):
        st = UpdateStats() if stats else None
        _check(load().vdbedt_update(self._h, ctypes.byref(st) if st is not None else None), "vdbedt_update", self._h)
        if st is not None:
            return {k: getattr(st, k) for k, _ in UpdateStats._fields_}
        return None

    def set_tuning(self, x_run: int = 0, y_run: int = 0, z_run: int = 0, variant: int = 0):
        t = Tuning(x_run, y_run, z_run, variant)
        _check(load().vdbedt_set_tuning(self._h, ctypes.byref(t)), "vdbedt_set_tuning", self._h)

    def set_profiling(self, on: bool = True):
        _check(load().vdbedt_set_profiling(self._h, int(on)), "vdbedt_set_profiling", self._h)

    def phase_times(self) -> dict:
        pt = PhaseTimes()
        _check(load().vdbedt_get_phase_times(self._h, ctypes.byref(pt)), "vdbedt_get_phase_times", self._h)
        return {k: getattr(pt, k) for k, _ in PhaseTimes._fields_}

    def synchronize(self):
        _check(load().vdbedt_synchronize(self._h), "vdbedt_synchronize", self._h)

    def info(self) -> dict:
        inf = Info()
        _check(load().vdbedt_get_info(self._h, ctypes.byref(inf)), "vdbedt_get_info", self._h)
        return {k: getattr(inf, k) for k, _ in Info._fields_}

    # -- reading --
    def query(self, xyz):
        lib = load()
        if isinstance(xyz, np.ndarray):
            x = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
            out = np.empty(x.shape[0], dtype=np.int32)
            _check(lib.vdbedt_query(self._h, _ptr_host(x), x.shape[0], _ptr_host(out), 0), "vdbedt_query", self._h)
            return out
        torch = _torch()
        x = xyz.to(torch.int32).contiguous().view(-1, 3)
        out = torch.empty(x.shape[0], dtype=torch.int32, device=x.device)
        self._enter(x, out)
        _check(lib.vdbedt_query(self._h, x.data_ptr(), x.shape[0], out.data_ptr(), 1), "vdbedt_query", self._h)
        self._leave()
        return out

    def query_nearest(self, xyz):
        """Nearest obstacle (x, y, z) of each voxel of xyz [n, 3] (numpy or CUDA tensor), -1s where
        none lies closer than dmax; ties to the smallest (z, y, x)."""
        lib = load()
        if isinstance(xyz, np.ndarray):
            x = np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3)
            out = np.empty_like(x)
            _check(lib.vdbedt_query_nearest(self._h, _ptr_host(x), x.shape[0], _ptr_host(out), 0),
                   "vdbedt_query_nearest", self._h)
            return out
        torch = _torch()
        x = xyz.to(torch.int32).contiguous().view(-1, 3)
        out = torch.empty_like(x)
        self._enter(x, out)
        _check(lib.vdbedt_query_nearest(self._h, x.data_ptr(), x.shape[0], out.data_ptr(), 1), "vdbedt_query_nearest",
               self._h)
        self._leave()
        return out

    def export_dense(self, on_device: bool = False):
        lib = load()
        nx, ny, nz = self.shape_xyz
        if not on_device:
            out = np.empty((nz, ny, nx), dtype=np.int32)
            _check(lib.vdbedt_export_dense(self._h, _ptr_host(out), 0), "vdbedt_export_dense", self._h)
            return out
        torch = _torch()
        out = torch.empty((nz, ny, nx), dtype=torch.int32, device=f"cuda:{self.device}")
        self._enter(out)
        _check(lib.vdbedt_export_dense(self._h, out.data_ptr(), 1), "vdbedt_export_dense", self._h)
        self._leave()
        return out

    def export_occupancy(self, z_lo: int, z_hi: int, dz: int = 0, changed_only: bool = False, max_n: int = 0):
        """Occupancy of planes [z_lo, z_hi) as packed 64-bit records (int64 CUDA tensor) with z
        shifted by dz: every occupied voxel, or (changed_only) every voxel of the bricks the last
        update changed.  Grows its buffer and retries once when max_n is too small."""
        torch = _torch()
        lib = load()
        n = ctypes.c_int64(0)
        cap = int(max_n) if max_n > 0 else 1 << 16
        for _ in range(2):
            out = torch.empty(cap, dtype=torch.int64, device=f"cuda:{self.device}")
            self._enter(out)
            st = lib.vdbedt_export_occupancy(self._h, int(z_lo), int(z_hi), int(dz), int(bool(changed_only)),
                                             out.data_ptr(), cap, ctypes.byref(n))
            if st == 5 and n.value > cap:  # EOVERFLOW: retry with room for every record
                cap = int(n.value)
                continue
            _check(st, "vdbedt_export_occupancy", self._h)
            return out[: n.value]
        raise VdbedtError(5, "vdbedt_export_occupancy", "record count changed between attempts")

    def distance_at(self, pts, with_grad: bool = True):
        """Trilinear distance (metres) at points [..., 3] (float32 CUDA tensor, metres) and, with
        with_grad, its gradient [..., 3] (the field a planner descends away from obstacles)."""
        torch = _torch()
        p = pts.contiguous().view(-1, 3)
        if p.dtype != torch.float32 or not p.is_cuda:
            raise TypeError("pts must be a float32 CUDA tensor [..., 3]")
        d = torch.empty(p.shape[0], dtype=torch.float32, device=p.device)
        g = torch.empty_like(p) if with_grad else None
        self._enter(p, d, *([g] if with_grad else []))
        _check(load().vdbedt_distance_at(self._h, p.data_ptr(), p.shape[0], d.data_ptr(),
                                         g.data_ptr() if with_grad else None), "vdbedt_distance_at", self._h)
        self._leave()
        shape = pts.shape[:-1]
        return (d.view(shape), g.view(*shape, 3)) if with_grad else d.view(shape)

    def clearance_forward(self, pts, tau: float):
        torch = _torch()
        p = pts.contiguous()
        T, P = p.shape[0], p.shape[1]
        cost = torch.empty(T, dtype=torch.float32, device=p.device)
        self._enter(p, cost)
        _check(load().vdbedt_clearance_forward(self._h, p.data_ptr(), T, P, float(tau), cost.data_ptr()),
               "vdbedt_clearance_forward", self._h)
        self._leave()
        return cost

    def clearance_backward(self, pts, tau: float, grad_cost):
        torch = _torch()
        p = pts.contiguous()
        gc = grad_cost.contiguous().to(torch.float32)
        T, P = p.shape[0], p.shape[1]
        g = torch.empty_like(p)
        self._enter(p, gc, g)
        _check(load().vdbedt_clearance_backward(self._h, p.data_ptr(), T, P, float(tau), gc.data_ptr(), g.data_ptr()),
               "vdbedt_clearance_backward", self._h)
        self._leave()
        return g


class _CapturedStep:
    """Shared machinery of the captured forms: fixed device input buffers (records and their
    count) and one CUDA graph of the library calls of `_body`, replayed on the map's stream."""

    def __init__(self, m: Map, max_records: int):
        torch = _torch()
        self.m = m
        self.max_records = int(max_records)
        dev = f"cuda:{m.device}"
        self.xyz = torch.zeros((self.max_records, 3), dtype=torch.int32, device=dev)
        self.occ = torch.zeros(self.max_records, dtype=torch.uint8, device=dev)
        self.count = torch.zeros(1, dtype=torch.int32, device=dev)
        m._enter()
        with torch.cuda.stream(m.stream):
            # one uncaptured run with an empty frame: reserves the stage and the ingest scratch
            self._body()
            m.stream.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=m.stream):
                self._body()
        m.synchronize()

    def _stage(self):
        lib = load()
        h = self.m._h
        _check(lib.vdbedt_set_occupancy_counted(h, self.xyz.data_ptr(), self.occ.data_ptr(), self.count.data_ptr(),
                                                self.max_records), "vdbedt_set_occupancy_counted", h)

    def load(self, xyz, occ):
        """Writes one set of records into the input buffers (stream-ordered on the map's stream)
        without replaying; xyz [n, 3] int32 and occ [n] uint8, CUDA tensors or numpy.  A producer
        may instead write xyz[:n], occ[:n] and count[0] itself."""
        torch = _torch()
        n = int(occ.shape[0])
        if n > self.max_records:
            raise ValueError(f"{n} records exceed the captured maximum {self.max_records}")
        if isinstance(xyz, np.ndarray):
            xyz = torch.from_numpy(np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3))
            occ = torch.from_numpy(np.ascontiguousarray(occ, dtype=np.uint8).reshape(-1))
        self.m._enter()
        with torch.cuda.stream(self.m.stream):
            if n:
                self.xyz[:n].copy_(xyz.view(-1, 3), non_blocking=True)
                self.occ[:n].copy_(occ.view(-1), non_blocking=True)
            self.count.fill_(n)
        self.m._leave()

    def run(self, xyz, occ):
        """Replay for one set of records; xyz [n, 3] int32 and occ [n] uint8, CUDA tensors or numpy."""
        self.load(xyz, occ)
        self.replay()

    def replay(self):
        """Replay with the records already in the input buffers (xyz, occ, count)."""
        torch = _torch()
        self.m._enter()
        with torch.cuda.stream(self.m.stream):
            self.graph.replay()
        self.m._leave()


class GlobalGraph(_CapturedStep):
    """The global transform from a fresh occupancy -- vdbedt_reset, staging of up to max_records
    device records with a device-side count, vdbedt_global -- captured once into a CUDA graph.
    run(xyz, occ) equals reset() + set_occupancy(xyz, occ) + global_() bit for bit."""

    def _body(self):
        lib = load()
        h = self.m._h
        _check(lib.vdbedt_reset(h), "vdbedt_reset", h)
        self._stage()
        _check(lib.vdbedt_global(h), "vdbedt_global", h)


class UpdateGraph(_CapturedStep):
    """One incremental update of a Map -- staging of up to max_records device records with a
    device-side count, then vdbedt_update -- captured once into a CUDA graph.  run(xyz, occ)
    writes a frame's records into the graph's fixed input buffers and replays the graph on the
    map's stream; the result equals set_occupancy(xyz, occ) + update() bit for bit.  The map must
    not be reset, given a dense grid or retuned while the graph is in use (the graph holds the
    launches of the incremental form with the tuning of capture time); the first, uncaptured call
    runs the global transform if the map has none yet."""

    def _body(self):
        lib = load()
        h = self.m._h
        self._stage()
        _check(lib.vdbedt_update(h, None), "vdbedt_update", h)


class BatchUpdateGraph:
    """One incremental update of every grid of a Batch -- counted staging of up to max_records
    device records per grid, then vdbedt_batch_update -- captured once into a CUDA graph.
    run(frames) takes one (xyz [n, 3] int32, occ [n] uint8) pair per grid (CUDA tensors or numpy),
    writes them into the graph's fixed input buffers and replays the graph on the batch's stream;
    the result equals set_occupancy on each grid + Batch.update() bit for bit."""

    def __init__(self, batch: "Batch", max_records: int):
        torch = _torch()
        self.b = batch
        self.max_records = int(max_records)
        k = len(batch.maps)
        dev = f"cuda:{batch.device}"
        self.xyz = torch.zeros((k, self.max_records, 3), dtype=torch.int32, device=dev)
        self.occ = torch.zeros((k, self.max_records), dtype=torch.uint8, device=dev)
        self.count = torch.zeros(k, dtype=torch.int32, device=dev)
        m0 = batch.maps[0]
        m0._enter()
        with torch.cuda.stream(batch.stream):
            # one uncaptured run with empty frames: reserves every grid's stage and scratch and
            # uploads the grids' update arguments
            self._body()
            batch.stream.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=batch.stream):
                self._body()
        batch.synchronize()

    def _body(self):
        lib = load()
        for i, m in enumerate(self.b.maps):
            _check(lib.vdbedt_set_occupancy_counted(m._h, self.xyz[i].data_ptr(), self.occ[i].data_ptr(),
                                                    self.count[i:i + 1].data_ptr(), self.max_records),
                   "vdbedt_set_occupancy_counted", m._h)
        self.b._chk(lib.vdbedt_batch_update(self.b._b, None), "vdbedt_batch_update")

    def run(self, frames):
        torch = _torch()
        if len(frames) != len(self.b.maps):
            raise ValueError("one (xyz, occ) pair per grid")
        counts = []
        m0 = self.b.maps[0]
        m0._enter()
        with torch.cuda.stream(self.b.stream):
            for i, (xyz, occ) in enumerate(frames):
                n = int(occ.shape[0])
                if n > self.max_records:
                    raise ValueError(f"{n} records exceed the captured maximum {self.max_records}")
                if isinstance(xyz, np.ndarray):
                    xyz = torch.from_numpy(np.ascontiguousarray(xyz, dtype=np.int32).reshape(-1, 3))
                    occ = torch.from_numpy(np.ascontiguousarray(occ, dtype=np.uint8).reshape(-1))
                if n:
                    self.xyz[i, :n].copy_(xyz.view(-1, 3), non_blocking=True)
                    self.occ[i, :n].copy_(occ.view(-1), non_blocking=True)
                counts.append(n)
            self.count.copy_(torch.tensor(counts, dtype=torch.int32), non_blocking=True)
            self.graph.replay()
        m0._leave()

    def replay(self):
        """Replay with the records already in the input buffers (xyz, occ, count)."""
        torch = _torch()
        m0 = self.b.maps[0]
        m0._enter()
        with torch.cuda.stream(self.b.stream):
            self.graph.replay()
        m0._leave()


NOALLOC_MAX_VOXELS = 1 << 21


def edt_dense_noalloc(occ, dmax: int, out=None):
    """D of a small dense grid occ [nz, ny, nx] (CUDA tensor) through vdbedt_edt_dense_noalloc, which
    allocates nothing on the device (its scratch is a fixed array of the library); returns int32
    [nz, ny, nx] on occ's device and that device's current torch stream.  `out` (a contiguous int32
    CUDA tensor of shape [nz, ny, nx] on occ's device) may be given preallocated, so that the call
    itself allocates nothing.  Bad tensors raise TypeError / ValueError before the C call."""
    torch = _torch()
    if not isinstance(occ, torch.Tensor) or not occ.is_cuda:
        raise TypeError("occ must be a CUDA tensor [nz, ny, nx]")
    if occ.dim() != 3:
        raise ValueError(f"occ must have 3 dimensions [nz, ny, nx], got shape {tuple(occ.shape)}")
    if out is not None:
        if not isinstance(out, torch.Tensor) or not out.is_cuda or out.dtype != torch.int32:
            raise TypeError("out must be an int32 CUDA tensor")
        if out.device != occ.device:
            raise ValueError(f"out is on {out.device}, occ on {occ.device}")
        if tuple(out.shape) != tuple(occ.shape) or not out.is_contiguous():
            raise ValueError(f"out must be contiguous with shape {tuple(occ.shape)}")
    with torch.cuda.device(occ.device):
        o = occ if (occ.dtype == torch.uint8 and occ.is_contiguous()) else occ.to(torch.uint8).contiguous()
        nz, ny, nx = o.shape
        if out is None:
            out = torch.empty((nz, ny, nx), dtype=torch.int32, device=o.device)
        st = torch.cuda.current_stream(o.device).cuda_stream
        _check(load().vdbedt_edt_dense_noalloc(o.data_ptr(), nx, ny, nz, int(dmax), out.data_ptr(), st),
               "vdbedt_edt_dense_noalloc")
    return out


def kernel_launches() -> int:
    return int(load().vdbedt_kernel_launches())


def global_batched(maps):
    """vdbedt_global_batched over Map objects (one launch per step when they are one Batch's grids)."""
    lib = load()
    arr = (ctypes.c_void_p * len(maps))(*[m.handle for m in maps])
    _check(lib.vdbedt_global_batched(arr, len(maps)), "vdbedt_global_batched")


class Batch:
    """k grids of uneven size created together (vdbedt_batch_create); maps[i] is grid i as a Map.
    set_occupancy_dense(grids) and global_() run each step once for all grids."""

    def __init__(self, dims_xyz, dmax: int, voxel_size: float = 0.1, device: int = 0, stream=None):
        lib = load()
        torch = _torch()
        if stream is None:
            stream = torch.cuda.Stream(device)
        self.device, self.stream, self.dmax = device, stream, dmax
        k = len(dims_xyz)
        cfgs = (Config * k)(*[Config(int(nx), int(ny), int(nz), int(dmax), voxel_size, device,
                                     ctypes.c_void_p(stream.cuda_stream), 0, 0) for nx, ny, nz in dims_xyz])
        b = ctypes.c_void_p()
        st = lib.vdbedt_batch_create(cfgs, k, ctypes.byref(b))
        if st != 0:
            raise VdbedtError(st, "vdbedt_batch_create", (lib.vdbedt_batch_last_error(None) or b"").decode())
        self._b = b
        self.maps = []
        for i, (nx, ny, nz) in enumerate(dims_xyz):
            h = ctypes.c_void_p()
            self._chk(lib.vdbedt_batch_map(b, i, ctypes.byref(h)), "vdbedt_batch_map")
            self.maps.append(Map(int(nx), int(ny), int(nz), dmax, voxel_size, device, stream, _borrow=h))

    def _chk(self, status, where):
        if status != 0:
            msg = load().vdbedt_batch_last_error(self._b)
            raise VdbedtError(status, where, msg.decode() if msg else "")

    def close(self):
        if getattr(self, "_b", None):
            for m in self.maps:
                m._h = None
            load().vdbedt_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __len__(self):
        return len(self.maps)

    def set_occupancy_dense(self, grids):
        """grids[i]: grid i's occupancy [nz, ny, nx]; all numpy arrays (host) or all CUDA tensors."""
        lib = load()
        k = len(self.maps)
        if all(isinstance(g, np.ndarray) for g in grids):
            keep = [np.ascontiguousarray(g, dtype=np.uint8) for g in grids]
            arr = (ctypes.c_void_p * k)(*[_ptr_host(g) for g in keep])
            self._chk(lib.vdbedt_batch_set_occupancy_dense(self._b, arr, 0), "vdbedt_batch_set_occupancy_dense")
            return
        torch = _torch()
        keep = [g.to(torch.uint8).contiguous() for g in grids]
        self.maps[0]._enter(*keep)
        arr = (ctypes.c_void_p * k)(*[g.data_ptr() for g in keep])
        self._chk(lib.vdbedt_batch_set_occupancy_dense(self._b, arr, 1), "vdbedt_batch_set_occupancy_dense")

    def global_(self):
        self._chk(load().vdbedt_batch_global(self._b), "vdbedt_batch_global")

    def update(self, stats: bool = False):
        """vdbedt_batch_update: every grid applies its staged records incrementally, each step
        launched once for the whole batch; with stats, one dict per grid."""
        k = len(self.maps)
        st = (UpdateStats * k)() if stats else None
        self._chk(load().vdbedt_batch_update(self._b, st), "vdbedt_batch_update")
        if st is not None:
            return [{f: getattr(st[i], f) for f, _ in UpdateStats._fields_} for i in range(k)]
        return None

    def set_tuning(self, x_run: int = 0, y_run: int = 0, z_run: int = 0, variant: int = 0):
        t = Tuning(x_run, y_run, z_run, variant)
        self._chk(load().vdbedt_batch_set_tuning(self._b, ctypes.byref(t)), "vdbedt_batch_set_tuning")

    def synchronize(self):
        self._chk(load().vdbedt_batch_synchronize(self._b), "vdbedt_batch_synchronize")

    def set_profiling(self, on: bool = True):
        self._chk(load().vdbedt_batch_set_profiling(self._b, int(on)), "vdbedt_batch_set_profiling")

    def phase_times(self) -> dict:
        pt = PhaseTimes()
        self._chk(load().vdbedt_batch_get_phase_times(self._b, ctypes.byref(pt)), "vdbedt_batch_get_phase_times")
        return {k: getattr(pt, k) for k, _ in PhaseTimes._fields_}


def _make_clearance_fn():
    torch = _torch()

    class _Clearance(torch.autograd.Function):
        @staticmethod
        def forward(ctx, pts, m, tau):
            if pts.dtype != torch.float32 or not pts.is_cuda:
                raise TypeError("pts must be a float32 CUDA tensor [T, P, 3]")
            p = pts.detach().contiguous()
            ctx.m, ctx.tau = m, tau
            ctx.save_for_backward(p)
            return m.clearance_forward(p, tau)

        @staticmethod
        def backward(ctx, gcost):
            (p,) = ctx.saved_tensors
            return ctx.m.clearance_backward(p, ctx.tau, gcost), None, None

    return _Clearance


_clearance_fn = None


def clearance_cost(m: Map, pts, tau: float = 1.0):
    """Per-trajectory clearance cost sum_p max(0, tau - d(p))^2 (Eq. 2's clearance term as a squared
    hinge) with d the trilinear distance in metres; differentiable with respect to pts [T, P, 3]."""
    global _clearance_fn
    if _clearance_fn is None:
        _clearance_fn = _make_clearance_fn()
    return _clearance_fn.apply(pts, m, tau)
