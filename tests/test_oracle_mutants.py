"""Planted mistakes: the oracle's pins must catch plausible errors in the oracle itself.

Each case copies ``oracle/edt_oracle.c``, plants one mistake (a dropped term, an off-by-one
window, a wrong index, a missing saturation, a reversed sort), compiles the copy into a temporary
library and runs the pins of ``test_oracle_edt`` (scipy's exact transform, closed forms,
invariants) against it.  The unmodified source must pass the same pins.
"""
import ctypes
import os
import resource
import subprocess
import sys

import numpy as np
import pytest

import oracle as O
from test_oracle_edt import check_invariants, scipy_sq_edt

SRC = os.path.join(os.path.dirname(O.__file__), "edt_oracle.c")

MUTANTS = {
    "window_off_by_one": ("edt", "const int w = dmax - 1; /* largest", "const int w = dmax - 2; /* largest"),
    "y_square_dropped": ("edt", "int32_t c = d * d + g1[", "int32_t c = g1["),
    "z_wrong_index": ("edt", "int32_t c = d * d + g2[((i64)zz * ny + y)", "int32_t c = d * d + g2[((i64)z * ny + y)"),
    "wrong_saturation": ("edt", "const int32_t cap = dmax * dmax;\n  const int w = dmax - 1; /* largest",
                         "const int32_t cap = dmax * dmax + 1;\n  const int w = dmax - 1; /* largest"),
    "naive_dz_dropped": ("naive", "i64 d2 = dx * dx + dy * dy + dz * dz;", "i64 d2 = dx * dx + dy * dy;"),
    "naive_axes_swapped": ("naive", "int x = (int)(i % nx), y = (int)((i / nx) % ny)",
                           "int y = (int)(i % nx), x = (int)((i / nx) % ny)"),
    "at_sort_reversed": ("at", "return (p->d2 > q->d2) - (p->d2 < q->d2);", "return (p->d2 < q->d2) - (p->d2 > q->d2);"),
    "alg1_sqdist_dz_dropped": ("alg1", " + (az - bz) * (az - bz);", ";"),
    "alg1_stops_early": ("alg1", "if (dnew < s->dmax2) {", "if (dnew < s->dmax2 / 2) {"),
    "alg1_raise_inverted": ("alg1inc", "if (!is_obst(s, n->obst)) {", "if (is_obst(s, n->obst)) {"),
    "alg1_remove_ignored": ("alg1inc", "if (s->occ[i] && !c->queued) {", "if (0) {"),
}


def build_variant(tmp_path, name, old, new):
    src = open(SRC).read()
    if old is not None:
        assert src.count(old) == 1, f"mutation anchor for {name} not unique"
        src = src.replace(old, new)
    c = tmp_path / f"{name}.c"
    so = tmp_path / f"{name}.so"
    c.write_text(src)
    subprocess.check_call(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-o", str(so), str(c)])
    return str(so)


def load_variant(so):
    lib = ctypes.CDLL(so)
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    for f in (lib.oracle_edt_naive, lib.oracle_edt_factorised):
        f.restype = i32
        f.argtypes = [vp, i32, i32, i32, i32, vp, i32]
    lib.oracle_edt_at.restype = i32
    lib.oracle_edt_at.argtypes = [vp, i32, i32, i32, i32, vp, i64, vp, i32]
    lib.alg1_create.restype = vp
    lib.alg1_create.argtypes = [i32, i32, i32, i32]
    lib.alg1_global.argtypes = [vp, vp]
    lib.alg1_update.argtypes = [vp, vp, vp, i64]
    lib.alg1_read.argtypes = [vp, vp, vp]
    lib.alg1_destroy.argtypes = [vp]
    return lib


def run_field(lib, which, occ, dmax):
    occ = np.ascontiguousarray(occ, np.uint8)
    nz, ny, nx = occ.shape
    out = np.empty(occ.shape, np.int32)
    if which == "edt":
        lib.oracle_edt_factorised(occ.ctypes.data, nx, ny, nz, dmax, out.ctypes.data, 2)
    elif which == "naive":
        lib.oracle_edt_naive(occ.ctypes.data, nx, ny, nz, dmax, out.ctypes.data, 2)
    elif which == "at":
        z, y, x = np.indices(occ.shape)
        xyz = np.ascontiguousarray(np.stack([x.ravel(), y.ravel(), z.ravel()], 1).astype(np.int32))
        flat = np.empty(xyz.shape[0], np.int32)
        lib.oracle_edt_at(occ.ctypes.data, nx, ny, nz, dmax, xyz.ctypes.data, xyz.shape[0], flat.ctypes.data, 2)
        out = flat.reshape(occ.shape)
    elif which == "alg1":
        h = lib.alg1_create(nx, ny, nz, dmax)
        lib.alg1_global(h, occ.ctypes.data)
        lib.alg1_read(h, out.ctypes.data, None)
        lib.alg1_destroy(h)
    elif which == "alg1inc":
        # start from a shifted copy of occ, then edit it into occ: removals and additions
        start = np.ascontiguousarray(np.roll(occ, 2, axis=2))
        h = lib.alg1_create(nx, ny, nz, dmax)
        lib.alg1_global(h, start.ctypes.data)
        diff = np.argwhere(start != occ)
        xyz = np.ascontiguousarray(diff[:, ::-1].astype(np.int32))
        val = np.ascontiguousarray(occ[diff[:, 0], diff[:, 1], diff[:, 2]].astype(np.uint8))
        lib.alg1_update(h, xyz.ctypes.data, val.ctypes.data, xyz.shape[0])
        lib.alg1_read(h, out.ctypes.data, None)
        lib.alg1_destroy(h)
    return out


def pins_pass(lib, which):
    """True iff every pin holds for the given library's function."""
    rs = np.random.default_rng(1234)
    try:
        for shape, p, dmax in (((9, 12, 15), 0.02, 5), ((14, 7, 11), 0.05, 3), ((6, 10, 8), 0.0, 4)):
            occ = (rs.random(shape) < p).astype(np.uint8)
            if occ.sum() == 0 and p > 0:
                occ[0, 0, 0] = 1
            D = run_field(lib, which, occ, dmax)
            if not np.array_equal(D, scipy_sq_edt(occ, dmax)):
                return False
            check_invariants(occ, D, dmax)
        # single obstacle off-centre in a non-cubic grid
        occ = np.zeros((5, 9, 13), np.uint8)
        occ[1, 6, 3] = 1
        z, y, x = np.indices(occ.shape)
        if not np.array_equal(run_field(lib, which, occ, 6),
                              np.minimum((x - 3) ** 2 + (y - 6) ** 2 + (z - 1) ** 2, 36)):
            return False
    except AssertionError:
        return False
    return True


def _limits():
    resource.setrlimit(resource.RLIMIT_AS, (2 << 30, 2 << 30))


def pins_pass_isolated(so, which):
    """Run the pins in a child process (2 GiB, 60 s): a mutant that never terminates or blows up
    its queue counts as caught."""
    here = os.path.dirname(os.path.abspath(__file__))
    env = dict(os.environ, PYTHONPATH=os.pathsep.join([here, os.path.dirname(here)]), OMP_NUM_THREADS="2")
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), so, which], cwd=here, timeout=60,
                           preexec_fn=_limits, capture_output=True, env=env)
    except subprocess.TimeoutExpired:
        return False
    return r.returncode == 0


@pytest.mark.parametrize("which", ["edt", "naive", "at", "alg1", "alg1inc"])
def test_unmodified_passes(tmp_path, which):
    so = build_variant(tmp_path, f"orig_{which}", None, None)
    assert pins_pass_isolated(so, which)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    which, old, new = MUTANTS[name]
    so = build_variant(tmp_path, name, old, new)
    assert not pins_pass_isolated(so, which), f"planted mistake {name} was not caught by the pins"


if __name__ == "__main__":
    sys.exit(0 if pins_pass(load_variant(sys.argv[1]), sys.argv[2]) else 1)
