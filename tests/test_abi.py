"""The C-ABI library builds, loads and exports every entry point that include/vdbedt.h declares
(no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "vdbedt.h")


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vdbedt_[a-z_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2105_04419_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("vdbedt_create", "vdbedt_set_occupancy", "vdbedt_global", "vdbedt_update", "vdbedt_query",
                     "vdbedt_destroy", "vdbedt_last_error", "vdbedt_global_batched", "vdbedt_clearance_forward",
                     "vdbedt_clearance_backward"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_the_header():
    from paper_2105_04419_gb300 import lib as L
    assert set(declared_functions()) <= set(L.SIGNATURES)


def test_struct_layouts_match_header(tmp_path):
    """ctypes structures match the C header: sizes and field offsets from a gcc-compiled probe."""
    import subprocess
    from paper_2105_04419_gb300 import lib as L
    structs = {"vdbedt_config": L.Config, "vdbedt_info": L.Info, "vdbedt_update_stats": L.UpdateStats,
               "vdbedt_tuning": L.Tuning, "vdbedt_phase_times": L.PhaseTimes}
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "vdbedt.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append(f'printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines.append("return 0; }")
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(c)])
    out = subprocess.check_output([str(exe)], text=True).split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)


def test_create_without_device_is_einval(lib):
    """Handle-less failure paths return codes (no abort) even where no GPU is visible."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is visible")
    from paper_2105_04419_gb300 import lib as L
    lb = L.load()
    cfg = L.Config(8, 8, 8, 4, 0.1, 0, None, 0, 0)
    h = ctypes.c_void_p()
    assert lb.vdbedt_create(ctypes.byref(cfg), ctypes.byref(h)) == 1
    assert lb.vdbedt_last_error(None)
    assert lb.vdbedt_destroy(None) == 0
    bad = L.Config(0, 8, 8, 4, 0.1, 0, None, 0, 0)
    assert lb.vdbedt_create(ctypes.byref(bad), ctypes.byref(h)) == 1


def test_header_constants_match_binding(tmp_path):
    """The binding's copies of the header's macros (flags, sentinels, limits) hold the same values."""
    import subprocess
    from paper_2105_04419_gb300 import lib as L
    pairs = {"VDBEDT_FLAG_UNBOUNDED": L.FLAG_UNBOUNDED, "VDBEDT_FLAG_UNTRUNCATED": L.FLAG_UNTRUNCATED,
             "VDBEDT_D_NONE": L.D_NONE, "VDBEDT_UNBOUNDED_OFFSET": L.UNBOUNDED_OFFSET,
             "VDBEDT_UNBOUNDED_MIN": L.UNBOUNDED_MIN, "VDBEDT_UNBOUNDED_MAX": L.UNBOUNDED_MAX,
             "VDBEDT_DMAX_LIMIT": L.VDBEDT_DMAX_LIMIT}
    lines = ['#include <stdio.h>', '#include "vdbedt.h"', "int main(void) {"]
    lines += [f'printf("{k} %lld\\n", (long long)({k}));' for k in pairs]
    lines.append("return 0; }")
    c = tmp_path / "consts.c"
    c.write_text("\n".join(lines))
    exe = tmp_path / "consts"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(c)])
    got = {l.split()[0]: int(l.split()[1]) for l in subprocess.check_output([str(exe)], text=True).split("\n") if l}
    assert got == pairs
