"""Autotuner of the transform passes' work-item shapes.

The brick is fixed at 8^3 voxels (the storage layout); what is tuned is the tile each pass works
on -- the run of bricks one work item covers along the pass axis (4, 8 or 16 bricks: longer runs
re-read less halo per output brick but give fewer, larger items) -- and the algorithm: the windowed
minimum of the in-plane and z passes (1: full window; 3: window with early exit and skips of
windows without finite input) or the lower-envelope form of all three passes (variant 8: O(1)
amortised work per voxel whatever the window, on runs of 16 bricks; the only form above dmax 45).
Every choice computes the same exact field; only the time differs.

The tuner times the map's (or batch's) own global transform under each candidate with the
library's phase events, picks per axis the fastest run, and stores the choice in a JSON cache keyed
by GPU, brick radius and workload size, so that later maps of the same kind reuse it without
timing.  The windowed passes are independent per axis, so 3 variants x 3 runs = 9 timed
configurations cover every combination (the x pass also has two kernels: the bulk-copy ring and
plain loads); the envelope form is one more, compared with the windowed choice on the whole
transform (x + y + z), since it replaces all three passes.
"""
from __future__ import annotations

import json
import os
import statistics
import threading

RUNS = (4, 8, 16)
# 1: full window; 3: pruned window; 7: pruned window with the x pass on plain loads (+4)
VARIANTS = (1, 3, 7)
X_DIRECT = 4
ENVELOPE = 8  # the lower-envelope form (runs of 16 bricks; the run settings do not apply)
ENVELOPE_KEY = (ENVELOPE, 16)
WINDOW_DMAX = 45  # above it, the envelope is the only form
# Candidates within TIE of the fastest count as equal, and the first of them in preference order
# wins (the library defaults first), so that timing noise does not flip the choice between runs.
TIE = 0.02
RUN_PREF = (8, 16, 4)
VARIANT_PREF = (3, 7, 1)
_lock = threading.Lock()


def default_cache_path() -> str:
    base = os.environ.get("VDBEDT_TUNING_CACHE")
    if base:
        return base
    root = os.environ.get("XDG_CACHE_HOME") or os.path.join(os.path.expanduser("~"), ".cache")
    return os.path.join(root, "vdbedt", "tuning.json")


def _round_sig(v: int, digits: int = 2) -> int:
    if v <= 0:
        return 0
    s = len(str(int(v)))
    q = 10 ** max(0, s - digits)
    return int(round(v / q) * q)


def signature(target) -> str:
    """Cache key: GPU name, brick radius R, grid count and allocated bricks (2 significant
    digits) of a Map or Batch after a transform."""
    import torch
    maps = getattr(target, "maps", None) or [target]
    dev = torch.cuda.get_device_name(maps[0].device)
    infos = [m.info() for m in maps]
    bricks = sum(i["allocated_bricks"] for i in infos)
    return f"{dev}|R={infos[0]['R']}|grids={len(maps)}|bricks~{_round_sig(bricks)}"


def _pick(cands, cost):
    """The first candidate (in preference order) whose cost is within TIE of the lowest."""
    best = min(cost(c) for c in cands)
    return next(c for c in cands if cost(c) <= best * (1.0 + TIE))


def choose(table: dict, joint_yz: bool = False) -> dict:
    """Pick the tuning from timed phases.  table[(variant, run)] = {"x_ms", "y_ms", "z_ms"}
    (medians), with the envelope form at ENVELOPE_KEY when it was timed.  The x pass takes its
    fastest (kernel, run) over every windowed candidate (its time depends only on the X_DIRECT bit
    of the variant and the run); the window variant is the one whose best y + z is lowest; then y
    and z each take their fastest run under it (jointly when the phases are timed together, as for
    batches).  The envelope form replaces that choice when its whole transform (x + y + z) is
    faster than the windowed choice's.  Near-ties (TIE) go to the preferred candidate (the windowed
    form before the envelope)."""
    env = {"x_run": 16, "y_run": 16, "z_run": 16, "variant": ENVELOPE}
    if not any(k != ENVELOPE_KEY for k in table):
        return env
    xv, x_run = _pick([(v, r) for v in VARIANT_PREF for r in RUN_PREF], lambda vr: table[vr]["x_ms"])

    def yz_best(v):
        if joint_yz:
            r = _pick(RUN_PREF, lambda r: table[(v, r)]["z_ms"])
            return table[(v, r)]["z_ms"], r, r
        ry = _pick(RUN_PREF, lambda r: table[(v, r)]["y_ms"])
        rz = _pick(RUN_PREF, lambda r: table[(v, r)]["z_ms"])
        return table[(v, ry)]["y_ms"] + table[(v, rz)]["z_ms"], ry, rz

    window = _pick(VARIANT_PREF, lambda v: yz_best(v)[0])
    yz, y_run, z_run = yz_best(window)
    variant = (window & 3) | (xv & X_DIRECT)
    if ENVELOPE_KEY in table:
        e = table[ENVELOPE_KEY]
        if (e["x_ms"] + e["y_ms"] + e["z_ms"]) * (1.0 + TIE) < table[(xv, x_run)]["x_ms"] + yz:
            return env
    return {"x_run": x_run, "y_run": y_run, "z_run": z_run, "variant": variant}


def _load(path: str) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def _store(path: str, key: str, value: dict) -> None:
    with _lock:
        data = _load(path)
        data[key] = value
        os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(data, f, indent=1, sort_keys=True)
        os.replace(tmp, path)


def measure(target, reps: int = 5) -> dict:
    """Median phase times of target.global_() under each candidate: every (variant, run) of the
    windowed form when the target's dmax allows it, and the envelope form."""
    cands = [ENVELOPE_KEY]
    if getattr(target, "dmax", 0) <= WINDOW_DMAX:
        cands = [(v, r) for v in VARIANTS for r in RUNS] + cands
    table = {}
    target.set_profiling(True)
    try:
        for v, r in cands:
            target.set_tuning(r, r, r, v)
            target.global_()  # warm-up (also applies any staged records)
            samples = []
            for _ in range(reps):
                target.global_()
                samples.append(target.phase_times())
            table[(v, r)] = {k: statistics.median(s[k] for s in samples) for k in ("x_ms", "y_ms", "z_ms")}
    finally:
        target.set_profiling(False)
    return table


def autotune(target, reps: int = 5, cache_path: str | None = None, use_cache: bool = True) -> dict:
    """Tune a Map or Batch on its current occupancy; applies and returns the tuning
    {"x_run", "y_run", "z_run", "variant", "source": "cache" | "measured"}.  The field is left
    recomputed (global transform) under the chosen tuning."""
    if getattr(target, "untruncated", False):
        raise ValueError("an untruncated grid has no tuning: its whole-line passes take no work-item shapes")
    path = cache_path or default_cache_path()
    target.global_()
    key = signature(target)
    if use_cache:
        hit = _load(path).get(key)
        if hit:
            t = {k: int(hit[k]) for k in ("x_run", "y_run", "z_run", "variant")}
            target.set_tuning(**t)
            target.global_()
            return dict(t, source="cache", key=key)
    table = measure(target, reps)
    t = choose(table, joint_yz=hasattr(target, "maps"))
    target.set_tuning(**t)
    target.global_()
    _store(path, key, dict(t, table={f"v{v}_r{r}": ms for (v, r), ms in table.items()}))
    return dict(t, source="measured", key=key)
