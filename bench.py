#!/usr/bin/env python
"""Benchmark of the exact truncated EDT on a sparse brick grid (one JSON line on rank 0).

Workload (default): the synthetic tunnel scene, 1024 x 1024 x 256 voxels, 40 spline tunnels of
radius 8-24 voxels whose walls are occupied shells, dmax = 32 (clamp 1024), seed 1.  One step =
one global transform from the occupied-voxel list already resident on the device: reset the grid,
stage the records, build the sparse grid (sort / unique / compaction), activate, run the in-plane
and z passes.  value = active voxels (bricks with some D < dmax^2, times 512) per second, in
Mvoxels/s, summed over ranks.

Rows reported beside the headline: roofline of the dominant kernel and of the whole step, the CPU
oracle on the host cores (bounded sample), the end-to-end number through the C ABI with host
buffers, clocks sampled during the timed region, and the library's kernel-launch count; then the
clearance cost (queries/s, forward and forward + backward, 8192 x 128 points in free space) on
the same field; the incremental update along 300 lidar frames (ms/frame of the CUDA-graph
replay and of the eager calls, against the global transform of the final occupancy); and the
batched transform of 96 maps of uneven size (one batch against 96 single handles).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload tunnel|bernoulli64]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "EDT Mvoxels/s and % HBM roofline; incremental update ms/frame; queries/s"
L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2

WORKLOADS = {
    "tunnel": dict(dims=(1024, 1024, 256), dmax=32, seed=1, kind="tunnel",
                   name="tunnel scene 1024x1024x256, 40 tunnels r 8-24, shell walls, dmax 32"),
    "tunnel512": dict(dims=(512, 512, 256), dmax=32, seed=1, kind="tunnel", ntunnels=20,
                      name="tunnel scene 512x512x256, 20 tunnels r 8-24, shell walls, dmax 32 (profiling size)"),
    "bernoulli64": dict(dims=(64, 64, 64), dmax=16, seed=0, kind="bernoulli", p=0.02,
                        name="dense 64^3 Bernoulli(0.02), dmax 16"),
}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="tunnel")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-incremental", action="store_true")
    ap.add_argument("--no-clearance", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-crossover", action="store_true")
    ap.add_argument("--no-untruncated", action="store_true")
    ap.add_argument("--shard", choices=["replicas", "slabs"], default="replicas",
                    help="replicas: every rank transforms the whole scene; slabs: the scene's grid is split "
                         "into z-slabs over the ranks (sparse halo exchange of band records)")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default work-item tuning")
    ap.add_argument("--frames", type=int, default=300, help="lidar frames of the incremental measurement")
    ap.add_argument("--incr-run", type=int, default=4, choices=(4, 8, 16),
                    help="bricks per work item of the incremental maps (default: the library's 4)")
    ap.add_argument("--alg1-frames", type=int, default=1,
                    help="time the paper's Alg. 1 (the oracle's single-threaded transcription) on the first K "
                         "lidar frames (about 20 s for the first frame and 7 GB of host memory; 0: skip)")
    ap.add_argument("--variant", type=int, default=0, help="pass variant (0 automatic; see vdbedt_set_tuning)")
    ap.add_argument("--x-run", type=int, default=0)
    ap.add_argument("--y-run", type=int, default=0)
    ap.add_argument("--z-run", type=int, default=0)
    return ap.parse_args()


def make_occupancy(wl):
    import workloads as W
    nx, ny, nz = wl["dims"]
    if wl["kind"] == "tunnel":
        return W.tunnel_scene(wl["seed"], (nx, ny, nz), ntunnels=wl.get("ntunnels", 40))
    return W.bernoulli_grid(wl["seed"], (nz, ny, nx), wl["p"])


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def traffic_for(kernel: str, tuning: dict):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    source of the kernel (hash of the pass source file) with the same work-item runs."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            t = json.load(f)
        src = open(os.path.join(ROOT, "paper_2105_04419_gb300", "csrc", "passes.cu"), "rb").read()
        h = hashlib.sha256(src).hexdigest()[:16]
        e = t.get(kernel)
        runs = "x_run {x_run}, y_run {y_run}, z_run {z_run}, variant {variant}".format(
            **{k: tuning.get(k) for k in ("x_run", "y_run", "z_run", "variant")})
        if e and e.get("source_sha") == h and runs in t.get("_note", ""):
            return e
    except Exception:
        pass
    return None


def max_over_ranks(x: float) -> float:
    """Largest value of x over the ranks of the default process group (x itself without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_summary(v):
    v = sorted(v)
    if not v:
        return None
    return {"median": statistics.median(v), "p95": v[min(len(v) - 1, int(round(0.95 * (len(v) - 1))))],
            "max": v[-1], "min": v[0], "mean": statistics.mean(v)}


def alg1_frames(truth, frames, dmax, k):
    """The paper's Alg. 1 (the oracle's transcription, one thread as in the paper) on the first k
    frames of the sequence, from the same empty map: milliseconds and queue counters per frame."""
    import oracle as O
    a = O.Alg1(truth.shape, dmax)
    try:
        a.global_(np.zeros(truth.shape, np.uint8))
        out = []
        for xyz, val in frames[:k]:
            a.reset_counters()
            t0 = time.perf_counter()
            a.update(xyz, val)
            out.append(dict(ms=1e3 * (time.perf_counter() - t0), records=int(len(val)), **a.counters()))
        return {"frames": out, "threads": 1, "kind": "oracle (Alg. 1)",
                "note": "the same records as the GPU frames; the GPU's fields equal Eq. 1, Alg. 1 may overshoot it"}
    finally:
        a.close()


def bench_incremental(V, torch, wl, truth, stream, flush, nframes, INCR_RUN=4, alg1_k=0):
    """Per-frame incremental update along the lidar sequence (map starts empty): eager calls and
    the CUDA-graph replay, each frame event-timed on the map's stream with L2 flushed before it,
    against the global transform of the final occupancy."""
    import workloads as W
    nx, ny, nz = wl["dims"]
    dmax = wl["dmax"]
    _, lines = W.tunnel_lines(wl["seed"], (nx, ny, nz), ntunnels=wl.get("ntunnels", 40))
    seq = W.LidarSequence(truth, wl["seed"], lines[0], nframes=nframes)
    frames = [seq.next() for _ in range(nframes)]
    alg1 = alg1_frames(truth, frames, dmax, alg1_k) if alg1_k > 0 else None
    hits = [int(v.sum()) for _, v in frames]  # "set" records: one per ray that meets a wall in range
    final_occ = seq.map
    counts = [len(v) for _, v in frames]
    offs = np.concatenate([[0], np.cumsum(counts)])
    xyz_d = torch.from_numpy(np.concatenate([x for x, _ in frames])).cuda()
    val_d = torch.from_numpy(np.concatenate([v for _, v in frames])).cuda()
    sl = [(xyz_d[offs[k]:offs[k + 1]], val_d[offs[k]:offs[k + 1]]) for k in range(nframes)]

    # untimed pass with statistics (records, net flips, dirty runs per frame); every incremental
    # map works on runs of INCR_RUN bricks (default: the library's 4), pruned windows
    ms = V.Map(nx, ny, nz, dmax, voxel_size=0.1, stream=stream)
    ms.set_tuning(INCR_RUN, INCR_RUN, INCR_RUN, 3)
    ms.global_()
    ms.set_profiling(True)
    stats, phases = [], []
    for x, v in sl:
        ms.set_occupancy(x, v)
        stats.append(ms.update(stats=True))
        phases.append(ms.phase_times())
    info_final = ms.info()
    ms.close()
    # update phases: ingest = records applied with flip tracking, activation = changed bricks, their
    # dilation and the dirty runs, items = slot lists of the dirty runs
    phase_med = {k: statistics.median(p[k] for p in phases) for k in phases[0]}

    def timed(run_frame, label, before=None):
        # an NVTX range per timed sequence, so that a profiler can take just these frames; `before`
        # runs ahead of each frame's first event (stream-ordered, untimed)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nframes)]
        torch.cuda.nvtx.range_push(label)
        for k in range(nframes):
            flush.fill_(k & 255)
            if before is not None:
                before(k)
            ev[k][0].record(stream)
            run_frame(k)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        torch.cuda.nvtx.range_pop()
        return [a.elapsed_time(b) for a, b in ev]

    me = V.Map(nx, ny, nz, dmax, voxel_size=0.1, stream=stream)
    me.set_tuning(INCR_RUN, INCR_RUN, INCR_RUN, 3)
    me.global_()
    launches0 = V.kernel_launches()

    def eager(k):
        me.set_occupancy(*sl[k])
        me.update()

    eager_ms = timed(eager, "incremental_eager_frames")
    eager_launches = (V.kernel_launches() - launches0) / nframes
    D_eager = me.export_dense(on_device=True)
    me.close()

    mg = V.Map(nx, ny, nz, dmax, voxel_size=0.1, stream=stream)
    mg.set_tuning(INCR_RUN, INCR_RUN, INCR_RUN, 3)
    mg.global_()
    graph = V.UpdateGraph(mg, max(counts))
    # the frame's records written into the graph's input buffers before the frame (as a producer
    # writing there would), then the replay timed: staging, ingest and transform
    graph_ms = timed(lambda k: graph.replay(), "incremental_graph_frames", before=lambda k: graph.load(*sl[k]))
    D_graph = mg.export_dense(on_device=True)
    same = bool(torch.equal(D_eager, D_graph))
    del D_eager, D_graph
    mg.close()
    # UpdateGraph.run on the same frames: the copies into the input buffers inside each frame
    mr = V.Map(nx, ny, nz, dmax, voxel_size=0.1, stream=stream)
    mr.set_tuning(INCR_RUN, INCR_RUN, INCR_RUN, 3)
    mr.global_()
    graph_r = V.UpdateGraph(mr, max(counts))
    graph_run_ms = timed(lambda k: graph_r.run(*sl[k]), "incremental_graph_run_frames")
    mr.close()

    # global transform of the final occupancy (same step as the headline: reset + records + global)
    fx = torch.from_numpy(W.occupied_coords(final_occ)).cuda()
    fo = torch.ones(fx.shape[0], dtype=torch.uint8, device="cuda")
    mf = V.Map(nx, ny, nz, dmax, voxel_size=0.1, stream=stream)
    gms = []
    for k in range(8):
        flush.fill_(k & 255)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        mf.reset()
        mf.set_occupancy(fx, fo)
        mf.global_()
        b.record(stream)
        torch.cuda.synchronize()
        if k >= 3:
            gms.append(a.elapsed_time(b))
    mf.close()
    glob = statistics.median(gms)
    g = dist_summary(graph_ms)
    # algorithmic bytes of a frame: the unfused three-pass model (21 B per voxel) over the bricks the
    # z pass recomputes (its dirty runs, INCR_RUN bricks each: an upper bound on the influence
    # region), plus 16 B per record
    peak, peak_src = peaks()
    fbytes = [21 * 512 * s["z_items"] * INCR_RUN + 16 * s["records"] for s in stats]
    fgbs = [b / (t * 1e-3) / 1e9 for b, t in zip(fbytes, graph_ms)]
    # the same frames on the bricks each pass actually recomputed (stored bricks of the dirty runs),
    # at the stored widths (x: mask in + g1 out; y: g1 + g2; z: g2 + int32 D) and under the 21 B model
    sbytes = [1088 * s["x_bricks"] + 2048 * s["y_bricks"] + 3072 * s["z_bricks"] + 16 * s["records"] for s in stats]
    mbytes = [21 * 512 * s["z_bricks"] + 16 * s["records"] for s in stats]
    sgbs = [b / (t * 1e-3) / 1e9 for b, t in zip(sbytes, graph_ms)]
    mgbs = [b / (t * 1e-3) / 1e9 for b, t in zip(mbytes, graph_ms)]
    return {"frames": nframes, "workload": "lidar sequence along tunnel 0 of the scene, 64 beams x 1024 azimuths, "
                                           "range 400 voxels, 1 % noise; map starts empty",
            "records_per_frame": dist_summary([s["records"] for s in stats]),
            "set_records_per_frame": dist_summary(hits),
            "records_note": "set records are the rays' wall hits within range (at most 64 x 1024 per frame); the "
                            "other records clear the map-occupied voxels the rays traverse",
            "net_flips_per_frame": dist_summary([s["net_flips"] for s in stats]),
            "changed_bricks_per_frame": dist_summary([s["changed_bricks"] for s in stats]),
            "z_runs_per_frame": dist_summary([s["z_items"] for s in stats]),
            "runs": INCR_RUN, "graph_ms_per_frame": g, "eager_ms_per_frame": dist_summary(eager_ms),
            "graph_run_ms_per_frame": dist_summary(graph_run_ms),
            "graph_note": "graph: replay with the frame's records already in the graph's input buffers; graph_run: "
                          "UpdateGraph.run, which copies them there inside the frame (two device copies, one fill)",
            "roofline_frames": {"model": "21 B x 512 x bricks of the z pass's dirty runs + 16 B x records, per frame",
                                "bytes_per_frame": dist_summary(fbytes), "achieved_median": statistics.median(fgbs),
                                "unit": "GB/s", "peak": peak, "peak_source": peak_src,
                                "frac_median": statistics.median(fgbs) / peak},
            "roofline_frames_recomputed": {
                "model": "bricks each pass recomputed (stored bricks of its dirty runs) at stored widths: "
                         "1,088 B x, 2,048 B y, 3,072 B z per brick + 16 B per record",
                "bytes_per_frame": dist_summary(sbytes), "achieved_median": statistics.median(sgbs),
                "frac_median": statistics.median(sgbs) / peak, "unit": "GB/s", "peak": peak, "peak_source": peak_src,
                "model_21B": {"bytes_per_frame": dist_summary(mbytes), "achieved_median": statistics.median(mgbs),
                              "frac_median": statistics.median(mgbs) / peak},
                "bricks_per_frame": {a: dist_summary([s[a + "_bricks"] for s in stats]) for a in "xyz"}},
            "eager_phase_ms_median": phase_med,
            "eager_launches_per_frame": eager_launches,
            "global_ms_final_occupancy": glob, "global_over_graph_median": glob / g["median"],
            "final_map": {"occupied_voxels": int(final_occ.sum()), "allocated_bricks": info_final["allocated_bricks"]},
            "graph_equals_eager": same, "l2": "flushed before every frame (untimed)",
            **({"cpu_alg1": alg1} if alg1 else {})}, frames


def bench_crossover(V, torch, wl, occ, xyz_d, stream, flush, fractions=(1e-4, 3e-4, 1e-3, 3e-3, 1e-2, 3e-2, 0.1, 0.25, 0.5),
                    seed=17, untruncated=False):
    """Global against incremental transform after edits of growing size (the paper's ablation shape,
    Sec. V-A: remove a fraction of the obstacles at random and add as many new ones, uniform in the
    domain).  For each fraction the map holds the scene's field; the same records are staged and
    either vdbedt_update or vdbedt_global applies them (event-timed, L2 flushed before, 3 repeats,
    median); the two fields are compared.  untruncated: the same on the map without truncation."""
    nx, ny, nz = wl["dims"]
    dmax = None if untruncated else wl["dmax"]
    rs = np.random.default_rng(seed)
    n_obs = xyz_d.shape[0]
    ones = torch.ones(n_obs, dtype=torch.uint8, device="cuda")
    m = V.Map(nx, ny, nz, dmax, voxel_size=0.1, stream=stream)
    rows = []
    for f in fractions:
        k = max(1, int(round(f * n_obs)))
        rm = xyz_d[torch.from_numpy(rs.choice(n_obs, k, replace=False)).cuda()]
        add = torch.from_numpy(np.stack([rs.integers(0, nx, k), rs.integers(0, ny, k), rs.integers(0, nz, k)],
                                        1).astype(np.int32)).cuda()
        rec = torch.cat([rm, add])
        val = torch.cat([torch.zeros(k, dtype=torch.uint8, device="cuda"), torch.ones(k, dtype=torch.uint8, device="cuda")])
        res = {}
        for form in ("update", "global"):
            ts = []
            for r in range(3):
                m.reset()
                m.set_occupancy(xyz_d, ones)
                m.global_()
                m.set_occupancy(rec, val)
                flush.fill_(r)
                a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                if form == "update":
                    m.update()
                else:
                    m.global_()
                e.record(stream)
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(e))
            res[form] = statistics.median(ts)
            res[form + "_field"] = m.export_dense(on_device=True)
        m.reset()
        m.set_occupancy(xyz_d, ones)
        m.global_()
        m.set_occupancy(rec, val)
        st = m.update(stats=True)
        same = bool(torch.equal(res.pop("update_field"), res.pop("global_field")))
        row = {"fraction": f, "removed": k, "added": k, "net_flips": st["net_flips"],
               "changed_bricks": st["changed_bricks"], "z_bricks": st["z_bricks"],
               "update_ms": res["update"], "global_ms": res["global"],
               "global_over_update": res["global"] / res["update"], "same_field": same}
        if untruncated:
            del row["z_bricks"]
            row.update(x_rows=st["x_items"], y_lines=st["y_items"], z_lines=st["z_items"])
        rows.append(row)
    m.close()
    return {"workload": "the scene's obstacles; a fraction removed at random and as many added uniformly in the domain",
            "step": "staged records applied by vdbedt_update or by vdbedt_global on the same map", "rows": rows}


def bench_clearance(V, torch, m, occ, stream, reps=20):
    """Clearance cost of 8192 trajectories x 128 points in free space on the field of the headline
    workload: raw forward, raw forward + backward and the autograd path, event-timed."""
    import workloads as W
    T, P, tau = 8192, 128, 1.0
    pts = torch.from_numpy(W.free_points(11, occ, 0.1, T * P).reshape(T, P, 3)).cuda()
    ones = torch.ones(T, dtype=torch.float32, device="cuda")

    def time_it(fn):
        for _ in range(3):
            fn()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    fwd = time_it(lambda: m.clearance_forward(pts, tau))
    fb = time_it(lambda: (m.clearance_forward(pts, tau), m.clearance_backward(pts, tau, ones)))

    def autograd():
        p = pts.detach().requires_grad_(True)
        V.clearance_cost(m, p, tau).sum().backward()
        return p.grad

    ag = time_it(autograd)
    dg = time_it(lambda: m.distance_at(pts, with_grad=True))
    gr = m.clearance_backward(pts, tau, ones)
    active = float((gr.abs().sum(-1) > 0).float().mean().item())
    q = T * P
    return {"trajectories": T, "points_per_trajectory": P, "tau_m": tau, "voxel_m": 0.1,
            "fwd_ms": fwd, "fwd_queries_per_s": q / (fwd / 1e3),
            "fwd_bwd_ms": fb, "fwd_bwd_queries_per_s": q / (fb / 1e3),
            "autograd_fwd_bwd_ms": ag, "autograd_overhead_ms": ag - fb,
            "distance_gradient_ms": dg, "distance_gradient_queries_per_s": q / (dg / 1e3),
            "hinge_active_fraction": active,
            "hinge_active_rule": "points with a nonzero gradient (d < tau and a nonzero distance gradient)"}


def bench_batched(V, torch, stream, flush, autotuned=True, steps=5, warmup=3):
    """96 maps of uneven size (cubes of log-uniform side 32..512, Bernoulli(0.01..0.05) plus up to
    20 solid boxes, dmax 24, seed 7) from dense device grids: the batch (each step launched once
    for all maps) against the same maps as 96 single handles (every step launched per map)."""
    import workloads as W
    k, dmax, seed = 96, 24, 7
    grids_h = [W.batched_map(seed, i) for i in range(k)]
    dims = [(g.shape[2], g.shape[1], g.shape[0]) for g in grids_h]
    grids = [torch.from_numpy(g).cuda() for g in grids_h]
    del grids_h
    voxels = sum(int(g.numel()) for g in grids)
    b = V.Batch(dims, dmax, stream=stream)
    singles = [V.Map(nx, ny, nz, dmax, stream=stream) for nx, ny, nz in dims]
    b.set_occupancy_dense(grids)
    tuning = {"source": "default"}
    if autotuned:
        from paper_2105_04419_gb300.autotune import autotune
        tuning = autotune(b)  # untimed
        for m in singles:
            m.set_tuning(tuning["x_run"], tuning["y_run"], tuning["z_run"], tuning["variant"])

    def run_batch():
        b.set_occupancy_dense(grids)
        b.global_()

    def run_singles():
        for m, g in zip(singles, grids):
            m.set_occupancy_dense(g)
            m.global_()

    def timed(fn):
        for _ in range(warmup):
            fn()
        ms = []
        l0 = V.kernel_launches()
        for i in range(steps):
            flush.fill_(i & 255)
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            e.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(e))
        return statistics.median(ms), (V.kernel_launches() - l0) / steps

    batch_ms, batch_launches = timed(run_batch)
    single_ms, single_launches = timed(run_singles)
    b.set_profiling(True)
    a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a0.record(stream)
    b.set_occupancy_dense(grids)
    a1.record(stream)
    b.global_()
    phases = b.phase_times()
    dense_ms = a0.elapsed_time(a1)
    b.set_profiling(False)
    same = True
    active = 0
    allocated = 0
    for i in range(k):
        a = b.maps[i].export_dense(on_device=True)
        c = singles[i].export_dense(on_device=True)
        same &= bool(torch.equal(a, c))
        inf_i = b.maps[i].info()
        active += inf_i["finite_bricks"] * 512
        allocated += inf_i["allocated_bricks"]
        del a, c
    # bytes of the step: the unfused three-pass model (21 B per active voxel), and the stored widths
    # (dense uint8 grids in; per allocated brick 1,088 B x, 2,048 B y, 3,072 B z); the passes alone
    # against their phase times
    peak, peak_src = peaks()
    stored = voxels + 6208 * allocated
    pass_bytes = {"x": 1088 * allocated, "y_and_z": 5120 * allocated}
    roof = {"model_21B": {"bytes": 21 * active, "achieved": 21 * active / (batch_ms * 1e-3) / 1e9,
                          "frac": 21 * active / (batch_ms * 1e-3) / 1e9 / peak},
            "stored_widths": {"bytes": stored, "achieved": stored / (batch_ms * 1e-3) / 1e9,
                              "frac": stored / (batch_ms * 1e-3) / 1e9 / peak},
            "passes_stored_widths": {
                key: {"bytes": v, "achieved": v / (ph * 1e-3) / 1e9, "frac": v / (ph * 1e-3) / 1e9 / peak}
                for key, v, ph in (("x", pass_bytes["x"], phases["x_ms"]),
                                   ("y_and_z", pass_bytes["y_and_z"], phases["z_ms"]))},
            "allocated_bricks": allocated, "unit": "GB/s", "peak": peak, "peak_source": peak_src}
    upd = bench_batched_update(V, torch, b, singles, stream, flush, dims)
    for m in singles:
        m.close()
    b.close()
    return {"maps": k, "dmax": dmax, "seed": seed, "domain_voxels": voxels, "active_voxels": active,
            "update": upd,
            "sides": {"min": min(d[0] for d in dims), "max": max(d[0] for d in dims)},
            "step": "dense occupancy from device grids + global transform of every map",
            "batch_ms": batch_ms, "batch_mvoxels_per_s": active / (batch_ms / 1e3) / 1e6,
            "batch_domain_mvoxels_per_s": voxels / (batch_ms / 1e3) / 1e6, "batch_launches": batch_launches,
            "single_handles_ms": single_ms, "single_handles_mvoxels_per_s": active / (single_ms / 1e3) / 1e6,
            "single_handles_launches": single_launches, "single_over_batch": single_ms / batch_ms,
            "batch_phases_ms": {"reset_and_dense_ingest": dense_ms, "activation": phases["activation_ms"], "items": phases["items_ms"],
                                "x": phases["x_ms"], "y_and_z": phases["z_ms"]},
            "batch_equals_single_handles": same, "l2": "flushed between timed steps (untimed)",
            "roofline": roof, "tuning": {k: v for k, v in tuning.items() if k != "key"}}


def bench_batched_update(V, torch, b, singles, stream, flush, dims, records=2000, frames=8, warm=3, seed=13):
    """Incremental frames on the 96 maps: each map gets `records` random records per frame (2/3 set,
    1/3 clear, uniform in its grid).  The batch's update (each step one launch for all maps) replayed
    from one CUDA graph, against the 96 single handles' updates each replayed from its own graph;
    same records, same starting fields; event-timed per frame, L2 flushed before each."""
    k = len(dims)
    rs = np.random.default_rng(seed)
    fr = []
    for f in range(frames):
        per = []
        for nx, ny, nz in dims:
            xyz = np.stack([rs.integers(0, nx, records), rs.integers(0, ny, records), rs.integers(0, nz, records)],
                           1).astype(np.int32)
            val = (rs.random(records) < 2.0 / 3.0).astype(np.uint8)
            per.append((torch.from_numpy(xyz).cuda(), torch.from_numpy(val).cuda()))
        fr.append(per)
    bg = V.BatchUpdateGraph(b, records)
    sg = [V.UpdateGraph(m, records) for m in singles]

    def fill_batch(f):
        for i, (xyz, val) in enumerate(fr[f]):
            bg.xyz[i].copy_(xyz)
            bg.occ[i].copy_(val)
        bg.count.fill_(records)

    def fill_singles(f):
        for g, (xyz, val) in zip(sg, fr[f]):
            g.xyz.copy_(xyz)
            g.occ.copy_(val)
            g.count.fill_(records)

    def timed(fill, run):
        ms = []
        for f in range(frames):
            fill(f)
            flush.fill_(f & 255)
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            run()
            e.record(stream)
            torch.cuda.synchronize()
            if f >= warm:
                ms.append(a.elapsed_time(e))
        return statistics.median(ms)

    batch_ms = timed(fill_batch, bg.replay)

    def run_singles():
        for g in sg:
            g.replay()

    single_ms = timed(fill_singles, run_singles)
    same = all(bool(torch.equal(b.maps[i].export_dense(on_device=True), singles[i].export_dense(on_device=True)))
               for i in range(k))
    del bg, sg
    return {"frames_timed": frames - warm, "records_per_map_per_frame": records,
            "records": "uniform in each map, 2/3 set, 1/3 clear",
            "batch_graph_ms_per_frame": batch_ms, "single_graphs_ms_per_frame": single_ms,
            "single_over_batch": single_ms / batch_ms, "batch_equals_single_handles": same,
            "step": "one frame of incremental updates on every map (graph replays; records already on the device)"}


def bench_untruncated(V, torch, wl, xyz, ones, stream, flush, steps=5, warm=3):
    """The same scene with no truncation (the paper's dmax = infinity runs, Table II): reset + stage
    device records + global transform over whole lines of the grid, event-timed with the L2
    flushed before each step.  Bytes per voxel of the line passes (model, every value finite): x
    5 (g1 written once, 4; a carry per row and brick written and read back, 1), y and z 24 each
    (input 4, stack pushed and read 8 + 8, output 4)."""
    nx, ny, nz = wl["dims"]
    m = V.Map(nx, ny, nz, None, voxel_size=0.1, stream=stream)

    def step():
        m.reset()
        m.set_occupancy(xyz, ones)
        m.global_()

    for _ in range(warm):
        step()
    m.set_profiling(True)
    ms, ph = [], {"ingest_ms": [], "x_ms": [], "y_ms": [], "z_ms": []}
    for k in range(steps):
        flush.fill_(k & 255)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        pt = m.phase_times()
        for key in ph:
            ph[key].append(pt[key])
    m.set_profiling(False)
    info = m.info()
    probe = m.query(np.array([[nx // 2, ny // 2, nz // 2]], np.int32))
    m.close()
    vox = nx * ny * nz
    t = statistics.mean(ms)
    phm = {k: statistics.mean(v) for k, v in ph.items()}
    peak, peak_src = peaks()
    per_vox = {"x_ms": 5, "y_ms": 24, "z_ms": 24}
    return {"workload": wl["name"].replace(", dmax 32", "") + ", no truncation", "dmax": "none (untruncated)",
            "ms_per_step": t, "value": vox / (t / 1e3) / 1e6, "unit": "Mvoxels/s (every voxel of the grid)",
            "phases_ms": phm, "stored_bricks": info["allocated_bricks"], "finite_bricks": info["finite_bricks"],
            "centre_voxel_D": int(probe[0]),
            "passes_gbs_model": {k: vox * per_vox[k] / (phm[k] / 1e3) / 1e9 for k in per_vox},
            "bytes_per_voxel_model": per_vox, "peak": peak, "peak_source": peak_src,
            "l2": "flushed before every step (untimed)", "steps": steps}


def bench_untruncated_frames(V, torch, wl, frames, stream, flush):
    """The lidar frames of the incremental measurement on the untruncated map (the paper's Table II
    setting: per-frame updates with dmax = infinity), map starting empty: an untimed pass with
    statistics (lines each pass recomputes), the eager frames and the captured update's replays
    (records placed in its input buffers before each frame), each frame event-timed with the L2
    flushed before it; then the field against a global transform of the final occupancy."""
    nx, ny, nz = wl["dims"]
    nframes = len(frames)
    counts = [len(v) for _, v in frames]
    offs = np.concatenate([[0], np.cumsum(counts)])
    xyz_d = torch.from_numpy(np.concatenate([x for x, _ in frames])).cuda()
    val_d = torch.from_numpy(np.concatenate([v for _, v in frames])).cuda()
    sl = [(xyz_d[offs[k]:offs[k + 1]], val_d[offs[k]:offs[k + 1]]) for k in range(nframes)]

    def fresh():
        m = V.Map(nx, ny, nz, None, voxel_size=0.1, stream=stream)
        m.global_()
        return m

    m = fresh()
    stats = []
    for x, v in sl:
        m.set_occupancy(x, v)
        stats.append(m.update(stats=True))
    m.close()

    def timed(run_frame, before=None):
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nframes)]
        for k in range(nframes):
            flush.fill_(k & 255)
            if before is not None:
                before(k)
            ev[k][0].record(stream)
            run_frame(k)
            ev[k][1].record(stream)
        torch.cuda.synchronize()
        return [a.elapsed_time(b) for a, b in ev]

    m = fresh()

    def eager(k):
        m.set_occupancy(*sl[k])
        m.update()

    eager_ms = timed(eager)
    D_eager = m.export_dense(on_device=True)
    # the global transform of the final occupancy on the same map, timed (reset + records + global)
    final = m.export_occupancy(0, nz)
    u = final.view(torch.int64)
    fx = torch.stack([u & ((1 << 21) - 1), (u >> 21) & ((1 << 21) - 1), (u >> 42) & ((1 << 21) - 1)], 1)
    fx = fx.to(torch.int32).contiguous()
    fo = torch.ones(fx.shape[0], dtype=torch.uint8, device="cuda")
    gms = []
    for k in range(4):
        flush.fill_(k & 255)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        m.reset()
        m.set_occupancy(fx, fo)
        m.global_()
        b.record(stream)
        torch.cuda.synchronize()
        if k >= 1:
            gms.append(a.elapsed_time(b))
    same_global = bool(torch.equal(D_eager, m.export_dense(on_device=True)))
    m.close()
    mg = fresh()
    graph = V.UpdateGraph(mg, max(counts))
    graph_ms = timed(lambda k: graph.replay(), before=lambda k: graph.load(*sl[k]))
    same_graph = bool(torch.equal(D_eager, mg.export_dense(on_device=True)))
    mg.close()
    del D_eager
    glob = statistics.median(gms)
    g = dist_summary(graph_ms)
    return {"frames": nframes, "workload": "the incremental measurement's lidar frames on the untruncated map "
                                           "(map starts empty)",
            "net_flips_per_frame": dist_summary([s["net_flips"] for s in stats]),
            "lines_per_frame": {"x_rows": dist_summary([s["x_items"] for s in stats]),
                                "y_lines": dist_summary([s["y_items"] for s in stats]),
                                "z_lines": dist_summary([s["z_items"] for s in stats]),
                                "of": {"x_rows": ny * nz, "y_lines": nx * nz, "z_lines": nx * ny}},
            "global_form_frames": int(sum(s["global_form"] for s in stats)),
            "graph_ms_per_frame": g, "eager_ms_per_frame": dist_summary(eager_ms),
            "global_ms_final_occupancy": glob, "global_over_graph_median": glob / g["median"],
            "equals_global_of_final_occupancy": same_global, "graph_equals_eager": same_graph,
            "l2": "flushed before every frame (untimed)"}


def bench_nearest(V, torch, m, dims, stream, reps=20):
    """Nearest-obstacle query of 2^20 voxels uniform in the grid, device in and out, event-timed."""
    nx, ny, nz = dims
    g = torch.Generator(device="cuda").manual_seed(5)
    n = 1 << 20
    q = torch.stack([torch.randint(0, nx, (n,), generator=g, device="cuda"),
                     torch.randint(0, ny, (n,), generator=g, device="cuda"),
                     torch.randint(0, nz, (n,), generator=g, device="cuda")], 1).to(torch.int32).contiguous()
    for _ in range(3):
        out = m.query_nearest(q)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(reps):
        out = m.query_nearest(q)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    found = float((out[:, 0] >= 0).float().mean().item())
    return {"queries": n, "ms": ms, "queries_per_s": n / (ms / 1e3), "with_obstacle_fraction": found,
            "rule": "nearest occupied voxel, ties to the smallest (z, y, x); voxels uniform in the grid"}


def host_cpu():
    """The host's cores: os.sched_getaffinity and lscpu."""
    info = {"affinity_cores": len(os.sched_getaffinity(0))}
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            key, _, v = ln.partition(":")
            key = key.strip()
            if key in ("Architecture", "CPU(s)", "Model name", "Thread(s) per core", "Core(s) per socket",
                       "Socket(s)", "CPU max MHz"):
                info[key] = v.strip()
    except Exception:
        info["lscpu"] = "unavailable"
    return info


def cpu_baseline(occ, dmax, budget_s=12.0):
    """The CPU oracle (Eq. 1 factorised, OpenMP on all host cores) on a z-slab of the workload."""
    import oracle as O
    nz = occ.shape[0]
    cores = O.num_threads()
    # size the slab so the run takes roughly budget_s: calibrate on a thin slab first
    t0 = time.perf_counter()
    thin = np.ascontiguousarray(occ[: min(8, nz)])
    O.edt_factorised(thin, dmax)
    per_plane = (time.perf_counter() - t0) / thin.shape[0]
    planes = int(max(8, min(nz, budget_s / max(per_plane, 1e-6))))
    slab = np.ascontiguousarray(occ[:planes])
    t0 = time.perf_counter()
    D = O.edt_factorised(slab, dmax)
    dt = time.perf_counter() - t0
    active = active_voxels_of(D, dmax)
    ny, nx = slab.shape[1:]
    return {"value": active / dt / 1e6, "unit": "Mvoxels/s", "cores": cores, "kind": "oracle",
            "sample": f"Eq. 1 factorised (OpenMP) on the first {planes} z-planes ({nx}x{ny}x{planes}) of the "
                      f"workload; {active} active voxels in {dt:.2f} s"}


def cpu_baselines_other(frames_first, truth, dmax3, budget4_voxels=300_000_000):
    """The oracle on the other workloads, timed on the host cores: Eq. 1 factorised (OpenMP) on the
    dense 64^3 cube (median of 5) and on the first maps of the 96-map batch (about 3e8 voxels); the
    paper's Alg. 1 (one thread, as the paper runs it) global on the 64^3 cube and on the first lidar
    frame from an empty map."""
    import oracle as O
    import workloads as W
    out = {"o1": {}, "o2_alg1": {}}
    occ1 = W.bernoulli_grid(0, (64, 64, 64), 0.02)
    ts = []
    for _ in range(5):
        t0 = time.perf_counter()
        D1 = O.edt_factorised(occ1, 16)
        ts.append(time.perf_counter() - t0)
    a1 = active_voxels_of(D1, 16)
    out["o1"]["cube64_dmax16"] = {"ms": 1e3 * statistics.median(ts), "mvoxels_per_s": a1 / statistics.median(ts) / 1e6,
                                  "active_voxels": a1, "threads": O.num_threads()}
    voxels, act, dt, maps = 0, 0, 0.0, 0
    while voxels < budget4_voxels and maps < 96:
        g = W.batched_map(7, maps)
        t0 = time.perf_counter()
        D = O.edt_factorised(g, 24)
        dt += time.perf_counter() - t0
        act += active_voxels_of(D, 24)
        voxels += g.size
        maps += 1
        del D, g
    out["o1"]["batch96_dmax24_first_maps"] = {"maps": maps, "domain_voxels": voxels, "active_voxels": act,
                                              "s": dt, "mvoxels_per_s": act / dt / 1e6, "threads": O.num_threads()}
    a = O.Alg1(occ1.shape, 16)
    try:
        t0 = time.perf_counter()
        a.global_(occ1)
        ms = 1e3 * (time.perf_counter() - t0)
        exact = bool(np.array_equal(a.dist(), D1))
        out["o2_alg1"]["cube64_dmax16_global"] = dict(ms=ms, mvoxels_per_s=a1 / (ms / 1e3) / 1e6, threads=1,
                                                      equals_eq1=exact, **a.counters())
    finally:
        a.close()
    if frames_first:
        out["o2_alg1"]["lidar_first_frames_dmax32"] = alg1_frames(truth, frames_first, dmax3, len(frames_first))
    return out


def active_voxels_of(D, dmax):
    nz, ny, nx = D.shape
    bz, by, bx = -(-nz // 8), -(-ny // 8), -(-nx // 8)
    pad = np.full((bz * 8, by * 8, bx * 8), dmax * dmax, dtype=D.dtype)
    pad[:nz, :ny, :nx] = D
    fin = (pad < dmax * dmax).reshape(bz, 8, by, 8, bx, 8).any(axis=(1, 3, 5))
    return int(fin.sum()) * 512


def run_reference(args, wl):
    """The oracle as the reference arm: each step is the CPU factorised transform of a bounded
    sample (a z-slab) of the workload, on the host cores of rank 0."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle as O
    occ = make_occupancy(wl)
    dmax = wl["dmax"]
    nz = occ.shape[0]
    budget = 150.0 / max(1, args.steps + args.warmup)
    t0 = time.perf_counter()
    O.edt_factorised(np.ascontiguousarray(occ[: min(8, nz)]), dmax)
    per_plane = (time.perf_counter() - t0) / min(8, nz)
    planes = int(max(8, min(nz, budget / max(per_plane, 1e-6))))
    slab = np.ascontiguousarray(occ[:planes])
    for _ in range(args.warmup):
        O.edt_factorised(slab, dmax)
    times = []
    D = None
    for _ in range(args.steps):
        t0 = time.perf_counter()
        D = O.edt_factorised(slab, dmax)
        times.append(time.perf_counter() - t0)
    active = active_voxels_of(D, dmax)
    ms = 1e3 * statistics.mean(times)
    value = active / (ms / 1e3) / 1e6
    ny, nx = slab.shape[1:]
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "Mvoxels/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": wl["name"], "sample": f"{nx}x{ny}x{planes} z-slab"},
            "cpu_baseline": {"value": value, "unit": "Mvoxels/s", "cores": O.num_threads(), "kind": "oracle",
                             "sample": f"Eq. 1 factorised (OpenMP) on the first {planes} z-planes"},
            "e2e": {"value": value, "unit": "Mvoxels/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_shard_slabs(args, wl, V, torch, dist, rank, world, local):
    """One grid over the ranks: z-slabs (paper_2105_04419_gb300.slabs.SlabMap).  One step = every
    rank's own global transform, export of its halo bands, the record exchange with its neighbours
    (NCCL point-to-point), the staging of the neighbours' records and an incremental update.
    value = active voxels of the whole grid / the slowest rank's step time (L2 flushed between
    steps); bytes exchanged are reported per rank."""
    import workloads as W
    from paper_2105_04419_gb300 import slabs as S
    nx, ny, nz = wl["dims"]
    dmax = wl["dmax"]
    occ = make_occupancy(wl)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    sm = S.SlabMap(nx, ny, nz, dmax, rank, world, device=local, stream=stream)
    z, y, x = np.nonzero(occ[sm.z0:sm.z1])
    own = torch.from_numpy(np.stack([x, y, z + (sm.z0 - sm.h0)], 1).astype(np.int32)).cuda()
    ones = torch.ones(own.shape[0], dtype=torch.uint8, device="cuda")
    del occ
    group = dist.group.WORLD if world > 1 else None

    def step():
        if world > 1:
            sm.global_(own, ones, group=group)
        else:
            sm.finish(sm.begin_global(own, ones))

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    ms = []
    b0 = sm.bytes_sent
    for k in range(args.steps):
        flush.fill_(k & 255)
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        e.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(e))
    if world > 1:
        dist.barrier()
    step_ms = max_over_ranks(statistics.mean(ms))
    sent = (sm.bytes_sent - b0) / max(1, args.steps)
    d = sm.owned_field()
    nzo = d.shape[0]
    bz, by, bx = -(-nzo // 8), -(-ny // 8), -(-nx // 8)
    pad = torch.full((bz * 8, by * 8, bx * 8), dmax * dmax, dtype=torch.int32, device="cuda")
    pad[:nzo, :ny, :nx] = d
    act = torch.tensor([float((pad < dmax * dmax).view(bz, 8, by, 8, bx, 8).any(5).any(3).any(1).sum().item()) * 512],
                       dtype=torch.float64, device="cuda")
    per_rank = torch.tensor([float(sent), float(sm.h1 - sm.h0)], dtype=torch.float64, device="cuda")
    if world > 1:
        dist.all_reduce(act)
        allr = [torch.zeros_like(per_rank) for _ in range(world)]
        dist.all_gather(allr, per_rank)
    else:
        allr = [per_rank]
    sm.close()
    if rank == 0:
        line = {"metric": METRIC, "value": act.item() / (step_ms / 1e3) / 1e6, "unit": "Mvoxels/s", "n_gpus": world,
                "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": step_ms, "higher_is_better": True,
                "scaling": "strong", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
                "config": {"workload": wl["name"], "parallelism": f"z-slabs x{world}",
                           "step": "own global + band export + record exchange + incremental update of the halos",
                           "l2": "flushed between timed steps (256 MiB write, untimed)"},
                "shard": {"bytes_sent_per_step_per_rank": [r[0].item() for r in allr],
                          "extended_planes_per_rank": [int(r[1].item()) for r in allr],
                          "halo_planes": S.halo_planes(dmax)}}
        print(json.dumps(line), flush=True)


def main():
    args = parse()
    wl = WORKLOADS[args.workload]
    if args.impl == "reference":
        run_reference(args, wl)
        return
    import torch
    import torch.distributed as dist
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    from paper_2105_04419_gb300 import build as B
    if not B.up_to_date():
        if rank == 0 or world == 1:
            B.build()
        if world > 1:
            dist.barrier()
    import paper_2105_04419_gb300 as V

    if args.shard == "slabs":
        run_shard_slabs(args, wl, V, torch, dist, rank, world, local)
        if world > 1:
            dist.destroy_process_group()
        return
    occ = make_occupancy(wl)
    nx, ny, nz = wl["dims"]
    dmax = wl["dmax"]
    import workloads as W
    xyz_h = W.occupied_coords(occ)
    n = len(xyz_h)
    ones_h = np.ones(n, np.uint8)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)  # everything below (torch and the library) runs on this stream
    xyz = torch.from_numpy(xyz_h).cuda()
    ones = torch.from_numpy(ones_h).cuda()
    m = V.Map(nx, ny, nz, dmax, voxel_size=0.1, stream=stream)
    tuning = {"source": "default"}
    if args.variant or args.x_run or args.y_run or args.z_run:
        m.set_tuning(args.x_run, args.y_run, args.z_run, args.variant)
        tuning = {"source": "command line", "x_run": args.x_run, "y_run": args.y_run, "z_run": args.z_run,
                  "variant": args.variant}
    elif not args.no_autotune:
        from paper_2105_04419_gb300.autotune import autotune
        m.set_occupancy(xyz, ones)
        tuning = autotune(m)  # untimed; leaves the chosen tuning set

    def step():
        m.reset()
        m.set_occupancy(xyz, ones)
        m.global_()

    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    info = m.info()
    active = info["finite_bricks"] * 512
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")

    m.set_profiling(True)
    phases = {k: [] for k in ("ingest_ms", "activation_ms", "items_ms", "x_ms", "y_ms", "z_ms")}
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = V.kernel_launches()
    for k in range(args.steps):
        flush.fill_(k & 255)  # evict the previous step's data from L2 (not timed)
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
        pt = m.phase_times()  # waits for this step; device times are unaffected
        for key in phases:
            phases[key].append(pt[key])
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    launches = V.kernel_launches() - launches0
    clocks = sampler.stop()
    m.set_profiling(False)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = max_over_ranks(statistics.mean(step_ms))
    value = active * world / (ms / 1e3) / 1e6
    ph = {k: statistics.mean(v) for k, v in phases.items()}

    # roofline: dominant kernel with its compulsory bytes at the stored widths
    peak, peak_src = peaks()
    allocated = info["allocated_bricks"]
    # compulsory bytes per brick: x pass mask in + g1 out; y pass g1 in + g2 out; z pass g2 in + D out
    per_brick = {"x_ms": 64 + 1024, "y_ms": 1024 + 1024, "z_ms": 1024 + 2048}
    dom = max(per_brick, key=lambda k: ph[k])
    kname = {"x_ms": "k_pass<x>", "y_ms": "k_pass<y>", "z_ms": "k_pass<z>"}[dom]
    achieved = allocated * per_brick[dom] / (ph[dom] / 1e3) / 1e9
    tr = traffic_for(kname, tuning)
    roofline = {"kernel": kname, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src,
                "bytes_per_brick": per_brick[dom], "bricks_per_launch": allocated,
                "traffic": (tr["dram_bytes_per_launch"] if tr else None)}
    # whole step against the unfused three-pass model (21 B per active voxel) and the compulsory
    # bytes (bit mask in, int32 out: 4.125 B per active voxel)
    roof_step = {"model_B_per_active_voxel": 21.0, "achieved": active * 21.0 / (ms / 1e3) / 1e9,
                 "frac": active * 21.0 / (ms / 1e3) / 1e9 / peak,
                 "compulsory_B_per_active_voxel": 4.125,
                 "frac_compulsory": active * 4.125 / (ms / 1e3) / 1e9 / peak, "peak": peak, "unit": "GB/s"}

    # the same step captured once into a CUDA graph (reset + counted staging + global) and replayed
    graph = V.GlobalGraph(m, n)
    graph.xyz.copy_(xyz)
    graph.occ.copy_(ones)
    graph.count.fill_(n)
    for _ in range(max(3, args.warmup)):
        graph.replay()
    gev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    launches_g0 = V.kernel_launches()
    for k in range(args.steps):
        flush.fill_(k & 255)
        gev[k][0].record(stream)
        graph.replay()
        gev[k][1].record(stream)
    torch.cuda.synchronize()
    graph_ms = max_over_ranks(statistics.mean(a.elapsed_time(b) for a, b in gev))
    graph_launches = V.kernel_launches() - launches_g0  # host launches inside the graph replays: 0
    del graph

    line = {"metric": METRIC, "value": value, "unit": "Mvoxels/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": {"workload": wl["name"], "dims_xyz": list(wl["dims"]), "dmax": dmax, "occupied_voxels": n,
                       "active_bricks": info["finite_bricks"], "allocated_bricks": allocated,
                       "obstacle_bricks": info["obstacle_bricks"], "parallelism": f"replicas x{world}",
                       "l2": "flushed between timed steps (256 MiB write, untimed)",
                       "step": "reset + stage device records + global transform",
                       "tuning": {k: v for k, v in tuning.items() if k != "key"}},
            "phases_ms": ph, "roofline": roofline, "roofline_step": roof_step, "gpu_launches": launches,
            "clocks": clocks,
            "graph_replay": {"ms_per_step": graph_ms, "value": active * world / (graph_ms / 1e3) / 1e6,
                             "unit": "Mvoxels/s", "library_launches_per_step": launches / args.steps,
                             "host_launches_during_replay": graph_launches,
                             "step": "the same step captured once into a CUDA graph and replayed"}}

    if not args.no_e2e:
        # end to end through the C ABI with host buffers (pinned): the occupancy host -> device (the
        # occupied bricks as 64-byte masks; packed 64-bit records and the (x, y, z) + occ form
        # beside it), the transform, and a host consumer's read-back: D at 2^20 voxels uniform in the
        # grid, queried from host memory into host memory (coordinates in, distances out), with the
        # grid's counters
        nq = 1 << 20
        rq = np.random.default_rng(21)
        q_h = torch.from_numpy(np.stack([rq.integers(0, nx, nq), rq.integers(0, ny, nq), rq.integers(0, nz, nq)],
                                        1).astype(np.int32)).pin_memory().numpy()
        d_h = torch.empty(nq, dtype=torch.int32).pin_memory().numpy()
        packed_h = torch.from_numpy(V.pack_records(xyz_h, ones_h).view(np.int64)).pin_memory().numpy().view(np.uint64)
        xyz_p = torch.from_numpy(xyz_h).pin_memory().numpy()
        ones_p = torch.from_numpy(ones_h).pin_memory().numpy()
        bk_h, bm_h = V.brick_masks(occ)
        nb = len(bk_h)
        bk_p = torch.from_numpy(bk_h).pin_memory().numpy()
        bm_p = torch.from_numpy(bm_h.view(np.int64)).pin_memory().numpy().view(np.uint64)
        lib = V.load()

        def e2e(stage):
            ms = []
            for k in range(max(3, args.warmup) + args.steps):
                flush.fill_(k & 255)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                m.reset()
                stage()
                m.global_()
                V.lib._check(lib.vdbedt_query(m.handle, q_h.ctypes.data, nq, d_h.ctypes.data, 0), "vdbedt_query",
                             m.handle)
                inf2 = m.info()
                ms.append(1e3 * (time.perf_counter() - t0))
            return max_over_ranks(statistics.mean(ms[max(3, args.warmup):])), inf2

        emsb, inf2 = e2e(lambda: m.set_occupancy_bricks(bk_p, bm_p))
        qref = m.query(q_h)
        same_b = bool(np.array_equal(qref, d_h))
        ems, _ = e2e(lambda: m.set_occupancy_packed(packed_h))
        ems3, _ = e2e(lambda: m.set_occupancy(xyz_p, ones_p))
        act = inf2["finite_bricks"] * 512 * world
        line["e2e"] = {"value": act / (emsb / 1e3) / 1e6, "unit": "Mvoxels/s",
                       "ms_per_step": emsb, "host_buffers": "pinned",
                       "records": f"occupied bricks as 64-byte masks + brick coordinates ({nb} bricks)",
                       "h2d_bytes_per_step": int(nb * 76 + nq * 12), "d2h_bytes_per_step": int(nq * 4 + 4 * 19 + 16),
                       "readback": f"D at {nq} voxels (vdbedt_query, host in and out) + grid counters",
                       "readback_equals_device_query": same_b,
                       "packed_form": {"ms_per_step": ems, "value": act / (ems / 1e3) / 1e6,
                                       "h2d_bytes_per_step": int(n * 8 + nq * 12)},
                       "triples_form": {"ms_per_step": ems3, "value": act / (ems3 / 1e3) / 1e6,
                                        "h2d_bytes_per_step": int(n * 13 + nq * 12)}}

    if wl["kind"] == "tunnel" and not args.no_clearance:
        line["clearance"] = bench_clearance(V, torch, m, occ, stream)
        line["nearest"] = bench_nearest(V, torch, m, wl["dims"], stream)
    if wl["kind"] == "tunnel" and not args.no_crossover:
        line["crossover"] = bench_crossover(V, torch, wl, occ, xyz, stream, flush)
    if wl["kind"] == "tunnel" and not args.no_batched:
        line["batched"] = bench_batched(V, torch, stream, flush, autotuned=not args.no_autotune)
    frames = None
    if wl["kind"] == "tunnel" and not args.no_incremental:
        line["incremental"], frames = bench_incremental(V, torch, wl, occ, stream, flush, args.frames,
                                                        args.incr_run, 0)
    if wl["kind"] == "tunnel" and not args.no_untruncated:
        line["untruncated"] = bench_untruncated(V, torch, wl, xyz, ones, stream, flush)
        if frames:
            line["untruncated"]["incremental"] = bench_untruncated_frames(V, torch, wl, frames, stream, flush)
        if not args.no_crossover:
            line["untruncated"]["crossover"] = bench_crossover(V, torch, wl, occ, xyz, stream, flush,
                                                               fractions=(1e-4, 1e-3, 1e-2, 0.1), untruncated=True)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(occ, dmax)
        line["cpu_baseline"]["host"] = host_cpu()
        first = frames[:args.alg1_frames] if (frames and args.alg1_frames > 0 and wl["kind"] == "tunnel") else None
        line["cpu_baseline"].update(cpu_baselines_other(first, occ, dmax))
    if rank == 0:
        print(json.dumps(line), flush=True)
    m.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
