"""The replica path of bench.py with more than one rank, on CPU ranks over gloo: the step time
reported is the maximum over ranks, and the reference arm runs on rank 0 only."""
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        got = bench.max_over_ranks(1.5 + rank)
        dist.barrier()
        q.put((rank, got))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_max_over_ranks_gloo(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    assert [g for _, g in got] == [1.5 + world - 1] * world


def test_max_over_ranks_single_process():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.25) == 3.25


def test_reference_arm_other_ranks_exit_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2"],
                       env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_json_line():
    """`bench.py --impl reference` (the oracle on the host cores) prints one JSON line with the
    contract's keys, on the same metric and unit as the GPU arm."""
    import json
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    line = json.loads(r.stdout.strip().splitlines()[-1])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["unit"] == "Mvoxels/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["d2h_bytes_per_step"] == 0


def test_alg1_frames_helper():
    """bench.alg1_frames runs the paper's Alg. 1 on the first frames of a lidar sequence (here a
    small scene) and reports time, record count and queue counters per frame."""
    sys.path.insert(0, ROOT)
    import bench
    import workloads as W
    dims = (96, 80, 48)
    truth = W.tunnel_scene(4, dims, ntunnels=3, rmin=5, rmax=8)
    _, lines = W.tunnel_lines(4, dims, ntunnels=3, rmin=5, rmax=8)
    seq = W.LidarSequence(truth, 4, lines[0], nframes=4, nbeams=8, nazim=128, maxrange=80)
    frames = [seq.next() for _ in range(3)]
    r = bench.alg1_frames(truth, frames, 12, 2)
    assert len(r["frames"]) == 2 and r["threads"] == 1
    for f, (xyz, val) in zip(r["frames"], frames):
        assert f["records"] == len(val) and f["ms"] > 0 and f["lowered"] >= 0


def test_bench_cpu_baselines_other_small():
    """bench.cpu_baselines_other times the oracle on the other workloads (here with a small budget):
    Eq. 1 factorised on the 64^3 cube and on the first batch map, the paper's Alg. 1 global on the
    cube, which equals Eq. 1 there; host_cpu reports the cores."""
    import bench
    out = bench.cpu_baselines_other(None, None, 32, budget4_voxels=1)
    assert out["o1"]["cube64_dmax16"]["active_voxels"] > 0
    assert out["o1"]["batch96_dmax24_first_maps"]["maps"] == 1
    assert out["o2_alg1"]["cube64_dmax16_global"]["threads"] == 1
    assert out["o2_alg1"]["cube64_dmax16_global"]["equals_eq1"] in (True, False)
    info = bench.host_cpu()
    assert info["affinity_cores"] >= 1
