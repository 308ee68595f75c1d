"""The autotuner's choice logic and cache (CPU; a fake target stands in for a map), and on the GPU
that a tuned map still gives the oracle's exact field."""
import json

import numpy as np
import pytest

from paper_2105_04419_gb300 import autotune as A


def table_from(fn, envelope=None):
    t = {(v, r): fn(v, r) for v in A.VARIANTS for r in A.RUNS}
    if envelope is not None:
        t[A.ENVELOPE_KEY] = envelope
    return t


def test_choose_envelope_only_when_faster_overall():
    # windowed best: x 1.0 (run 16) + y 4.0 (run 8) + z 4.0 (run 4) = 9.0
    def t(v, r):
        return {"x_ms": {4: 3.0, 8: 2.0, 16: 1.0}[r] + (0.5 if v & 4 else 0.0),
                "y_ms": {4: 5.0, 8: 4.0, 16: 6.0}[r] * (2.0 if v == 1 else 1.0),
                "z_ms": {4: 4.0, 8: 5.0, 16: 7.0}[r] * (2.0 if v == 1 else 1.0)}
    slower = {"x_ms": 1.0, "y_ms": 4.0, "z_ms": 4.1}       # 9.1: the windowed choice stays
    tie = {"x_ms": 1.0, "y_ms": 3.9, "z_ms": 3.95}          # 8.85, within 2 %: the windowed choice stays
    faster = {"x_ms": 0.5, "y_ms": 2.0, "z_ms": 2.0}       # 4.5: the envelope form wins
    win = {"x_run": 16, "y_run": 8, "z_run": 4, "variant": 3}
    assert A.choose(table_from(t, slower)) == win
    assert A.choose(table_from(t, tie)) == win
    assert A.choose(table_from(t, faster)) == {"x_run": 16, "y_run": 16, "z_run": 16, "variant": 8}
    # above dmax 45 only the envelope is timed
    assert A.choose({A.ENVELOPE_KEY: faster})["variant"] == 8


def test_choose_per_axis_minimum():
    # x best at run 16 with the ring kernel, y best at 8, z best at 4; pruned windows faster
    def t(v, r):
        return {"x_ms": {4: 3.0, 8: 2.0, 16: 1.0}[r] + (0.5 if v & 4 else 0.0),
                "y_ms": {4: 5.0, 8: 4.0, 16: 6.0}[r] * (2.0 if v == 1 else 1.0),
                "z_ms": {4: 4.0, 8: 5.0, 16: 7.0}[r] * (2.0 if v == 1 else 1.0)}
    assert A.choose(table_from(t)) == {"x_run": 16, "y_run": 8, "z_run": 4, "variant": 3}


def test_choose_x_direct_bit():
    # the plain-load x kernel wins at run 8; the window variant stays the full one
    def t(v, r):
        return {"x_ms": 1.0 if (v & 4 and r == 8) else 2.0,
                "y_ms": 1.0 if v == 1 else 3.0, "z_ms": 1.0 if v == 1 else 3.0}
    assert A.choose(table_from(t)) == {"x_run": 8, "y_run": 8, "z_run": 8, "variant": 5}  # equal runs: run 8


def test_choose_variant_by_best_yz_sum():
    # variant 1 wins on y + z at its best runs even though variant 3 wins y alone at run 4
    def t(v, r):
        if v & 3 == 3:
            return {"x_ms": 1.0, "y_ms": {4: 1.0, 8: 9.0, 16: 9.0}[r], "z_ms": 9.0}
        return {"x_ms": 1.0, "y_ms": 2.0, "z_ms": {4: 3.0, 8: 2.5, 16: 4.0}[r]}
    got = A.choose(table_from(t))
    assert got["variant"] == 1 and got["z_run"] == 8


def test_choose_near_ties_go_to_the_preferred_run():
    # z at run 16 is 1 % faster than at run 8 (noise-sized): run 8 is kept; y at run 4 is 10 %
    # faster than at run 8: run 4 wins
    def t(v, r):
        return {"x_ms": 1.0 + (v & 4), "y_ms": {4: 0.9, 8: 1.0, 16: 1.2}[r] + (v == 1),
                "z_ms": {4: 1.5, 8: 1.0, 16: 0.99}[r] + (v == 1)}
    got = A.choose(table_from(t))
    assert got == {"x_run": 8, "y_run": 4, "z_run": 8, "variant": 3}


def test_choose_joint_yz():
    def t(v, r):
        return {"x_ms": 1.0 + (v & 4), "y_ms": 0.0, "z_ms": {4: 3.0, 8: 1.0, 16: 2.0}[r] + (v == 1)}
    got = A.choose(table_from(t), joint_yz=True)
    assert got["y_run"] == got["z_run"] == 8 and got["variant"] == 3


class FakeTarget:
    """Records calls; phase times depend on the tuning like a pass that prefers run 8 (the
    envelope form, variant 8, is slower overall)."""

    device = 0
    dmax = 32

    def __init__(self):
        self.tuning = None
        self.globals = 0
        self.profiling = False

    def set_tuning(self, x_run, y_run, z_run, variant):
        self.tuning = (x_run, y_run, z_run, variant)

    def set_profiling(self, on=True):
        self.profiling = on

    def global_(self):
        self.globals += 1

    def phase_times(self):
        x, y, z, v = self.tuning
        if v == A.ENVELOPE:
            return {"x_ms": 1.0, "y_ms": 2.0, "z_ms": 2.0}
        cost = {4: 2.0, 8: 1.0, 16: 3.0}
        return {"x_ms": cost[x] + (v & 4), "y_ms": cost[y] + (v == 1), "z_ms": cost[z] + (v == 1)}


def test_autotune_measures_then_uses_cache(tmp_path, monkeypatch):
    monkeypatch.setattr(A, "signature", lambda target: "fake|R=4|grids=1|bricks~100")
    path = str(tmp_path / "tuning.json")
    t = FakeTarget()
    got = A.autotune(t, reps=2, cache_path=path)
    assert got["source"] == "measured"
    assert (got["x_run"], got["y_run"], got["z_run"], got["variant"]) == (8, 8, 8, 3)
    assert t.tuning == (8, 8, 8, 3) and not t.profiling
    data = json.load(open(path))
    assert data["fake|R=4|grids=1|bricks~100"]["variant"] == 3
    t2 = FakeTarget()
    got2 = A.autotune(t2, reps=2, cache_path=path)
    assert got2["source"] == "cache" and t2.tuning == (8, 8, 8, 3) and t2.globals == 2


def test_round_sig():
    assert A._round_sig(467113) == 470000 and A._round_sig(0) == 0 and A._round_sig(7) == 7


@pytest.mark.gpu
def test_autotuned_map_is_exact(tmp_path):
    import oracle as O
    import workloads as W
    import paper_2105_04419_gb300 as V
    from gpu_common import first_mismatch
    occ = W.tunnel_scene(2, (192, 160, 64), ntunnels=6, rmin=5, rmax=9)
    m = V.Map(192, 160, 64, 20)
    m.set_occupancy_dense(occ)
    got = A.autotune(m, reps=2, cache_path=str(tmp_path / "t.json"))
    assert got["source"] == "measured" and got["variant"] in (1, 3, 5, 7, 8)
    assert first_mismatch(m.export_dense(), O.edt_factorised(occ, 20)) is None
    again = A.autotune(m, reps=2, cache_path=str(tmp_path / "t.json"))
    assert again["source"] == "cache"


@pytest.mark.gpu
def test_autotuned_batch_is_exact(tmp_path):
    import oracle as O
    import workloads as W
    import paper_2105_04419_gb300 as V
    from gpu_common import first_mismatch
    grids = [W.batched_map(3, i, smin=32, smax=80) for i in range(5)]
    b = V.Batch([(g.shape[2], g.shape[1], g.shape[0]) for g in grids], 24)
    b.set_occupancy_dense(grids)
    got = A.autotune(b, reps=2, cache_path=str(tmp_path / "t.json"))
    assert got["y_run"] == got["z_run"]
    for i, g in enumerate(grids):
        assert first_mismatch(b.maps[i].export_dense(), O.edt_factorised(g, 24)) is None, i
