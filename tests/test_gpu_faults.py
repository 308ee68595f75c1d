"""Failure detection without a GPU fault: a bounded device-side wait that runs out (an mbarrier
phase that never completes; a node insertion left pending) gives up, sets the handle's error
word, and the host reads VDBEDT_ETIMEOUT; the context stays usable and, after a reset, the grid
transforms exactly again.  Invalid inputs are rejected with status codes."""
import time

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_common import first_mismatch

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("which", [0, 1])
def test_bounded_wait_reports_timeout(which):
    import paper_2105_04419_gb300 as V
    from paper_2105_04419_gb300 import lib as L
    occ = W.bernoulli_grid(3, (24, 30, 36), 0.01)
    m = V.Map(36, 30, 24, 9)
    m.set_occupancy_dense(occ)
    m.global_()
    m.synchronize()
    t0 = time.perf_counter()
    assert L.load().vdbedt_selftest_wait_timeout(m.handle, which) == 0
    with pytest.raises(V.VdbedtError) as e:
        m.synchronize()
    assert e.value.code == "ETIMEOUT"
    assert time.perf_counter() - t0 < 60
    # the context is still usable: reset, transform again, exact
    m.reset()
    m.set_occupancy_dense(occ)
    m.global_()
    m.synchronize()
    assert first_mismatch(m.export_dense(), O.edt_factorised(occ, 9)) is None
    # other CUDA work on the device is unaffected
    import torch
    assert float(torch.ones(8, device="cuda").sum().item()) == 8.0


def test_selftest_rejects_bad_argument():
    import paper_2105_04419_gb300 as V
    from paper_2105_04419_gb300 import lib as L
    m = V.Map(8, 8, 8, 3)
    assert L.load().vdbedt_selftest_wait_timeout(m.handle, 2) == 1
    m.synchronize()
