"""Failure detection without a GPU fault: a bounded device wait runs out.

With GPR_INJECT_LOOKBACK_STALL set, the first tile of the build's compaction
never publishes its prefix, so every later tile's decoupled look-back waits on
a flag nothing sets.  Each wait gives up after a bounded number of polls, the
kernel records the timeout and returns, and graph_build reports GPR_ETIMEOUT;
the context stays usable.
"""
import os
import time

import numpy as np
import pytest

import gen
import oracle
import paper_1606_07550_gb300 as gpr

pytestmark = pytest.mark.gpu


def test_lookback_wait_times_out_and_device_stays_usable():
    import torch
    src, dst = gen.rmat_coo(50_000, 400_000, seed=5)
    s, d = torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda()
    os.environ["GPR_INJECT_LOOKBACK_STALL"] = "1"
    try:
        t0 = time.time()
        with pytest.raises(gpr.GprError) as ei:
            gpr.graph_build(s, d, 50_000)
        assert ei.value.status == gpr.ETIMEOUT
        assert time.time() - t0 < 60
    finally:
        os.environ.pop("GPR_INJECT_LOOKBACK_STALL", None)
    g = gpr.graph_build(s, d, 50_000)
    ref = oracle.build_csc(50_000, src, dst)
    cp, ri, od = g.export()
    assert (cp == ref.col_ptr).all() and (ri == ref.row_idx).all()
