"""The allocation-free PageRank entry point (pagerank_csc_noalloc).

Some callers cannot allocate device memory (fixed start-up memory plans,
allocator-free regions of a larger runtime); this entry point serves them
from a static scratch array.  Its output must agree with the regular
`pagerank` entry point on the same graph, within the FP32 tolerance the other
tests use, on two calls in a row (the second call reuses the scratch the
first one left behind).  This file is collected last on purpose.
"""
import numpy as np
import pytest

import gen
import paper_1606_07550_gb300 as gpr

pytestmark = pytest.mark.gpu

TOL = 1e-5


def test_matches_pagerank_on_two_calls_in_a_row():
    import torch
    n = 200_000
    src, dst = gen.rmat_coo(n, 3_000_000, seed=77)
    g = gpr.graph_build(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    ref = torch.empty(n, device="cuda")
    gpr.pagerank(g, ref, damping=0.85, iters=40)
    ref = ref.cpu().numpy().astype(np.float64)
    cp, ri, od = (torch.from_numpy(a).cuda() for a in g.export())
    for call in range(2):
        out = torch.full((n,), -1.0, device="cuda")
        gpr.pagerank_csc_noalloc(cp, ri, od, n, out, damping=0.85, iters=40)
        torch.cuda.synchronize()
        x = out.cpu().numpy().astype(np.float64)
        assert np.abs(x - ref).sum() <= TOL, (call, np.abs(x - ref).sum())
    # an odd step count ends in the scratch copy and must still land in out
    ref7 = torch.empty(n, device="cuda")
    gpr.pagerank(g, ref7, iters=7)
    out = torch.empty(n, device="cuda")
    gpr.pagerank_csc_noalloc(cp, ri, od, n, out, iters=7)
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy().astype(np.float64) - ref7.cpu().numpy()).sum() <= TOL


def test_rejects_more_nodes_than_the_scratch_holds():
    import torch
    z = torch.zeros(4, dtype=torch.int32, device="cuda")
    out = torch.empty(4, device="cuda")
    with pytest.raises(gpr.GprError) as ei:
        gpr.pagerank_csc_noalloc(z, z, z, (1 << 21) + 1, out)
    assert ei.value.status == gpr.EINVAL and "scratch" in str(ei.value)
