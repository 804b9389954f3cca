"""The allocation-free PageRank entry point (pagerank_csc_noalloc).

Some callers cannot allocate device memory: hosts that fix their memory plan
at start-up, allocator-free regions of a larger runtime, code that shares the
device with an allocator it does not own.  This entry point serves them from a
static scratch array.  Its output is checked against the FP64 oracle on the
same CSC (L1 <= 1e-5, the FP32 tolerance of the other tests) and against the
regular `pagerank` entry point, on two calls in a row (the second call reuses
the scratch the first one left behind), with the device's free memory
unchanged around the second call.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import gen
import oracle
import paper_1606_07550_gb300 as gpr

from gpu_util import l1

TOL = 1e-5


@pytest.mark.gpu
def test_matches_oracle_and_pagerank_on_two_calls_in_a_row():
    import torch
    n = 200_000
    src, dst = gen.rmat_coo(n, 3_000_000, seed=77)
    g = gpr.graph_build(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    ref = torch.empty(n, device="cuda")
    gpr.pagerank(g, ref, damping=0.85, iters=40)
    ref = ref.cpu().numpy().astype(np.float64)
    cp_h, ri_h, od_h = g.export()
    want = oracle.pagerank(oracle.CSC(n, cp_h, ri_h, od_h), 0.85, 40)
    cp, ri, od = (torch.from_numpy(a).cuda() for a in (cp_h, ri_h, od_h))
    for call in range(2):
        out = torch.full((n,), -1.0, device="cuda")
        torch.cuda.synchronize()
        free0 = torch.cuda.mem_get_info()[0]
        launches0 = gpr.lib().gpr_kernel_launches()
        gpr.pagerank_csc_noalloc(cp, ri, od, n, out, damping=0.85, iters=40)
        torch.cuda.synchronize()
        if call == 1:  # the scratch is resident: nothing is allocated
            assert torch.cuda.mem_get_info()[0] == free0
        assert gpr.lib().gpr_kernel_launches() - launches0 == 42  # reset, start vector, 40 steps
        x = out.cpu().numpy().astype(np.float64)
        assert l1(x, want) <= TOL, (call, l1(x, want))
        assert l1(x, ref) <= TOL, (call, l1(x, ref))
    # an odd step count ends in the scratch copy and must still land in out
    out = torch.empty(n, device="cuda")
    gpr.pagerank_csc_noalloc(cp, ri, od, n, out, iters=7)
    torch.cuda.synchronize()
    assert l1(out.cpu().numpy(), oracle.pagerank(oracle.CSC(n, cp_h, ri_h, od_h), 0.85, 7)) <= TOL


@pytest.mark.gpu
@pytest.mark.parametrize("case", ["one node", "no edges", "zero iterations", "dangling hub"])
def test_edge_cases_against_oracle(case):
    import torch
    if case == "one node":
        n, src, dst, iters = 1, np.zeros(0, np.int32), np.zeros(0, np.int32), 10
    elif case == "no edges":
        n, src, dst, iters = 1000, np.zeros(0, np.int32), np.zeros(0, np.int32), 10
    elif case == "zero iterations":
        n, iters = 5000, 0
        src, dst = gen.rmat_coo(n, 40_000, seed=78)
    else:  # in-star: every leaf points to the dangling hub 0
        n, iters = 3000, 60
        src = np.arange(1, n, dtype=np.int32)
        dst = np.zeros(n - 1, np.int32)
    ref_g = oracle.build_csc(n, src, dst)
    want = oracle.pagerank(ref_g, 0.85, iters)
    cp, ri, od = (torch.from_numpy(np.ascontiguousarray(a, np.int32)).cuda()
                  for a in (ref_g.col_ptr, np.append(ref_g.row_idx, 0), ref_g.outdeg))
    out = torch.full((n,), -1.0, device="cuda")
    gpr.pagerank_csc_noalloc(cp, ri, od, n, out, iters=iters)
    torch.cuda.synchronize()
    assert l1(out.cpu().numpy(), want) <= TOL


@pytest.mark.gpu
def test_rejects_more_nodes_than_the_scratch_holds():
    import torch
    n = (1 << 21) + 1
    z = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    out = torch.empty(n, device="cuda")
    with pytest.raises(gpr.GprError) as ei:
        gpr.pagerank_csc_noalloc(z, z, z, n, out)
    assert ei.value.status == gpr.EINVAL and "scratch" in str(ei.value)


def test_binding_checks_types_and_sizes_before_the_library():
    # CPU tensors: the checks run before anything reaches the library
    import torch
    n = 10
    i32 = torch.zeros(n + 1, dtype=torch.int32)
    f32 = torch.zeros(n, dtype=torch.float32)
    for bad in (dict(col_ptr=i32.long()), dict(row_idx=i32.long()), dict(outdeg=i32[:n].long()),
                dict(out=f32.double()), dict(out=f32[: n - 1]), dict(col_ptr=i32[:n]), dict(outdeg=i32[: n - 1])):
        args = dict(col_ptr=i32, row_idx=i32, outdeg=i32[:n], out=f32)
        args.update(bad)
        with pytest.raises(ValueError):
            gpr.pagerank_csc_noalloc(args["col_ptr"], args["row_idx"], args["outdeg"], n, args["out"])
