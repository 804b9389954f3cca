"""In-place edge updates (graph_update) against a rebuild of the same edge set
by the oracle (bit-exact CSC), and warm-started PageRank against the oracle
started from the same vector."""
import numpy as np
import pytest

import gen
import oracle
import paper_1606_07550_gb300 as gpr

from gpu_util import l1

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def edge_set(src, dst):
    return {(int(u), int(v)) for u, v in zip(src, dst) if u != v}


def arrays(es):
    es = sorted(es)
    return (np.array([u for u, _ in es], np.int32), np.array([v for _, v in es], np.int32))


def check_export(g, n, es):
    s, d = arrays(es)
    ref = oracle.build_csc(n, s, d)
    cp, ri, od = g.export()
    assert (cp == ref.col_ptr).all() and (ri == ref.row_idx).all() and (od == ref.outdeg).all()
    return ref


def random_batch(rng, n, es, k_ins, k_del):
    ins_s = rng.integers(0, n, k_ins).astype(np.int32)
    ins_d = rng.integers(0, n, k_ins).astype(np.int32)
    ins_d[: k_ins // 20] = ins_s[: k_ins // 20]          # self-loops (dropped)
    r = k_ins // 10
    ins_s[k_ins - r:] = ins_s[:r]                        # repeats
    ins_d[k_ins - r:] = ins_d[:r]
    present = sorted(es)
    pick = rng.integers(0, len(present), k_del)
    del_s = np.array([present[i][0] for i in pick], np.int32)  # existing edges, some repeated
    del_d = np.array([present[i][1] for i in pick], np.int32)
    q = k_del // 10
    del_s[:q] = rng.integers(0, n, q)                        # and some that are not there
    del_d[:q] = rng.integers(0, n, q)
    del_s[-5:] = ins_s[-5:]                                  # deleted and inserted in one batch: inserted
    del_d[-5:] = ins_d[-5:]
    return ins_s, ins_d, del_s, del_d


@pytest.mark.parametrize("n,m_raw,seed", [(200, 1500, 1), (5000, 60_000, 2), (40_000, 600_000, 3)])
def test_batches_match_rebuild(torch, n, m_raw, seed):
    rng = np.random.default_rng(seed)
    src, dst = gen.rmat_coo(n, m_raw, seed=seed)
    g = gpr.graph_build(src, dst, n)
    es = edge_set(src, dst)
    for step in range(3):
        ins_s, ins_d, del_s, del_d = random_batch(rng, n, es, m_raw // 20 + 10, m_raw // 25 + 10)
        if step == 1:  # host arrays
            gpr.graph_update(g, (ins_s, ins_d), (del_s, del_d))
        else:
            gpr.graph_update(g, (torch.from_numpy(ins_s).cuda(), torch.from_numpy(ins_d).cuda()),
                             (torch.from_numpy(del_s).cuda(), torch.from_numpy(del_d).cuda()))
        es = (es - edge_set(del_s, del_d)) | edge_set(ins_s, ins_d)
        ref = check_export(g, n, es)
        assert g.info().m == len(es)
    # PageRank (pull and blocked), HITS and WCC on the updated graph
    x = torch.empty(n, device="cuda")
    for spmv in ("pull", "blocked"):
        gpr.pagerank(g, x, iters=30, spmv=spmv)
        assert l1(x.cpu().numpy(), oracle.pagerank(ref, 0.85, 30)) <= 1e-5
    hub, auth = torch.empty(n, device="cuda"), torch.empty(n, device="cuda")
    gpr.hits(g, hub, auth, iters=10)
    rh, ra = oracle.hits(ref, 10)
    assert np.linalg.norm(auth.cpu().numpy() - ra) <= 1e-5
    lab = torch.empty(n, dtype=torch.int32, device="cuda")
    gpr.wcc(g, lab)
    assert (lab.cpu().numpy() == oracle.wcc(ref)[0]).all()


def test_warm_start_after_update(torch):
    n = 30_000
    src, dst = gen.rmat_coo(n, 500_000, seed=21)
    g = gpr.graph_build(src, dst, n)
    x = torch.empty(n, device="cuda")
    gpr.pagerank(g, x, iters=60)
    es = edge_set(src, dst)
    rng = np.random.default_rng(5)
    ins_s, ins_d, del_s, del_d = random_batch(rng, n, es, 5000, 5000)
    gpr.graph_update(g, (ins_s, ins_d), (del_s, del_d))
    es = (es - edge_set(del_s, del_d)) | edge_set(ins_s, ins_d)
    ref = check_export(g, n, es)
    x0 = x.cpu().numpy().astype(np.float64)
    gpr.pagerank(g, x, iters=10, warm_start=True)        # x holds the start vector on input
    xr = oracle.pagerank(ref, 0.85, 10, x0=x0)
    assert l1(x.cpu().numpy(), xr) <= 1e-5
    # a warm start from the old ranks is closer to the new fixed point than a
    # cold start after the same number of steps
    xstar = oracle.pagerank(ref, 0.85, 200)
    cold = oracle.pagerank(ref, 0.85, 10)
    assert l1(x.cpu().numpy(), xstar) < l1(cold, xstar)
    # host vector in and out
    h = x0.astype(np.float32)
    gpr.pagerank(g, h, iters=10, warm_start=True)
    assert l1(h, xr) <= 1e-5


def test_invalid_and_empty_updates(torch):
    n = 3000
    src, dst = gen.rmat_coo(n, 30_000, seed=22)
    g = gpr.graph_build(src, dst, n)
    es = edge_set(src, dst)
    before = g.export()
    with pytest.raises(gpr.GprError) as ei:
        gpr.graph_update(g, (np.array([0, n], np.int32), np.array([1, 2], np.int32)))
    assert ei.value.status == gpr.EINVAL
    after = g.export()
    assert all((a == b).all() for a, b in zip(before, after))
    gpr.graph_update(g)  # nothing at all
    check_export(g, n, es)
    # delete every edge: uniform PageRank, every node its own component
    s, d = arrays(es)
    gpr.graph_update(g, None, (s, d))
    assert g.info().m == 0
    x = torch.empty(n, device="cuda")
    gpr.pagerank(g, x, iters=5)
    assert np.abs(x.cpu().numpy() - 1 / n).max() < 1e-9
    # and back
    gpr.graph_update(g, (s, d))
    check_export(g, n, es)
