"""GPU HITS and eigenvector centrality against the FP64 oracle.

Both return unit-L2 vectors; the bar is an L2 distance of at most 1e-5 from
the oracle's vector at the same step count (FP32 products, FP64 norms), and
entries that are exactly 0 in the oracle (no in- or out-edges) are 0 on the
GPU too.
"""
import numpy as np
import pytest

import gen
import oracle
import paper_1606_07550_gb300 as gpr

from gpu_util import l1, random_coo_with_dups

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def gpu_hits(torch, g, iters, spmv="auto"):
    hub = torch.empty(g.n, device="cuda")
    auth = torch.empty(g.n, device="cuda")
    gpr.hits(g, hub, auth, iters=iters, spmv=spmv)
    return hub.cpu().numpy().astype(np.float64), auth.cpu().numpy().astype(np.float64)


def gpu_eig(torch, g, iters, spmv="auto"):
    x = torch.empty(g.n, device="cuda")
    gpr.eigen_centrality(g, x, iters=iters, spmv=spmv)
    return x.cpu().numpy().astype(np.float64)


def close(x, ref):
    assert np.linalg.norm(x - ref) <= TOL, np.linalg.norm(x - ref)
    assert (x[ref == 0] == 0).all()


@pytest.mark.parametrize("spmv", ["pull", "blocked"])
@pytest.mark.parametrize("n,m_raw,seed", [(257, 3000, 12), (40_000, 600_000, 13)])
def test_both_schedules_match_oracle(torch, spmv, n, m_raw, seed):
    # the blocked schedule carries unit weights and L1-normalised vectors
    # through fixed-point sums; the pull schedule gathers FP32
    src, dst = gen.rmat_coo(n, m_raw, seed=seed)
    g = gpr.graph_build(src, dst, n)
    ref = oracle.build_csc(n, src, dst)
    for iters in (1, 7, 30):
        hub, auth = gpu_hits(torch, g, iters, spmv)
        rh, ra = oracle.hits(ref, iters)
        close(hub, rh)
        close(auth, ra)
        close(gpu_eig(torch, g, iters, spmv), oracle.eigen_centrality(ref, iters))
    # the schedules agree with each other too, and with PageRank run between them
    x = torch.empty(n, device="cuda")
    gpr.pagerank(g, x, iters=20, spmv=spmv)
    assert l1(x.cpu().numpy(), oracle.pagerank(ref, 0.85, 20)) <= 1e-5
    hub2, auth2 = gpu_hits(torch, g, 30, spmv)
    rh, ra = oracle.hits(ref, 30)
    close(hub2, rh)
    close(auth2, ra)
    g.free()


def test_conflicting_schedule_flags(torch):
    g = gpr.graph_build(np.array([0, 1], np.int32), np.array([1, 2], np.int32), 3)
    x = torch.empty(3, device="cuda")
    from paper_1606_07550_gb300 import SPMV_BLOCKED, SPMV_PULL, lib
    st = lib().eigen_centrality(g.handle, 3, x.data_ptr(), SPMV_PULL | SPMV_BLOCKED,
                                torch.cuda.current_stream().cuda_stream)
    assert st == gpr.EINVAL
    g.free()


@pytest.mark.parametrize("n,m_raw,seed", [(1, 5, 0), (2, 1, 1), (257, 3000, 2), (4099, 40_000, 3),
                                          (100_003, 1_000_000, 4)])
def test_random_graphs_match_oracle(torch, n, m_raw, seed):
    src, dst = random_coo_with_dups(np.random.default_rng(seed), n, m_raw)
    g = gpr.graph_build(src, dst, n)
    ref = oracle.build_csc(n, src, dst)
    for iters in (0, 1, 20):
        hub, auth = gpu_hits(torch, g, iters)
        rh, ra = oracle.hits(ref, iters)
        close(hub, rh)
        close(auth, ra)
        close(gpu_eig(torch, g, iters), oracle.eigen_centrality(ref, iters))
    g.free()


def test_power_law_graph_matches_oracle(torch):
    # hubs with long rows (chunked), many rows without in- or out-edges
    n = 30_000
    src, dst = gen.rmat_coo(n, 600_000, seed=31)
    g = gpr.graph_build(src, dst, n)
    ref = oracle.build_csc(n, src, dst)
    hub, auth = gpu_hits(torch, g, 50)
    rh, ra = oracle.hits(ref, 50)
    close(hub, rh)
    close(auth, ra)
    close(gpu_eig(torch, g, 50), oracle.eigen_centrality(ref, 50))


def test_closed_forms_on_gpu(torch):
    p, q = 3, 8
    src = np.repeat(np.arange(p), q).astype(np.int32)
    dst = (p + np.tile(np.arange(q), p)).astype(np.int32)
    g = gpr.graph_build(src, dst, p + q)
    hub, auth = gpu_hits(torch, g, 10)
    assert np.abs(hub[:p] - 1 / np.sqrt(p)).max() < 1e-7 and (hub[p:] == 0).all()
    assert np.abs(auth[p:] - 1 / np.sqrt(q)).max() < 1e-7 and (auth[:p] == 0).all()
    N = 1000
    cyc = np.arange(N, dtype=np.int32)
    g = gpr.graph_build(cyc, (cyc + 1) % N, N)
    assert np.abs(gpu_eig(torch, g, 30) - 1 / np.sqrt(N)).max() < 1e-7
    # no edges at all: every product is 0, and 0 stays 0
    z = np.zeros(0, np.int32)
    g = gpr.graph_build(z, z, 50)
    hub, auth = gpu_hits(torch, g, 3)
    assert (hub == 0).all() and (auth == 0).all()
    assert (gpu_eig(torch, g, 3) == 0).all()
    assert np.abs(gpu_eig(torch, g, 0) - 1 / np.sqrt(50)).max() < 1e-7


def test_deterministic_host_output_and_pagerank_after(torch):
    n = 20_000
    src, dst = gen.rmat_coo(n, 300_000, seed=8)
    g = gpr.graph_build(src, dst, n)
    a = gpu_hits(torch, g, 30)
    b = gpu_hits(torch, g, 30)
    assert (a[0] == b[0]).all() and (a[1] == b[1]).all()
    hh = np.empty(n, np.float32)
    ha = np.empty(n, np.float32)
    gpr.hits(g, hh, ha, iters=30)
    assert (hh == a[0]).all() and (ha == a[1]).all()
    xe = np.empty(n, np.float32)
    gpr.eigen_centrality(g, xe, iters=30)
    assert (xe == gpu_eig(torch, g, 30)).all()
    # PageRank on the same graph (shared workspace) is unaffected
    ref = oracle.build_csc(n, src, dst)
    out = torch.empty(n, device="cuda")
    gpr.pagerank(g, out, iters=25)
    assert l1(out.cpu().numpy(), oracle.pagerank(ref, 0.85, 25)) <= 1e-5
    hub, auth = gpu_hits(torch, g, 30)
    assert (hub == a[0]).all() and (auth == a[1]).all()


def test_rejects_bad_arguments(torch):
    g = gpr.graph_build(np.array([0], np.int32), np.array([1], np.int32), 2)
    out = torch.empty(2, device="cuda")
    with pytest.raises(gpr.GprError) as ei:
        gpr.eigen_centrality(g, out, iters=-1)
    assert ei.value.status == gpr.EINVAL
    with pytest.raises(gpr.GprError) as ei:
        gpr._check(gpr.lib().hits(g.handle, 5, None, out.data_ptr(), 0, None))
    assert ei.value.status == gpr.EINVAL
