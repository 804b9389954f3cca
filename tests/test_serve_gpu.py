"""Continuous-batching server: results against the oracle, the same bits alone
and in a mix, admission under a memory budget, and failure isolation."""
import time

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


@pytest.fixture(scope="module")
def pool(torch):
    specs = [(3000, 40_000, 61), (20_000, 320_000, 62), (1 << 16, 1 << 20, 63)]
    out = []
    for n, m, sd in specs:
        src, dst = gen.rmat_coo(n, m, seed=sd)
        out.append((gpr.graph_build(src, dst, n), oracle.build_csc(n, src, dst)))
    return out


def wait(srv, t, timeout_s=60):
    t0 = time.time()
    while time.time() - t0 < timeout_s:
        r = srv.poll(t, 100_000)
        if r is not None:
            return r
    raise AssertionError("request did not finish")


def result(torch, srv, t, r):
    out = torch.empty(r.n * r.num_seeds, device="cuda")
    srv.fetch(t, out)
    return out.cpu().numpy().reshape(r.n, r.num_seeds)


def test_single_request_matches_oracle(torch, pool):
    graphs = [g for g, _ in pool]
    srv = gpr.Server(graphs, budget_bytes=8 << 30)
    seeds = np.array([0, 17, 2999], np.int32)
    t = srv.submit(0, seeds, damping=0.85, max_iters=50)
    r = wait(srv, t)
    assert r.status == gpr.OK and r.iters_max == 50 and r.latency_ms > 0
    x = result(torch, srv, t, r)
    for k, s in enumerate(seeds):
        assert l1(x[:, k], oracle.ppr(pool[0][1], int(s), 0.85, 50)[0]) <= 1e-5
    srv.release(t)
    srv.close()


@pytest.mark.parametrize("dt,tol,storage", [(gpr.FP32, 1e-6, 1e-5), (gpr.FP32, 1e-3, 1e-5), (gpr.FP16, 1e-3, 1e-3),
                                             (gpr.BF16, 1e-3, 1e-3), (gpr.BF16, 1e-6, 1e-5)])
def test_served_columns_reach_the_oracle_fixed_point(torch, pool, dt, tol, storage):
    # a request with a tolerance stops once d/(1-d) ||x_k - x_{k-1}||_1 <= tol
    # (or its residual has stopped shrinking), so each served column lies
    # within tol of the fixed point, plus the error of its storage type
    graphs = [g for g, _ in pool]
    srv = gpr.Server(graphs, budget_bytes=8 << 30)
    rng = np.random.default_rng(int(tol * 1e9) + dt)
    for gi in (1, 2):
        seeds = rng.integers(0, graphs[gi].n, 5).astype(np.int32)
        t = srv.submit(gi, seeds, damping=0.82, tol=tol, max_iters=1000, dtype=dt)
        r = wait(srv, t)
        assert r.status == gpr.OK
        x = result(torch, srv, t, r)
        for k, s in enumerate(seeds):
            xstar, _ = oracle.ppr(pool[gi][1], int(s), 0.82, 300)
            err = l1(x[:, k], xstar)
            assert err <= tol + storage, (gi, int(s), err)
        srv.release(t)
    srv.close()


def test_alone_equals_mix_and_admission_mid_flight(torch, pool):
    graphs = [g for g, _ in pool]
    srv = gpr.Server(graphs, budget_bytes=8 << 30, steps_per_tick=4)
    probe = dict(graph_id=1, seeds=[5, 9, 19_999], damping=0.83, tol=1e-6, max_iters=1000)
    t = srv.submit(**probe)
    alone = result(torch, srv, t, wait(srv, t))
    srv.release(t)
    # a long request first, then a stream of others, the probe among them
    long_t = srv.submit(2, list(range(64)), damping=0.85, tol=0.0, max_iters=400)
    time.sleep(0.05)
    rng = np.random.default_rng(3)
    ts = []
    for i in range(20):
        g = int(rng.integers(0, 3))
        ts.append(srv.submit(g, rng.integers(0, graphs[g].n, int(rng.integers(1, 40))), damping=0.85,
                             tol=1e-3, max_iters=200, dtype=[gpr.FP32, gpr.BF16, gpr.FP16][i % 3]))
        if i == 10:
            tp = srv.submit(**probe)
    rp = wait(srv, tp)
    # the probe arrived after the long request was already running and
    # finished first: it was admitted into the running batches mid-flight
    assert srv.poll(long_t) is None
    mixed = result(torch, srv, tp, rp)
    assert (alone == mixed).all()
    for t in ts + [long_t, tp]:
        assert wait(srv, t).status == gpr.OK
        srv.release(t)
    st = srv.stats()
    assert st["completed"] == 23 and st["failed"] == 0
    srv.close()


def test_budget_admission_and_rejections(torch, pool):
    graphs = [g for g, _ in pool]
    g2 = graphs[2]
    pool_bytes = sum(g.info().device_bytes for g in graphs)
    slot = g2.n * 64 * 12
    res = g2.n * 64 * 4
    # room for one 64-seed request on graph 2 at a time
    srv = gpr.Server(graphs, budget_bytes=pool_bytes + slot + res + (1 << 20), max_queue=1)  # + small per-slot step state
    with pytest.raises(gpr.GprError) as ei:  # the pool alone exceeds the budget
        gpr.Server(graphs, budget_bytes=pool_bytes - 1)
    assert ei.value.status == gpr.ENOMEM
    small = gpr.Server(graphs, budget_bytes=pool_bytes + 1024)
    with pytest.raises(gpr.GprError) as ei:
        small.submit(2, [1])
    assert ei.value.status == gpr.ENOMEM
    small.close()
    t1 = srv.submit(2, list(range(64)), max_iters=300)
    t0 = time.time()
    while srv.stats()["admitted"] < 1 and time.time() - t0 < 30:  # t1 leaves the queue
        time.sleep(0.001)
    t2 = srv.submit(2, list(range(64, 128)), max_iters=10)   # waits: the budget holds one
    with pytest.raises(gpr.GprError) as ei:
        srv.submit(2, [7], max_iters=10)                      # queue (max 1) is full
    assert ei.value.status == gpr.EBUSY
    r1 = wait(srv, t1)
    assert r1.status == gpr.OK
    srv.release(t1)                                           # frees the budget for t2
    r2 = wait(srv, t2)
    assert r2.status == gpr.OK and r2.latency_ms >= r1.latency_ms * 0.5
    srv.release(t2)
    srv.close()


def test_injected_allocation_failure_fails_one_request(torch, pool):
    graphs = [g for g, _ in pool]
    srv = gpr.Server(graphs, budget_bytes=8 << 30, fail_alloc_at=1)
    t_bad = srv.submit(0, [1, 2], max_iters=20)
    r = wait(srv, t_bad)
    assert r.status == gpr.ENOMEM
    srv.release(t_bad)
    t_ok = srv.submit(0, [1, 2], max_iters=20)
    r = wait(srv, t_ok)
    assert r.status == gpr.OK
    x = result(torch, srv, t_ok, r)
    assert l1(x[:, 0], oracle.ppr(pool[0][1], 1, 0.85, 20)[0]) <= 1e-5
    srv.release(t_ok)
    srv.close()


def test_bad_requests_and_unknown_tickets(torch, pool):
    graphs = [g for g, _ in pool]
    srv = gpr.Server(graphs, budget_bytes=8 << 30)
    for kw in (dict(graph_id=3, seeds=[0]), dict(graph_id=0, seeds=[3000]), dict(graph_id=0, seeds=[]),
               dict(graph_id=0, seeds=list(range(65))), dict(graph_id=0, seeds=[0], damping=1.0)):
        with pytest.raises(gpr.GprError) as ei:
            srv.submit(**kw)
        assert ei.value.status == gpr.EINVAL
    with pytest.raises(gpr.GprError) as ei:
        srv.poll(12345)
    assert ei.value.status == gpr.ENOTFOUND
    srv.close()


def test_destroy_with_work_in_flight_does_not_hang(torch, pool):
    graphs = [g for g, _ in pool]
    srv = gpr.Server(graphs, budget_bytes=8 << 30)
    for i in range(10):
        srv.submit(2, list(range(i, i + 64)), max_iters=2000)
    t0 = time.time()
    srv.close()
    assert time.time() - t0 < 30
