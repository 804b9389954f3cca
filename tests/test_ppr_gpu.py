"""Batched personalised PageRank on the GPU against the FP64 CPU oracle.

Every column is compared with a single-seed oracle run at the same step count:
L1 <= 1e-5 with FP32 contributions, <= 1e-3 with scaled FP16 ones and <= 1e-3
with BF16 ones (sent as error-feedback deltas).  A column must give the same
bits alone as inside a batch.
"""
import numpy as np
import pytest

import gen
import oracle
import paper_1606_07550_gb300 as gpr

from gpu_util import l1, random_coo_with_dups

pytestmark = pytest.mark.gpu

TOL = {gpr.FP32: 1e-5, gpr.FP16: 1e-3, gpr.BF16: 1e-3}


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def make_graph(torch, n, m_raw, seed):
    src, dst = gen.rmat_coo(n, m_raw, seed=seed)
    g = gpr.graph_build(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    return g, oracle.build_csc(n, src, dst)


def run(torch, reqs, iters, tol=0.0, dt=gpr.FP32):
    outs = [torch.zeros((g.n, len(s)), dtype=torch.float32, device="cuda") for g, s, d in reqs]
    res = gpr.ppr_batch([(g, s, d, o) for (g, s, d), o in zip(reqs, outs)], max_iters=iters, tol=tol, dtype=dt)
    return [o.cpu().numpy() for o in outs], res


@pytest.mark.parametrize("dt", [gpr.FP32, gpr.FP16, gpr.BF16])
def test_columns_match_oracle(torch, dt):
    graphs = [make_graph(torch, n, m, 40 + i) for i, (n, m) in
              enumerate([(1000, 12_000), (5000, 90_000), (20_000, 500_000), (3001, 3000)])]
    rng = np.random.default_rng(1)
    reqs = []
    for g, ref in graphs:
        k = int(rng.integers(1, 65))
        seeds = rng.integers(0, g.n, k).astype(np.int32)
        dang = np.flatnonzero(ref.outdeg == 0)
        if len(dang):
            seeds[0] = dang[0]  # a dangling seed
        damp = rng.uniform(0.8, 0.9, k).astype(np.float32)
        reqs.append((g, seeds, damp))
    xs, res = run(torch, reqs, 50, dt=dt)
    worst = 0.0
    for (g, seeds, damp), (_, ref), x, (it, _) in zip(reqs, graphs, xs, res):
        assert (it == 50).all()
        for k, s in enumerate(seeds):
            xr, _ = oracle.ppr(ref, int(s), float(damp[k]), 50)
            err = l1(x[:, k], xr)
            worst = max(worst, err)
            assert err <= TOL[dt], (k, s, err)
    print(f"dtype {dt}: worst column L1 {worst:.3e}")


def test_bf16_deltas_correct_their_rounding(torch):
    # the error of a BF16 column is one rounding of the last step-to-step
    # change, not of the contributions: far below the 8-bit significand's
    # 2^-9 relative error once the iteration has settled
    g, ref = make_graph(torch, 20_000, 400_000, 44)
    seeds = np.array([0, 1, 2, 3, 100, 5000, 19_999], np.int32)
    xs, _ = run(torch, [(g, seeds, 0.85)], 100, dt=gpr.BF16)
    for k, s in enumerate(seeds):
        xr, _ = oracle.ppr(ref, int(s), 0.85, 100)
        assert l1(xs[0][:, k], xr) <= 1e-4


def test_alone_equals_in_mix_bitwise(torch):
    g1, _ = make_graph(torch, 8000, 150_000, 7)
    g2, _ = make_graph(torch, 2000, 20_000, 8)
    seeds = np.array([5, 17, 17, 1999], np.int32)
    alone, _ = run(torch, [(g2, seeds, 0.85)], 40)
    mixed, _ = run(torch, [(g1, np.arange(64, dtype=np.int32), 0.85), (g2, seeds, 0.85),
                           (g1, np.array([3], np.int32), 0.5)], 40)
    assert (alone[0] == mixed[1]).all()
    # one column alone vs the same column among 63 others of the same graph
    one, _ = run(torch, [(g2, seeds[1:2], 0.85)], 40)
    assert (one[0][:, 0] == mixed[1][:, 1]).all()


def test_more_than_64_seeds(torch):
    g, ref = make_graph(torch, 4000, 60_000, 9)
    seeds = np.arange(0, 4000, 31, dtype=np.int32)  # 130 seeds -> three jobs
    xs, _ = run(torch, [(g, seeds, 0.85)], 30)
    for k in (0, 63, 64, 100, len(seeds) - 1):
        xr, _ = oracle.ppr(ref, int(seeds[k]), 0.85, 30)
        assert l1(xs[0][:, k], xr) <= 1e-5


def test_heavy_rows_and_closed_form(torch):
    # in-star: every leaf points to the hub, whose row is one long block-processed row
    N = 60_000
    leaves = np.arange(1, N, dtype=np.int32)
    g = gpr.graph_build(torch.from_numpy(leaves).cuda(), torch.from_numpy(np.zeros_like(leaves)).cuda(), N)
    ref = oracle.build_csc(N, leaves, np.zeros_like(leaves))
    xs, _ = run(torch, [(g, np.array([0, 5, N - 1], np.int32), 0.85)], 60)
    for k, s in enumerate([0, 5, N - 1]):
        xr, _ = oracle.ppr(ref, s, 0.85, 60)
        assert l1(xs[0][:, k], xr) <= 1e-5
    # PPR on a directed cycle: x_v = (1-d) d^j / (1 - d^N)
    N = 500
    a = np.arange(N, dtype=np.int32)
    g = gpr.graph_build(torch.from_numpy(a).cuda(), torch.from_numpy((a + 1) % N).cuda(), N)
    xs, _ = run(torch, [(g, np.array([7], np.int32), 0.85)], 400)
    j = (np.arange(N) - 7) % N
    assert np.abs(xs[0][:, 0] - (1 - 0.85) * 0.85 ** j / (1 - 0.85 ** N)).max() < 1e-6


def test_tolerance_stop(torch):
    g, ref = make_graph(torch, 6000, 80_000, 10)
    seeds = np.array([1, 2, 3, 500, 5999], np.int32)
    for tol in (1e-3, 1e-6):
        xs, res = run(torch, [(g, seeds, 0.85)], 1000, tol=tol)
        it, resid = res[0]
        for k, s in enumerate(seeds):
            xr, k_ref = oracle.ppr(ref, int(s), 0.85, 1000, tol)
            assert abs(int(it[k]) - k_ref) <= 1
            assert 0.85 / 0.15 * resid[k] <= tol * (1 + 1e-3)
            xstar, _ = oracle.ppr(ref, int(s), 0.85, 400)
            assert l1(xs[0][:, k], xstar) <= tol + 1e-5


@pytest.mark.parametrize("dt,tol,err", [(gpr.FP32, 1e-12, 1e-5), (gpr.FP16, 1e-6, 1e-3), (gpr.BF16, 1e-9, 1e-3)])
def test_tolerance_below_the_storage_floor_stops_at_the_floor(torch, dt, tol, err):
    # the bound d/(1-d)||x_k - x_{k-1}||_1 cannot reach tol in this storage:
    # a column stops once its residual has stopped shrinking, long before
    # max_iters, at the fixed point within the storage's tolerance
    g, ref = make_graph(torch, 6000, 80_000, 12)
    seeds = np.array([1, 77, 5999], np.int32)
    xs, res = run(torch, [(g, seeds, 0.9)], 5000, tol=tol, dt=dt)
    it, resid = res[0]
    for k, s in enumerate(seeds):
        assert 20 < int(it[k]) < 1000, int(it[k])
        xstar, _ = oracle.ppr(ref, int(s), 0.9, 600)
        assert l1(xs[0][:, k], xstar) <= err


def test_zero_iterations_is_the_seed_vector(torch):
    g, _ = make_graph(torch, 1000, 10_000, 11)
    xs, res = run(torch, [(g, np.array([4, 999], np.int32), 0.85)], 0)
    e = np.zeros((1000, 2), np.float32)
    e[4, 0] = e[999, 1] = 1.0
    assert (xs[0] == e).all() and (res[0][0] == 0).all()


def test_random_small_graphs(torch):
    rng = np.random.default_rng(5)
    reqs, refs = [], []
    for i in range(10):
        n = int(rng.integers(1, 300))
        src, dst = random_coo_with_dups(rng, n, int(rng.integers(0, 3000)))
        g = gpr.graph_build(src, dst, n)
        refs.append(oracle.build_csc(n, src, dst))
        reqs.append((g, rng.integers(0, n, 3).astype(np.int32), 0.85))
    xs, _ = run(torch, reqs, 25)
    for (g, seeds, _), ref, x in zip(reqs, refs, xs):
        for k, s in enumerate(seeds):
            assert l1(x[:, k], oracle.ppr(ref, int(s), 0.85, 25)[0]) <= 1e-5


def test_rejects_bad_requests(torch):
    g, _ = make_graph(torch, 100, 500, 12)
    out = torch.zeros((100, 1), device="cuda")
    for seeds, d in (([100], 0.85), ([-1], 0.85), ([0], 1.0), ([0], 0.0)):
        with pytest.raises(gpr.GprError) as ei:
            gpr.ppr_batch([(g, seeds, d, out)])
        assert ei.value.status == gpr.EINVAL


def test_tuner_picks_a_shape_per_size_class_and_every_shape_is_correct(torch):
    import os
    sizes = [(1500, 20_000), (6000, 80_000), (40_000, 600_000)]  # ceil log2 n = 11, 13, 16: three classes
    graphs = [make_graph(torch, n, m, 70 + i) for i, (n, m) in enumerate(sizes)]
    reqs = [(g, (np.arange(64, dtype=np.int32) * 37) % g.n, 0.85) for g, _ in graphs]
    outs = [torch.zeros((g.n, 64), dtype=torch.float32, device="cuda") for g, _ in graphs]
    res = gpr.ppr_tune([(g, sd, d, o) for (g, sd, d), o in zip(reqs, outs)], trial_steps=5)
    assert [r["log2n_max"] for r in res] == [11, 13, 17]
    for r in res:
        assert r["jobs"] == 1 and r["cluster"] in (1, 2, 4, 8) and r["ms"] > 0 and r["ms_cluster8"] > 0
        assert r["ms"] <= r["ms_cluster8"]
    try:
        for shape in ("1", "2", "4", "8"):
            os.environ["GPR_PPR_CLUSTER"] = shape
            xs, res2 = run(torch, reqs, 30)
            for (g, sd, d), (_, ref), x in zip(reqs, graphs, xs):
                for k in (0, 17, 63):
                    xr, _ = oracle.ppr(ref, int(sd[k]), 0.85, 30)
                    assert l1(x[:, k], xr) <= 1e-5, (shape, g.n, k)
    finally:
        os.environ.pop("GPR_PPR_CLUSTER", None)
    with pytest.raises(gpr.GprError) as ei:
        gpr.ppr_tune([(graphs[0][0], [0], 0.85, outs[0][:, :1].contiguous())], trial_steps=0)
    assert ei.value.status == gpr.EINVAL
