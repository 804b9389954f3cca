"""GPU PageRank against the FP64 CPU oracle at the same iteration count.

Tolerance: L1 <= 1e-5 for FP32 rank storage and <= 1e-3 for BF16 storage
(FP32 accumulation in both).
"""
import os

import numpy as np
import pytest

import gen
import oracle
import paper_1606_07550_gb300 as gpr
from gen import workloads

from gpu_util import coo_for, l1, load_rmat25_oracle, max_rel, random_coo_with_dups, sampled_errors

pytestmark = pytest.mark.gpu

TOL = {gpr.FP32: 1e-5, gpr.BF16: 1e-3}


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def gpu_pr(torch, g, iters, d=0.85, dt=gpr.FP32, stats=False, spmv="auto"):
    out = torch.empty(g.n, dtype=torch.float32, device="cuda")
    st = gpr.pagerank(g, out, damping=d, iters=iters, dtype=dt, stats=stats, spmv=spmv)
    x = out.cpu().numpy()
    return (x, st) if stats else x


def check(torch, n, src, dst, iters, dt=gpr.FP32, d=0.85, buckets=None, hot=None, spmv="auto"):
    if buckets is not None:
        os.environ["GPR_BUCKETS"] = buckets
    if hot is not None:
        os.environ["GPR_HOT"] = hot
    try:
        g = gpr.graph_build(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    finally:
        os.environ.pop("GPR_BUCKETS", None)
        os.environ.pop("GPR_HOT", None)
    ref = oracle.pagerank(oracle.build_csc(n, src, dst), d, iters)
    x, st = gpu_pr(torch, g, iters, d, dt, stats=True, spmv=spmv)
    err = l1(x, ref)
    assert err <= TOL[dt], (err, max_rel(x, ref))
    # BF16 rounding of the gathered contributions moves the mass by up to ~2^-9 d
    assert abs(st.mass - 1.0) <= TOL[dt]
    g.free()
    return err


def test_er_10k_fp32_and_bf16(torch):
    spec = workloads.ER_10K
    src, dst = coo_for(spec)
    check(torch, spec.n, src, dst, spec.iters, gpr.FP32)
    check(torch, spec.n, src, dst, spec.iters, gpr.BF16)


@pytest.mark.parametrize("hot", [None, "100000", "256"])
@pytest.mark.parametrize("buckets", [None, "*:1", "*:4", "*:8", "*:32", "*:0", "0:1,3:2,9:16,100:32,*:0"])
def test_each_bucket_kernel_alone(torch, buckets, hot):
    # power-law graph with hubs, dangling nodes and isolated nodes; hot=None
    # runs without the shared-memory hot pass, "100000" puts every source in
    # it, "256" splits the rows between the two passes
    src, dst = gen.rmat_coo(30_000, 600_000, seed=31)
    for dt in (gpr.FP32, gpr.BF16):
        check(torch, 30_000, src, dst, 30, dt=dt, buckets=buckets, hot=hot)


def test_split_rows(torch):
    # rows longer than one chunk are split and finished by the fold kernel
    os.environ["GPR_CHUNK_EDGES"] = "1024"
    try:
        src, dst = gen.rmat_coo(20_000, 800_000, seed=32)
        check(torch, 20_000, src, dst, 20, buckets="16:8,*:0")
        check(torch, 20_000, src, dst, 20, buckets="16:8,*:0", hot="1000")
    finally:
        os.environ.pop("GPR_CHUNK_EDGES", None)


@pytest.mark.parametrize("n,m_raw,seed", [(1, 5, 0), (2, 1, 1), (257, 3000, 2), (4099, 40_000, 3),
                                          (100_003, 1_000_000, 4)])
def test_random_graphs(torch, n, m_raw, seed):
    rng = np.random.default_rng(seed)
    src, dst = random_coo_with_dups(rng, n, m_raw)
    for dt in (gpr.FP32, gpr.BF16):
        check(torch, n, src, dst, 25, dt)


@pytest.fixture
def block_bits():
    """Sets the blocked schedule's block sizes ("sb,w") for one test."""
    def set_bits(v):
        os.environ["GPR_BLOCK_BITS"] = v
    yield set_bits
    os.environ.pop("GPR_BLOCK_BITS", None)


# "sb,w[,log2 unit,dense sources]".  "4,5": 16-node source blocks and
# 32-row bins, so a 30k-node graph has ~1.8M segments, expand units cut at
# 1024 segments, and hub bins cut into several accumulate units meeting in the
# global accumulator.  Without a dense count the layout takes as many dense
# sources as it can (every whole block of a small graph); 0 sends every edge
# through the expand phase; "9,4,12,4096" splits the sources between the two.
@pytest.mark.parametrize("bits", ["15,14", "15,14,16,0", "4,5", "4,5,12,0", "9,4,12,4096", "13,13,14,8192"])
@pytest.mark.parametrize("n,m_raw,seed", [(1, 5, 0), (2, 1, 1), (257, 3000, 2), (30_000, 600_000, 31),
                                          (100_003, 3_000_000, 4)])
def test_blocked_schedule_matches_oracle(torch, block_bits, bits, n, m_raw, seed):
    block_bits(bits)
    if n == 30_000:
        src, dst = gen.rmat_coo(n, m_raw, seed=seed)
    else:
        src, dst = random_coo_with_dups(np.random.default_rng(seed), n, m_raw)
    for dt in (gpr.FP32, gpr.BF16):
        check(torch, n, src, dst, 25, dt, spmv="blocked")


@pytest.mark.parametrize("dt", [gpr.FP32, gpr.BF16])
def test_blocked_sums_do_not_depend_on_the_dense_sources(torch, block_bits, dt):
    # the row sums are exact integer sums of the same codes, whichever edges
    # read their code directly (dense sources) and which through the expand
    # phase: the results are bitwise identical
    n = 60_000
    src, dst = gen.rmat_coo(n, 1_500_000, seed=33)
    g = gpr.graph_build(src, dst, n)
    xs = []
    for bits in ("12,12,14,0", "12,12,14,4096", "12,12,14,16384", "12,12,14,-1"):
        block_bits(bits)
        xs.append(gpu_pr(torch, g, 25, dt=dt, spmv="blocked"))
    for x in xs[1:]:
        assert (x == xs[0]).all()
    ref = oracle.pagerank(oracle.build_csc(n, src, dst), 0.85, 25)
    assert l1(xs[0], ref) <= TOL[dt]


def test_blocked_schedule_rejects_block_sizes_that_do_not_fit(torch, block_bits):
    g = gpr.graph_build(np.array([0, 1], np.int32), np.array([1, 0], np.int32), 2)
    out = torch.empty(2, device="cuda")
    for bits in ("16,16", "3,8", "8,17"):  # shared memory too small / blocks out of range
        block_bits(bits)
        with pytest.raises(gpr.GprError) as ei:
            gpr.pagerank(g, out, iters=3, spmv="blocked")
        assert ei.value.status == gpr.EINVAL
    block_bits("8,8")
    gpr.pagerank(g, out, iters=3, spmv="blocked")
    assert np.abs(out.cpu().numpy() - 0.5).max() < 1e-7


def test_blocked_schedule_long_rows_and_split_bins(torch, block_bits):
    # a hub row with 2M in-edges (longer than an accumulate unit) and a
    # source block whose segment is longer than an expand unit
    n = 70_000
    rng = np.random.default_rng(12)
    src = rng.integers(0, n, 3_000_000).astype(np.int32)
    dst = np.where(rng.random(3_000_000) < 0.7, 5, rng.integers(0, n, 3_000_000)).astype(np.int32)
    for bits in ("15,14", "12,12"):
        block_bits(bits)
        check(torch, n, src, dst, 20, gpr.FP32, spmv="blocked")


def test_blocked_schedule_deterministic_and_switching(torch):
    src, dst = gen.rmat_coo(40_000, 900_000, seed=7)
    g = gpr.graph_build(src, dst, 40_000)
    a = gpu_pr(torch, g, 30, spmv="blocked")
    p = gpu_pr(torch, g, 30, spmv="pull")
    b = gpu_pr(torch, g, 30, spmv="blocked")
    assert (a == b).all()
    assert l1(a, p) <= 2e-6
    out = torch.empty(g.n, device="cuda")
    with pytest.raises(gpr.GprError) as ei:  # both schedules at once
        gpr._check(gpr.lib().pagerank(g.handle, 0.85, 3, gpr.FP32, gpr.SPMV_PULL | gpr.SPMV_BLOCKED,
                                      out.data_ptr(), None, None))
    assert ei.value.status == gpr.EINVAL


def test_tuner_records_its_choice_for_the_graph_and_its_shape(torch):
    # 2^18 nodes, 2^23 raw edges: above the size at which pagerank tunes
    n, m_raw = 1 << 18, 1 << 23
    src, dst = gen.rmat_coo(n, m_raw, seed=41)
    g = gpr.graph_build(src, dst, n)
    r = gpr.pagerank_tune(g, trial_steps=3)
    assert r.schedule in (gpr.SPMV_PULL, gpr.SPMV_BLOCKED)
    assert r.candidates >= 2 and r.ms_per_step > 0 and r.pull_ms_per_step >= r.ms_per_step
    if r.schedule == gpr.SPMV_BLOCKED:
        assert 4 <= r.sb_bits <= 16 and 4 <= r.w_bits <= 16 and r.unit_edges > 0
    x, st = gpu_pr(torch, g, 30, stats=True)
    assert st.schedule == r.schedule
    ref_g = oracle.build_csc(n, src, dst)
    assert l1(x, oracle.pagerank(ref_g, 0.85, 30)) <= 1e-5
    # another graph of the same shape takes the recorded choice without timing
    src2, dst2 = gen.rmat_coo(n, m_raw, seed=42)
    g2 = gpr.graph_build(src2, dst2, n)
    x2, st2 = gpu_pr(torch, g2, 30, stats=True)
    assert st2.schedule == r.schedule
    assert l1(x2, oracle.pagerank(oracle.build_csc(n, src2, dst2), 0.85, 30)) <= 1e-5
    for bad in (0, 1001):
        with pytest.raises(gpr.GprError) as ei:
            gpr.pagerank_tune(g, trial_steps=bad)
        assert ei.value.status == gpr.EINVAL


@pytest.mark.parametrize("spmv", ["pull", "blocked"])
def test_closed_forms_on_gpu(torch, spmv):
    N = 1000
    cyc = np.arange(N, dtype=np.int32)
    g = gpr.graph_build(torch.from_numpy(cyc).cuda(), torch.from_numpy((cyc + 1) % N).cuda(), N)
    x = gpu_pr(torch, g, 50, spmv=spmv)
    assert np.abs(x - 1.0 / N).max() < 1e-9
    # out-star: hub 0 -> leaves, fixed point x_hub = 1 / (N + d)
    leaves = np.arange(1, N, dtype=np.int32)
    g = gpr.graph_build(torch.from_numpy(np.zeros_like(leaves)).cuda(), torch.from_numpy(leaves).cuda(), N)
    x = gpu_pr(torch, g, 200, spmv=spmv)
    assert abs(x[0] - 1.0 / (N + 0.85)) < 1e-7
    # no edges at all: uniform
    z = torch.zeros(0, dtype=torch.int32, device="cuda")
    g = gpr.graph_build(z, z, 77)
    x = gpu_pr(torch, g, 10, spmv=spmv)
    assert np.abs(x - 1.0 / 77).max() < 1e-9


def test_zero_iterations_and_damping_values(torch):
    src, dst = gen.rmat_coo(5000, 60_000, seed=5)
    g = gpr.graph_build(src, dst, 5000)
    x = gpu_pr(torch, g, 0)
    assert np.abs(x - 1.0 / 5000).max() < 1e-12
    ref_g = oracle.build_csc(5000, src, dst)
    for d in (0.5, 0.99):
        x = gpu_pr(torch, g, 40, d=d)
        assert l1(x, oracle.pagerank(ref_g, d, 40)) <= 1e-5


def test_stats_match_oracle(torch):
    src, dst = gen.rmat_coo(20_000, 200_000, seed=6)
    g = gpr.graph_build(src, dst, 20_000)
    ref_g = oracle.build_csc(20_000, src, dst)
    xr, resid, _ = oracle.pagerank(ref_g, 0.85, 12, with_resid=True)
    x, st = gpu_pr(torch, g, 12, stats=True)
    assert st.iters_run == 12
    assert abs(st.residual_l1 - resid[-1]) <= 1e-6
    assert abs(st.mass - 1.0) <= 1e-6
    assert abs(st.dangling - xr[ref_g.outdeg == 0].sum()) <= 1e-5


def test_deterministic(torch):
    src, dst = gen.rmat_coo(40_000, 900_000, seed=7)
    g = gpr.graph_build(src, dst, 40_000)
    a = gpu_pr(torch, g, 30)
    b = gpu_pr(torch, g, 30)
    g2 = gpr.graph_build(src, dst, 40_000)
    c = gpu_pr(torch, g2, 30)
    assert (a == b).all() and (a == c).all()


def test_host_output_and_streams(torch):
    src, dst = gen.rmat_coo(8000, 90_000, seed=8)
    g = gpr.graph_build(src, dst, 8000)
    out = np.empty(8000, np.float32)
    s = torch.cuda.Stream()
    gpr.pagerank(g, out, iters=20, stream=s)
    ref = oracle.pagerank(oracle.build_csc(8000, src, dst), 0.85, 20)
    assert l1(out, ref) <= 1e-5


def test_rejects_bad_arguments(torch):
    g = gpr.graph_build(np.array([0], np.int32), np.array([1], np.int32), 2)
    out = torch.empty(2, device="cuda")
    for kw in ({"damping": 0.0}, {"damping": 1.0}, {"iters": -1}, {"dtype": 7}):
        with pytest.raises(gpr.GprError) as ei:
            gpr.pagerank(g, out, **kw)
        assert ei.value.status == gpr.EINVAL


@pytest.mark.slow
def test_rmat_lj_full_oracle(torch):
    """LiveJournal-shaped graph (4.8M ids, 69M raw edges), 100 iterations,
    full-vector comparison against the oracle."""
    spec = workloads.RMAT_LJ
    src, dst = coo_for(spec)
    err = check(torch, spec.n, src, dst, spec.iters)
    print(f"rmat-lj L1 = {err:.3e}")


@pytest.mark.slow
def test_rmat25_full_size_against_oracle(torch):
    """Billion-edge graph in the benchmark's launch configuration (R-MAT
    scale 25, edge factor 32, 100 iterations, the library's own schedule
    choice) against the FP64 oracle's stored x_100: L1 <= 1e-5 over the whole
    vector when its file is present, and always on the committed sample of
    2,048 nodes (L1 relative to the sampled mass, the estimate of the full
    L1) with the largest relative error bounded too."""
    spec = workloads.RMAT_25
    meta, full = load_rmat25_oracle()
    if meta is None:
        pytest.skip("oracle summary of the scale-25 workload not written")
    n, m_raw = spec.n, spec.m
    s_d = torch.empty(m_raw, dtype=torch.int32, device="cuda")
    d_d = torch.empty(m_raw, dtype=torch.int32, device="cuda")
    perm = torch.from_numpy(gen.permutation(n, spec.seed)).cuda()
    gen.rmat_coo_dev(n, m_raw, spec.seed, s_d.data_ptr(), d_d.data_ptr(), perm.data_ptr())
    g = gpr.graph_build(s_d, d_d, n)
    del s_d, d_d, perm
    torch.cuda.empty_cache()
    assert g.m == meta["m"]
    # the full-size CSC offsets and out-degrees are the oracle's, bit for bit
    import hashlib
    cp, _, od = g.export()
    assert hashlib.sha256(np.ascontiguousarray(cp, np.int32).tobytes()).hexdigest() == meta["sha256_col_ptr"]
    assert hashlib.sha256(np.ascontiguousarray(od, np.int32).tobytes()).hexdigest() == meta["sha256_outdeg"]
    del cp, od
    x = gpu_pr(torch, g, spec.iters)
    rel_l1, mr = sampled_errors(x, meta)
    print(f"rmat25 sampled: relative L1 {rel_l1:.3e}, max rel {mr:.3e}")
    assert rel_l1 <= 1e-5 and mr <= 1e-4
    if full is not None:
        err = l1(x, full)
        print(f"rmat25 full: L1 {err:.3e}, max rel {max_rel(x, full):.3e}")
        assert err <= 1e-5


@pytest.mark.slow
def test_rmat25_properties_at_full_size(torch):
    """Billion-edge graph: properties that hold at any size, in the benchmark's
    launch configuration: unit mass, the lower bound (1-d)/N on every entry,
    and one exact FP64 step on the GPU's own CSC carrying x_99 to within
    FP32 rounding of x_100."""
    spec = workloads.RMAT_25
    n, m_raw = spec.n, spec.m
    s_d = torch.empty(m_raw, dtype=torch.int32, device="cuda")
    d_d = torch.empty(m_raw, dtype=torch.int32, device="cuda")
    perm = torch.from_numpy(gen.permutation(n, spec.seed)).cuda()
    gen.rmat_coo_dev(n, m_raw, spec.seed, s_d.data_ptr(), d_d.data_ptr(), perm.data_ptr())
    g = gpr.graph_build(s_d, d_d, n)
    del s_d, d_d, perm
    torch.cuda.empty_cache()
    x99 = gpu_pr(torch, g, 99).astype(np.float64)
    x100, st = gpu_pr(torch, g, 100, stats=True)
    assert abs(x100.astype(np.float64).sum() - 1.0) <= 1e-5
    assert x100.min() >= (1 - 0.85) / n * (1 - 1e-5)
    cp, ri, od = g.export()
    s = x99.sum()
    dang = x99[od == 0].sum()
    contrib = np.where(od > 0, x99 / np.maximum(od, 1), 0.0) / s
    starts = np.minimum(cp[:-1].astype(np.int64), max(len(ri) - 1, 0))
    pulled = np.add.reduceat(contrib[ri], starts) if len(ri) else np.zeros(n)
    pulled[np.diff(cp) == 0] = 0.0
    step = (1 - 0.85) / n + 0.85 * (pulled + dang / s / n)
    assert l1(x100, step) <= 1e-5
