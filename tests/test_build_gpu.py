"""GPU COO -> CSC build against the CPU oracle: bit-exact arrays."""
import numpy as np
import pytest

import gen
import oracle
import paper_1606_07550_gb300 as gpr
from gen import workloads

from gpu_util import coo_for, random_coo_with_dups

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def build_and_compare(torch, n, src, dst, device=True):
    ref = oracle.build_csc(n, src, dst)
    if device:
        g = gpr.graph_build(torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda(), n)
    else:
        g = gpr.graph_build(src, dst, n)
    cp, ri, od = g.export()
    inf = g.info()
    assert inf.m == ref.m and inf.m_raw == len(src) and inf.n == n
    np.testing.assert_array_equal(cp, ref.col_ptr)
    np.testing.assert_array_equal(ri, ref.row_idx)
    np.testing.assert_array_equal(od, ref.outdeg)
    assert inf.n_dangling == int((ref.outdeg == 0).sum())
    g.free()
    return ref


@pytest.mark.parametrize("n,m_raw,seed", [
    (1, 10, 0), (2, 3, 1), (17, 500, 2), (1000, 4095, 3), (1000, 4097, 4), (5000, 50_001, 5),
    (70_000, 300_000, 6), (3, 20_000, 7), (1 << 16, 1 << 18, 8),
])
def test_random_coo_bit_exact(torch, n, m_raw, seed):
    rng = np.random.default_rng(seed)
    src, dst = random_coo_with_dups(rng, n, m_raw)
    build_and_compare(torch, n, src, dst)


def test_wide_ids_sort_with_nine_bit_digits(torch):
    # 2^25 + 3 nodes need 26-bit ids: the (dst, src) keys have 52 bits, sorted
    # in six passes of 8, 8, 9, 9, 9 and 9 bits, so digits start off byte
    # boundaries (bits 16, 25, 34, 43); the CSC must still be bit-exact
    n = (1 << 25) + 3
    rng = np.random.default_rng(12)
    src, dst = random_coo_with_dups(rng, n, 1 << 20)
    src[:1000] = n - 1 - np.arange(1000, dtype=np.int32)  # the highest ids take part
    build_and_compare(torch, n, src, dst)


def test_concurrent_builds_on_two_streams(torch):
    # builds from two threads at once: one borrows the device's sort scratch,
    # the other finds it lent and sorts in buffers of its own; both exact
    from concurrent.futures import ThreadPoolExecutor
    cases = [(200_000, 3_000_000, 21), (150_000, 2_500_000, 22)]
    inputs = []
    for n, m_raw, seed in cases:
        src, dst = random_coo_with_dups(np.random.default_rng(seed), n, m_raw)
        inputs.append((n, src, dst, oracle.build_csc(n, src, dst)))

    def run(case):
        n, src, dst, ref = case
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            s_d, d_d = torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda()
            stream.synchronize()
            outs = []
            for _ in range(3):
                g = gpr.graph_build(s_d, d_d, n, stream=stream)
                outs.append(g.export())
                g.free()
        return outs, ref

    with ThreadPoolExecutor(2) as ex:
        results = list(ex.map(run, inputs))
    for outs, ref in results:
        for cp, ri, od in outs:
            np.testing.assert_array_equal(cp, ref.col_ptr)
            np.testing.assert_array_equal(ri, ref.row_idx)
            np.testing.assert_array_equal(od, ref.outdeg)


def test_host_pointers(torch):
    rng = np.random.default_rng(11)
    src, dst = random_coo_with_dups(rng, 3000, 20_000)
    build_and_compare(torch, 3000, src, dst, device=False)


def test_edge_cases(torch):
    z = np.zeros(0, np.int32)
    build_and_compare(torch, 5, z, z)                                  # no edges
    build_and_compare(torch, 1, np.zeros(3, np.int32), np.zeros(3, np.int32))   # n = 1, loops only
    a = np.arange(1000, dtype=np.int32)
    build_and_compare(torch, 1000, a, a)                               # all self-loops
    build_and_compare(torch, 10, np.full(9000, 3, np.int32), np.full(9000, 7, np.int32))  # all duplicates
    hub_src = np.arange(1, 200_000, dtype=np.int32)
    build_and_compare(torch, 200_000, hub_src, np.zeros_like(hub_src))  # one in-hub, long row
    build_and_compare(torch, 200_000, np.zeros_like(hub_src), hub_src)  # one out-hub
    build_and_compare(torch, 1 << 20, np.array([0, (1 << 20) - 1], np.int32),
                      np.array([(1 << 20) - 1, 5], np.int32))            # id n - 1, huge gaps


def test_invalid_ids_are_rejected(torch):
    for bad in ([0, 5, 10], [0, -1, 3]):
        src = torch.tensor(bad, dtype=torch.int32, device="cuda")
        dst = torch.tensor([1, 2, 3], dtype=torch.int32, device="cuda")
        with pytest.raises(gpr.GprError) as ei:
            gpr.graph_build(src, dst, 10)
        assert ei.value.status == gpr.EINVAL
    # the device stays usable
    build_and_compare(torch, 4, np.array([0, 1], np.int32), np.array([1, 2], np.int32))


def test_er_10k_matches_oracle_and_golden(torch):
    import hashlib
    import json
    import os
    spec = workloads.ER_10K
    src, dst = gen.er_gnm(spec.n, spec.m, spec.seed)
    build_and_compare(torch, spec.n, src, dst)
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "er10k_pagerank50.json")))
    g = gpr.graph_build(src, dst, spec.n)
    cp, ri, od = g.export()
    assert hashlib.sha256(np.ascontiguousarray(ri).tobytes()).hexdigest() == gold["sha256_row_idx"]
    assert hashlib.sha256(np.ascontiguousarray(cp).tobytes()).hexdigest() == gold["sha256_col_ptr"]


def test_rmat_medium_bit_exact(torch):
    src, dst = gen.rmat_coo(1 << 18, 1 << 22, seed=21)
    build_and_compare(torch, 1 << 18, src, dst)


def test_device_generator_matches_host(torch):
    n, m = 100_000, 1_000_003
    s_h, d_h = gen.rmat_coo(n, m, seed=9)
    perm = torch.from_numpy(gen.permutation(n, 9)).cuda()
    s_d = torch.empty(m, dtype=torch.int32, device="cuda")
    d_d = torch.empty(m, dtype=torch.int32, device="cuda")
    gen.rmat_coo_dev(n, m, 9, s_d.data_ptr(), d_d.data_ptr(), perm.data_ptr())
    torch.cuda.synchronize()
    assert (s_d.cpu().numpy() == s_h).all() and (d_d.cpu().numpy() == d_h).all()
    u_h = gen.uniform_coo(n, m, seed=4)
    gen.uniform_coo_dev(n, m, 4, s_d.data_ptr(), d_d.data_ptr())
    torch.cuda.synchronize()
    assert (s_d.cpu().numpy() == u_h[0]).all() and (d_d.cpu().numpy() == u_h[1]).all()


def test_repeat_builds_identical(torch):
    src, dst = gen.rmat_coo(50_000, 700_000, seed=13)
    s, d = torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda()
    a = gpr.graph_build(s, d, 50_000).export()
    b = gpr.graph_build(s, d, 50_000).export()
    for x, y in zip(a, b):
        assert (x == y).all()


def _check_csc_invariants(cp, ri, od, n):
    assert cp[0] == 0 and (np.diff(cp.astype(np.int64)) >= 0).all() and cp[-1] == len(ri)
    assert int(od.astype(np.int64).sum()) == len(ri)
    assert ri.min() >= 0 and ri.max() < n


@pytest.mark.slow
@pytest.mark.parametrize("spec", [workloads.RMAT_LJ, workloads.RMAT_25], ids=lambda s: s.name)
def test_full_size_sampled_rows(torch, spec):
    """At the benchmark sizes, in the benchmark's launch configuration: sampled
    rows and out-degrees bit-exact against the oracle computed one by one
    from the raw COO, plus whole-array invariants."""
    n, m_raw = spec.n, spec.m
    s_d = torch.empty(m_raw, dtype=torch.int32, device="cuda")
    d_d = torch.empty(m_raw, dtype=torch.int32, device="cuda")
    perm = torch.from_numpy(gen.permutation(n, spec.seed)).cuda()
    gen.rmat_coo_dev(n, m_raw, spec.seed, s_d.data_ptr(), d_d.data_ptr(), perm.data_ptr())
    g = gpr.graph_build(s_d, d_d, n)
    cp, ri, od = g.export()
    g.free()
    src, dst = s_d.cpu().numpy(), d_d.cpu().numpy()
    del s_d, d_d
    torch.cuda.empty_cache()
    _check_csc_invariants(cp, ri, od, n)
    rng = np.random.default_rng(spec.seed)
    indeg = np.diff(cp.astype(np.int64))
    rows = np.unique(np.concatenate([rng.integers(0, n, 24), [int(indeg.argmax())], [0, n - 1]])).astype(np.int32)
    ref_rows = oracle.sample_in_rows(n, src, dst, rows)
    for v, ref in zip(rows, ref_rows):
        np.testing.assert_array_equal(ri[cp[v]:cp[v + 1]], ref)
    nodes = np.unique(np.concatenate([rng.integers(0, n, 24), [int(od.argmax())]])).astype(np.int32)
    np.testing.assert_array_equal(od[nodes], oracle.sample_outdeg(n, src, dst, nodes))
    # sources strictly ascending inside sampled rows, no self-loops anywhere sampled
    for v in rows:
        seg = ri[cp[v]:cp[v + 1]]
        assert (np.diff(seg) > 0).all() and not (seg == v).any()
