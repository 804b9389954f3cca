"""Generator sanity (no GPU): determinism, exact G(n, m), R-MAT quadrant rates."""
import numpy as np

import gen
from gen import workloads


def test_deterministic_and_seed_sensitive():
    a = gen.rmat_coo(1000, 5000, seed=1)
    b = gen.rmat_coo(1000, 5000, seed=1)
    c = gen.rmat_coo(1000, 5000, seed=2)
    assert (a[0] == b[0]).all() and (a[1] == b[1]).all()
    assert not (a[0] == c[0]).all()


def test_er_gnm_has_exactly_m_distinct_non_loop_edges():
    src, dst = gen.er_gnm(10_000, 100_000, seed=1)
    pairs = {(int(u), int(v)) for u, v in zip(src, dst) if u != v}
    assert len(pairs) == 100_000
    # the last draw is the one that completed the set
    pairs2 = {(int(u), int(v)) for u, v in zip(src[:-1], dst[:-1]) if u != v}
    assert len(pairs2) == 99_999
    assert len(src) > 100_000  # repeats and loops are in the raw stream


def test_uniform_prefix_property():
    s1, d1 = gen.uniform_coo(777, 100, seed=4)
    s2, d2 = gen.uniform_coo(777, 1000, seed=4)
    assert (s1 == s2[:100]).all() and (d1 == d2[:100]).all()
    assert s2.min() >= 0 and s2.max() < 777


def test_permutation_is_bijection():
    p = gen.permutation(100_000, seed=3)
    assert (np.sort(p) == np.arange(100_000)).all()


def test_rmat_quadrant_rates():
    # unpermuted, n = 2^scale: the top bit of the source is 1 with
    # probability c + d = 0.24, of the destination with b + d = 0.24,
    # and both with d = 0.05
    scale = 12
    src, dst = gen.rmat_coo(1 << scale, 200_000, seed=8, permute=False)
    top = 1 << (scale - 1)
    su = (src & top) != 0
    du = (dst & top) != 0
    assert abs(su.mean() - 0.24) < 0.005
    assert abs(du.mean() - 0.24) < 0.005
    assert abs((su & du).mean() - 0.05) < 0.003
    # node 0 is the heaviest source
    assert np.bincount(src).argmax() == 0


def test_rmat_rejection_keeps_ids_in_range():
    src, dst = gen.rmat_coo(4_800, 50_000, seed=2)
    assert src.max() < 4_800 and dst.max() < 4_800 and src.min() >= 0


def test_workload_specs():
    specs = workloads.batched_specs(64)
    ns = np.array([s.n for s in specs])
    assert ns.min() >= 1000 and ns.max() <= 200_000
    degs = np.array([s.m / s.n for s in specs])
    assert degs.min() >= 3.99 and degs.max() <= 32.01
    pool = workloads.serving_pool_specs(18)
    assert [p.scale for p in pool[:9]] == list(range(14, 23))
    reqs = workloads.serving_trace([p.n for p in pool], rate=2000, duration=0.5)
    assert 800 < len(reqs) < 1200
    assert all(1 <= len(r.seeds) <= 64 for r in reqs)
    assert all(0.8 <= r.damping <= 0.9 for r in reqs)
    assert all(not r.bf16 or r.tol == 1e-3 for r in reqs)
