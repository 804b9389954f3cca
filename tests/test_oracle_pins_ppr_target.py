"""Pins for the oracle's single-target personalised PageRank (section 4.3,
"Fast Random Walk Algorithms": a backward phase from the target, then random
walks forward from the sources).  No GPU.

The estimator targets pi_s(t), the personalised PageRank of oracle.ppr
(restart 1 - d, dangling mass back to the seed).  It rests on Q_s(t), the
chance that one excursion from s (stop with probability a = 1 - d at every
node, absorbed at a dangling node when it does not stop) stops at t:
pi_s(t) = Q_s(t) / sum_v Q_s(v).  The reverse push keeps
Q_s(t) = p(s) + sum_v Q_s(v) r(v), and the estimate averages, over PageRank
walks from s ending at V, the unbiased term p(s) (1 + (d/a) 1{V dangling}) + r(V).
The pins check, against independent dense solves, closed forms and sampling
bounds: the contributions, the ratio identity, the push invariant, the
estimates, and that planted slips in push or estimate fail them.
"""
import numpy as np
import pytest

import gen
import oracle

D = 0.85
A = 1.0 - D


def random_graph(rng, n, m):
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    return oracle.build_csc(n, src, dst)


def csc(n, edges):
    return oracle.build_csc(n, np.array([u for u, _ in edges], np.int32), np.array([v for _, v in edges], np.int32))


def dense_Q(g):
    """Q[s, v] = Q_s(v) = a (I - d P)^-1 with P[u, v] = 1/outdeg(u) for u -> v
    (rows of dangling nodes zero), from a dense solve."""
    n = g.n
    P = np.zeros((n, n))
    for v in range(n):
        for u in g.row_idx[g.col_ptr[v]:g.col_ptr[v + 1]]:
            P[u, v] = 1.0 / g.outdeg[u]
    return A * np.linalg.inv(np.eye(n) - D * P)


# ------------------------------------------------------------ contributions --

@pytest.mark.parametrize("seed", range(10))
def test_contributions_match_dense_solve(seed):
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(2, 60))
    g = random_graph(rng, n, int(rng.integers(0, 4 * n)))
    Q = dense_Q(g)
    for t in rng.integers(0, n, 3):
        q = oracle.ppr_contrib(g, int(t), D, 250)
        assert np.abs(q - Q[:, t]).max() <= 1e-14


@pytest.mark.parametrize("N", [3, 8, 25])
def test_contributions_cycle_closed_form(N):
    # directed cycle i -> i+1: the excursion from s stops at t after
    # k = (t - s) mod N steps plus whole laps
    g = csc(N, [(i, (i + 1) % N) for i in range(N)])
    t = N // 2
    q = oracle.ppr_contrib(g, t, D, 400)
    for s in range(N):
        k = (t - s) % N
        assert abs(q[s] - A * D ** k / (1 - D ** N)) < 1e-14


# ------------------------------------------------------------ ratio identity --

@pytest.mark.parametrize("seed", range(8))
def test_ppr_is_normalised_excursion_distribution(seed):
    # pi_s = Q_s / sum(Q_s): the walk with dangling mass returned to s is a
    # run of excursions until one stops (and Q_s = pi_s without dangling nodes)
    rng = np.random.default_rng(800 + seed)
    n = int(rng.integers(2, 50))
    g = random_graph(rng, n, int(rng.integers(n, 4 * n)))
    Q = dense_Q(g)
    for s in rng.integers(0, n, 3):
        x, _ = oracle.ppr(g, int(s), D, 300)
        assert np.abs(x - Q[s] / Q[s].sum()).max() <= 1e-13
    cyc = csc(n, [(i, (i + 1) % n) for i in range(n)] + [(i, (3 * i + 1) % n) for i in range(n)])
    assert (cyc.outdeg > 0).all()
    Qc = dense_Q(cyc)
    assert np.abs(Qc.sum(axis=1) - 1).max() <= 1e-13


# -------------------------------------------------------------- reverse push --

@pytest.mark.parametrize("seed", range(10))
@pytest.mark.parametrize("r_max", [0.3, 1e-3, 1e-7])
def test_reverse_push_invariant(seed, r_max):
    rng = np.random.default_rng(900 + seed)
    n = int(rng.integers(2, 60))
    g = random_graph(rng, n, int(rng.integers(0, 4 * n)))
    Q = dense_Q(g)
    t = int(rng.integers(0, n))
    p, r, pushes = oracle.reverse_push(g, t, D, r_max)
    assert (p >= 0).all() and (r >= 0).all() and r.max() <= r_max
    # Q_s(t) = p(s) + sum_v Q_s(v) r(v) for every s
    assert np.abs(Q[:, t] - (p + Q @ r)).max() <= 1e-14
    # hence 0 <= Q_s(t) - p(s) <= r_max sum_v Q_s(v) <= r_max
    gap = Q[:, t] - p
    assert gap.min() >= -1e-15 and (gap <= r_max * Q.sum(axis=1) + 1e-15).all()
    # pushes are taken only above the threshold: none when r_max >= 1
    p0, r0, k0 = oracle.reverse_push(g, t, D, 1.0)
    assert k0 == 0 and p0.sum() == 0 and r0[t] == 1 and r0.sum() == 1


def test_reverse_push_in_star_closed_form():
    # leaves 1..N-1 -> hub 0; one push at the hub gives every leaf d / 1
    N = 7
    g = csc(N, [(i, 0) for i in range(1, N)])
    p, r, k = oracle.reverse_push(g, 0, D, 0.9)
    assert k == 1 and p[0] == A and (r[1:] == D).all() and r[0] == 0
    p, r, k = oracle.reverse_push(g, 0, D, 1e-3)
    assert k == N and p[0] == A and np.allclose(p[1:], A * D, rtol=0, atol=1e-16) and r.max() == 0


# --------------------------------------------------------------- estimates --

def sampling_tol(p_s, W, r_max):
    """Six standard deviations of the estimate: it is the mean of W terms
    p(s) (d/a) 1{V dangling} + r(V), each in [0, p(s) d/a + min(r_max, 1)]."""
    return 3 * (p_s * D / A + min(r_max, 1.0)) / np.sqrt(W) + 1e-12


@pytest.mark.parametrize("r_max", [1.0, 1e-2, 1e-4])
def test_estimates_within_sampling_bound(r_max):
    n = 300
    src, dst = gen.rmat_coo(n, 2400, seed=11)
    g = oracle.build_csc(n, src, dst)
    assert (g.outdeg == 0).any()          # dangling nodes present
    Q = dense_Q(g)
    t = int(np.argmax(np.diff(g.col_ptr)))  # a well-reached target
    p, r, _ = oracle.reverse_push(g, t, D, r_max)
    sources = np.concatenate([np.arange(0, n, 7), [t]]).astype(np.int32)
    W = 4000
    est = oracle.ppr_target(g, t, sources, D, r_max, W, seed=5)
    for s, e in zip(sources, est):
        pi = Q[s, t] / Q[s].sum()
        assert abs(e - pi) <= sampling_tol(p[s], W, r_max), (s, e, pi)


def test_no_dangling_estimate_is_push_plus_walk_mean():
    # without dangling nodes pi_s = Q_s and the estimate is p(s) + mean r(V):
    # within 3 r_max / sqrt(W) of Q_s(t)
    n = 200
    edges = [(i, (i + 1) % n) for i in range(n)] + [(i, (i * 7 + 3) % n) for i in range(n)]
    g = csc(n, edges)
    Q = dense_Q(g)
    t, W = 17, 2000
    sources = np.arange(n, dtype=np.int32)
    for r_max in (1e-3, 1e-5):
        est = oracle.ppr_target(g, t, sources, D, r_max, W, seed=9)
        assert np.abs(est - Q[:, t]).max() <= 3 * r_max / np.sqrt(W) + 1e-13


def test_pure_walks_are_endpoint_frequencies():
    # r_max >= 1: no push, and the estimate is the fraction of the seeded
    # walks that end at t, reproducible exactly from the same streams
    n = 300
    src, dst = gen.rmat_coo(n, 2400, seed=12)
    g = oracle.build_csc(n, src, dst)
    sources = np.arange(0, n, 5, dtype=np.int32)
    W = 500
    a = oracle.ppr_target(g, 3, sources, D, 1.0, W, seed=77)
    b = oracle.ppr_target(g, 3, sources, D, 1.0, W, seed=77)
    c = oracle.ppr_target(g, 3, sources, D, 1.0, W, seed=78)
    assert (a == b).all() and not (a == c).all()
    assert np.abs(a * W - np.round(a * W)).max() < 1e-9
    # summed over all targets, every walk ends somewhere exactly once
    tot = sum(oracle.ppr_target(g, t, sources[:4], D, 1.0, 300, seed=3) for t in range(n))
    assert np.abs(tot - 1).max() <= 1e-12


def test_degenerate_sources():
    g = csc(4, [(0, 1), (1, 2), (2, 0)])      # node 3 isolated
    # an isolated source: every walk ends at s, which is dangling, so the
    # estimate is p(s) (1 + d/a) = a + d = 1; and 0 from anywhere else
    est = oracle.ppr_target(g, 3, np.array([3, 0], np.int32), D, 1e-4, 200, seed=1)
    assert abs(est[0] - 1.0) <= 1e-15 and est[1] == 0.0
    # source = target on a cycle: (1 - d) / (1 - d^3)
    est = oracle.ppr_target(g, 0, np.array([0], np.int32), D, 1e-9, 50, seed=1)
    assert abs(est[0] - A / (1 - D ** 3)) <= 1e-8
    with pytest.raises(ValueError):
        oracle.ppr_target(g, 0, np.array([4], np.int32), D, 1e-4, 10)
    with pytest.raises(ValueError):
        oracle.reverse_push(g, 4, D, 1e-4)
    with pytest.raises(ValueError):
        oracle.ppr_target(g, 0, np.array([0], np.int32), D, 1e-4, 0)


# ------------------------------------------------ planted mistakes are caught --

def _mutant_push(g, t, r_max, mutation):
    """Reverse push written out in Python with one deliberate slip."""
    n = g.n
    p, r = np.zeros(n), np.zeros(n)
    r[t] = 1.0
    out_lists = [[] for _ in range(n)]
    for v in range(n):
        for u in g.row_idx[g.col_ptr[v]:g.col_ptr[v + 1]]:
            out_lists[u].append(v)
    while r.max() > r_max:
        v = int(np.argmax(r))
        amt, r[v] = r[v], 0.0
        p[v] += A * amt
        if mutation == "push_to_out_neighbours":
            for w in out_lists[v]:
                r[w] += D * amt / len(out_lists[v])
        else:
            for u in g.row_idx[g.col_ptr[v]:g.col_ptr[v + 1]]:
                deg = g.outdeg[v] if mutation == "target_degree" else g.outdeg[u]
                r[u] += D * amt / max(deg, 1)
    return p, r


@pytest.mark.parametrize("mutation", ["push_to_out_neighbours", "target_degree"])
def test_pins_catch_planted_push_mistakes(mutation):
    rng = np.random.default_rng(4)
    g = random_graph(rng, 40, 160)
    Q = dense_Q(g)
    t = int(np.argmax(np.diff(g.col_ptr)))
    p, r = _mutant_push(g, t, 1e-6, mutation)
    assert np.abs(Q[:, t] - (p + Q @ r)).max() > 1e-6
    p, r = _mutant_push(g, t, 1e-6, "none")
    assert np.abs(Q[:, t] - (p + Q @ r)).max() <= 1e-14


@pytest.mark.parametrize("mutation", ["dangling_as_stop", "no_dangling_factor"])
def test_sampling_bound_catches_estimator_mistakes(mutation):
    # the exact expectation of a slipped estimator, from the dense solve and
    # the oracle's own push, misses pi_s(t) by more than the sampling
    # tolerance for some source of this graph
    n = 300
    src, dst = gen.rmat_coo(n, 2400, seed=11)
    g = oracle.build_csc(n, src, dst)
    Q = dense_Q(g)
    dang = g.outdeg == 0
    t = int(np.argmax(np.diff(g.col_ptr)))
    r_max, W = 1e-4, 4000
    p, r, _ = oracle.reverse_push(g, t, D, r_max)
    worst = 0.0
    for s in range(n):
        pi_row = Q[s] / Q[s].sum()
        if mutation == "dangling_as_stop":
            # walks end at a dangling node instead of going back to s: the
            # endpoint law is that of one excursion, absorbed mass included
            L = Q[s] + np.where(dang, Q[s] * D / A, 0.0)
            expect = p[s] * (1 + D / A * L[dang].sum()) + L @ r
        else:
            # the estimate without the dangling factor on p(s)
            expect = p[s] + pi_row @ r
        worst = max(worst, abs(expect - pi_row[t]) / sampling_tol(p[s], W, r_max))
    assert worst > 1.0
    # the unslipped expectation meets pi_s(t) to rounding
    for s in range(0, n, 3):
        pi_row = Q[s] / Q[s].sum()
        assert abs(p[s] * (1 + D / A * pi_row[dang].sum()) + pi_row @ r - pi_row[t]) <= 1e-13
