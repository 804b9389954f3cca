"""Single-target personalised PageRank on the GPU (ppr_reverse_push,
ppr_target) against the oracle.

The push runs in rounds on the GPU and in FIFO order in the oracle, so p and r
differ in their last digits and in which nodes ended just below r_max; what
both must meet is the push's bound against the oracle's contributions q
(q(s) = Q_s(t), an independent fixed-point solve): 0 <= q(s) - p(s) <= r_max
for every s, all residuals in [0, r_max].  The walks replay the same seeded
streams on both sides, so with no push (r_max >= 1) the estimates, which are
then endpoint counts / W, agree bit for bit; with a push they agree with the
exact pi_s(t) within the estimator's sampling bound.
"""
import numpy as np
import pytest

import gen
import oracle
import paper_1606_07550_gb300 as gpr

pytestmark = pytest.mark.gpu

D = 0.85
A = 1 - D


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


@pytest.fixture(scope="module")
def graphs(torch):
    out = {}
    for name, (n, m_raw, seed) in {"rmat5k": (5000, 60_000, 31), "rmat40k": (40_000, 600_000, 32)}.items():
        src, dst = gen.rmat_coo(n, m_raw, seed=seed)
        g = gpr.graph_build(src, dst, n)
        out[name] = (g, oracle.build_csc(n, src, dst))
    # a small graph with the degenerate cases: isolated nodes, a node without
    # in-edges, a dangling sink
    edges = [(0, 1), (1, 2), (2, 0), (3, 0), (1, 4), (5, 4)]
    s = np.array([u for u, _ in edges], np.int32)
    d = np.array([v for _, v in edges], np.int32)
    out["tiny"] = (gpr.graph_build(s, d, 8), oracle.build_csc(8, s, d))
    return out


_Q = {}


def contrib(name, ref, t):
    if (name, t) not in _Q:
        _Q[name, t] = oracle.ppr_contrib(ref, t, D, 260)
    return _Q[name, t]


def targets_of(ref, rng, k=3):
    indeg = np.diff(ref.col_ptr)
    ts = [int(np.argmax(indeg)), int(np.argmin(indeg))]          # the hub and a node without in-edges
    ts += [int(t) for t in rng.integers(0, ref.n, k)]
    if (ref.outdeg == 0).any():
        ts.append(int(np.flatnonzero(ref.outdeg == 0)[0]))      # a dangling target
    return ts


@pytest.mark.parametrize("name", ["tiny", "rmat5k", "rmat40k"])
@pytest.mark.parametrize("r_max", [1e-3, 1e-6, 1e-10])
def test_push_bound_against_contributions(torch, graphs, name, r_max):
    g, ref = graphs[name]
    rng = np.random.default_rng(3)
    n = ref.n
    for t in targets_of(ref, rng):
        p = torch.empty(n, dtype=torch.float64, device="cuda")
        r = torch.empty(n, dtype=torch.float64, device="cuda")
        st = gpr.ppr_reverse_push(g, t, r_max, p, r)
        k = st.pushes
        p, r = p.cpu().numpy(), r.cpu().numpy()
        q = contrib(name, ref, t)
        assert (r >= 0).all() and r.max() <= r_max and (p >= 0).all()
        gap = q - p
        assert gap.min() >= -1e-13 and gap.max() <= r_max + 1e-13, (t, gap.min(), gap.max())
        # against the oracle's own push: both within r_max of q
        po, ro, ko = oracle.reverse_push(ref, t, D, r_max)
        assert np.abs(p - po).max() <= r_max + 1e-13
        assert k >= 1 and (k == 1) == (ko == 1)
        # each push scans the in-edges of its node; at least one per round
        assert st.rounds >= 1 and st.pushes >= st.rounds and st.edges >= 0 and st.push_ms > 0
        if k == 1:
            assert st.edges == np.diff(ref.col_ptr)[t] and st.rounds == 1


def test_push_host_buffers_and_no_push(torch, graphs):
    g, ref = graphs["rmat5k"]
    n = ref.n
    t = int(np.argmax(np.diff(ref.col_ptr)))
    p = np.empty(n)
    r = np.empty(n)
    k = gpr.ppr_reverse_push(g, t, 1e-5, p, r).pushes
    q = oracle.ppr_contrib(ref, t, D, 260)
    assert k > 1 and np.abs(q - p).max() <= 1e-5 + 1e-13 and r.max() <= 1e-5
    # r_max >= 1: nothing to push
    st = gpr.ppr_reverse_push(g, t, 1.0, p, r)
    k = st.pushes
    assert st.rounds == 0 and st.edges == 0 and k == 0 and p.max() == 0 and r[t] == 1 and r.sum() == 1
    # only one output wanted
    k2 = gpr.ppr_reverse_push(g, t, 1e-5, p, None).pushes
    assert k2 > 1 and np.abs(q - p).max() <= 1e-5 + 1e-13


@pytest.mark.parametrize("name", ["tiny", "rmat5k", "rmat40k"])
def test_pure_walks_bit_exact(torch, graphs, name):
    # no push: each estimate is (walks ending at t) / W of the same seeded walks
    g, ref = graphs[name]
    rng = np.random.default_rng(4)
    n = ref.n
    sources = np.unique(np.concatenate([rng.integers(0, n, 40), np.flatnonzero(ref.outdeg == 0)[:5],
                                        [int(np.argmax(np.diff(ref.col_ptr)))]])).astype(np.int32)
    W = 700
    for t in targets_of(ref, rng, 2):
        want = oracle.ppr_target(ref, t, sources, D, 1.0, W, seed=123)
        out = torch.empty(len(sources), dtype=torch.float64, device="cuda")
        st = gpr.ppr_target(g, t, torch.from_numpy(sources).cuda(), out, 1.0, W, seed=123)
        assert (out.cpu().numpy() == want).all(), t
        # a walk stops with probability a per step: about len * W * d / a steps
        N = len(sources) * W
        assert abs(st.walk_steps / N - D / A) < 6 * np.sqrt(D) / A / np.sqrt(N)
        assert st.pushes == 0 and st.walk_ms > 0 and st.total_ms >= st.walk_ms
        # host buffers
        h = np.empty(len(sources))
        gpr.ppr_target(g, t, sources, h, 1.0, W, seed=123)
        assert (h == want).all()


def test_dangling_factor_exact(torch, graphs):
    # a target without in-edges: one push, p = a e_t, r = 0, and the estimate
    # from s = t is a (1 + (d/a) #dangling endpoints / W), exact up to rounding
    g, ref = graphs["rmat5k"]
    indeg = np.diff(ref.col_ptr)
    cand = np.flatnonzero((indeg == 0) & (ref.outdeg > 0))
    t = int(cand[0])
    srcs = np.array([t, int(cand[1])], np.int32)
    want = oracle.ppr_target(ref, t, srcs, D, 1e-4, 3000, seed=9)
    got = np.empty(2)
    gpr.ppr_target(g, t, srcs, got, 1e-4, 3000, seed=9)
    assert abs(got[0] - want[0]) <= 1e-15 * want[0] and got[1] == 0 and want[1] == 0
    assert want[0] > A  # some walks ended on dangling nodes


@pytest.mark.parametrize("name,r_max", [("rmat5k", 1e-3), ("rmat5k", 1e-5), ("rmat40k", 1e-5)])
def test_estimates_within_sampling_bound(torch, graphs, name, r_max):
    g, ref = graphs[name]
    rng = np.random.default_rng(6)
    n = ref.n
    t = int(np.argmax(np.diff(ref.col_ptr)))
    sources = np.unique(np.concatenate([rng.integers(0, n, 24), [t]])).astype(np.int32)
    W = 4000
    est = np.empty(len(sources))
    gpr.ppr_target(g, t, sources, est, r_max, W, seed=77)
    po, _, _ = oracle.reverse_push(ref, t, D, r_max)
    mine = oracle.ppr_target(ref, t, sources, D, r_max, W, seed=77)
    for s, e, o in zip(sources, est, mine):
        pi = oracle.ppr(ref, int(s), D, 200)[0][t]
        tol = 3 * ((po[s] + r_max) * D / A + r_max) / np.sqrt(W) + 1e-12
        assert abs(e - pi) <= tol, (s, e, pi, tol)
        # the same seeded walks on both sides: the estimates differ only
        # through the pushes, |dp(s)| <= r_max and |dr(V)| <= r_max
        assert abs(e - o) <= r_max * (2 + D / A) + 1e-13


@pytest.mark.parametrize("W", [1, 31, 256, 1000])
def test_walk_runs_split_across_sources(torch, graphs, W):
    # a thread runs several consecutive walks, which may span sources; many
    # sources and few walks each put those seams everywhere
    g, ref = graphs["rmat5k"]
    rng = np.random.default_rng(W)
    k = 20_000 // W + 3
    sources = rng.integers(0, ref.n, k).astype(np.int32)
    t = int(np.argmax(np.diff(ref.col_ptr)))
    want = oracle.ppr_target(ref, t, sources, D, 1.0, W, seed=5)
    out = np.empty(k)
    gpr.ppr_target(g, t, sources, out, 1.0, W, seed=5)
    assert (out == want).all()


def test_repeatable(torch, graphs):
    g, ref = graphs["rmat40k"]
    t = int(np.argmax(np.diff(ref.col_ptr)))
    sources = np.arange(0, ref.n, 401, dtype=np.int32)
    a, b = np.empty(len(sources)), np.empty(len(sources))
    gpr.ppr_target(g, t, sources, a, 1e-6, 500, seed=3)
    gpr.ppr_target(g, t, sources, b, 1e-6, 500, seed=3)
    assert np.abs(a - b).max() <= 1e-12      # the push's atomics may round differently


def test_errors_and_empty(torch, graphs):
    g, ref = graphs["tiny"]
    n = ref.n
    out = np.empty(2)
    for bad in [dict(target=n), dict(target=-1), dict(r_max=0.0), dict(r_max=float("nan")), dict(walks=0),
                dict(damping=1.0), dict(sources=np.array([0, n], np.int32))]:
        kw = dict(target=0, sources=np.array([0, 1], np.int32), r_max=1e-3, walks=10, damping=D)
        kw.update(bad)
        with pytest.raises(gpr.GprError) as ei:
            gpr.ppr_target(g, kw["target"], kw["sources"], out, kw["r_max"], kw["walks"], damping=kw["damping"])
        assert ei.value.status == gpr.EINVAL
    with pytest.raises(gpr.GprError):
        gpr.ppr_reverse_push(g, n, 1e-3, np.empty(n), None)
    gpr.ppr_target(g, 0, np.empty(0, np.int32), np.empty(0), 1e-3, 10)  # no sources: nothing to do
    # still usable after the errors
    est = np.empty(3)
    srcs = np.array([0, 3, 6], np.int32)
    gpr.ppr_target(g, 0, srcs, est, 1e-9, 64, seed=1)
    want = oracle.ppr_target(ref, 0, srcs, D, 1e-9, 64, seed=1)
    assert np.abs(est - want).max() <= 1e-9 * (2 + D / A) + 1e-13


def test_after_update_and_load(torch, tmp_path):
    # the out-adjacency cached for the walks follows edge updates and loads
    n = 3000
    src, dst = gen.rmat_coo(n, 30_000, seed=41)
    g = gpr.graph_build(src, dst, n)
    sources = np.arange(0, n, 37, dtype=np.int32)
    out = np.empty(len(sources))
    gpr.ppr_target(g, 5, sources, out, 1.0, 300, seed=2)
    ins = (np.arange(100, dtype=np.int32), (np.arange(100, dtype=np.int32) * 7 + 1) % n)
    gpr.graph_update(g, ins)
    es = {(int(u), int(v)) for u, v in zip(src, dst) if u != v} | {(int(u), int(v)) for u, v in zip(*ins) if u != v}
    es = sorted(es)
    ref = oracle.build_csc(n, np.array([u for u, _ in es], np.int32), np.array([v for _, v in es], np.int32))
    gpr.ppr_target(g, 5, sources, out, 1.0, 300, seed=2)
    assert (out == oracle.ppr_target(ref, 5, sources, D, 1.0, 300, seed=2)).all()
    path = str(tmp_path / "g.bin")
    g.save(path)
    g2 = gpr.graph_load(path)
    out2 = np.empty(len(sources))
    gpr.ppr_target(g2, 5, sources, out2, 1.0, 300, seed=2)
    assert (out2 == out).all()
