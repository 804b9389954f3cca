"""Pins for the CPU oracle against what mathematics fixes (no GPU).

The paper prints no PageRank values, no worked example and no error bound
(section 6 reports only timings), so every pin here is a closed form, a brute
force, an independent dense linear solve or an invariant.  Each is chosen so
that a plausible slip in the oracle (a dropped dangling term, a wrong
teleport, a transposed adjacency, an off-by-one in the CSC) fails one of them.
"""
import numpy as np
import pytest

import gen
import oracle

D = 0.85


# ---------------------------------------------------------------- helpers --

def brute_csc(n, src, dst):
    """Simple directed graph by Python sets: distinct (u, v), u != v."""
    edges = sorted({(int(u), int(v)) for u, v in zip(src, dst) if u != v}, key=lambda e: (e[1], e[0]))
    col_ptr = [0] * (n + 1)
    for _, v in edges:
        col_ptr[v + 1] += 1
    for v in range(n):
        col_ptr[v + 1] += col_ptr[v]
    row_idx = [u for u, _ in edges]
    outdeg = [0] * n
    for u, _ in edges:
        outdeg[u] += 1
    return np.array(col_ptr), np.array(row_idx, dtype=np.int64), np.array(outdeg), edges


def dense_google(n, edges, t):
    """Column-stochastic M with M[v, u] = 1/outdeg(u) for u -> v and the
    column of a dangling u replaced by the teleport vector t."""
    outdeg = np.zeros(n)
    for u, _ in edges:
        outdeg[u] += 1
    M = np.zeros((n, n))
    for u, v in edges:
        M[v, u] += 1.0 / outdeg[u]
    for u in range(n):
        if outdeg[u] == 0:
            M[:, u] = t
    return M


def dense_fixed_point(n, edges, t, d=D):
    """Solve (I - d M) x = (1 - d) t."""
    M = dense_google(n, edges, t)
    return np.linalg.solve(np.eye(n) - d * M, (1.0 - d) * t)


def dense_power(n, edges, t, x0, k, d=D):
    M = dense_google(n, edges, t)
    x = x0.copy()
    for _ in range(k):
        x = (1.0 - d) * t + d * (M @ x)
    return x


def csc_from_edges(n, edges):
    src = np.array([u for u, _ in edges], np.int32)
    dst = np.array([v for _, v in edges], np.int32)
    return oracle.build_csc(n, src, dst)


def random_coo(rng, n, m_raw, p_loop=0.1, p_dup=0.2):
    src = rng.integers(0, n, m_raw)
    dst = rng.integers(0, n, m_raw)
    for i in range(m_raw):
        r = rng.random()
        if r < p_loop:
            dst[i] = src[i]
        elif r < p_loop + p_dup and i > 0:
            j = rng.integers(0, i)
            src[i], dst[i] = src[j], dst[j]
    return src.astype(np.int32), dst.astype(np.int32)


# ------------------------------------------------------------- CSC build --

@pytest.mark.parametrize("seed", range(40))
def test_build_matches_brute_force(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 14))
    m_raw = int(rng.integers(0, 70))
    src, dst = random_coo(rng, n, m_raw)
    g = oracle.build_csc(n, src, dst)
    cp, ri, od, edges = brute_csc(n, src, dst)
    assert g.m == len(edges)
    np.testing.assert_array_equal(g.col_ptr, cp)
    np.testing.assert_array_equal(g.row_idx, ri)
    np.testing.assert_array_equal(g.outdeg, od)
    assert g.outdeg.sum() == g.m == g.col_ptr[-1]


def test_build_invariant_under_coo_order_duplicates_and_loops():
    rng = np.random.default_rng(7)
    n, m_raw = 50, 400
    src, dst = random_coo(rng, n, m_raw, p_loop=0.0, p_dup=0.0)
    g0 = oracle.build_csc(n, src, dst)
    perm = rng.permutation(m_raw)
    loops = rng.integers(0, n, 60).astype(np.int32)
    src2 = np.concatenate([src[perm], src[:100], loops])
    dst2 = np.concatenate([dst[perm], dst[:100], loops])
    g1 = oracle.build_csc(n, src2, dst2)
    np.testing.assert_array_equal(g0.col_ptr, g1.col_ptr)
    np.testing.assert_array_equal(g0.row_idx, g1.row_idx)
    np.testing.assert_array_equal(g0.outdeg, g1.outdeg)


def test_build_edge_cases():
    # empty edge list: all nodes isolated
    g = oracle.build_csc(5, np.zeros(0, np.int32), np.zeros(0, np.int32))
    assert g.m == 0 and list(g.col_ptr) == [0] * 6 and list(g.outdeg) == [0] * 5
    # only self-loops
    g = oracle.build_csc(3, np.array([0, 1, 2, 2], np.int32), np.array([0, 1, 2, 2], np.int32))
    assert g.m == 0
    # one node
    g = oracle.build_csc(1, np.array([0], np.int32), np.array([0], np.int32))
    assert g.m == 0 and list(g.col_ptr) == [0, 0]
    # largest id n - 1
    g = oracle.build_csc(4, np.array([3, 3, 0], np.int32), np.array([0, 0, 3], np.int32))
    assert list(g.col_ptr) == [0, 1, 1, 1, 2] and list(g.row_idx) == [3, 0] and list(g.outdeg) == [1, 0, 0, 1]


def test_build_rejects_out_of_range_ids():
    for s, d in [([0, 5], [1, 1]), ([0, 1], [1, -1]), ([-1], [0])]:
        with pytest.raises(ValueError):
            oracle.build_csc(5, np.array(s, np.int32), np.array(d, np.int32))


def test_sampled_rows_and_outdeg_match_full_build():
    src, dst = gen.rmat_coo(3000, 40000, seed=11)
    g = oracle.build_csc(3000, src, dst)
    rows = np.array([0, 5, 17, 2999, 1234, 777], np.int32)
    lists = oracle.sample_in_rows(3000, src, dst, rows)
    for v, lst in zip(rows, lists):
        np.testing.assert_array_equal(lst, g.row_idx[g.col_ptr[v]:g.col_ptr[v + 1]])
    od = oracle.sample_outdeg(3000, src, dst, rows)
    np.testing.assert_array_equal(od, g.outdeg[rows])


# -------------------------------------------------------- closed forms --

@pytest.mark.parametrize("N", [1, 2, 3, 10, 257])
def test_cycle_uniform_every_iteration(N):
    edges = [(i, (i + 1) % N) for i in range(N)] if N > 1 else []
    g = csc_from_edges(N, edges)
    for k in [0, 1, 2, 7, 50]:
        x = oracle.pagerank_uniform(g, D, k)
        np.testing.assert_allclose(x, 1.0 / N, rtol=0, atol=1e-15)


@pytest.mark.parametrize("N", [2, 3, 6, 20])
def test_complete_digraph_uniform(N):
    edges = [(u, v) for u in range(N) for v in range(N) if u != v]
    g = csc_from_edges(N, edges)
    x = oracle.pagerank_uniform(g, D, 30)
    np.testing.assert_allclose(x, 1.0 / N, rtol=0, atol=1e-15)


@pytest.mark.parametrize("N", [2, 3, 5, 40])
def test_in_star_fixed_point(N):
    # leaves -> hub 0; the hub is dangling.  x_hub = (1 + (N-1)d) / (N + (N-1)d)
    edges = [(i, 0) for i in range(1, N)]
    g = csc_from_edges(N, edges)
    x = oracle.pagerank_uniform(g, D, 250)
    hub = (1 + (N - 1) * D) / (N + (N - 1) * D)
    leaf = (1 - hub) / (N - 1)
    assert abs(x[0] - hub) < 1e-13
    np.testing.assert_allclose(x[1:], leaf, rtol=0, atol=1e-13)


def test_in_star_two_nodes_value():
    # N = 2, d = 0.85: 1.85 / 2.85 and 1 / 2.85
    g = csc_from_edges(2, [(1, 0)])
    x = oracle.pagerank_uniform(g, D, 250)
    assert abs(x[0] - 1.85 / 2.85) < 1e-14 and abs(x[1] - 1.0 / 2.85) < 1e-14
    assert abs(x[0] - 0.6491228070175439) < 1e-13


@pytest.mark.parametrize("N", [2, 3, 5, 40])
def test_out_star_fixed_point(N):
    # hub 0 -> leaves; the leaves are dangling.  x_hub = 1 / (N + d)
    edges = [(0, i) for i in range(1, N)]
    g = csc_from_edges(N, edges)
    x = oracle.pagerank_uniform(g, D, 250)
    assert abs(x[0] - 1.0 / (N + D)) < 1e-13
    np.testing.assert_allclose(x[1:], (N + D - 1) / ((N - 1) * (N + D)), rtol=0, atol=1e-13)


@pytest.mark.parametrize("N,s", [(5, 0), (7, 3), (30, 29)])
def test_ppr_cycle_closed_form(N, s):
    # x_v = (1 - d) d^j / (1 - d^N), j = forward distance from s to v
    edges = [(i, (i + 1) % N) for i in range(N)]
    g = csc_from_edges(N, edges)
    x, k = oracle.ppr(g, s, D, 400)
    j = (np.arange(N) - s) % N
    np.testing.assert_allclose(x, (1 - D) * D ** j / (1 - D ** N), rtol=0, atol=1e-14)


def test_ppr_dangling_mass_returns_to_seed():
    # 0 -> 1, 1 dangling, seed 0: x0 = (1-d) + d x1, x1 = d x0 -> x0 = (1-d)/(1-d^2)
    g = csc_from_edges(3, [(0, 1)])
    x, _ = oracle.ppr(g, 0, D, 400)
    assert abs(x[0] - (1 - D) / (1 - D * D)) < 1e-14
    assert abs(x[1] - D * (1 - D) / (1 - D * D)) < 1e-14
    assert x[2] == 0.0


# --------------------------------------------------------- dense solves --

def _random_small_graph(rng, n):
    m = int(rng.integers(0, 3 * n + 1))
    src, dst = random_coo(rng, n, m, p_loop=0.1, p_dup=0.1)
    _, _, _, edges = brute_csc(n, src, dst)
    return src, dst, edges


@pytest.mark.parametrize("seed", range(25))
def test_fixed_point_matches_dense_solve(seed):
    rng = np.random.default_rng(100 + seed)
    n = int(rng.integers(1, 65))
    src, dst, edges = _random_small_graph(rng, n)
    g = oracle.build_csc(n, src, dst)
    t = np.full(n, 1.0 / n)
    xs = dense_fixed_point(n, edges, t)
    x = oracle.pagerank_uniform(g, D, 250)
    assert np.abs(x - xs).sum() <= 1e-12
    # personalised, random seed
    s = int(rng.integers(0, n))
    e = np.zeros(n)
    e[s] = 1.0
    xs = dense_fixed_point(n, edges, e)
    xp, _ = oracle.ppr(g, s, D, 250)
    assert np.abs(xp - xs).sum() <= 1e-12
    # another damping
    xs = dense_fixed_point(n, edges, t, d=0.5)
    x = oracle.pagerank(g, d=0.5, iters=120)
    assert np.abs(x - xs).sum() <= 1e-12


@pytest.mark.parametrize("seed", range(15))
def test_finite_k_matches_dense_power_iteration(seed):
    rng = np.random.default_rng(300 + seed)
    n = int(rng.integers(1, 65))
    src, dst, edges = _random_small_graph(rng, n)
    g = oracle.build_csc(n, src, dst)
    t = np.full(n, 1.0 / n)
    for k in [1, 2, 5, 50]:
        x = oracle.pagerank_uniform(g, D, k)
        xd = dense_power(n, edges, t, t, k)
        assert np.abs(x - xd).sum() <= 1e-13


# ---------------------------------------------------------- invariants --

def test_mass_and_lower_bound_every_iterate():
    src, dst = gen.rmat_coo(2000, 16000, seed=5)
    g = oracle.build_csc(2000, src, dst)
    assert (g.outdeg == 0).any()  # dangling nodes present
    for k in range(0, 12):
        x = oracle.pagerank_uniform(g, D, k)
        assert abs(x.sum() - 1.0) <= 1e-12
        assert x.min() >= (1 - D) / 2000 - 1e-18


def test_geometric_convergence_bound():
    rng = np.random.default_rng(9)
    n = 60
    src, dst, edges = _random_small_graph(rng, n)
    g = oracle.build_csc(n, src, dst)
    xs = dense_fixed_point(n, edges, np.full(n, 1.0 / n))
    for k in range(1, 40):
        x = oracle.pagerank_uniform(g, D, k)
        assert np.abs(x - xs).sum() <= 2 * D ** k + 1e-14


@pytest.mark.parametrize("tol", [1e-3, 1e-6, 1e-9])
def test_tolerance_stop_rule_bounds_error(tol):
    rng = np.random.default_rng(21)
    n = 50
    src, dst, edges = _random_small_graph(rng, n)
    g = oracle.build_csc(n, src, dst)
    for s in [0, 7, 49]:
        e = np.zeros(n)
        e[s] = 1.0
        xs = dense_fixed_point(n, edges, e)
        x, k = oracle.ppr(g, s, D, 1000, tol)
        assert k < 1000
        assert np.abs(x - xs).sum() <= tol + 1e-13
        # and it stopped at the first step that met the rule
        _, resid, k2 = oracle.pagerank(g, D, 1000, t=e, tol=tol, with_resid=True)
        assert k2 == k and (D / (1 - D)) * resid[-1] <= tol
        assert all((D / (1 - D)) * r > tol for r in resid[:-1])


def test_per_step_residual_is_l1_change():
    src, dst = gen.rmat_coo(500, 3000, seed=3)
    g = oracle.build_csc(500, src, dst)
    prev = oracle.pagerank_uniform(g, D, 0)
    _, resid, k = oracle.pagerank(g, D, 6, with_resid=True)
    for i in range(6):
        cur = oracle.pagerank_uniform(g, D, i + 1)
        assert abs(np.abs(cur - prev).sum() - resid[i]) <= 1e-13  # summation order differs
        prev = cur


# ------------------------------------------ planted mistakes are caught --

def _mutant_pagerank(g, iters, mutation):
    """The oracle's update written out in Python with one deliberate slip,
    to show the pins above would catch it."""
    n = g.n
    x = np.full(n, 1.0 / n)
    t = np.full(n, 1.0 / n)
    for _ in range(iters):
        dang = x[g.outdeg == 0].sum()
        xn = np.empty(n)
        for v in range(n):
            srcs = g.row_idx[g.col_ptr[v]:g.col_ptr[v + 1]]
            pulled = sum(x[u] / g.outdeg[u] for u in srcs)
            if mutation == "drop_dangling":
                xn[v] = (1 - D) * t[v] + D * pulled
            elif mutation == "teleport_sign":
                xn[v] = (1 + D) * t[v] + D * (pulled + dang * t[v])
            elif mutation == "no_outdeg":
                xn[v] = (1 - D) * t[v] + D * (sum(x[u] for u in srcs) + dang * t[v])
            else:
                xn[v] = (1 - D) * t[v] + D * (pulled + dang * t[v])
        x = xn
    return x


@pytest.mark.parametrize("mutation", ["drop_dangling", "teleport_sign", "no_outdeg"])
def test_pins_catch_planted_mistakes(mutation):
    # out-star: dangling leaves and a hub of out-degree N - 1
    N = 6
    g = csc_from_edges(N, [(0, i) for i in range(1, N)])
    x = _mutant_pagerank(g, 250, mutation)
    ok_hub = abs(x[0] - 1.0 / (N + D)) < 1e-13
    ok_mass = abs(x.sum() - 1.0) <= 1e-12
    assert not (ok_hub and ok_mass)
    # and the unmutated transcription passes the same pins
    x = _mutant_pagerank(g, 250, "none")
    assert abs(x[0] - 1.0 / (N + D)) < 1e-13 and abs(x.sum() - 1.0) <= 1e-12


# ------------------------------------------- HITS and eigenvector centrality --
# Pins: closed forms of bipartite and star graphs, the principal
# eigenvectors of A^T A, A A^T and A^T from a dense eigen-decomposition,
# unit norms and supports, and the zero-vector rule.

def dense_adj(g):
    """A[u, v] = 1 for each edge u -> v, from the CSC."""
    A = np.zeros((g.n, g.n))
    for v in range(g.n):
        for u in g.row_idx[g.col_ptr[v]:g.col_ptr[v + 1]]:
            A[u, v] = 1.0
    return A


@pytest.mark.parametrize("p,q", [(1, 1), (2, 5), (7, 3)])
def test_hits_complete_bipartite_closed_form(p, q):
    # every source points to every sink: one step reaches the fixed point
    edges = [(u, p + v) for u in range(p) for v in range(q)]
    g = csc_from_edges(p + q, edges)
    for k in (1, 2, 30):
        hub, auth = oracle.hits(g, k)
        assert np.allclose(hub[:p], 1 / np.sqrt(p), atol=1e-15, rtol=0) and (hub[p:] == 0).all()
        assert np.allclose(auth[p:], 1 / np.sqrt(q), atol=1e-15, rtol=0) and (auth[:p] == 0).all()


@pytest.mark.parametrize("N", [2, 5, 40])
def test_hits_stars(N):
    out_star = csc_from_edges(N, [(0, i) for i in range(1, N)])
    hub, auth = oracle.hits(out_star, 5)
    assert abs(hub[0] - 1) < 1e-15 and (hub[1:] == 0).all()
    assert auth[0] == 0 and np.allclose(auth[1:], 1 / np.sqrt(N - 1), atol=1e-15, rtol=0)
    in_star = csc_from_edges(N, [(i, 0) for i in range(1, N)])
    hub, auth = oracle.hits(in_star, 5)
    assert abs(auth[0] - 1) < 1e-15 and (auth[1:] == 0).all()
    assert hub[0] == 0 and np.allclose(hub[1:], 1 / np.sqrt(N - 1), atol=1e-15, rtol=0)


def test_hits_zero_steps_and_no_edges():
    g = csc_from_edges(9, [(0, 1), (3, 2)])
    hub, auth = oracle.hits(g, 0)
    assert np.allclose(hub, 1 / 3) and np.allclose(auth, 1 / 3)
    hub, auth = oracle.hits(csc_from_edges(4, []), 3)
    assert (hub == 0).all() and (auth == 0).all()


def principal(M):
    """Principal eigenpair of a symmetric PSD matrix, vector made nonnegative."""
    w, V = np.linalg.eigh(M)
    v = V[:, -1]
    v = v if v.sum() >= 0 else -v
    return w, v


@pytest.mark.parametrize("seed", range(12))
def test_hits_matches_dense_principal_eigenvectors(seed):
    rng = np.random.default_rng(300 + seed)
    N = int(rng.integers(5, 40))
    src, dst = rng.integers(0, N, N * 6), rng.integers(0, N, N * 6)
    g = oracle.build_csc(N, src, dst)
    A = dense_adj(g)
    wa, va = principal(A.T @ A)
    wh, vh = principal(A @ A.T)
    if wa[-1] <= 0 or wa[-2] / wa[-1] > 0.9:  # need a spectral gap for 400 steps to settle
        pytest.skip("no spectral gap")
    hub, auth = oracle.hits(g, 400)
    assert np.abs(auth - va).max() < 1e-9
    assert np.abs(hub - vh).max() < 1e-9
    # unit norms, nonnegative, supported on nodes with in- / out-edges
    assert abs(np.linalg.norm(auth) - 1) < 1e-12 and abs(np.linalg.norm(hub) - 1) < 1e-12
    assert (auth >= 0).all() and (hub >= 0).all()
    assert (auth[A.sum(0) == 0] == 0).all() and (hub[A.sum(1) == 0] == 0).all()


def test_hits_finite_steps_match_dense_products():
    rng = np.random.default_rng(7)
    g = oracle.build_csc(30, rng.integers(0, 30, 150), rng.integers(0, 30, 150))
    A = dense_adj(g)
    h = np.full(30, 1 / np.sqrt(30))
    for _ in range(6):
        a = A.T @ h
        a /= np.linalg.norm(a)
        h = A @ a
        h /= np.linalg.norm(h)
    hub, auth = oracle.hits(g, 6)
    assert np.abs(hub - h).max() < 1e-14 and np.abs(auth - a).max() < 1e-14


@pytest.mark.parametrize("N", [3, 17])
def test_eigen_centrality_cycle_and_complete_uniform(N):
    cyc = csc_from_edges(N, [(i, (i + 1) % N) for i in range(N)])
    comp = csc_from_edges(N, [(u, v) for u in range(N) for v in range(N) if u != v])
    for g in (cyc, comp):
        for k in (1, 7, 50):
            assert np.allclose(oracle.eigen_centrality(g, k), 1 / np.sqrt(N), atol=1e-15, rtol=0)


def test_eigen_centrality_in_star_and_zero_rule():
    # leaves -> hub 0: one step puts everything on the hub; the hub points
    # nowhere, so the next product is 0 and stays 0
    g = csc_from_edges(6, [(i, 0) for i in range(1, 6)])
    x1 = oracle.eigen_centrality(g, 1)
    assert abs(x1[0] - 1) < 1e-15 and (x1[1:] == 0).all()
    assert (oracle.eigen_centrality(g, 2) == 0).all()


@pytest.mark.parametrize("seed", range(10))
def test_eigen_centrality_matches_perron_vector(seed):
    rng = np.random.default_rng(500 + seed)
    N = int(rng.integers(6, 40))
    g = oracle.build_csc(N, rng.integers(0, N, N * 8), rng.integers(0, N, N * 8))
    A = dense_adj(g)
    w, V = np.linalg.eig(A.T)
    order = np.argsort(-np.abs(w))
    lead, second = w[order[0]], w[order[1]]
    if abs(lead.imag) > 1e-12 or abs(second) / abs(lead) > 0.9:
        pytest.skip("no dominant real eigenvalue with a gap")
    v = np.real(V[:, order[0]])
    v = v / np.linalg.norm(v)
    v = v if v.sum() >= 0 else -v
    x = oracle.eigen_centrality(g, 600)
    assert np.abs(x - v).max() < 1e-9
    # and it is an eigenvector of A^T: A^T x = lambda x
    assert np.abs(A.T @ x - np.real(lead) * x).max() < 1e-8


def _mutant_hits(g, iters, mutation):
    """HITS written out with one deliberate slip."""
    A = dense_adj(g)
    h = np.full(g.n, 1 / np.sqrt(g.n))
    a = h.copy()
    for _ in range(iters):
        a = (A @ h) if mutation == "authority_from_out_edges" else (A.T @ h)
        a /= np.linalg.norm(a) or 1.0
        h = (A.T @ a) if mutation == "hub_from_in_edges" else (A @ a)
        if mutation != "no_hub_norm":
            h /= np.linalg.norm(h) or 1.0
    return h, a


@pytest.mark.parametrize("mutation", ["authority_from_out_edges", "hub_from_in_edges", "no_hub_norm"])
def test_hits_pins_catch_planted_mistakes(mutation):
    p, q = 2, 5
    g = csc_from_edges(p + q, [(u, p + v) for u in range(p) for v in range(q)])
    hub, auth = _mutant_hits(g, 3, mutation)
    ok = (np.allclose(hub[:p], 1 / np.sqrt(p)) and np.allclose(auth[p:], 1 / np.sqrt(q))
          and (hub[p:] == 0).all() and (auth[:p] == 0).all())
    assert not ok
    hub, auth = _mutant_hits(g, 3, "none")
    assert np.allclose(hub[:p], 1 / np.sqrt(p)) and np.allclose(auth[p:], 1 / np.sqrt(q))


# ------------------------------------------ weakly connected components --
# Pins: brute-force search over the undirected edge set, scipy's weak
# components (compared as partitions), closed forms and invariants.

def brute_wcc(n, src, dst):
    adj = [set() for _ in range(n)]
    for u, v in zip(src, dst):
        if u != v:
            adj[int(u)].add(int(v))
            adj[int(v)].add(int(u))
    lab = [-1] * n
    for s in range(n):
        if lab[s] >= 0:
            continue
        lab[s] = s
        stack = [s]
        while stack:
            u = stack.pop()
            for w in adj[u]:
                if lab[w] < 0:
                    lab[w] = s
                    stack.append(w)
    return np.array(lab, np.int32)


@pytest.mark.parametrize("seed", range(25))
def test_wcc_matches_brute_force_and_scipy(seed):
    import scipy.sparse
    import scipy.sparse.csgraph
    rng = np.random.default_rng(700 + seed)
    n = int(rng.integers(1, 300))
    m_raw = int(rng.integers(0, 2 * n))
    src, dst = random_coo(rng, n, m_raw)
    g = oracle.build_csc(n, src, dst)
    lab, k = oracle.wcc(g)
    ref = brute_wcc(n, src, dst)
    assert (lab == ref).all()
    A = scipy.sparse.csr_matrix((np.ones(len(src)), (src, dst)), shape=(n, n))
    k2, sl = scipy.sparse.csgraph.connected_components(A, directed=True, connection="weak")
    assert k == k2
    # the same partition: equal scipy labels <=> equal oracle labels
    pairs = set(zip(sl.tolist(), lab.tolist()))
    assert len(pairs) == k
    # invariants: a label is the smallest id of its component and labels itself
    assert (lab <= np.arange(n)).all() and (lab[lab] == lab).all()


def test_wcc_closed_forms():
    N = 50
    path = csc_from_edges(N, [(i + 1, i) if i % 2 else (i, i + 1) for i in range(N - 1)])
    lab, k = oracle.wcc(path)
    assert k == 1 and (lab == 0).all()
    lab, k = oracle.wcc(csc_from_edges(N, []))
    assert k == N and (lab == np.arange(N)).all()
    # two stars joined by nothing, hub ids larger than their leaves
    edges = [(10, i) for i in range(5)] + [(i, 30) for i in range(20, 25)]
    lab, k = oracle.wcc(csc_from_edges(40, edges))
    assert k == 40 - 5 - 5
    assert (lab[[0, 1, 2, 3, 4, 10]] == 0).all() and (lab[[20, 21, 22, 23, 24, 30]] == 20).all()
    assert lab[39] == 39
