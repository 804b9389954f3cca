"""CPU models of the index logic of three CUDA kernels (no GPU).

Each model replays, lane by lane, how a kernel walks its data: which edge or
walk a lane takes and what it derives from it.  They check, on small and
awkward shapes, the properties the kernels rely on: every edge visited once
with its own row (the edge-chunk helper of the key kernels), every walk run
once (the warp pools of the walk kernel), and the union-find scheme of WCC
giving the components the oracle gives.  They do not exercise the CUDA code;
the GPU tests do.
"""
import numpy as np
import pytest

import oracle

# ---------------------------------------------- for_each_edge_with_row ----


def edge_rows_model(col_ptr, nwarps, chunk=4096):
    """Every (edge, row) the helper hands to its callback."""
    n = len(col_ptr) - 1
    m = int(col_ptr[n])
    seen = {}
    for w in range(nwarps):
        cb = w * chunk
        while cb < m:
            ce = min(cb + chunk, m)
            p, hi = 0, n  # binary search: col_ptr[p] <= cb < col_ptr[hi]
            while hi - p > 1:
                mid = p + (hi - p) // 2
                if col_ptr[mid] <= cb:
                    p = mid
                else:
                    hi = mid
            for e0 in range(cb, ce, 32):
                rows = [-1] * 32
                while True:
                    start = [int(col_ptr[min(p + lane, n)]) for lane in range(32)]
                    wend = int(col_ptr[min(p + 32, n)])
                    for lane in range(32):
                        e = e0 + lane
                        q = 0
                        for step in (16, 8, 4, 2, 1):
                            if start[q + step] <= e:
                                q += step
                        if e < ce and rows[lane] < 0 and e < wend:
                            rows[lane] = p + q
                    if not any(e0 + lane < ce and rows[lane] < 0 for lane in range(32)):
                        break
                    p += 32
                for lane in range(32):
                    if e0 + lane < ce:
                        assert e0 + lane not in seen
                        seen[e0 + lane] = rows[lane]
                if rows[31] >= 0:
                    p = rows[31]
            cb += nwarps * chunk
    return seen


@pytest.mark.parametrize("seed", range(12))
def test_edge_chunks_visit_every_edge_with_its_row(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 300))
    deg = rng.integers(0, 4, n) * rng.integers(0, 2, n)
    if seed % 3 == 0:
        deg[rng.integers(0, n)] = int(rng.integers(3000, 9000))  # a hub row longer than a chunk
    if seed % 4 == 1:
        deg[:] = 0
        deg[-1] = 70  # a long run of empty rows first
    col_ptr = np.concatenate([[0], np.cumsum(deg)])
    seen = edge_rows_model(col_ptr, nwarps=int(rng.integers(1, 4)), chunk=int(rng.choice([64, 4096])))
    assert len(seen) == col_ptr[-1]
    for e, r in seen.items():
        assert col_ptr[r] <= e < col_ptr[r + 1]


# ------------------------------------------------- walk kernel pools ------


def walk_pool_model(total, per_warp, lengths):
    """Walk indices each lane runs, and in which order, under the warp's
    refill rule; lengths[idx] = steps of walk idx."""
    warps = (total + per_warp - 1) // per_warp
    done = []
    for wp in range(warps):
        w0, w1 = wp * per_warp, min(wp * per_warp + per_warp, total)
        nxt = w0 + 32
        idx = [w0 + lane if w0 + lane < w1 else -1 for lane in range(32)]
        left = [lengths[i] if i >= 0 else 0 for i in idx]
        guard = 0
        while any(i >= 0 for i in idx):
            guard += 1
            assert guard < 10 * per_warp * (max(lengths) + 2)
            finished = [lane for lane in range(32) if idx[lane] >= 0 and left[lane] == 0]
            for lane in range(32):
                if idx[lane] >= 0 and left[lane] > 0:
                    left[lane] -= 1
            if finished:
                for rank, lane in enumerate(finished):  # lanes in ascending order, as popc(mask & lt)
                    done.append(idx[lane])
                    q = nxt + rank
                    idx[lane] = q if q < w1 else -1
                    left[lane] = lengths[q] if q < w1 else 0
                nxt += len(finished)
    return done


@pytest.mark.parametrize("total,per_warp", [(1, 64), (31, 64), (64, 64), (65, 64), (1000, 64), (5000, 432),
                                            (33 * 64 + 5, 64)])
def test_walk_pools_run_every_walk_once(total, per_warp):
    rng = np.random.default_rng(total)
    lengths = rng.geometric(0.15, total) - 1  # steps before the stop draw succeeds
    done = walk_pool_model(total, per_warp, lengths)
    assert sorted(done) == list(range(total))


def test_walk_pool_size_rule():
    # about two resident waves of warps, pools of 64 .. 4096 walks
    sms = 152
    for total in (1, 1000, 8_388_608, 2_000_000_000):
        per = max(64, min(4096, total // (2 * sms * 64)))
        warps = (total + per - 1) // per
        assert 64 <= per <= 4096 and warps * per >= total
        assert (warps * 32 + 255) // 256 < 2 ** 31


# ------------------------------------------------------ WCC union-find ----


def wcc_model(n, col_ptr, row_idx, rng, skip_rows_outside=False):
    """Sampled links, the giant root c ranked lowest, one pass that links
    only edges with an endpoint outside c (taken in a random order, as the
    GPU's threads may), then labels = min caller id per tree."""
    parent = list(range(n))

    def root(x):
        while parent[x] != x:
            x = parent[x]
        return x

    def above(a, b, c):
        return b == c or (a != c and a > b)

    def link(u, v, c):
        a, b = root(u), root(v)
        while a != b:
            hi, lo = (a, b) if above(a, b, c) else (b, a)
            if parent[hi] == hi:  # the compare-and-swap succeeds
                parent[hi] = lo
                return
            a, b = root(hi), root(lo)

    for v in range(n):
        for e in range(col_ptr[v], min(col_ptr[v] + 2, col_ptr[v + 1])):
            link(int(row_idx[e]), v, -1)
    parent[:] = [root(v) for v in range(n)]
    k = min(1024, n)
    stride = max(1, n // k) | 1  # odd: spreads over [0, n)
    sample = [parent[(i * stride) % n] for i in range(k)]
    vals, counts = np.unique(sample, return_counts=True)
    c = int(vals[np.argmax(counts)])
    inc = [parent[x] == c for x in range(n)]
    edges = [(int(row_idx[e]), v) for v in range(n) for e in range(col_ptr[v], col_ptr[v + 1])]
    todo = [(u, v) for (u, v) in edges if not inc[u]]
    if not skip_rows_outside:  # the pass over rows outside c
        todo += [(u, v) for (u, v) in edges if inc[u] and not inc[v]]
    rng.shuffle(todo)
    for u, v in todo:
        link(u, v, c)
    assert parent[c] == c  # c is never hooked under another root
    roots = [root(v) for v in range(n)]
    low = {}
    for v in range(n):
        low[roots[v]] = min(low.get(roots[v], v), v)
    return np.array([low[roots[v]] for v in range(n)])


@pytest.mark.parametrize("seed", range(15))
def test_wcc_scheme_matches_oracle(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 120))
    m = int(rng.integers(0, 3 * n))
    src = rng.integers(0, n, m).astype(np.int32)
    dst = rng.integers(0, n, m).astype(np.int32)
    if seed % 5 == 0:  # two equal cycles: the sampled mode may pick either
        h = max(1, n // 2)
        a = np.arange(h)
        src = np.concatenate([a, a + h]).astype(np.int32) % n
        dst = np.concatenate([(a + 1) % h, (a + 1) % h + h]).astype(np.int32) % n
    g = oracle.build_csc(n, src, dst)
    labels = wcc_model(n, g.col_ptr, g.row_idx, rng)
    ref, _ = oracle.wcc(g)
    assert (labels == ref).all()


def test_wcc_scheme_needs_the_rows_outside_the_giant():
    # node 2's first two in-neighbours (0 and 1) have no in-edges, so the
    # sampled links leave {0, 1, 2} outside the giant cycle 5..19; its only
    # tie to the giant is the edge 10 -> 2, whose source is inside c.  Without
    # the pass over rows outside c that edge is lost.
    n = 20
    cyc = np.arange(5, 20)
    src = np.concatenate([cyc, [0, 1, 10]]).astype(np.int32)
    dst = np.concatenate([np.roll(cyc, -1), [2, 2, 2]]).astype(np.int32)
    g = oracle.build_csc(n, src, dst)
    ref, k = oracle.wcc(g)
    assert k == 3 and ref[2] == 0 and ref[10] == 0       # {0,1,2,5..19}, {3}, {4}
    rng = np.random.default_rng(0)
    assert (wcc_model(n, g.col_ptr, g.row_idx, rng) == ref).all()
    assert not (wcc_model(n, g.col_ptr, g.row_idx, rng, skip_rows_outside=True) == ref).all()
