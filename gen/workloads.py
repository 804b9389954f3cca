"""The synthetic workloads that stand in for the paper's benchmark graphs.

Each entry states sizes, seeds and the generator recipe only.  The paper's
LiveJournal (4.8M nodes, 69M edges; section 6, Table "exp_algs") and
Twitter2010 (42M nodes, 1.5B edges; section 6, Table "exp_parallel") graphs are
not available; R-MAT graphs of the same shape stand in for them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

from . import RMAT_ABC, scale_for, unit_draws

# Streams for workload-level draws (edge streams use the constants in rng.h).
STREAM_SIZES = 5
STREAM_ARRIVALS = 6


@dataclass(frozen=True)
class GraphSpec:
    name: str
    kind: str  # "er" (exact G(n, m)), "uniform" (raw draws) or "rmat"
    n: int
    m: int  # er: distinct edges wanted; uniform / rmat: raw COO length
    seed: int
    iters: int = 0
    abc: tuple = RMAT_ABC

    @property
    def scale(self) -> int:
        return scale_for(self.n)


# Directed G(10,000, 100,000), 50 iterations.
ER_10K = GraphSpec("er-10k-100k", "er", 10_000, 100_000, seed=1, iters=50)
# LiveJournal-shaped R-MAT: 4.8M ids, 69M raw edges, 100 iterations.
RMAT_LJ = GraphSpec("rmat-lj-4.8m-69m", "rmat", 4_800_000, 69_000_000, seed=2, iters=100)
# Twitter2010-scale R-MAT: scale 25, edge factor 32, 100 iterations.
RMAT_25 = GraphSpec("rmat-s25-ef32", "rmat", 1 << 25, 1 << 30, seed=3, iters=100)
# The same recipe at scale 23 (a quarter of the edges): the case the step
# kernels' DRAM traffic is measured on, larger than L2 and small enough for
# multi-pass counter captures.
RMAT_23 = GraphSpec("rmat-s23-ef32", "rmat", 1 << 23, 1 << 28, seed=3, iters=100)


def batched_specs(num_graphs: int = 4096, n_lo: float = 1e3, n_hi: float = 2e5,
                  deg_lo: float = 4.0, deg_hi: float = 32.0, base_seed: int = 1000):
    """Graph g: n log-uniform on [n_lo, n_hi], mean out-degree uniform on
    [deg_lo, deg_hi], m_raw = round(n * deg), R-MAT with seed base_seed + g."""
    out = []
    for g in range(num_graphs):
        u = unit_draws(base_seed + g, STREAM_SIZES, 2)
        n = int(round(math.exp(math.log(n_lo) + u[0] * (math.log(n_hi) - math.log(n_lo)))))
        deg = deg_lo + u[1] * (deg_hi - deg_lo)
        out.append(GraphSpec(f"batch-{g}", "rmat", n, int(round(n * deg)), seed=base_seed + g, iters=50))
    return out


def batched_seed_base(g: int) -> int:
    """Seed of graph g's personalised-PageRank seed nodes."""
    return 2_000_000 + g


def serving_pool_specs(num_graphs: int = 256, base_seed: int = 5000, scale_lo: int = 14,
                       scale_span: int = 9, edge_factor: int = 16):
    """Pool graph j: R-MAT scale scale_lo + (j mod scale_span), n = 2^scale,
    m_raw = edge_factor * n, seed base_seed + j."""
    out = []
    for j in range(num_graphs):
        s = scale_lo + (j % scale_span)
        out.append(GraphSpec(f"pool-{j}", "rmat", 1 << s, edge_factor << s, seed=base_seed + j))
    return out


@dataclass(frozen=True)
class Request:
    t_arrive: float  # seconds from the start of the trace
    graph: int
    seeds: np.ndarray
    damping: float
    tol: float
    bf16: bool


def serving_trace(pool_n, rate: float = 2000.0, duration: float = 65.0, seed: int = 7,
                  max_seeds: int = 64):
    """Poisson arrivals at `rate` per second.  Each request: graph uniform
    over the pool, 1..max_seeds seeds uniform, seed nodes uniform over the
    graph, damping uniform on [0.80, 0.90], tol 1e-6 or 1e-3 with
    probability 1/2, BF16 state with probability 1/2 when tol is 1e-3."""
    reqs = []
    t = 0.0
    i = 0
    while True:
        u = unit_draws(seed * 1_000_003 + i, STREAM_ARRIVALS, 8)
        t += -math.log1p(-u[0]) / rate
        if t >= duration:
            break
        g = min(int(u[1] * len(pool_n)), len(pool_n) - 1)
        k = 1 + min(int(u[2] * max_seeds), max_seeds - 1)
        n = pool_n[g]
        su = unit_draws(seed * 1_000_003 + i, STREAM_ARRIVALS + 1, k)
        seeds = np.minimum((su * n).astype(np.int64), n - 1).astype(np.int32)
        damping = 0.80 + 0.10 * u[3]
        tol = 1e-6 if u[4] < 0.5 else 1e-3
        bf16 = bool(tol == 1e-3 and u[5] < 0.5)
        reqs.append(Request(t, g, seeds, damping, tol, bf16))
        i += 1
    return reqs
