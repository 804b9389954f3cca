"""Writes the stored expected values under tests/golden/ from the oracle alone.

Run from the repository root:  python tests/golden/make_golden.py
Inputs come from the seeded generators; every number written here is computed
by the CPU oracle (never by the CUDA path).
"""
import hashlib
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import gen  # noqa: E402
import oracle  # noqa: E402
from gen import workloads  # noqa: E402


def sha(a):
    return hashlib.sha256(np.ascontiguousarray(a, np.int32).tobytes()).hexdigest()


def main():
    spec = workloads.ER_10K
    src, dst = gen.er_gnm(spec.n, spec.m, spec.seed)
    g = oracle.build_csc(spec.n, src, dst)
    x, resid, k = oracle.pagerank(g, oracle.DAMPING, spec.iters, with_resid=True)
    top = np.argsort(-x, kind="stable")[:20]
    out = {
        "workload": spec.name,
        "n": spec.n,
        "m_raw": int(len(src)),
        "m": g.m,
        "dangling": int((g.outdeg == 0).sum()),
        "sha256_col_ptr": sha(g.col_ptr),
        "sha256_row_idx": sha(g.row_idx),
        "sha256_outdeg": sha(g.outdeg),
        "damping": oracle.DAMPING,
        "iters": spec.iters,
        "final_l1_change": float(resid[-1]),
        "top20_nodes": [int(v) for v in top],
        "top20_x": [float(x[v]) for v in top],
    }
    with open(os.path.join(HERE, "er10k_pagerank50.json"), "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
