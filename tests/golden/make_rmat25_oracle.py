"""Writes the FP64 oracle's PageRank of the R-MAT scale-25 workload.

Run from the repository root (about 10 GB of host memory per 2^29 raw edges,
half an hour of one core at scale 25):

    python tests/golden/make_rmat25_oracle.py [--scale 25]

The input is the seeded R-MAT stream of the workload (R-MAT scale 25, edge
factor 32, seed 3: 2^25 ids, 2^30 raw edges); every number written is
computed by the CPU oracle alone (``oracle.build_csc`` then 100 steps of
``oracle.pagerank``), never by the CUDA path.  Two outputs:

  tests/golden/big/<workload>_pagerank<iters>.f64   the whole FP64 vector in
      caller ids (2^25 doubles, 256 MiB; kept out of git: ``big/`` is ignored)
  tests/golden/<workload>_pagerank<iters>.json      committed: the vector
      file's sha256, the CSC's sizes and hashes, the oracle's last L1 change,
      the sum of x, and x at 2,048 sampled nodes (sample seed 11) plus the
      64 largest entries, so that a check can run where the big file is absent.

The paper's benchmark this stands in for is per-iteration PageRank on
Twitter2010 (section 6, Table "exp_parallel").
"""
import argparse
import hashlib
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import gen  # noqa: E402
import oracle  # noqa: E402
from gen import workloads  # noqa: E402

N_SAMPLES = 2048
SAMPLE_SEED = 11
N_TOP = 64


def sha_bytes(b: bytes) -> str:
    return hashlib.sha256(b).hexdigest()


def sample_nodes(n: int) -> np.ndarray:
    """N_SAMPLES distinct node ids, ascending, from the seeded generator."""
    out = np.unique(gen.seed_nodes(n, 4 * N_SAMPLES, SAMPLE_SEED))
    return np.sort(out[:N_SAMPLES]).astype(np.int64)


def paths(spec, scale_tag: str):
    base = f"{spec.name}{scale_tag}_pagerank{spec.iters}"
    return (os.path.join(HERE, "big", base + ".f64"), os.path.join(HERE, base + ".json"))


def spec_for(scale: int):
    s = workloads.RMAT_25
    if scale == 25:
        return s, ""
    return workloads.GraphSpec(s.name, "rmat", 1 << scale, 32 << scale, seed=s.seed, iters=s.iters), f"-s{scale}"


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--scale", type=int, default=25, help="R-MAT scale (25 is the workload; smaller for a dry run)")
    a = ap.parse_args()
    spec, tag = spec_for(a.scale)
    big, js = paths(spec, tag)
    os.makedirs(os.path.dirname(big), exist_ok=True)
    t0 = time.time()
    src, dst = gen.rmat_coo(spec.n, spec.m, spec.seed)
    print(f"generated {len(src)} raw edges in {time.time() - t0:.1f} s", flush=True)
    t1 = time.time()
    g = oracle.build_csc(spec.n, src, dst)
    del src, dst
    print(f"oracle build: m = {g.m} in {time.time() - t1:.1f} s", flush=True)
    t2 = time.time()
    x, resid, k = oracle.pagerank(g, oracle.DAMPING, spec.iters, with_resid=True)
    print(f"oracle PageRank: {k} steps in {time.time() - t2:.1f} s", flush=True)
    raw = np.ascontiguousarray(x, np.float64).tobytes()
    with open(big, "wb") as f:
        f.write(raw)
    nodes = sample_nodes(spec.n)
    top = np.argsort(-x, kind="stable")[:N_TOP]
    out = {
        "workload": spec.name,
        "generator": {"kind": "rmat", "n": spec.n, "m_raw": spec.m, "seed": spec.seed, "abc": list(spec.abc)},
        "n": spec.n,
        "m": int(g.m),
        "dangling": int((g.outdeg == 0).sum()),
        "sha256_col_ptr": sha_bytes(np.ascontiguousarray(g.col_ptr, np.int32).tobytes()),
        "sha256_outdeg": sha_bytes(np.ascontiguousarray(g.outdeg, np.int32).tobytes()),
        "damping": oracle.DAMPING,
        "iters": spec.iters,
        "final_l1_change": float(resid[-1]),
        "sum_x": float(x.sum()),
        "vector_file": os.path.relpath(big, os.path.dirname(os.path.dirname(HERE))),
        "vector_sha256": sha_bytes(raw),
        "vector_dtype": "float64, little-endian, caller ids",
        "sample_seed": SAMPLE_SEED,
        "sample_nodes": [int(v) for v in nodes],
        "sample_x": [float(x[v]) for v in nodes],
        "top_nodes": [int(v) for v in top],
        "top_x": [float(x[v]) for v in top],
        "oracle_seconds": {"build": round(t2 - t1, 1), "pagerank": round(time.time() - t2, 1)},
    }
    with open(js, "w") as f:
        json.dump(out, f, indent=0)
        f.write("\n")
    print(f"wrote {big} and {js}", flush=True)


if __name__ == "__main__":
    main()
