"""The oracle reproduces its stored regression values (no GPU)."""
import hashlib
import json
import os

import numpy as np

import gen
import oracle
from gen import workloads

GOLD = os.path.join(os.path.dirname(__file__), "golden", "er10k_pagerank50.json")


def test_er10k_golden():
    ref = json.load(open(GOLD))
    spec = workloads.ER_10K
    src, dst = gen.er_gnm(spec.n, spec.m, spec.seed)
    assert len(src) == ref["m_raw"]
    g = oracle.build_csc(spec.n, src, dst)
    assert g.m == ref["m"] == spec.m
    for name, arr in [("col_ptr", g.col_ptr), ("row_idx", g.row_idx), ("outdeg", g.outdeg)]:
        assert hashlib.sha256(np.ascontiguousarray(arr, np.int32).tobytes()).hexdigest() == ref["sha256_" + name]
    x = oracle.pagerank_uniform(g, ref["damping"], ref["iters"])
    np.testing.assert_allclose(x[ref["top20_nodes"]], ref["top20_x"], rtol=1e-14, atol=0)
