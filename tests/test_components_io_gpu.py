"""GPU weakly connected components against the oracle (bit-exact labels:
the smallest node id of each component), and binary save / load round trips
(bit-identical graphs, rejected malformed files)."""
import os

import numpy as np
import pytest

import gen
import oracle
import paper_1606_07550_gb300 as gpr

from gpu_util import random_coo_with_dups

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    import torch
    return torch


def gpu_wcc(torch, g):
    out = torch.empty(g.n, dtype=torch.int32, device="cuda")
    k = gpr.wcc(g, out)
    return out.cpu().numpy(), k


@pytest.mark.parametrize("n,m_raw,seed", [(1, 3, 0), (2, 1, 1), (300, 200, 2), (5000, 4000, 3), (5000, 20_000, 4),
                                          (200_003, 150_000, 5), (100_000, 2_000_000, 6)])
def test_wcc_random_graphs_bit_exact(torch, n, m_raw, seed):
    # sparse cases have many components, dense ones a giant component
    src, dst = random_coo_with_dups(np.random.default_rng(seed), n, m_raw)
    g = gpr.graph_build(src, dst, n)
    lab, k = gpu_wcc(torch, g)
    ref, kr = oracle.wcc(oracle.build_csc(n, src, dst))
    assert k == kr and (lab == ref).all()


def test_wcc_power_law_and_chains(torch):
    # R-MAT: long rows (chunked), a giant component and many isolated nodes
    n = 60_000
    src, dst = gen.rmat_coo(n, 500_000, seed=9)
    g = gpr.graph_build(src, dst, n)
    lab, k = gpu_wcc(torch, g)
    ref, kr = oracle.wcc(oracle.build_csc(n, src, dst))
    assert k == kr and (lab == ref).all()
    # a long path with alternating directions and shuffled ids: many rounds
    N = 50_000
    perm = np.random.default_rng(4).permutation(N).astype(np.int32)
    a, b = perm[:-1], perm[1:]
    flip = np.arange(N - 1) % 2 == 1
    s_ = np.where(flip, b, a)
    d_ = np.where(flip, a, b)
    g = gpr.graph_build(s_, d_, N)
    lab, k = gpu_wcc(torch, g)
    assert k == 1 and (lab == 0).all()
    host = np.empty(N, np.int32)
    assert gpr.wcc(g, host) == 1 and (host == 0).all()
    # no edges: every node its own component
    z = np.zeros(0, np.int32)
    lab, k = gpu_wcc(torch, gpr.graph_build(z, z, 77))
    assert k == 77 and (lab == np.arange(77)).all()


def test_wcc_giant_choice_and_ties(torch):
    # two equal cycles (the sampled mode may pick either), a hub whose long
    # in-row is cut into chunks, nodes reachable only along out-edges into the
    # giant component, and isolated nodes between them
    n = 30_000
    a = np.arange(0, 10_000, dtype=np.int32) * 2            # even ids 0..19998: one cycle
    b = a + 1                                               # odd ids: another
    src = [a, b, np.arange(20_000, 29_000, dtype=np.int32)]  # 20000.. point into the hub 5
    dst = [np.roll(a, 1), np.roll(b, 1), np.full(9_000, 5, np.int32)]
    src.append(np.array([29_500], np.int32))                 # 29500 -> 3 (only an out-edge)
    dst.append(np.array([3], np.int32))
    s_, d_ = np.concatenate(src), np.concatenate(dst)
    g = gpr.graph_build(s_, d_, n)
    lab, k = gpu_wcc(torch, g)
    ref, kr = oracle.wcc(oracle.build_csc(n, s_, d_))
    assert k == kr and (lab == ref).all()
    assert lab[29_500] == 1 and lab[25_000] == 1 and lab[0] == 0 and lab[29_999] == 29_999 and k == 1001


def test_wcc_edge_into_a_node_outside_the_giant(torch):
    # node 2's first two in-neighbours (0, 1) have no in-edges, so sampling
    # leaves {0, 1, 2} outside the giant cycle 5..19; the only tie is 10 -> 2,
    # an edge whose source is inside the giant: the rows-outside pass links it
    n = 20
    cyc = np.arange(5, 20)
    src = np.concatenate([cyc, [0, 1, 10]]).astype(np.int32)
    dst = np.concatenate([np.roll(cyc, -1), [2, 2, 2]]).astype(np.int32)
    g = gpr.graph_build(src, dst, n)
    lab, k = gpu_wcc(torch, g)
    ref, kr = oracle.wcc(oracle.build_csc(n, src, dst))
    assert k == kr == 3 and (lab == ref).all()


def test_save_load_round_trip(torch, tmp_path):
    n = 40_000
    src, dst = gen.rmat_coo(n, 700_000, seed=12)
    g = gpr.graph_build(src, dst, n)
    path = str(tmp_path / "g.bin")
    g.save(path)
    h = gpr.graph_load(path)
    a, b = g.export(), h.export()
    assert all((x == y).all() for x, y in zip(a, b))
    ia, ib = g.info(), h.info()
    assert (ia.n, ia.m, ia.m_raw, ia.n_dangling, ia.max_in_degree, ia.max_out_degree) == \
           (ib.n, ib.m, ib.m_raw, ib.n_dangling, ib.max_in_degree, ib.max_out_degree)
    # the same internal layout: identical bits from every computation
    xa = torch.empty(n, device="cuda")
    xb = torch.empty(n, device="cuda")
    gpr.pagerank(g, xa, iters=30)
    gpr.pagerank(h, xb, iters=30)
    assert (xa.cpu() == xb.cpu()).all()
    assert (gpu_wcc(torch, g)[0] == gpu_wcc(torch, h)[0]).all()
    # a graph with no edges round-trips too
    z = np.zeros(0, np.int32)
    e = gpr.graph_build(z, z, 5)
    e.save(path)
    assert gpr.graph_load(path).info().m == 0


def test_load_rejects_malformed_files(torch, tmp_path):
    n = 3000
    src, dst = gen.rmat_coo(n, 30_000, seed=13)
    g = gpr.graph_build(src, dst, n)
    path = str(tmp_path / "g.bin")
    g.save(path)
    raw = bytearray(open(path, "rb").read())
    m = g.info().m
    bad = str(tmp_path / "bad.bin")

    def expect(data, status):
        open(bad, "wb").write(bytes(data))
        with pytest.raises(gpr.GprError) as ei:
            gpr.graph_load(bad)
        assert ei.value.status == status

    expect(raw[:-4], gpr.EINVAL)                         # truncated
    expect(b"X" + raw[1:], gpr.EINVAL)                   # not our magic
    hdr, off_rows = 40, 40 + 4 * (n + 1)
    r = bytearray(raw)
    r[off_rows:off_rows + 4] = np.int32(n + 5).tobytes()  # a source id out of range
    expect(r, gpr.EINVAL)
    r = bytearray(raw)
    r[hdr + 4:hdr + 8] = np.int32(m + 1).tobytes()       # offsets not a CSC
    expect(r, gpr.EINVAL)
    r = bytearray(raw)
    off_perm = off_rows + 4 * m
    r[off_perm:off_perm + 4] = r[off_perm + 4:off_perm + 8]  # new2old not a permutation
    expect(r, gpr.EINVAL)
    with pytest.raises(gpr.GprError) as ei:
        gpr.graph_load(str(tmp_path / "missing.bin"))
    assert ei.value.status == gpr.ENOTFOUND
    assert os.path.exists(path) and gpr.graph_load(path).info().m == m
