"""The multi-rank path of bench.py on CPU, world size 2 over gloo (no GPU).

bench.py runs plain PageRank as independent replicas, one per GPU (that path
has no data-path collective), and shares the independent units of batched
and served personalised PageRank out by index (graph g on rank g % world).
What crosses ranks is host-side: a barrier around the timed region, the
maximum of the per-rank times, the sum of the per-rank work and the gathered
latency lists.  These tests run those helpers, and the reference arm under
torchrun, as two processes on this machine.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


RANK_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import bench
world, rank, local = bench.dist_setup()
bench.barrier(world)
mx = bench.max_over_ranks(world, 1.5 + rank)          # per-rank step times
sm = bench.sum_over_ranks(world, 10.0 * (rank + 1))   # per-rank work
bench.barrier(world)
print(json.dumps({{"rank": rank, "world": world, "local": local, "max": mx, "sum": sm}}), flush=True)
import torch.distributed as dist
dist.destroy_process_group()
"""


def test_replica_helpers_two_ranks():
    port = free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", RANK_SCRIPT.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for r, d in enumerate(outs):
        assert d["rank"] == r and d["world"] == 2 and d["local"] == r
        assert d["max"] == 2.5          # the slowest rank's time
        assert d["sum"] == 30.0         # all ranks' work


SHARD_SCRIPT = r"""
import json, os, sys
sys.path.insert(0, {root!r})
import bench
world, rank, local = bench.dist_setup()
mine = bench.shard_indices(4096, world, rank)
allg = bench.gather_lists(world, mine)
lat = [float(10 * rank + i) for i in range(3)]  # this rank's latencies
raw = {{"lat": lat, "unfinished": rank, "solves": 64 * len(mine), "offered": 100, "arrived": 5,
        "rejected": {{"busy": 1, "nomem": 0}}, "server": {{}}}}
merged = bench.merge_serve(world, raw, 2000.0, 2.0)
print(json.dumps({{"rank": rank, "mine_head": mine[:3], "n_mine": len(mine), "all_sorted": sorted(allg) == list(range(4096)),
                  "merged": merged}}), flush=True)
import torch.distributed as dist
dist.destroy_process_group()
"""


def test_sharded_units_and_merged_results_two_ranks():
    port = free_port()
    procs = []
    for r in range(2):
        env = dict(os.environ, RANK=str(r), LOCAL_RANK=str(r), WORLD_SIZE="2", MASTER_ADDR="127.0.0.1",
                   MASTER_PORT=str(port), CUDA_VISIBLE_DEVICES="")
        procs.append(subprocess.Popen([sys.executable, "-c", SHARD_SCRIPT.format(root=ROOT)], env=env,
                                      stdout=subprocess.PIPE, stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        o, e = p.communicate(timeout=120)
        assert p.returncode == 0, e
        outs.append(json.loads(o.strip().splitlines()[-1]))
    for r, d in enumerate(outs):
        # graph g on rank g % 2: disjoint halves that together cover every graph once
        assert d["mine_head"] == [r, r + 2, r + 4] and d["n_mine"] == 2048 and d["all_sorted"]
        m = d["merged"]
        assert m["solves_per_s"] == 64 * 4096 / 2.0      # every rank's solves over the window
        assert m["offered_solves_per_s"] == 200 / 2.0
        assert m["arrived_in_window"] == 10 and m["unfinished_after_drain"] == 1
        assert m["completed_in_window"] == 6             # both ranks' latencies
        assert m["p50_ms"] == 10.0 and m["p99_ms"] == 12.0
        assert m["rejected"] == {"busy": 2, "nomem": 0}


def test_single_rank_helpers_are_identities():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1, 3.25) == 3.25 and bench.sum_over_ranks(1, 7.0) == 7.0
    bench.barrier(1)
    assert bench.shard_indices(5, 1, 0) == [0, 1, 2, 3, 4] and bench.gather_lists(1, [3, 1]) == [3, 1]


@pytest.mark.timeout(600)
def test_reference_arm_under_torchrun_two_ranks():
    # rank 0 alone times the oracle and prints one JSON line; rank 1 exits 0
    port = free_port()
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", f"--master-port={port}", os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0", "--cpu-sample-scale", "12"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, r.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["cpu_baseline"]["kind"] == "oracle"
    # a workload the reference arm does not time says so and exits 0
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "wcc"],
                       cwd=ROOT, env=env, capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and json.loads(r.stdout.strip().splitlines()[-1])["unavailable"]
