#!/usr/bin/env python
"""Benchmark: COO -> CSC graph build + PageRank power iteration on one GB300.

One step = the whole hot path once: graph_build from a raw COO edge stream
already resident in HBM (pack, radix sort, dedupe, CSC offsets, out-degrees,
execution layout) followed by `iters` PageRank steps (pull SpMV, fused
teleport / dangling / residual step, FP64 reductions) and the write-back of
the rank vector.  Default workload: the Twitter2010-scale stand-in, R-MAT
scale 25 with edge factor 32 (33.5M ids, 2^30 raw edges), 100 iterations.

value = PageRank GTEPS over the whole step = m * iters / (build + iterate
time), m the deduplicated edge count.  The JSON line also carries the
iteration-only rate, the build time, an end-to-end figure through the C-ABI
with host buffers, a roofline object for the PageRank iteration and the CPU
oracle timed on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gpr|reference]
Under torchrun (N > 1) each rank runs an independent replica on its own GPU
(the plain PageRank path is not sharded); value sums all ranks' edges over
the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FALLBACK_HBM_GBS = 6800.0
DAMPING = 0.85


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gpr", "reference"], default="gpr")
    ap.add_argument("--workload", choices=["rmat25", "rmat23", "rmat-lj", "er10k", "batched", "serve", "hits", "wcc", "dynamic",
                                           "target"],
                    default="rmat25")
    ap.add_argument("--graphs", type=int, default=4096, help="batched: number of graphs")
    ap.add_argument("--dtypes", default="fp32,bf16,fp16", help="batched: contribution storage types")
    ap.add_argument("--serve-seconds", type=float, default=60.0)
    ap.add_argument("--serve-warmup", type=float, default=5.0)
    ap.add_argument("--serve-rate", type=float, default=2000.0)
    ap.add_argument("--pool", type=int, default=256)
    ap.add_argument("--stable-rates", default="", help="serve: lower request rates to find the max stable load")
    ap.add_argument("--stable-seconds", type=float, default=20.0)
    ap.add_argument("--e2e-steps", type=int, default=3)
    ap.add_argument("--spmv", choices=["auto", "pull", "blocked"], default="auto",
                    help="schedule of the PageRank step (auto: the library's choice)")
    ap.add_argument("--target-sources", type=int, default=1024, help="target: sources per query")
    ap.add_argument("--target-walks", type=int, default=8192, help="target: walks per source")
    ap.add_argument("--target-rmax", type=float, default=1e-5, help="target: reverse-push threshold")
    ap.add_argument("--target-scale", "--scale", type=int, default=25,
                    help="target, wcc: R-MAT scale (edge factor 32)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-scale", type=int, default=19)
    return ap.parse_args()


def rmat_spec(scale):
    """R-MAT, edge factor 32, seed 3: the scale-25 benchmark graph or a smaller one of the same recipe."""
    if scale == 25:
        return workload("rmat25")
    from gen.workloads import GraphSpec
    return GraphSpec(f"rmat-s{scale}-ef32", "rmat", 1 << scale, 1 << (scale + 5), seed=3)


def workload(name):
    from gen import workloads
    return {"rmat25": workloads.RMAT_25, "rmat23": workloads.RMAT_23, "rmat-lj": workloads.RMAT_LJ,
            "er10k": workloads.ER_10K}[name]


# sources of the kernels a recorded DRAM-traffic figure depends on (the
# graph layout and the PageRank step)
TRAFFIC_SOURCES = ("blocked_kernels.cuh", "pr_step.cuh")  # the measured kernels and the layout kernels


def src_hash():
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1606_07550_gb300", "csrc")
    for f in TRAFFIC_SOURCES:
        h.update(open(os.path.join(csrc, f), "rb").read())
    return h.hexdigest()[:16]


def measured_peak():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        for k in ("hbm_gbs", "hbm_GBs", "hbm_copy_gbs"):
            if k in d:
                return float(d[k]), "measured"
    except Exception:
        pass
    return FALLBACK_HBM_GBS, "fallback"


def recorded_traffic(wl_name):
    """DRAM bytes per PageRank iteration from a committed ncu summary, or None
    if the kernels changed since it was taken."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
        e = d.get(wl_name)
        if e and e.get("src_hash") == src_hash():
            return e
    except Exception:
        pass
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.f = None

    def __enter__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id is not None:
            cmd += ["-i", str(self.gpu_id)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        try:
            lines = open(self.f.name).read().strip().splitlines()
            os.unlink(self.f.name)
        except Exception:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(scale, iters, seed=3):
    """The CPU oracle as it stands (single-threaded FP64 C), on a bounded
    sample of the same workload recipe: R-MAT scale `scale`, edge factor 32,
    build + `iters` iterations.  Returns (GTEPS, seconds, m, description)."""
    import gen
    import oracle
    n = 1 << scale
    src, dst = gen.rmat_coo(n, 32 * n, seed=seed)
    t0 = time.perf_counter()
    g = oracle.build_csc(n, src, dst)
    oracle.pagerank_uniform(g, DAMPING, iters)
    dt = time.perf_counter() - t0
    desc = (f"R-MAT scale {scale}, edge factor 32 ({n} ids, {32 * n} raw edges, m={g.m}), same generator "
            f"recipe; build + {iters} iterations, single-threaded FP64 oracle")
    return g.m * iters / dt / 1e9, dt, g.m, desc


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("gloo", rank=rank, world_size=world)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, v):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def shard_indices(count, world, rank):
    """The independent units (graphs of the batch, graphs of the serving
    pool) this rank owns: index % world == rank."""
    return [i for i in range(count) if i % world == rank]


def gather_lists(world, items):
    """Every rank's list, concatenated in rank order (gloo object gather)."""
    if world == 1:
        return list(items)
    import torch.distributed as dist
    out = [None] * world
    dist.all_gather_object(out, list(items))
    return [x for part in out for x in part]


def gpu_index_of(local):
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    return vis.split(",")[local] if vis else str(local)


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle, as it stands, on the host cores."""
    if rank != 0:
        return
    if args.workload not in ("rmat25", "rmat23", "rmat-lj", "er10k"):
        print(json.dumps({"impl": "reference", "unavailable": "the reference arm times the oracle on the PageRank "
                                                             "workloads only (rmat25, rmat23, rmat-lj, er10k)"}), flush=True)
        return
    spec = workload(args.workload)
    scale = min(args.cpu_sample_scale - 1, spec.scale)
    for _ in range(args.warmup):
        cpu_baseline(scale, spec.iters)
    vals, secs = [], 0.0
    desc = ""
    for _ in range(args.steps):
        v, dt, m, desc = cpu_baseline(scale, spec.iters)
        vals.append(v)
        secs += dt
    value = statistics.median(vals)
    line = {
        "impl": "reference", "metric": "PageRank GTEPS", "value": value, "unit": "GTEPS", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": spec.name, "sample": desc, "iters": spec.iters},
        "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def headline_accuracy(spec, x):
    """L1 and max relative error of the ranks x (caller ids) against the FP64
    oracle: for the scale-25 workload, the oracle's stored x_100 (written by
    tests/golden/make_rmat25_oracle.py; the whole vector when its file is
    present, else its committed sample of 2,048 nodes, where the L1 relative
    to the sampled mass estimates the full L1); for the G(n, m) workload, an
    oracle run here.  None for the others."""
    import numpy as np
    x = np.asarray(x, np.float64)
    if spec.name == "rmat-s25-ef32":
        js = os.path.join(ROOT, "tests", "golden", f"{spec.name}_pagerank{spec.iters}.json")
        if not os.path.exists(js):
            return {"vs": "oracle summary not written", "l1": None, "max_rel": None}
        meta = json.load(open(js))
        path = os.path.join(ROOT, meta["vector_file"])
        if os.path.exists(path):
            raw = open(path, "rb").read()
            if hashlib.sha256(raw).hexdigest() == meta["vector_sha256"]:
                ref = np.frombuffer(raw, np.float64)
                nz = ref > 0
                return {"vs": "FP64 oracle x_100, whole vector", "l1": float(np.abs(x - ref).sum()),
                        "max_rel": float(np.max(np.abs(x[nz] - ref[nz]) / ref[nz]))}
        nodes = np.asarray(meta["sample_nodes"], np.int64)
        ref = np.asarray(meta["sample_x"], np.float64)
        got = x[nodes]
        return {"vs": f"FP64 oracle x_100 at {len(nodes)} sampled nodes (L1 relative to the sampled mass)",
                "l1": float(np.abs(got - ref).sum() / ref.sum()),
                "max_rel": float(np.max(np.abs(got - ref) / ref))}
    if spec.kind == "er":
        import gen
        import oracle
        src, dst = gen.er_gnm(spec.n, spec.m, spec.seed)
        ref = oracle.pagerank(oracle.build_csc(spec.n, src, dst), DAMPING, spec.iters)
        return {"vs": "FP64 oracle, whole vector", "l1": float(np.abs(x - ref).sum()),
                "max_rel": float(np.max(np.abs(x - ref) / ref))}
    return None


def make_coo_device(torch, spec):
    import gen
    if spec.kind == "rmat":
        s = torch.empty(spec.m, dtype=torch.int32, device="cuda")
        d = torch.empty(spec.m, dtype=torch.int32, device="cuda")
        perm = torch.from_numpy(gen.permutation(spec.n, spec.seed)).cuda()
        gen.rmat_coo_dev(spec.n, spec.m, spec.seed, s.data_ptr(), d.data_ptr(), perm.data_ptr(),
                         stream=torch.cuda.current_stream().cuda_stream, abc=spec.abc)
        torch.cuda.synchronize()
        return s, d
    src, dst = gen.er_gnm(spec.n, spec.m, spec.seed)
    return torch.from_numpy(src).cuda(), torch.from_numpy(dst).cuda()


def run_gpr(args, world, rank, local):
    import torch

    import paper_1606_07550_gb300 as gpr

    torch.cuda.set_device(local)
    spec = workload(args.workload)
    iters = spec.iters
    cpu = None
    if rank == 0 and world >= 1 and not args.no_cpu_baseline:
        # before any GPU work in this process
        cpu = cpu_baseline(args.cpu_sample_scale, iters)

    stream = torch.cuda.current_stream()
    src, dst = make_coo_device(torch, spec)
    m_raw = int(src.numel())  # the raw stream (G(n,m) draws until m distinct edges)
    out = torch.empty(spec.n, dtype=torch.float32, device="cuda")
    L = gpr.lib()

    stats = []

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        g = gpr.graph_build(src, dst, spec.n, stream=stream)
        if ev:
            ev[1].record(stream)
        st = gpr.pagerank(g, out, damping=DAMPING, iters=iters, dtype=gpr.FP32, stream=stream, stats=True,
                          spmv=args.spmv)
        if ev:
            ev[2].record(stream)
            stats.append(st)
        return g

    g = None
    for _ in range(args.warmup):
        g = step()
        inf = g.info()
        g.free()
    torch.cuda.synchronize()
    m = inf.m
    n = spec.n

    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[local] if os.environ.get(
        "CUDA_VISIBLE_DEVICES") else str(local)
    launches0 = L.gpr_kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(gpu_index) as clk:
        t0 = time.perf_counter()
        for k in range(args.steps):
            g = step(evs[k])
            g.free()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    barrier(world)
    launches = L.gpr_kernel_launches() - launches0
    t_build = sum(e[0].elapsed_time(e[1]) for e in evs) / args.steps
    t_iter = sum(e[1].elapsed_time(e[2]) for e in evs) / args.steps
    t_step = sum(e[0].elapsed_time(e[2]) for e in evs) / args.steps
    t_step_max = max_over_ranks(world, t_step)
    edges_all = sum_over_ranks(world, float(m))
    value = edges_all * iters / (t_step_max * 1e-3) / 1e9
    pr_gteps = m * iters / (t_iter * 1e-3) / 1e9

    # roofline of the PageRank iteration: modelled bytes 8m + 12n + 4 per
    # step over the device time of the iteration loop alone (the library's
    # CUDA events around its graph launch), without the per-graph setup
    # (workspace, blocked edge layout, graph capture) that t_iter includes
    t_loop = sum(st.t_iter_ms for st in stats) / len(stats)
    t_setup = sum(st.t_setup_ms for st in stats) / len(stats)
    schedule = {gpr.SPMV_PULL: "pull", gpr.SPMV_BLOCKED: "blocked"}.get(stats[-1].schedule, "?")
    bytes_per_iter = 8 * m + 12 * n + 4
    achieved = bytes_per_iter * iters / (t_loop * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    tr = recorded_traffic(spec.name)

    # end to end through the C-ABI with host buffers: H2D of the COO and D2H
    # of the ranks inside the timed region
    e2e = None
    if args.e2e_steps > 0:
        hs = torch.empty(m_raw, dtype=torch.int32, pin_memory=True)
        hd = torch.empty(m_raw, dtype=torch.int32, pin_memory=True)
        hs.copy_(src)
        hd.copy_(dst)
        hout = torch.empty(n, dtype=torch.float32, pin_memory=True)
        del src, dst
        torch.cuda.empty_cache()
        g = gpr.graph_build(hs, hd, n, stream=stream)
        gpr.pagerank(g, hout, damping=DAMPING, iters=iters, stream=stream, spmv=args.spmv)
        g.free()
        # the host link's pinned host-to-device rate (1 GiB of the source
        # buffer), probed after each step outside its time: on a machine
        # shared with other jobs it varies from copy to copy
        probe = torch.empty(1 << 28, dtype=torch.int32, device="cuda")

        def link_gbs():
            torch.cuda.synchronize()
            tp = time.perf_counter()
            probe.copy_(hs[:1 << 28], non_blocking=True)
            torch.cuda.synchronize()
            return (1 << 30) / (time.perf_counter() - tp) / 1e9

        barrier(world)
        each, link = [], [link_gbs()]
        for _ in range(args.e2e_steps):
            torch.cuda.synchronize()
            ts = time.perf_counter()
            g = gpr.graph_build(hs, hd, n, stream=stream)
            gpr.pagerank(g, hout, damping=DAMPING, iters=iters, stream=stream, spmv=args.spmv)
            g.free()
            torch.cuda.synchronize()
            each.append((time.perf_counter() - ts) * 1e3)
            link.append(link_gbs())
        del probe
        t_e2e = sum(each) / len(each) * 1e-3
        t_e2e = max_over_ranks(world, t_e2e)
        e2e = {"value": edges_all * iters / t_e2e / 1e9, "unit": "GTEPS",
               "h2d_bytes_per_step": 8 * m_raw, "d2h_bytes_per_step": 4 * n, "ms_per_step": t_e2e * 1e3,
               "ms_each": each, "host_link_gbs": link}

    if rank != 0:
        return
    accuracy = headline_accuracy(spec, out.cpu().numpy())
    line = {
        "metric": "PageRank GTEPS", "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_step_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {
            "workload": spec.name, "n": n, "m_raw": m_raw, "m": m, "iters": iters, "damping": DAMPING,
            "step": "graph_build (COO resident in HBM) + PageRank iterations + rank write-back",
            "value_counts": "m * iters / (build + iterate) per step",
            "l2": (f"inputs larger than L2 (COO {8 * m_raw / 2**30:.3g} GiB, CSC {4 * m / 2**30:.3g} GiB per replica)"
                   if m_raw > (1 << 25) else
                   "small graph: L2-resident (launch-bound)"),
            "parallelism": f"replicas x{world}",
        },
        "build_ms": t_build, "iterate_ms": t_iter, "pagerank_gteps": pr_gteps,
        "schedule": schedule, "iteration_loop_ms": t_loop, "pagerank_setup_host_ms": t_setup,
        "loop_gteps": m * iters / (t_loop * 1e-3) / 1e9,
        "build_edges_per_s": m_raw / (t_build * 1e-3),
        "roofline": {
            "kernel": ("PageRank iteration loop (bucketed pull SpMV + fused step + fold)" if schedule == "pull"
                       else "PageRank iteration loop (blocked expand + accumulate + fused step + fold)"),
            "timed": "CUDA events around the iteration graph launch, per call, averaged over the timed steps",
            "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "peak_source": peak_kind, "bytes_model": "8m + 12n + 4 per iteration",
            "traffic": (tr["dram_bytes_per_iter"] if tr and tr.get("schedule", "pull") == schedule else None),
        },
        "clocks": clk.summary(),
        "gpu_launches": launches,
        "wall_s_timed": wall,
        "accuracy": accuracy,
    }
    if e2e:
        line["e2e"] = e2e
    if cpu:
        line["cpu_baseline"] = {"value": cpu[0], "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": cpu[3],
                                "seconds": cpu[1]}
    print(json.dumps(line), flush=True)


def build_graph_dev(torch, gpr, spec, stream=None):
    """Device-generated R-MAT COO of `spec` -> graph (the COO is freed)."""
    import gen
    s = torch.empty(spec.m, dtype=torch.int32, device="cuda")
    d = torch.empty(spec.m, dtype=torch.int32, device="cuda")
    perm = torch.from_numpy(gen.permutation(spec.n, spec.seed)).cuda()
    gen.rmat_coo_dev(spec.n, spec.m, spec.seed, s.data_ptr(), d.data_ptr(), perm.data_ptr(),
                     stream=torch.cuda.current_stream().cuda_stream, abc=spec.abc)
    return gpr.graph_build(s, d, spec.n)


def ppr_bytes_per_step(n, m, dt_name, cols=64):
    """Modelled bytes of one personalised-PageRank step of a 64-column job:
    indices 4m, offsets 4(n+1), the state read and written per row and column
    (x: 8 B with FP32 and FP16 storage; with BF16 deltas the running and sent
    sums: 16 B), and the contributions written and gathered once per edge and
    column (s bytes each: 4 FP32, 2 FP16 / BF16)."""
    sz = 4 if dt_name == "fp32" else 2
    state = 16 if dt_name == "bf16" else 8
    return 4 * m + 4 * (n + 1) + cols * n * (state + sz) + cols * m * sz


def run_batched(args, world, rank, local):
    """Config: 4,096 R-MAT graphs (n log-uniform in [1e3, 2e5], mean out-degree
    uniform in [4, 32]), 64 personalised-PageRank seeds each, damping 0.85,
    50 steps, one persistent launch per storage type.  Under torchrun the
    graphs are shared out (graph g on rank g % world, no data-path
    collective); value = all ranks' solves over the slowest rank's time.
    Baselines on the same GPU: one solve per call (ppr_batch with one seed)
    and plain PageRank (pagerank, one vector) per solve, each timed on a
    sample and expressed in solves/s.  Accuracy: sampled columns against the
    FP64 oracle."""
    import numpy as np
    import torch

    import gen
    import oracle
    import paper_1606_07550_gb300 as gpr
    from gen import workloads

    torch.cuda.set_device(local)
    specs_all = workloads.batched_specs(args.graphs)
    mine = shard_indices(len(specs_all), world, rank)
    specs = [specs_all[g] for g in mine]
    t0 = time.perf_counter()
    graphs = [build_graph_dev(torch, gpr, sp) for sp in specs]
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    seeds = [gen.seed_nodes(sp.n, 64, workloads.batched_seed_base(g)) for g, sp in zip(mine, specs)]
    outs = [torch.empty((sp.n, 64), dtype=torch.float32, device="cuda") for sp in specs]
    reqs = [(g, s, 0.85, o) for g, s, o in zip(graphs, seeds, outs)]
    iters = 50
    n_solves_all = 64 * len(specs_all)
    refs = []  # (local graph, column, oracle x) on about every 256th graph of the batch
    for i in range(0, len(specs), max(1, 256 // world)):
        sp = specs[i]
        src, dst = gen.rmat_coo(sp.n, sp.m, seed=sp.seed)
        csc = oracle.build_csc(sp.n, src, dst)
        for k in (0, 21, 42, 63):
            refs.append((i, k, oracle.ppr(csc, int(seeds[i][k]), 0.85, iters)[0]))
    dts = {"fp32": gpr.FP32, "bf16": gpr.BF16, "fp16": gpr.FP16}
    res = {}
    stream = torch.cuda.current_stream()
    peak, peak_kind = measured_peak()
    launches0 = gpr.lib().gpr_kernel_launches()
    def timed_runs(dt):
        times = []
        for _ in range(args.steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            gpr.ppr_batch(reqs, max_iters=iters, dtype=dt)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        return statistics.median(times)

    for name in args.dtypes.split(","):
        dt = dts[name]
        # the autotuner: CTAs per cluster for each graph-size class
        tuned = gpr.ppr_tune(reqs, dtype=dt, trial_steps=8)
        for _ in range(max(1, args.warmup)):
            gpr.ppr_batch(reqs, max_iters=iters, dtype=dt)
        torch.cuda.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        with ClockSampler(gpu_index_of(local)) as clk:
            ms_rank = timed_runs(dt)
        barrier(world)
        ms = max_over_ranks(world, ms_rank)
        # the same batch with the fixed shape (8 CTAs per cluster for every class)
        os.environ["GPR_PPR_CLUSTER"] = "8"
        try:
            gpr.ppr_batch(reqs, max_iters=iters, dtype=dt)
            torch.cuda.synchronize()
            ms8 = max_over_ranks(world, timed_runs(dt))
        finally:
            os.environ.pop("GPR_PPR_CLUSTER", None)
        gpr.ppr_batch(reqs, max_iters=iters, dtype=dt)  # outputs of the tuned shapes for the accuracy check
        torch.cuda.synchronize()
        # accuracy on sampled graphs, 4 seeds each, against the FP64 oracle
        l1s, mrs = [], []
        for g, k, xr in refs:
            x = outs[g][:, k].cpu().numpy()
            l1s.append(float(np.abs(x - xr).sum()))
            nz = xr > 0
            mrs.append(float(np.max(np.abs(x[nz] - xr[nz]) / xr[nz])) if nz.any() else 0.0)
        l1s, mrs = gather_lists(world, l1s), gather_lists(world, mrs)
        bytes_rank = sum(ppr_bytes_per_step(sp.n, g.m, name) for sp, g in zip(specs, graphs)) * iters
        achieved = bytes_rank / (ms_rank * 1e-3) / 1e9
        res[name] = {"ms": ms, "solves_per_s": n_solves_all / (ms * 1e-3),
                     "tuner": {"classes": tuned, "ms_fixed_8_cta_clusters": ms8,
                               "speedup_vs_fixed_8_cta_clusters": ms8 / ms},
                     "l1_max": max(l1s),
                     "l1_mean": statistics.mean(l1s), "max_rel_err_max": max(mrs), "sampled_columns": len(l1s),
                     "clocks": clk.summary(),
                     "roofline": {"kernel": "ppr_kernel (one persistent cluster launch over every job)",
                                  "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                                  "frac": achieved / peak, "peak_source": peak_kind,
                                  "bytes_model": "per step and job: 4m + 4(n+1) + 64n(state + s) + 64ms, state 8 (x) or "
                                                 "16 (BF16 running and sent sums), s = stored bytes per contribution; "
                                                 "gathers counted once per edge and column (cache hits count as bytes)",
                                  "traffic": None}}
    launches = gpr.lib().gpr_kernel_launches() - launches0
    # baselines: one solve at a time, on a sample of (graph, seed) pairs
    sample = list(range(0, len(specs), max(1, len(specs) // 64)))
    one_out = [torch.empty((specs[g].n, 1), dtype=torch.float32, device="cuda") for g in sample]
    for i, g in enumerate(sample[:4]):
        gpr.ppr_batch([(graphs[g], seeds[g][:1], 0.85, one_out[i])], max_iters=iters)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, g in enumerate(sample):
        gpr.ppr_batch([(graphs[g], seeds[g][:1], 0.85, one_out[i])], max_iters=iters)
    torch.cuda.synchronize()
    one_ppr = sum_over_ranks(world, len(sample) / (time.perf_counter() - t0))
    pr_out = [torch.empty(specs[g].n, dtype=torch.float32, device="cuda") for g in sample]
    for i, g in enumerate(sample[:4]):
        gpr.pagerank(graphs[g], pr_out[i], iters=iters)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i, g in enumerate(sample):
        gpr.pagerank(graphs[g], pr_out[i], iters=iters)
    torch.cuda.synchronize()
    one_pr = sum_over_ranks(world, len(sample) / (time.perf_counter() - t0))
    sum_n = sum(sp.n for sp in specs_all)
    sum_m = int(sum_over_ranks(world, float(sum(g.m for g in graphs))))
    best = res.get("fp32") or next(iter(res.values()))
    line = {
        "metric": "PPR solves/s (batched)", "value": best["solves_per_s"], "unit": "solves/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batched-ppr-4096x64", "graphs": len(specs_all), "seeds_per_graph": 64,
                   "iters": iters, "damping": 0.85, "sum_n": sum_n, "sum_m": sum_m,
                   "sum_m_raw": sum(sp.m for sp in specs_all),
                   "step": "one ppr_batch call: every column of every graph (of this rank), one persistent launch",
                   "parallelism": f"graphs sharded over {world} rank(s), g % world",
                   "l2": "per-job state 0.3-77 MB; the batch's working set far above L2"},
        "by_dtype": res,
        "clocks": best["clocks"],
        "roofline": best["roofline"],
        "accuracy": {"l1_max": best["l1_max"], "max_rel": best["max_rel_err_max"], "vs": "FP64 oracle, sampled columns",
                     "columns": best["sampled_columns"]},
        "gpu_launches": launches,
        "one_at_a_time": {"ppr_single_seed_solves_per_s": one_ppr, "plain_pagerank_solves_per_s": one_pr,
                          "sample_pairs": len(sample),
                          "speedup_vs_single_seed": best["solves_per_s"] / one_ppr,
                          "speedup_vs_plain_pagerank": best["solves_per_s"] / one_pr},
        "setup_s": t_setup,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def serve_window(torch, gpr, graphs, specs, rate, warm, window, budget, seed=7, world=1, rank=0, bf16_all=True):
    """One run of the server on a Poisson trace at `rate` requests/s:
    `warm` seconds of warm-up, then a `window`-second measured window, then
    up to 30 s to drain.  `graphs` are this rank's pool graphs (pool graph j
    on rank j % world); the rank serves the requests of the trace that name
    them.  Returns (raw results of this rank, completed-request steps)."""
    import threading

    trace = [q for q in workloads_trace(specs, rate, warm + window, seed) if q.graph % world == rank]
    srv = gpr.Server(graphs, budget_bytes=budget, max_queue=1 << 20)
    info = {}     # ticket -> (arrival s, seeds)
    done = {}     # ticket -> (latency ms, status, steps, completion s)
    rejected = {"busy": 0, "nomem": 0}
    stop = threading.Event()
    tstart = time.perf_counter()

    def collector():
        while True:
            ts = srv.completed(timeout_us=20_000)
            now = time.perf_counter() - tstart
            for t in ts:
                r = srv.poll(t)
                done[t] = (r.latency_ms, r.status, r.iters_max, now)
                srv.release(t)
            if stop.is_set() and not ts:
                return

    th = threading.Thread(target=collector, daemon=True)
    th.start()
    i = 0
    tickets = []
    while i < len(trace):
        now = time.perf_counter() - tstart
        while i < len(trace) and trace[i].t_arrive <= now:
            q = trace[i]
            try:
                # 16-bit contributions (BF16 error-feedback deltas) for the
                # 1e-3 requests: all of them with bf16_all, else the trace's half
                use_bf16 = q.bf16 or (bf16_all and q.tol >= 1e-3)
                t = srv.submit(q.graph // world, q.seeds, damping=q.damping, tol=q.tol, max_iters=1000,
                               dtype=gpr.BF16 if use_bf16 else gpr.FP32)
                info[t] = (q.t_arrive, len(q.seeds))
                tickets.append((t, q))
            except gpr.GprError as e:
                rejected["busy" if e.status == gpr.EBUSY else "nomem"] += 1
            i += 1
        if i < len(trace):
            time.sleep(max(0.0, min(0.002, trace[i].t_arrive - (time.perf_counter() - tstart))))
    t_submitted = time.perf_counter() - tstart
    drain_limit = 30.0
    while len(done) < len(info) and time.perf_counter() - tstart < t_submitted + drain_limit:
        time.sleep(0.05)
    stop.set()
    th.join(timeout=10)
    st = srv.stats()
    srv.close()
    in_window = [t for t, (a, _) in info.items() if warm <= a < warm + window]
    lat = [done[t][0] for t in in_window if t in done and done[t][1] == gpr.OK]
    unfinished = sum(1 for t in in_window if t not in done)
    solves = sum(info[t][1] for t, d in done.items() if d[1] == gpr.OK and warm <= d[3] < warm + window)
    offered = sum(info[t][1] for t in in_window)
    raw = {"lat": lat, "unfinished": unfinished, "solves": solves, "offered": offered,
           "arrived": len(in_window), "rejected": rejected, "server": st}
    steps = [(q, done[t][2]) for t, q in tickets if t in done and done[t][1] == gpr.OK]
    return raw, steps


def merge_serve(world, raw, rate, window):
    """All ranks' results of one serving run: latency percentiles over every
    rank's requests, solves and offered work summed."""
    lat = sorted(gather_lists(world, raw["lat"]))

    def pct(a, q):
        return a[min(len(a) - 1, int(q * len(a)))] if a else None

    solves = sum_over_ranks(world, float(raw["solves"]))
    offered = sum_over_ranks(world, float(raw["offered"]))
    return {"rate_req_per_s": rate, "window_s": window, "solves_per_s": solves / window,
            "offered_solves_per_s": offered / window,
            "arrived_in_window": int(sum_over_ranks(world, float(raw["arrived"]))),
            "completed_in_window": len(lat),
            "unfinished_after_drain": int(sum_over_ranks(world, float(raw["unfinished"]))),
            "p50_ms": pct(lat, 0.50), "p99_ms": pct(lat, 0.99),
            "rejected": {k: int(sum_over_ranks(world, float(v))) for k, v in raw["rejected"].items()},
            "server_rank0": raw["server"]}


def workloads_trace(specs, rate, duration, seed):
    from gen import workloads
    return workloads.serving_trace([sp.n for sp in specs], rate=rate, duration=duration, seed=seed)


def run_serve(args, world, rank, local):
    """Config: a resident pool of 256 R-MAT graphs (scales 14-22, edge factor
    16); Poisson arrivals at 2,000 requests/s, each naming a graph, 1-64 seeds,
    damping in [0.80, 0.90] and tolerance 1e-6 (FP32 contributions) or 1e-3
    (BF16 contributions, sent as error-feedback deltas); admission under a
    40 GB device budget per GPU that includes the pool.  Under torchrun the
    pool is shared out (graph j on rank j % world, with the requests that name
    it; no data-path collective).  Reports submit-to-completion p50/p99 over
    the requests that arrived in the measured window, solves/s completed in
    the window (one seed = one solve), rejections and the backlog, with the
    clocks seen during the window.  The offered load is far above capacity,
    so the same measurement is repeated at the lower rates of --stable-rates:
    the highest rate whose window drains (no request left unfinished,
    completions keeping up with arrivals) is the maximum stable load, with its
    latencies.  Baseline on the same GPU: one-at-a-time plain PageRank, one
    call per solve with the step count the request needed, on a sample of the
    trace."""
    import numpy as np
    import torch

    import gen
    import oracle
    import paper_1606_07550_gb300 as gpr
    from gen import workloads

    torch.cuda.set_device(local)
    specs = workloads.serving_pool_specs(args.pool)
    mine = shard_indices(len(specs), world, rank)
    t0 = time.perf_counter()
    graphs = [build_graph_dev(torch, gpr, specs[j]) for j in mine]
    torch.cuda.synchronize()
    torch.cuda.empty_cache()
    t_setup = time.perf_counter() - t0
    budget = 40 << 30
    launches0 = gpr.lib().gpr_kernel_launches()
    barrier(world)
    with ClockSampler(gpu_index_of(local)) as clk:
        raw, steps = serve_window(torch, gpr, graphs, specs, args.serve_rate, args.serve_warmup,
                                  args.serve_seconds, budget, world=world, rank=rank)
    barrier(world)
    launches = gpr.lib().gpr_kernel_launches() - launches0
    main_run = merge_serve(world, raw, args.serve_rate, args.serve_seconds)
    sweep = []
    for r in [float(x) for x in args.stable_rates.split(",") if x]:
        with ClockSampler(gpu_index_of(local)) as sclk:
            rr, _ = serve_window(torch, gpr, graphs, specs, r, args.serve_warmup, args.stable_seconds, budget,
                                 world=world, rank=rank)
        res = merge_serve(world, rr, r, args.stable_seconds)
        res["stable"] = res["unfinished_after_drain"] == 0 and res["solves_per_s"] >= 0.9 * res[
            "offered_solves_per_s"]
        res["clocks"] = sclk.summary()
        sweep.append(res)
    stable = [r for r in sweep if r["stable"]]
    max_stable = max(stable, key=lambda r: r["rate_req_per_s"]) if stable else None

    # accuracy of served columns against the FP64 oracle's fixed point, on
    # this rank's smallest pool graphs: FP32 at tol 1e-6, BF16 at tol 1e-3
    acc = []
    srv = gpr.Server(graphs, budget_bytes=budget)
    small = [i for i, j in enumerate(mine) if specs[j].n <= (1 << 16)][:2]
    for li in small:
        sp = specs[mine[li]]
        src, dst = gen.rmat_coo(sp.n, sp.m, seed=sp.seed)
        csc = oracle.build_csc(sp.n, src, dst)
        sd = gen.seed_nodes(sp.n, 4, 900 + mine[li])
        for dt, tol in ((gpr.FP32, 1e-6), (gpr.BF16, 1e-3)):
            t = srv.submit(li, sd, damping=0.85, tol=tol, max_iters=1000, dtype=dt)
            r = None
            while r is None:
                r = srv.poll(t, 100_000)
            o = torch.empty(r.n * r.num_seeds, device="cuda")
            srv.fetch(t, o)
            x = o.cpu().numpy().reshape(r.n, r.num_seeds)
            srv.release(t)
            for k, s_ in enumerate(sd):
                xs, _ = oracle.ppr(csc, int(s_), 0.85, 400)
                acc.append((int(dt), tol, float(np.abs(x[:, k] - xs).sum())))
    srv.close()
    acc = gather_lists(world, acc)

    # baseline: one-at-a-time plain PageRank, one call per solve, each with
    # the step count the served request needed; sampled requests of the
    # trace, at most ~10 s of GPU time per rank
    sample = steps[:: max(1, len(steps) // 200)]
    # the library tunes the step's schedule once per graph shape: do that
    # before the timed baseline
    tuned = set()
    for g in graphs:
        key = (int(g.n).bit_length(), int(g.info().m).bit_length())
        if g.info().m >= (1 << 22) and key not in tuned:
            gpr.pagerank_tune(g)
            tuned.add(key)
    torch.cuda.synchronize()
    b0 = time.perf_counter()
    nb = 0
    for q, k in sample:
        o = torch.empty(graphs[q.graph // world].n, dtype=torch.float32, device="cuda")
        for _ in q.seeds:
            gpr.pagerank(graphs[q.graph // world], o, damping=q.damping, iters=max(1, k))
            nb += 1
        torch.cuda.synchronize()
        if time.perf_counter() - b0 > 10.0:
            break
    base_rank = nb / (time.perf_counter() - b0) if nb else 0.0
    base = sum_over_ranks(world, base_rank)
    nb_all = int(sum_over_ranks(world, float(nb)))
    value = main_run["solves_per_s"]
    line = {
        "metric": "PPR solves/s (served)", "value": value, "unit": "solves/s", "n_gpus": world,
        "steps": 1, "warmup": 1, "ms_per_step": args.serve_seconds * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+bf16", "data": "synthetic",
        "config": {"workload": "serving-pool256-poisson", "pool_graphs": len(specs),
                   "pool_raw_edges": sum(sp.m for sp in specs), "rate_req_per_s": args.serve_rate,
                   "warmup_s": args.serve_warmup, "window_s": args.serve_seconds, "budget_bytes_per_gpu": budget,
                   "steps_per_tick": 8, "edges_per_part": 1 << 18, "max_iters": 1000,
                   "storage": "FP32 contributions for tol 1e-6 requests, BF16 error-feedback deltas for tol 1e-3",
                   "parallelism": f"pool sharded over {world} rank(s), graph j on rank j % world"},
        "latency_ms": {"p50": main_run["p50_ms"], "p99": main_run["p99_ms"],
                       "completed": main_run["completed_in_window"],
                       "arrived_in_window": main_run["arrived_in_window"],
                       "unfinished_after_drain": main_run["unfinished_after_drain"]},
        "offered_solves_per_s": main_run["offered_solves_per_s"],
        "rejected": main_run["rejected"],
        "server": main_run["server_rank0"],
        "clocks": clk.summary(),
        "gpu_launches": launches,
        "stable_load_sweep": sweep,
        "max_stable_load": ({"rate_req_per_s": max_stable["rate_req_per_s"],
                             "solves_per_s": max_stable["solves_per_s"], "p50_ms": max_stable["p50_ms"],
                             "p99_ms": max_stable["p99_ms"]} if max_stable else None),
        "accuracy": {"vs": "FP64 oracle fixed point (400 steps), served requests on small pool graphs",
                     "columns": [{"dtype": "bf16" if d == int(gpr.BF16) else "fp32", "tol": t, "l1": e}
                                 for d, t, e in acc],
                     "max_l1_minus_tol": max((e - t for _, t, e in acc), default=None)},
        "one_at_a_time_solves_per_s": base, "baseline_sample_solves": nb_all,
        "speedup_vs_one_at_a_time": value / base if base else None,
        "speedup_at_max_stable_load": (max_stable["solves_per_s"] / base if max_stable and base else None),
        "setup_s": t_setup,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_hits(args, world, rank, local):
    """HITS on the R-MAT scale-25 graph (edge factor 32): each step is one
    `hits` call of 20 iterations (authorities from the in-edges, hubs from the
    out-edges, both L2-normalised) on a graph built before the timed region
    (its out-adjacency is built by the first, untimed call).  GTEPS counts 2m
    edge traversals per iteration."""
    import torch

    import gen
    import oracle
    import paper_1606_07550_gb300 as gpr

    iters = 20
    torch.cuda.set_device(local)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        n_s = 1 << args.cpu_sample_scale
        s_h, d_h = gen.rmat_coo(n_s, 32 * n_s, seed=3)
        gs = oracle.build_csc(n_s, s_h, d_h)
        t0 = time.perf_counter()
        oracle.hits(gs, iters)
        dt = time.perf_counter() - t0
        cpu = (2 * gs.m * iters / dt / 1e9, dt,
               f"R-MAT scale {args.cpu_sample_scale}, edge factor 32 (m={gs.m}); {iters} HITS iterations, "
               "single-threaded FP64 oracle")
    spec = workload("rmat25")
    src, dst = make_coo_device(torch, spec)
    g = gpr.graph_build(src, dst, spec.n)
    del src, dst
    torch.cuda.empty_cache()
    m, n = g.info().m, spec.n
    stream = torch.cuda.current_stream()
    hub = torch.empty(n, device="cuda")
    auth = torch.empty(n, device="cuda")
    for _ in range(args.warmup):
        gpr.hits(g, hub, auth, iters=iters, stream=stream, spmv=args.spmv)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[local] if os.environ.get(
        "CUDA_VISIBLE_DEVICES") else str(local)
    launches0 = gpr.lib().gpr_kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(gpu_index) as clk:
        for k in range(args.steps):
            evs[k][0].record(stream)
            gpr.hits(g, hub, auth, iters=iters, stream=stream, spmv=args.spmv)
            evs[k][1].record(stream)
        torch.cuda.synchronize()
    barrier(world)
    launches = gpr.lib().gpr_kernel_launches() - launches0
    t = sum(a.elapsed_time(b) for a, b in evs) / args.steps
    t = max_over_ranks(world, t)
    value = sum_over_ranks(world, float(m)) * 2 * iters / (t * 1e-3) / 1e9
    bytes_iter = 2 * (8 * m + 12 * n + 4)
    achieved = bytes_iter * iters / (t * 1e-3) / 1e9
    peak, peak_kind = measured_peak()
    if rank != 0:
        return
    line = {
        "metric": "HITS GTEPS", "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "hits-rmat-s25-ef32", "n": n, "m": m, "iters": iters,
                   "step": "one hits call: 20 iterations (two products each) + L2 output",
                   "schedule": "blocked" if args.spmv != "pull" and m >= (1 << 22) else "pull",
                   "value_counts": "2 m iters / time", "l2": "inputs larger than L2 (CSC 4 GiB x 2)"},
        "roofline": {"kernel": "HITS iteration (two products, on the CSC and its transpose, + folds)",
                     "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "peak_source": peak_kind, "bytes_model": "2 x (8m + 12n + 4) per iteration", "traffic": None},
        "clocks": clk.summary(), "gpu_launches": launches,
    }
    if cpu:
        line["cpu_baseline"] = {"value": cpu[0], "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": cpu[2],
                                "seconds": cpu[1]}
    print(json.dumps(line), flush=True)


def run_wcc(args, world, rank, local):
    """Weakly connected components of the R-MAT scale-25 graph (edge factor
    32), built before the timed region; each step is one `wcc` call.  GTEPS
    counts m edges per call.  Also times a binary save and load of the same
    graph through a temporary file (the paper's save/load measurement)."""
    import tempfile

    import torch

    import gen
    import oracle
    import paper_1606_07550_gb300 as gpr

    torch.cuda.set_device(local)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        n_s = 1 << args.cpu_sample_scale
        s_h, d_h = gen.rmat_coo(n_s, 32 * n_s, seed=3)
        gs = oracle.build_csc(n_s, s_h, d_h)
        t0 = time.perf_counter()
        oracle.wcc(gs)
        dt = time.perf_counter() - t0
        cpu = (gs.m / dt / 1e9, dt, f"R-MAT scale {args.cpu_sample_scale}, edge factor 32 (m={gs.m}); union-find, "
                                    "single-threaded oracle")
    spec = rmat_spec(args.target_scale)
    src, dst = make_coo_device(torch, spec)
    g = gpr.graph_build(src, dst, spec.n)
    del src, dst
    torch.cuda.empty_cache()
    m, n = g.info().m, spec.n
    stream = torch.cuda.current_stream()
    labels = torch.empty(n, dtype=torch.int32, device="cuda")
    for _ in range(args.warmup):
        k = gpr.wcc(g, labels, stream=stream)
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[local] if os.environ.get(
        "CUDA_VISIBLE_DEVICES") else str(local)
    launches0 = gpr.lib().gpr_kernel_launches()
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(gpu_index) as clk:
        for i in range(args.steps):
            evs[i][0].record(stream)
            k = gpr.wcc(g, labels, stream=stream)
            evs[i][1].record(stream)
        torch.cuda.synchronize()
    barrier(world)
    launches = gpr.lib().gpr_kernel_launches() - launches0
    t = max_over_ranks(world, sum(a.elapsed_time(b) for a, b in evs) / args.steps)
    value = sum_over_ranks(world, float(m)) / (t * 1e-3) / 1e9
    io = None
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "g.bin")
        t0 = time.perf_counter()
        g.save(path)
        t_save = time.perf_counter() - t0
        size = os.path.getsize(path)
        t0 = time.perf_counter()
        h = gpr.graph_load(path)
        torch.cuda.synchronize()
        t_load = time.perf_counter() - t0
        h.free()
        io = {"file_bytes": size, "save_s": t_save, "load_s": t_load, "save_gb_per_s": size / t_save / 1e9,
              "load_gb_per_s": size / t_load / 1e9}
    if rank != 0:
        return
    line = {
        "metric": "WCC GTEPS", "value": value, "unit": "GTEPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": f"wcc-rmat-s{spec.scale}-ef32", "n": n, "m": m, "components": k,
                   "step": "one wcc call: sampled links, giant component skipped in one edge pass, labels by "
                           "caller id",
                   "value_counts": "m / time"},
        "clocks": clk.summary(), "gpu_launches": launches, "save_load": io,
    }
    if cpu:
        line["cpu_baseline"] = {"value": cpu[0], "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": cpu[2],
                                "seconds": cpu[1]}
    print(json.dumps(line), flush=True)


def run_dynamic(args, world, rank, local):
    """Dynamic graph (the paper's section 5 theme; Table "exp_del" times
    deletions): the R-MAT scale-25 graph (edge factor 32) takes, per step, one
    graph_update of 2^20 random insertions and 2^20 deletions of existing
    edges, then a 10-step PageRank warm-started from the previous ranks.
    value = updated edges per second of graph_update; the warm PageRank is
    reported beside it."""
    import torch

    import paper_1606_07550_gb300 as gpr

    torch.cuda.set_device(local)
    spec = workload("rmat25")
    src, dst = make_coo_device(torch, spec)
    g = gpr.graph_build(src, dst, spec.n)
    n = spec.n
    k = 1 << 20
    gen_ = torch.Generator(device="cuda")
    gen_.manual_seed(11)
    x = torch.empty(n, device="cuda")
    gpr.pagerank(g, x, iters=30)
    stream = torch.cuda.current_stream()

    def batch():
        pick = torch.randint(0, src.numel(), (k,), device="cuda", generator=gen_)
        ins_s = torch.randint(0, n, (k,), device="cuda", dtype=torch.int32, generator=gen_)
        ins_d = torch.randint(0, n, (k,), device="cuda", dtype=torch.int32, generator=gen_)
        return (ins_s, ins_d), (src[pick].contiguous(), dst[pick].contiguous())

    for _ in range(args.warmup):
        ins, dels = batch()
        gpr.graph_update(g, ins, dels, stream=stream)
        gpr.pagerank(g, x, iters=10, warm_start=True, stream=stream)
    torch.cuda.synchronize()
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[local] if os.environ.get(
        "CUDA_VISIBLE_DEVICES") else str(local)
    launches0 = gpr.lib().gpr_kernel_launches()
    t_upd, t_pr = [], []
    barrier(world)
    with ClockSampler(gpu_index) as clk:
        for _ in range(args.steps):
            ins, dels = batch()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            c = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            gpr.graph_update(g, ins, dels, stream=stream)
            b.record(stream)
            gpr.pagerank(g, x, iters=10, warm_start=True, stream=stream)
            c.record(stream)
            torch.cuda.synchronize()
            t_upd.append(a.elapsed_time(b))
            t_pr.append(b.elapsed_time(c))
    barrier(world)
    launches = gpr.lib().gpr_kernel_launches() - launches0
    tu = max_over_ranks(world, sum(t_upd) / len(t_upd))
    tp = sum(t_pr) / len(t_pr)
    value = sum_over_ranks(world, 2.0 * k) / (tu * 1e-3)
    if rank != 0:
        return
    line = {
        "metric": "edge updates/s", "value": value, "unit": "edges/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tu, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "int32", "data": "synthetic",
        "config": {"workload": "dynamic-rmat-s25-ef32", "n": n, "m_after": g.info().m, "insertions": k,
                   "deletions": k, "step": "graph_update (2^20 inserts + 2^20 deletes), then 10 warm PageRank steps"},
        "warm_pagerank_ms": tp, "clocks": clk.summary(), "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)


def run_target(args, world, rank, local):
    """Single-target personalised PageRank (section 4.3, bidirectional): on the
    R-MAT scale-25 graph (edge factor 32), each step answers one query: a
    random target, `--target-sources` random sources, reverse push to
    `--target-rmax`, then `--target-walks` walks per source.  value = (source,
    target) estimates per second.  The push alone is timed beside it."""
    import numpy as np
    import torch

    import gen
    import oracle
    import paper_1606_07550_gb300 as gpr

    torch.cuda.set_device(local)
    k, W, r_max = args.target_sources, args.target_walks, args.target_rmax
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        n_s = 1 << args.cpu_sample_scale
        s_h, d_h = gen.rmat_coo(n_s, 32 * n_s, seed=3)
        gs = oracle.build_csc(n_s, s_h, d_h)
        rng = np.random.default_rng(5)
        ks = 8
        t0 = time.perf_counter()
        done = 0
        while time.perf_counter() - t0 < 10.0 and done < 64:
            t = int(rng.integers(0, n_s))
            oracle.ppr_target(gs, t, rng.integers(0, n_s, ks).astype(np.int32), 0.85, r_max, W, seed=done)
            done += ks
        dt = time.perf_counter() - t0
        cpu = (done / dt, dt, f"R-MAT scale {args.cpu_sample_scale}, edge factor 32; {done // ks} targets x {ks} "
                              f"sources, r_max {r_max:g}, {W} walks; single-threaded oracle")
    spec = rmat_spec(args.target_scale)
    src, dst = make_coo_device(torch, spec)
    g = gpr.graph_build(src, dst, spec.n)
    del src, dst
    torch.cuda.empty_cache()
    n = spec.n
    stream = torch.cuda.current_stream()
    gen_ = torch.Generator(device="cpu")
    gen_.manual_seed(17 + rank)
    queries = [(int(torch.randint(0, n, (1,), generator=gen_)),
                torch.randint(0, n, (k,), generator=gen_, dtype=torch.int32).cuda())
               for _ in range(args.warmup + args.steps)]
    est = torch.empty(k, dtype=torch.float64, device="cuda")
    for i in range(args.warmup):
        t, srcs = queries[i]
        gpr.ppr_target(g, t, srcs, est, r_max, W, seed=i, stream=stream)
    torch.cuda.synchronize()
    gpu_index = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[local] if os.environ.get(
        "CUDA_VISIBLE_DEVICES") else str(local)
    launches0 = gpr.lib().gpr_kernel_launches()
    times, stats = [], []
    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(gpu_index) as clk:
        for i in range(args.warmup, args.warmup + args.steps):
            t, srcs = queries[i]
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            stats.append(gpr.ppr_target(g, t, srcs, est, r_max, W, seed=i, stream=stream))
            b.record(stream)
            torch.cuda.synchronize()
            times.append(a.elapsed_time(b))
    barrier(world)
    launches = gpr.lib().gpr_kernel_launches() - launches0
    tq = max_over_ranks(world, sum(times) / len(times))
    value = sum_over_ranks(world, float(k)) / (tq * 1e-3)
    # end to end: sources from pinned host memory, estimates back to the host
    h_src = [queries[i][1].cpu().pin_memory() for i in range(args.warmup, args.warmup + args.steps)]
    h_est = torch.empty(k, dtype=torch.float64).pin_memory()
    e2e_t = []
    for q, i in enumerate(range(args.warmup, args.warmup + args.steps)):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        gpr.ppr_target(g, queries[i][0], h_src[q].numpy(), h_est.numpy(), r_max, W, seed=i, stream=stream)
        e2e_t.append(time.perf_counter() - t0)
    e2e_ms = max_over_ranks(world, 1e3 * sum(e2e_t) / len(e2e_t))
    if rank != 0:
        return
    mean = lambda f: sum(f(x) for x in stats) / len(stats)
    walk_ms, push_ms = mean(lambda x: x.walk_ms), mean(lambda x: x.push_ms)
    # algorithmic bytes: a walk step reads the out-offsets of its node (8 B)
    # and one out-neighbour (4 B); each walk also reads its start offsets and
    # writes its endpoint (12 B).  A push scans its in-edges (source id 4 B,
    # its out-degree 4 B, the residual's atomic read and write 16 B per edge)
    # and takes its own residual, p, amount and offsets (72 B).
    walk_bytes = mean(lambda x: 12.0 * x.walk_steps + 12.0 * k * W)
    push_bytes = mean(lambda x: 24.0 * x.edges + 72.0 * x.pushes)
    peak = measured_peak()
    phases = {
        "walk": {"ms": walk_ms, "bytes": walk_bytes, "gbs": walk_bytes / (walk_ms * 1e6)},
        "push": {"ms": push_ms, "bytes": push_bytes, "gbs": push_bytes / (push_ms * 1e6),
                 "pushes": mean(lambda x: x.pushes), "edges": mean(lambda x: x.edges),
                 "rounds": mean(lambda x: x.rounds)},
    }
    top = "walk" if walk_ms >= push_ms else "push"
    line = {
        "metric": "single-target PPR estimates/s", "value": value, "unit": "estimates/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": tq, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"ppr-target-rmat-s{spec.scale}-ef32", "n": n, "m": g.info().m, "sources": k, "walks": W,
                   "r_max": r_max, "damping": 0.85,
                   "step": "one ppr_target call: reverse push from a random target beside walks from k random "
                           "sources, then the estimates",
                   "l2": "graph 4.3 GB + walk adjacency 4.3 GB >> L2; each query a new target and sources"},
        "roofline": {"bound": "hbm", "kernel": "walk_kernel" if top == "walk" else "push_take+push_scatter",
                     "achieved": phases[top]["gbs"], "peak": peak[0], "unit": "GB/s",
                     "frac": phases[top]["gbs"] / peak[0], "traffic": None, "peak_source": peak[1]},
        "phases": phases, "walk_steps_mean": mean(lambda x: x.walk_steps),
        "e2e": {"value": k / (e2e_ms * 1e-3), "unit": "estimates/s", "h2d_bytes_per_step": 4 * k,
                "d2h_bytes_per_step": 8 * k},
        "query_ms_each": times, "clocks": clk.summary(), "gpu_launches": launches,
    }
    if cpu:
        line["cpu_baseline"] = {"value": cpu[0], "unit": "estimates/s", "cores": 1, "kind": "oracle",
                                "sample": cpu[2], "seconds": cpu[1]}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "batched":
        run_batched(args, world, rank, local)
    elif args.workload == "serve":
        run_serve(args, world, rank, local)
    elif args.workload == "hits":
        run_hits(args, world, rank, local)
    elif args.workload == "wcc":
        run_wcc(args, world, rank, local)
    elif args.workload == "dynamic":
        run_dynamic(args, world, rank, local)
    elif args.workload == "target":
        run_target(args, world, rank, local)
    else:
        run_gpr(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
