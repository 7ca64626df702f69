"""Benchmark: PageRank GTEPS and fraction of the HBM roofline on one GB300,
fused (nonblocking, whole loop on the GPU) vs op-by-op (blocking mode).

Workload: R-MAT scale 22 (2^22 vertices, 2^26 raw edges, a,b,c,d =
.57,.19,.19,.05, duplicates and self loops dropped, labels scrambled),
FP32 ranks with an FP64 residual, damping 0.85, dangling rank spread
uniformly, 50 fixed iterations, seed 1.  A step is one PageRank solve
(50 fused iterations) on the graph resident in HBM; GTEPS = m x 50 / time.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  With --impl reference the FP64 CPU oracle (the
baseline arm) is timed on the host cores instead.
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "PageRank GTEPS & % HBM peak, fused vs op-by-op on 1 GB300, at L1 ≤1e-6 vs FP64"
SCALE, EDGE_FACTOR, SEED, ITERS, DAMPING = 22, 16, 1, 50, 0.85
WORKLOAD = ("R-MAT scale 22 (4,194,304 vertices, 67,108,864 raw edges, a=.57 b=.19 c=.19 d=.05, dedup, "
            "no self loops), FP32 ranks, FP64 residual, damping 0.85, uniform dangling, 50 fixed iterations, seed 1")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "pr_persistent_kernel_rmat22.md")
KERNEL_SOURCE = os.path.join(ROOT, "paper_2509_14211_gb300", "csrc", "kernels_pr.cu")


def _traffic_per_launch():
    """DRAM bytes (read + write) of one 50-body launch of the persistent
    kernel, from the committed ncu summary (a 2-body capture scaled by the
    bodies), or None when the kernel source has changed since the capture."""
    import hashlib
    import re

    try:
        with open(KERNEL_SOURCE, "rb") as f:
            digest = hashlib.sha256(f.read()).hexdigest()
        with open(PROFILE_SUMMARY) as f:
            text = f.read()
    except OSError:
        return None
    m_hash = re.search(r"kernels_pr\.cu sha256: ([0-9a-f]{64})", text)
    m_traffic = re.search(r"traffic per 50-body launch: (\d+) bytes", text)
    if not m_hash or not m_traffic or m_hash.group(1) != digest:
        return None
    return int(m_traffic.group(1))


def _start_clock_sampler(path):
    cmd = ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
           "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
           "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
           "--format=csv,noheader,nounits", "-lms", "200"]
    try:
        return subprocess.Popen(cmd, stdout=open(path, "w"), stderr=subprocess.DEVNULL)
    except Exception:
        return None


def _clocks_summary(path, device_index):
    sm, mx, reasons = [], [], set()
    try:
        with open(path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9 or parts[0] != str(device_index):
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for name, v in zip(("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"),
                                   parts[5:9]):
                    if v.lower() == "active":
                        reasons.add(name)
    except FileNotFoundError:
        pass
    if not sm:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons)}


def _max_over_ranks(x: float) -> float:
    """Max of x over the ranks of the process group (x itself without one).
    The bench's step time is the slowest rank's."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_gteps(world_size: int, m: int, iters: int, ms: float) -> float:
    """Whole-job throughput: every rank solves its own replica of the graph
    (weak scaling), so the job does world_size * m * iters edge updates in
    the slowest rank's time."""
    return world_size * m * iters / (ms * 1e-3) / 1e9


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_reference(args):
    """Baseline arm: the FP64 CPU oracle as it stands, on the host cores."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import graphgen
    import oracle

    src, dst = graphgen.rmat_edges(SCALE, EDGE_FACTOR, seed=SEED)
    n = 1 << SCALE
    ptr, col = oracle.build_at(n, src, dst)
    outdeg = oracle.out_degree(ptr, col)
    m = int(len(col))
    # each step: 2 iterations of the oracle's pagerank on the full graph
    iters_per_step = 2
    for _ in range(args.warmup):
        oracle.pagerank(ptr, col, outdeg, damping=DAMPING, tol=-1.0, itermax=iters_per_step, mode="uniform")
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.pagerank(ptr, col, outdeg, damping=DAMPING, tol=-1.0, itermax=iters_per_step, mode="uniform")
        times.append(time.perf_counter() - t0)
    t = sum(times) / len(times)
    value = m * iters_per_step / t / 1e9
    sample = f"{iters_per_step} FP64 oracle iterations per step on the full R-MAT scale 22 graph (CSR build untimed)"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "m": m, "iterations_per_step": iters_per_step},
        "cpu_baseline": {"value": value, "unit": "GTEPS", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GTEPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def run_profile_case_ppr(args):
    """Profiling run of the batched personalised PageRank: R-MAT --scale,
    --slots queries (1-32 seeds, seed 3), --iters bodies per run."""
    import torch

    import graphgen
    import paper_2509_14211_gb300 as grb
    from paper_2509_14211_gb300.pagerank import BUILD_FLAGS

    torch.cuda.set_device(0)
    n = 1 << args.scale
    src, dst = graphgen.rmat_edges(args.scale, EDGE_FACTOR, seed=3)
    sets = graphgen.ppr_seed_sets(n, args.slots, 1, 32, seed=3)
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    AT = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, n, n, src, dst, None, BUILD_FLAGS)
    m = grb.grb_matrix_nvals(AT)
    P = grb.grb_ppr_new(AT, DAMPING, args.slots)
    if args.vw:
        grb.grb_ppr_layout(P, args.vw)
    ms = 0.0
    for rep in range(args.warmup + args.steps):
        for s, S in enumerate(sets):
            grb.grb_ppr_set(P, s, S, -1.0, args.iters)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        grb.grb_ppr_run(P, args.iters)
        e1.record()
        torch.cuda.synchronize()
        if rep >= args.warmup:
            ms += e0.elapsed_time(e1) / args.steps
    print(json.dumps({"profile_case": "ppr", "scale": args.scale, "n": n, "m": m, "slots": args.slots,
                      "vector_width": args.vw or 1,
                      "bodies": args.iters, "ms": ms, "ms_per_body": ms / args.iters,
                      "edge_query_updates_per_s_G": m * args.slots * args.iters / (ms * 1e-3) / 1e9}), flush=True)
    grb.grb_free(P)
    grb.grb_free(AT)
    grb.grb_free(ctx)


def run_profile_case_batch(args):
    """Profiling run of the 512-graph batch (scale 8-16, edge factor 8-32,
    seed 3): --iters bodies per run."""
    import torch

    import graphgen
    import paper_2509_14211_gb300 as grb
    from paper_2509_14211_gb300.pagerank import BUILD_FLAGS

    torch.cuda.set_device(0)
    graphs = []
    for scale, ef, s in graphgen.batch_graph_specs(512, 8, 16, 8, 32, seed=3):
        src, dst = graphgen.rmat_edges(scale, ef, seed=s)
        graphs.append((1 << scale, src, dst))
    n, src, dst, vptr = grb.block_diagonal_edges(graphs)
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    grb.grb_context_set(ctx, grb.GRB_OPT_RELABEL, 0 if args.no_relabel else 1)
    AT = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, n, n, src, dst, None, BUILD_FLAGS)
    m = grb.grb_matrix_nvals(AT)
    B = grb.grb_prbatch_new(AT, vptr, DAMPING)
    _, chosen = grb.grb_prbatch_tune(B, 2)
    ms = 0.0
    for rep in range(args.warmup + args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        grb.grb_prbatch_run(B, -1.0, args.iters, args.iters)
        e1.record()
        torch.cuda.synchronize()
        if rep >= args.warmup:
            ms += e0.elapsed_time(e1) / args.steps
    print(json.dumps({"profile_case": "batch", "graphs": len(graphs), "n": n, "m": m, "bodies": args.iters,
                      "chosen_ctas_per_sm": chosen, "ms": ms,
                      "gteps": m * args.iters / (ms * 1e-3) / 1e9}), flush=True)
    grb.grb_free(B)
    grb.grb_free(AT)
    grb.grb_free(ctx)


def run_profile_case(args):
    """A small run of the fused device loop for ncu captures: builds R-MAT
    --scale, runs --warmup + --steps loops of --iters fused iterations."""
    import torch

    import graphgen
    import paper_2509_14211_gb300 as grb
    from paper_2509_14211_gb300.pagerank import BUILD_FLAGS, PageRankProblem

    torch.cuda.set_device(0)
    n = 1 << args.scale
    if args.graph == "er":
        src, dst = graphgen.er_edges(n, 16, p_dangling=0.02, seed=2)
    else:
        src, dst = graphgen.rmat_edges(args.scale, EDGE_FACTOR, seed=SEED, permute=not args.unpermuted)
    if args.degree_sorted:   # relabel by descending out-degree (host side, for the experiment)
        order = np.argsort(-np.bincount(src, minlength=n), kind="stable")
        new_id = np.empty(n, dtype=np.int32)
        new_id[order] = np.arange(n, dtype=np.int32)
        src, dst = new_id[src], new_id[dst]
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    grb.grb_context_set(ctx, grb.GRB_OPT_PERSISTENT, args.loop_mode)
    grb.grb_context_set(ctx, grb.GRB_OPT_RELABEL, 0 if args.no_relabel else 1)
    if args.hot_bytes is not None:
        grb.grb_context_set(ctx, grb.GRB_OPT_HOT_BYTES, args.hot_bytes)
    if args.tma_stages is not None:
        grb.grb_context_set(ctx, grb.GRB_OPT_TMA_STAGES, args.tma_stages)
    grb.grb_context_set(ctx, grb.GRB_OPT_ROW_BINS, 1 if args.row_bins else 0)
    grb.grb_context_set(ctx, grb.GRB_OPT_MIXED, 2 if args.mixed else 0)
    AT = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, n, n, src, dst, None, BUILD_FLAGS)
    m = grb.grb_matrix_nvals(AT)
    P = PageRankProblem(ctx, AT, n, DAMPING, grb.GRB_FP32, grb.GRB_FP64, "uniform")
    for _ in range(args.warmup):
        P.run(args.tol, args.iters, "device")
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    done = 0
    for _ in range(args.steps):
        done = P.run(args.tol, args.iters, "device")
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    kms = grb.grb_context_stats(ctx)["last_loop_kernel_ns"] / 1e6
    print(json.dumps({"profile_case": True, "graph": args.graph, "mixed": args.mixed, "scale": args.scale, "n": n,
                      "m": m, "iters": done,
                      "loop_mode": args.loop_mode, "relabel": not args.no_relabel, "hot_bytes": args.hot_bytes,
                      "tma_stages": args.tma_stages, "row_bins": args.row_bins,
                      "ms_per_loop": ms, "kernel_ms": kms, "gteps": m * done / (ms * 1e-3) / 1e9,
                      "kernel_gteps": m * done / (kms * 1e-3) / 1e9}), flush=True)
    P.free()
    grb.grb_free(AT)
    grb.grb_free(ctx)


MIXED_TOL = 1e-6 * (1 - DAMPING) / DAMPING


def run_mixed_leg(grb, torch, stream, log2n, modes):
    """Mixed precision on Erdos-Renyi 2^log2n (out-degree 16, 2% sinks, seed
    2): BF16 gathers until the residual falls below 1e-3 (or stalls), then
    FP32, to an L1 change of 1e-6 (1-d)/d, beside the FP32-only loop to the
    same stop.  `modes` are GRB_OPT_MIXED values: 1 lets the planner decide
    (BF16 only when the FP32 gather vector exceeds L2), 2 forces BF16, 0 is
    FP32 throughout.  Times are CUDA events around grb_iterate_end (graph
    resident)."""
    import graphgen
    from paper_2509_14211_gb300.pagerank import BUILD_FLAGS, PageRankProblem

    n = 1 << log2n
    src, dst = graphgen.er_edges(n, 16, p_dangling=0.02, seed=2)
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    grb.grb_context_set(ctx, grb.GRB_OPT_PERSISTENT, 1)
    AT = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, n, n, src, dst, None, BUILD_FLAGS)
    del src, dst
    m = grb.grb_matrix_nvals(AT)
    P = PageRankProblem(ctx, AT, n, DAMPING, grb.GRB_FP32, grb.GRB_FP64, "uniform")
    out = {"workload": f"Erdos-Renyi 2^{log2n} vertices, out-degree 16, 2% sinks, seed 2, uniform dangling",
           "n": n, "m": m, "stop_l1_change": MIXED_TOL, "fp32_gather_vector_bytes": 4 * n,
           "l2_bytes": int(torch.cuda.get_device_properties(torch.cuda.current_device()).L2_cache_size)}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    names = {0: "fp32_only", 1: "planner", 2: "bf16_forced"}
    for mixed in modes:
        grb.grb_context_set(ctx, grb.GRB_OPT_MIXED, mixed)
        P.run(MIXED_TOL, 500, "device")          # warm-up (builds plans, sink bits)
        times, iters = [], 0
        for _ in range(3):
            e0.record(stream)
            iters = P.run(MIXED_TOL, 500, "device")
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        hist, phase = grb.grb_iterate_history(ctx)
        r = P.rank().astype(np.float64)
        ms = sorted(times)[1]
        out[names[mixed]] = {"ms": ms, "iterations": int(iters), "gteps": m * iters / (ms * 1e-3) / 1e9,
                             "final_l1_change": float(hist[-1]), "bf16_phase_used": phase >= 0,
                             "switched_to_fp32": bool(phase == 1) if phase >= 0 else None,
                             "rank_sum": float(np.sum(r)), "rank_min": float(np.min(r))}
    for name in ("planner", "bf16_forced"):
        if name in out and "fp32_only" in out:
            out[name + "_speedup"] = out["fp32_only"]["ms"] / out[name]["ms"]
    P.free()
    grb.grb_free(AT)
    grb.grb_free(ctx)
    return out


def run_ppr_leg(grb, torch, stream):
    """Batched personalised PageRank: R-MAT scale 20, 64 queries with 1-32
    uniformly drawn seeds (seed 3), 50 bodies, as one slot batch (SpMM over
    64 right-hand sides).  CUDA events around the enqueued CUDA graph."""
    import graphgen
    from paper_2509_14211_gb300.pagerank import BUILD_FLAGS

    n, k, iters = 1 << 20, 64, 50
    src, dst = graphgen.rmat_edges(20, 16, seed=3)
    sets = graphgen.ppr_seed_sets(n, k, 1, 32, seed=3)
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    AT = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, n, n, src, dst, None, BUILD_FLAGS)
    m = grb.grb_matrix_nvals(AT)
    P = grb.grb_ppr_new(AT, DAMPING, k)
    tune_ms, vw = grb.grb_ppr_tune(P, 2)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for rep in range(4):
        for s, S in enumerate(sets):
            grb.grb_ppr_set(P, s, S, -1.0, iters)
        torch.cuda.synchronize()
        e0.record(stream)
        grb.grb_ppr_run(P, iters)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep > 0:                       # the first run captures the graph
            times.append(e0.elapsed_time(e1))
    ms = sorted(times)[len(times) // 2]
    out = {"workload": "R-MAT scale 20 (1,048,576 vertices, edge factor 16, seed 3), 64 personalised queries with "
                       "1-32 uniform seeds each, FP32, 50 bodies, uniform dangling",
           "n": n, "m": m, "k": k, "bodies": iters, "ms": ms, "ms_per_body": ms / iters,
           "autotune_ms_per_body_by_vector_width": {"1": float(tune_ms[0]), "2": float(tune_ms[1]),
                                                    "4": float(tune_ms[2])}, "vector_width": vw,
           "edge_query_updates_per_s_G": m * k * iters / (ms * 1e-3) / 1e9,
           "algorithmic_bytes_per_body": 4 * m + 4 * (n + 1) + 4 * k * 4 * n}
    out["hbm_frac_of_measured"] = out["algorithmic_bytes_per_body"] / (out["ms_per_body"] * 1e-3) / 1e9 / _peaks()[0]
    grb.grb_free(P)
    grb.grb_free(AT)
    grb.grb_free(ctx)
    return out


def run_batch_leg(grb, torch, stream):
    """512 independent R-MAT graphs (scale 8-16, edge factor 8-32, seed 3) as
    one block-diagonal batch: autotuned launch shape, 50 bodies captured in
    one CUDA graph; beside it the same graphs solved one after another with
    the single-graph persistent loop."""
    import graphgen
    from paper_2509_14211_gb300.pagerank import BUILD_FLAGS, PageRankProblem

    specs = graphgen.batch_graph_specs(512, 8, 16, 8, 32, seed=3)
    graphs = []
    for scale, ef, s in specs:
        src, dst = graphgen.rmat_edges(scale, ef, seed=s)
        graphs.append((1 << scale, src, dst))
    n, src, dst, vptr = grb.block_diagonal_edges(graphs)
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    AT = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, n, n, src, dst, None, BUILD_FLAGS)
    m = grb.grb_matrix_nvals(AT)
    B = grb.grb_prbatch_new(AT, vptr, DAMPING)
    tune_ms, chosen = grb.grb_prbatch_tune(B, 3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    grb.grb_prbatch_run(B, -1.0, ITERS, ITERS)           # warm-up (captures the graph)
    times = []
    for _ in range(3):
        e0.record(stream)
        grb.grb_prbatch_run(B, -1.0, ITERS, ITERS)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = sorted(times)[1]
    grb.grb_prbatch_run(B, MIXED_TOL, 1000, 16)
    _, its, _ = grb.grb_prbatch_result(B, n, len(graphs))
    out = {"workload": "512 R-MAT graphs, scale 8-16, edge factor 8-32 (seed 3), FP32, uniform dangling, 50 bodies "
                       "in one CUDA-graph launch", "graphs": len(graphs), "n": n, "m": m,
           "autotune_ms_per_body_by_ctas_per_sm": [round(float(x), 4) for x in tune_ms],
           "chosen_ctas_per_sm": chosen, "ms": ms, "gteps": m * ITERS / (ms * 1e-3) / 1e9,
           "bodies_to_l1_change_1.76e-7": {"min": int(its.min()), "median": float(np.median(its)),
                                           "max": int(its.max())}}
    grb.grb_free(B)
    grb.grb_free(AT)
    # one graph at a time through the single-graph device loop
    mats, probs = [], []
    for ng, s_, d_ in graphs:
        A1 = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, ng, ng, s_, d_, None, BUILD_FLAGS)
        mats.append(A1)
        probs.append(PageRankProblem(ctx, A1, ng, DAMPING, grb.GRB_FP32, grb.GRB_FP64, "uniform"))
    for P1 in probs:
        P1.run(-1.0, ITERS, "device")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    e0.record(stream)
    for P1 in probs:
        P1.run(-1.0, ITERS, "device")
    e1.record(stream)
    torch.cuda.synchronize()
    out["one_by_one_ms"] = e0.elapsed_time(e1)
    out["one_by_one_wall_ms"] = (time.perf_counter() - t0) * 1e3
    out["batch_speedup"] = out["one_by_one_ms"] / ms
    for P1 in probs:
        P1.free()
    for A1 in mats:
        grb.grb_free(A1)
    grb.grb_free(ctx)
    return out


def run_serve_leg(grb):
    """Serving: R-MAT scale 24 resident on the device, Poisson query streams
    (seed 4) with 1-64 log-uniform seeds, FP32 ranks with FP64 residual to an
    L1 change of 1e-6, continuous batching in 64 slots with one body per
    scheduling step; while no slot is busy and at most 2 queries wait, a
    query runs alone on the fused single-vector loop."""
    import graphgen
    from paper_2509_14211_gb300.pagerank import BUILD_FLAGS

    n = 1 << 24
    src, dst = graphgen.rmat_edges(24, 16, seed=4)
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    AT = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, n, n, src, dst, None, BUILD_FLAGS)
    del src, dst
    m = grb.grb_matrix_nvals(AT)
    out = {"workload": "R-MAT scale 24 (16,777,216 vertices, edge factor 16, seed 4); queries with 1-64 log-uniform "
                       "seeds; stop at L1 change 1e-6; 64 slots; one body per scheduling step; single-vector loop "
                       "while no slot is busy and at most 2 queries wait",
           "n": n, "m": m, "levels": []}
    for rate, count in ((10.0, 24), (200.0, 600), (1000.0, 1000), (2000.0, 1000)):
        sets = graphgen.ppr_seed_sets(n, count, 1, 64, seed=4, log_uniform=True)
        arr = graphgen.poisson_arrivals(rate, count, seed=4)
        r = grb.grb_ppr_serve(AT, arr, sets, damping=DAMPING, tol=1e-6, itermax=1000, chunk=1, slots=64,
                              mem_fraction=0.5, single_max=2)
        lat = r["latency_s"]
        q = max(count // 4, 1)
        out["levels"].append({"offered_qps": rate, "queries": count,
                              "answered_qps": count / r["wall_s"],
                              "answered_qps_over_arrivals": count / max(float(arr[-1]), 1e-9),
                              "p50_ms": float(np.percentile(lat, 50) * 1e3),
                              "p99_ms": float(np.percentile(lat, 99) * 1e3),
                              "p99_first_quarter_ms": float(np.percentile(lat[:q], 99) * 1e3),
                              "p99_last_quarter_ms": float(np.percentile(lat[-q:], 99) * 1e3),
                              "mean_bodies": float(np.mean(r["iters"])), "single_queries": int(r["single_queries"]),
                              "slots": r["slots"], "vector_width": r["vector_width"],
                              "max_in_flight": int(r["max_in_flight"]), "steps": int(r["steps"])})
    grb.grb_free(AT)
    grb.grb_free(ctx)
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-oracle", action="store_true", help="skip the FP64 oracle (error and CPU baseline)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision Erdos-Renyi 2^24 leg")
    ap.add_argument("--no-ppr", action="store_true", help="skip the batched personalised PageRank leg")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving leg")
    ap.add_argument("--no-batch", action="store_true", help="skip the 512-graph batch leg")
    ap.add_argument("--profile-case", action="store_true",
                    help="profiling run: only the fused device loop, on --scale/--iters (no JSON contract)")
    ap.add_argument("--scale", type=int, default=SCALE)
    ap.add_argument("--iters", type=int, default=ITERS)
    ap.add_argument("--loop-mode", type=int, default=1, help="1 persistent kernel, 2 CUDA graph of fused kernels")
    ap.add_argument("--unpermuted", action="store_true", help="profiling run on R-MAT without label scrambling")
    ap.add_argument("--degree-sorted", action="store_true", help="profiling run with vertices relabeled by out-degree")
    ap.add_argument("--no-relabel", action="store_true", help="profiling run on the matrix in its input vertex order")
    ap.add_argument("--hot-bytes", type=int, default=None, help="profiling run: shared-memory hot copy size")
    ap.add_argument("--tma-stages", type=int, default=None, help="profiling run: bulk-copy staging depth (0, 2, 3)")
    ap.add_argument("--row-bins", action="store_true", help="profiling run: the row-length-binned body")
    ap.add_argument("--graph", default="rmat", choices=["rmat", "er"], help="profiling run: graph family")
    ap.add_argument("--case", default="pagerank", choices=["pagerank", "ppr", "batch"],
                    help="profiling run: the device PageRank loop, batched personalised PageRank, or the graph batch")
    ap.add_argument("--slots", type=int, default=64, help="profiling run (ppr): number of queries")
    ap.add_argument("--vw", type=int, default=0, help="profiling run (ppr): slots per lane (0: 1)")
    ap.add_argument("--mixed", action="store_true", help="profiling run: BF16 gather, then FP32")
    ap.add_argument("--tol", type=float, default=-1.0, help="profiling run: stop at this L1 change")
    args = ap.parse_args()
    if args.profile_case:
        if args.case == "ppr":
            return run_profile_case_ppr(args)
        if args.case == "batch":
            return run_profile_case_batch(args)
        return run_profile_case(args)
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)

    import torch

    ws, rank, local = _dist()
    if ws > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()

    import graphgen
    import paper_2509_14211_gb300 as grb
    from paper_2509_14211_gb300.pagerank import BUILD_FLAGS, PageRankProblem

    n = 1 << SCALE
    src, dst = graphgen.rmat_edges(SCALE, EDGE_FACTOR, seed=SEED)
    src_pin = torch.from_numpy(src).pin_memory()
    dst_pin = torch.from_numpy(dst).pin_memory()
    stream = torch.cuda.current_stream()

    def barrier():
        torch.cuda.synchronize()
        if ws > 1:
            torch.distributed.barrier()

    # ------------------------------------------------------------ fused
    ctx = grb.grb_context_new(grb.GRB_NONBLOCKING)
    grb.grb_context_set(ctx, grb.GRB_OPT_PERSISTENT, 1)
    AT = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, n, n, src, dst, None, BUILD_FLAGS)
    m = grb.grb_matrix_nvals(AT)
    P = PageRankProblem(ctx, AT, n, DAMPING, grb.GRB_FP32, grb.GRB_FP64, "uniform")
    for _ in range(args.warmup):
        assert P.run(-1.0, ITERS, "device") == ITERS
    clock_path = tempfile.mktemp(suffix=".csv")
    sampler = _start_clock_sampler(clock_path)
    time.sleep(0.3)
    launches0 = grb.grb_context_stats(ctx)["kernel_launches"]
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    t_wall = time.perf_counter()
    for k in range(args.steps):
        # a fixed-count device loop only enqueues its work (nonblocking
        # mode), so the host records step k+1 while the GPU runs step k
        ev[k][0].record(stream)
        P.run(-1.0, ITERS, "device")
        ev[k][1].record(stream)
    barrier()
    t_wall = time.perf_counter() - t_wall
    kernel_ms_steps = [float(x) for x in grb.grb_context_loop_times(ctx, args.steps)]
    launches = grb.grb_context_stats(ctx)["kernel_launches"] - launches0
    if sampler:
        sampler.terminate()
        sampler.wait()
    clocks = _clocks_summary(clock_path, dev)
    step_ms = [a.elapsed_time(b) for a, b in ev]
    ms = _max_over_ranks(sum(step_ms) / len(step_ms))
    r_fused = P.rank().astype(np.float64)
    rdiff = P.residual()
    hist, _ = grb.grb_iterate_history(ctx)
    value = _job_gteps(ws, m, ITERS, ms)

    # graph-of-kernels variant of the device loop
    grb.grb_context_set(ctx, grb.GRB_OPT_PERSISTENT, 2)
    for _ in range(2):
        P.run(-1.0, ITERS, "device")
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        P.run(-1.0, ITERS, "device")
    e1.record(stream)
    torch.cuda.synchronize()
    graph_ms = e0.elapsed_time(e1) / 3
    grb.grb_context_set(ctx, grb.GRB_OPT_PERSISTENT, 1)

    # the persistent loop on the matrix in its input vertex order
    grb.grb_context_set(ctx, grb.GRB_OPT_RELABEL, 0)
    for _ in range(2):
        P.run(-1.0, ITERS, "device")
    e0.record(stream)
    for _ in range(3):
        P.run(-1.0, ITERS, "device")
    e1.record(stream)
    torch.cuda.synchronize()
    input_order_ms = e0.elapsed_time(e1) / 3
    grb.grb_context_set(ctx, grb.GRB_OPT_RELABEL, 1)

    # host loop with per-wait fusion (the paper's nonblocking mode)
    P.run(-1.0, 5, "host")
    e0.record(stream)
    P.run(-1.0, ITERS, "host")
    e1.record(stream)
    torch.cuda.synchronize()
    perwait_ms = e0.elapsed_time(e1)
    P.free()

    # ---------------------------------------------------------- unfused
    ctxb = grb.grb_context_new(grb.GRB_BLOCKING)
    ATb = grb.grb_matrix_build_csr(ctxb, grb.GRB_FP32, n, n, src, dst, None, BUILD_FLAGS)
    Pb = PageRankProblem(ctxb, ATb, n, DAMPING, grb.GRB_FP32, grb.GRB_FP64, "uniform")
    Pb.run(-1.0, 5, "host")
    unfused_runs = []
    for _ in range(3):
        ub0 = grb.grb_context_stats(ctxb)["kernel_launches"]
        e0.record(stream)
        Pb.run(-1.0, ITERS, "host")
        e1.record(stream)
        torch.cuda.synchronize()
        unfused_runs.append(e0.elapsed_time(e1))
        unfused_launches = grb.grb_context_stats(ctxb)["kernel_launches"] - ub0
    unfused_ms = float(np.median(unfused_runs))
    r_unfused = Pb.rank().astype(np.float64)
    Pb.free()
    grb.grb_free(ATb)
    grb.grb_free(ctxb)

    # -------------------------------------------------------------- e2e
    # through the public API from pinned host COO: the CSR build call takes
    # the HOST arrays and uploads them itself, then 50 fused iterations and
    # the ranks read back into pinned host memory
    e2e_ms = []
    h2d = int(src_pin.numel() * 4 * 2)
    d2h = n * 4
    out_host = torch.empty(n, dtype=torch.float32).pin_memory()
    # the host-side steps are in the timed region here: no garbage-collector
    # pauses inside it
    gc.collect()
    gc.disable()
    for k in range(args.warmup + args.steps):
        barrier()
        t0 = time.perf_counter()
        A2 = grb.grb_matrix_build_csr(ctx, grb.GRB_FP32, n, n, src_pin, dst_pin, None, BUILD_FLAGS)
        P2 = PageRankProblem(ctx, A2, n, DAMPING, grb.GRB_FP32, grb.GRB_FP64, "uniform")
        P2.run(-1.0, ITERS, "device")
        grb.grb_vector_extract_dense(P2.r, grb.GRB_FP32, out=out_host, present=False)
        barrier()
        dt = time.perf_counter() - t0
        P2.free()
        grb.grb_free(A2)
        if k >= args.warmup:
            e2e_ms.append(dt * 1e3)
    gc.enable()
    e2e_t = _max_over_ranks(sum(e2e_ms) / len(e2e_ms))
    grb.grb_free(AT)
    grb.grb_free(ctx)

    # the extension legs are single-GPU measurements: with several ranks only
    # the replicated main metric runs, so the N GPUs are held no longer
    legs = ws == 1
    mixed_leg = mixed_leg26 = None
    if legs and not args.no_mixed:
        mixed_leg = run_mixed_leg(grb, torch, stream, 24, (1, 2, 0))
        mixed_leg26 = run_mixed_leg(grb, torch, stream, 26, (1, 0))
    ppr_leg = run_ppr_leg(grb, torch, stream) if legs and not args.no_ppr else None
    serve_leg = run_serve_leg(grb) if legs and not args.no_serve else None
    batch_leg = run_batch_leg(grb, torch, stream) if legs and not args.no_batch else None

    # ---------------------------------------------------------- roofline
    # algorithmic bytes of one launch of the persistent kernel: per body
    # 4(n+1) row_ptr + 4m col_idx + 4n w gathered once + 4n d + 4n r_old +
    # 4n r_new + 4n w_new + n/8 sink bits; the prologue reads r_0, d, the
    # sink bits and writes w_0.
    body_bytes = 4 * (n + 1) + 4 * m + 4 * n * 5 + n // 8
    launch_bytes = ITERS * body_bytes + 12 * n + n // 8
    peak, peak_kind = _peaks()
    kernel_ms = sum(kernel_ms_steps) / len(kernel_ms_steps)
    achieved = launch_bytes / (kernel_ms * 1e-3) / 1e9
    # the operation's own minimum per body: B = 4m + 20n + 4 (col_idx once; r_old, r, w_old, w, d once each; the residual)
    min_bytes = ITERS * (4 * m + 20 * n + 4)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": _traffic_per_launch(), "peak_source": peak_kind,
                "kernel": "pr_persistent_kernel<float,float,768,1,0> (degree-ordered matrix, shared-memory hot "
                          "copy, gathers one tile deep)",
                "kernel_ms_per_launch": kernel_ms,
                "kernel_ms_min_median_max": [min(kernel_ms_steps), float(np.median(kernel_ms_steps)),
                                             max(kernel_ms_steps)],
                "algorithmic_bytes_per_launch": launch_bytes,
                "frac_of_nominal_8tbs": achieved / 8000.0,
                "frac_min_bytes_4m_20n": min_bytes / (kernel_ms * 1e-3) / 1e9 / peak}

    out = {
        "metric": METRIC, "value": value, "unit": "GTEPS", "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "n": n, "m": m, "iterations": ITERS,
                   "timing": "CUDA events on the launching stream; inputs larger than L2 (CSR 0.29 GB)",
                   "parallelism": "replicas" if ws > 1 else "1 GPU"},
        # the extension legs first (long), the main step's evidence last
        "mixed_er24": mixed_leg,
        "mixed_er26": mixed_leg26,
        "batched_ppr_rmat20_k64": ppr_leg,
        "serving_rmat24": serve_leg,
        "graph_batch_512": batch_leg,
        "vertex_order": ("device loops run on a copy of A^T with vertices numbered by descending out-degree, "
                         "built once per matrix inside the library (cost in e2e); ranks are permuted in and out "
                         "inside the timed step"),
        "wall_s_timed_region": t_wall,
        "clocks": clocks,
        "gpu_launches": launches,
        "e2e": {"value": _job_gteps(ws, m, ITERS, e2e_t), "unit": "GTEPS", "ms_per_step": e2e_t,
                "step_ms_min_median_max": [min(e2e_ms), float(np.median(e2e_ms)), max(e2e_ms)],
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "includes": "grb_matrix_build_csr on the pinned HOST COO arrays (the library uploads them), "
                            "GPU CSR build, setup, 50 fused iterations, rank read-back into pinned memory"},
        "roofline": roofline,
        "step_ms_min_median_max": [min(step_ms), float(np.median(step_ms)), max(step_ms)],
        "fused_graph_ms": graph_ms,
        "fused_persistent_input_order_ms": input_order_ms,
        "fused_per_wait_host_loop_ms": perwait_ms,
        "residual_after_50": rdiff,
        "unfused_gpu_launches": unfused_launches,
        "unfused_op_by_op_ms_runs": unfused_runs,
        "unfused_op_by_op_ms": unfused_ms,
        "fused_persistent_ms": ms,
        "fused_vs_unfused": unfused_ms / ms,
    }
    if ws == 1 and not args.no_oracle:   # the CPU baseline: one process, N = 1 only
        import oracle

        t0 = time.perf_counter()
        ptr, col = oracle.build_at(n, src, dst)
        outdeg = oracle.out_degree(ptr, col)
        t_build = time.perf_counter() - t0
        t0 = time.perf_counter()
        ref, _, ref_hist = oracle.pagerank(ptr, col, outdeg, damping=DAMPING, tol=-1.0, itermax=ITERS,
                                           mode="uniform")
        t_pr = time.perf_counter() - t0
        cores = oracle.par_threads()
        t0 = time.perf_counter()
        ref_par, _, _ = oracle.pagerank_par(ptr, col, outdeg, damping=DAMPING, tol=-1.0, itermax=ITERS,
                                            mode="uniform")
        t_par = time.perf_counter() - t0
        out["l1_unfused_vs_fp64"] = float(np.sum(np.abs(r_unfused - ref)))
        out["l1_vs_fp64"] = float(np.sum(np.abs(r_fused - ref)))
        out["cpu_baseline"] = {"value": m * ITERS / t_pr / 1e9, "unit": "GTEPS", "cores": 1, "kind": "oracle",
                               "sample": f"the FP64 oracle's 50 iterations on the same graph ({t_pr:.1f} s; its "
                                         f"CSR build, {t_build:.1f} s, untimed)",
                               "all_cores": {"value": m * ITERS / t_par / 1e9, "unit": "GTEPS", "cores": cores,
                                             "kind": "oracle, OpenMP over rows",
                                             "sample": f"the same 50 iterations ({t_par:.1f} s), max-abs "
                                                       f"{float(np.max(np.abs(ref_par - ref))):.1e} from the "
                                                       f"one-core oracle"}}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
