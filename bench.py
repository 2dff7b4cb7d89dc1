"""Benchmark of the PAKR expansion hot path on one or more GB300s.

One step = one ``pakr_expand`` (sample, cost-pruned NN, propagate + collide,
append) of the 3D double-integrator workload: 6D state, 50 random boxes,
1024 parents x 8 controls = 8192 rollouts, tree prefilled to 1,000,000 nodes
(cap 2^20).  Before each timed step the tree is truncated back to 1,000,000
nodes and L2 is flushed (a 256 MB write), so every step does the same work
from DRAM.

Printed JSON line: tree expansions/s (rollouts per second) over all ranks, the
rooflines of the nearest-neighbour kernel (tensor bound) and of the
propagate-collide kernel (FP32 ALU bound), the e2e rate through the C ABI with
the per-step info read back to the host, p50 time to first solution and the
AO-x cost after 100 ms on the three planning workloads (with a cost-vs-time
curve), the batched, adjoint and refinement measurements, a reduced Table 4
sweep, expansions/s on a tree from real growth, the CPU oracle timed on a bounded sample (one thread and all host
cores), and clocks.  Everything that runs the oracle sits in the CPU leg at
the end (timing, and the oracle's checks of gradients and paths).

``--impl reference`` times the FP64 CPU oracle on the same workload instead.
Multi-GPU (torchrun): independent replicas, one per GPU, weak scaling.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "di3"
N_PREFILL = 1_000_000
METRIC = "tree expansions/s"
UNIT = "rollouts/s"
WORKLOAD_DESC = ("3D double integrator (6D state, pos [0,1]^3, vel [-1,1]^3, accel [-1,1]^3), RK4 dt=0.05, "
                 "1-20 substeps per edge, 50 random boxes, B=1024 parents x k=8 controls = 8192 rollouts per "
                 "expansion, tree cap 2^20 prefilled to 1,000,000 uniform nodes, cost bound +inf")


def _dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(local_units, local_seconds, group=None):
    """Whole-job throughput: units summed over ranks / the slowest rank's time."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized():
        return local_units / local_seconds, local_seconds, local_units
    dev = "cuda" if dist.get_backend(group) == "nccl" else "cpu"
    t = torch.tensor([local_seconds], dtype=torch.float64, device=dev)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    dist.all_reduce(u, op=dist.ReduceOp.SUM, group=group)
    return u.item() / t.item(), t.item(), u.item()


class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.th.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# dram__bytes_read.sum + dram__bytes_write.sum of one tensor-core nearest-neighbour launch
# (k_nn_tc) on the bench workload (n = 1,000,000 nodes, d = 6), from the ncu capture named in
# NN_DRAM_SOURCE.  None when the kernel has changed since that capture.
NN_DRAM_BYTES_NCU = 36.885248e6 + 3584.0
NN_DRAM_SOURCE = ("profiles/k_nn_tc_di3_n1M.md, current kernel (FP16 operands, CTA-wide resolve, paired "
                  "chunks, suspending waits in every role, readers two tiles per trip): "
                  "dram__bytes_read.sum + dram__bytes_write.sum of one launch")

# Bytes of the planner's device control block that pakr_expand and pakr_plan read back.
CTL_BYTES = 216

# Nominal dense FP16 / BF16 tensor throughput ratio (both 2.25 PFLOP/s): the FP16 peak is the
# measured BF16 GEMM rate.
FP16_PER_BF16 = 1.0


def nn_flops_per_launch(K, n, d):
    """Algorithmic work of one nearest-neighbour pass, the method's own count: a subtract,
    a multiply and an add per coordinate of every (query, node) pair."""
    return 3.0 * K * n * d


def nn_tc_filter_flops_per_launch(K, n, d, kt):
    """Tensor-core work of the filter as the kernel forms it: per (query, node) pair kt
    FP16 multiply-adds (the hi/lo partial products and the two |x|^2 columns)."""
    return 2.0 * K * n * kt


def nn_tc_mma_flops_per_launch(K, n, d, kt, mma_steps):
    """Tensor-core work as issued: queries padded to 128-row blocks, nodes to 256-node
    tiles, mma_steps MMAs of K = 16 per 128 x 128 block."""
    return 2.0 * (-(-K // 128) * 128) * (-(-n // 256) * 256) * 16 * mma_steps


def tc_shape(d):
    """(columns of the packed node row, MMA k-steps per 128-node stage) of k_nn_tc: FP16
    operands, K = 16 per MMA; the split layout (x_hi, x_lo, |x|^2 hi, lo) with a second query
    operand against the x_hi columns where it stores fewer columns without more MMAs
    (d = 5, 6, 12), else (x_hi, x_lo, x_hi, |x|^2 hi, lo) (d = 3, 4)."""
    r16 = lambda c: (c + 15) // 16 * 16
    joint, split, ka2 = r16(3 * d + 2), r16(2 * d + 2), r16(d)
    if split < joint and split // 16 + ka2 // 16 <= joint // 16:
        return split, split // 16 + ka2 // 16
    return joint, joint // 16


def nn_uses_tensor_cores(spec, n):
    """Whether the planner's default nearest-neighbour choice (nn_mode auto) takes the
    tensor-core kernel for a tree of n nodes."""
    mode = spec.get("nn_mode", 0)
    if mode == 2:
        return True
    return mode == 0 and spec["K"] >= 256 and n >= 28672


# Algorithmic FP32 work of one propagate-collide substep (an FMA counts 2, an add, multiply or
# compare 1): the RK4 combination (3 stage points and 3 accumulations of d FMAs, a final add and
# FMA of d: 15 d), four evaluations of the dynamics (double integrator 0; quadrotor 77 flops
# and 3 sincos at 20 each, 137), the state-box test (2 d compares), the obstacle tests (2 pdim
# compares per box), the path-length increment (10) and the heuristic with the prune test (10).
F_EVAL_FLOPS = {"di2": 0, "di3": 0, "quad12": 137}


def propagate_flops_per_substep(spec):
    d, pdim = spec["d"], spec["pdim"]
    n_obs = len(spec["boxes"]) + len(spec["spheres"])
    return 15 * d + 4 * F_EVAL_FLOPS[spec["name"]] + 2 * d + 2 * pdim * n_obs + 10 + 10


def nn_bytes_per_launch(n, d):
    """Algorithmic DRAM bytes: every node's d coordinates and its f-cost, once."""
    return 4.0 * n * (d + 1)


# ---- the CPU leg: the FP64 oracle as it stands, on the host cores --------------------------
_ORA = {}


def _ora_init(workload, n_prefill, tree_seed):
    """Pool worker set-up: the oracle problem and the prefilled tree, once per process."""
    import oracle
    from paper_2607_03987_gb300 import workloads as W

    spec = W.problem(workload, env_seed=0)
    tree = W.prefilled_tree(spec, n_prefill, seed=tree_seed)
    _ORA["spec"] = spec
    _ORA["tree"] = oracle.OracleTree.from_arrays(spec["d"], spec["m"], spec["cap"], tree["states"],
                                                 tree["controls"], tree["parents"], tree["costs"], tree["steps"])
    _ORA["n"] = n_prefill


def _ora_expand(args):
    """One oracle expansion with K parents from the prefilled tree; (rollouts, seconds)."""
    import oracle
    from paper_2607_03987_gb300 import workloads as W

    K, seed = args
    s = W.with_sizes(_ORA["spec"], K=K)
    prob = oracle.OracleProblem(s)
    prob.set_goal(s["x_goal"])
    ot = _ORA["tree"]
    ot.T.count = _ORA["n"]
    t0 = time.perf_counter()
    oracle.expand(prob, ot, np.inf, seed)
    return K * s["k"], time.perf_counter() - t0


def oracle_pool(workers, tree_seed):
    """A process pool (spawn: no process is forked from one that holds a CUDA context) whose
    workers each hold the oracle's copy of the benchmark tree."""
    import multiprocessing as mp

    ctx = mp.get_context("spawn")
    pool = ctx.Pool(workers, initializer=_ora_init, initargs=(WORKLOAD, N_PREFILL, tree_seed))
    pool.map(_ora_expand, [(1, 0)] * workers)  # every worker has built its tree
    return pool


def cpu_baseline(spec, tree_seed, seed, target_s=10.0):
    """The FP64 oracle as it stands on a bounded sample of the workload: expansions with fewer
    parents on the same 1,000,000-node tree, single-threaded and then one process per host
    core (each expanding its own sample concurrently); about target_s of CPU work each."""
    cores = os.cpu_count() or 1
    pool = oracle_pool(cores, tree_seed)
    try:
        K0 = 16
        r0, t0 = pool.apply(_ora_expand, ((K0, seed),))
        K1 = int(max(K0, min(spec["K"], K0 * target_s / max(t0, 1e-3))))
        r1, t1 = pool.apply(_ora_expand, ((K1, seed),))
        single = r1 / t1
        w0 = time.perf_counter()
        res = pool.map(_ora_expand, [(K1, seed + 1 + w) for w in range(cores)], chunksize=1)
        wall = time.perf_counter() - w0
    finally:
        pool.close()
        pool.join()
    rollouts = sum(r for r, _ in res)
    return {"value": rollouts / wall, "unit": UNIT, "cores": cores, "kind": "oracle",
            "single_thread_value": single,
            "sample": f"{cores} processes (all host cores), each one expansion with {K1} of {spec['K']} parents x "
                      f"{spec['k']} controls on the same {N_PREFILL}-node tree ({rollouts} rollouts in {wall:.1f} s "
                      f"wall); single-threaded: {r1} rollouts in {t1:.1f} s, FP64"}


def oracle_checks(pending):
    """The oracle's checks of results the GPU measurements produced (run in the CPU leg):
    relative error of sampled adjoint gradients against the FP64 reverse mode, and an FP64
    replay of every plain and refined AO-x path (valid at every substep, continuous misses of
    the substep check counted exactly for the double integrator, in the goal ball, length)."""
    import oracle
    from paper_2607_03987_gb300 import refine

    out = {}
    adj = pending.get("adjoint")
    if adj:
        spec = adj["spec"]
        prob = oracle.OracleProblem(spec)
        prob.set_goal(spec["x_goal"])
        w = dict(refine.DEFAULT_WEIGHTS)
        ow = oracle.traj_params(w_dur=w["w_duration"], w_u=w["w_control"], w_obs=w["w_obstacle"], beta=w["beta"],
                                margin=w["margin"], w_goal=w["w_goal"], w_len=w["w_length"], len_eps=w["length_eps"])
        errs = []
        for x0, U, dU in adj["samples"]:
            _, dUo, _ = oracle.traj_grad(prob, x0, U, ow)
            errs.append(float(np.abs(dU - dUo).max() / np.abs(dUo).max()))
        out["adjoint"] = {"max_rel_grad_error_vs_fp64_oracle": max(errs), "sampled_sequences": len(errs)}
    for key, paths in pending.get("paths", {}).items():
        spec = paths["spec"]
        prob = oracle.OracleProblem(spec)
        prob.set_goal(spec["x_goal"])
        summary = {}
        for kind in ("plain", "refined"):
            n = valid = in_goal = misses = edges = exempt = 0
            for x0, U, steps, length in paths[kind]:
                x = np.asarray(x0, np.float64)
                g, ok = 0.0, True
                for e in range(len(steps)):
                    u = np.asarray(U[e], np.float64)
                    r = oracle.propagate(prob, x, g, u, int(steps[e]))
                    if r["collided"]:
                        if r["face_margin"] < 1e-5:
                            exempt += 1
                        else:
                            ok = False
                    elif oracle.di_edge_hits_exact(prob, x, u, int(steps[e])):
                        misses += 1
                    x, g = r["x_end"], r["cost_end"]
                    edges += 1
                n += 1
                valid += ok
                pd = spec["pdim"]
                in_goal += bool(np.linalg.norm(x[:pd] - spec["x_goal"][:pd]) <= spec["goal_r"])
            summary[kind] = {"paths": n, "valid_at_every_substep": valid, "in_goal": in_goal, "edges": edges,
                             "face_exempt_edges": exempt, "continuous_misses": misses}
        out[key] = summary
    return out


def table4_sweep(dev, stream, trials=20, budget_s=1.0):
    """Batch size and branching factor sensitivity on the 12D quadrotor
    (Table 4): for batch B in {4k, 8k, 16k, 32k} rollouts and branching
    factor A in {2, 16, 64, 128}, K = B / A parents per expansion.  Each
    trial plans from a fresh tree to the first solution with the device AO-x
    graph (budget_s per trial, seeds 0..trials-1); reported per cell: success
    rate, median device time to the first solution, median expansions and
    median tree size at that moment, and the median time per expansion
    iteration (the rate the sweep compares across hardware)."""
    from paper_2607_03987_gb300 import pakr
    from paper_2607_03987_gb300 import workloads as W

    out = []
    for B in (4096, 8192, 16384, 32768):
        for A in (2, 16, 64, 128):
            spec = W.problem("quad12", env_seed=0, K=B // A, k=A)
            planner = pakr.Planner(spec, device=dev, stream=stream)
            planner.plan(spec["x_init"], spec["x_goal"], budget_s=0.2, seed=999, stop_at_first=True)
            t_ms, iters, nodes, per_it, solved = [], [], [], [], 0
            for sd in range(trials):
                r = planner.plan(spec["x_init"], spec["x_goal"], budget_s=budget_s, seed=sd, stop_at_first=True)
                if r["n_solutions"]:
                    solved += 1
                    t_ms.append(r["t_first_solution_s"] * 1e3)
                    iters.append(r["iterations_first_solution"])
                    nodes.append(r["nodes_first_solution"])
                    per_it.append(r["t_first_solution_s"] * 1e3 / max(r["iterations_first_solution"], 1))
            planner.close()
            med = (lambda v: float(np.median(v)) if v else None)
            out.append({"batch": B, "branching": A, "parents": B // A, "success": solved / trials,
                        "time_ms_p50": med(t_ms), "iterations_p50": med(iters), "nodes_p50": med(nodes),
                        "ms_per_iteration_p50": med(per_it)})
    return {"workload": "12D quadrotor, 100-pillar forest, hover (0.1,0.1,0.5) -> goal ball (0.9,0.9,0.5) "
                        "r=0.05, cap 4M, plan to the first solution", "trials": trials, "budget_s": budget_s,
            "cells": out}


def tree_size_sweep(dev, stream, steps=10, warmup=3):
    """Expansions/s at fixed tree sizes: the paper's tier sizes 4^6..4^10 for the
    3D double integrator, and up to 4,000,000 nodes for the 12D quadrotor
    (4096 parents x 16 controls), each tree prefilled uniformly, L2 flushed
    before every timed step."""
    import torch

    from paper_2607_03987_gb300 import pakr
    from paper_2607_03987_gb300 import workloads as W

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")
    out = []
    cases = [("di3", [4 ** 6, 4 ** 7, 4 ** 8, 4 ** 9, 4 ** 10 - 8192], {}),
             ("quad12", [4 ** 6, 4 ** 8, 4 ** 10, 4_000_000 - 65536], {})]
    for name, sizes, over in cases:
        spec = W.problem(name, env_seed=0, **over)
        tree = W.prefilled_tree(spec, max(sizes), seed=3)
        planner = pakr.Planner(spec, device=dev, stream=stream)
        planner.tree_import(tree, spec["x_goal"])
        R = spec["K"] * spec["k"]
        for n in sorted(sizes, reverse=True):  # truncation only shrinks the tree: largest size first
            for w in range(warmup):
                planner.tree_truncate(n)
                planner.expand(np.inf, 900 + w, info=False)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            for s_, (a, b) in enumerate(ev):
                planner.tree_truncate(n)
                flush.zero_()
                a.record(stream)
                planner.expand(np.inf, s_, info=False)
                b.record(stream)
            torch.cuda.synchronize(dev)
            ms = sum(a.elapsed_time(b) for a, b in ev) / steps
            planner.set_profiling(True)  # per-kernel times: a second pass with per-launch events
            for s_ in range(steps):
                planner.tree_truncate(n)
                flush.zero_()
                planner.expand(np.inf, 500 + s_, info=False)
            kt = planner.kernel_times()
            planner.set_profiling(False)
            nk = "k_nn_tc" if nn_uses_tensor_cores(spec, n) else "k_nn"
            nn_ms = kt[nk]["ms"] / max(kt[nk]["launches"], 1)
            out.append({"workload": name, "n": n, "parents": spec["K"], "branching": spec["k"],
                        "rollouts_per_s": R / (ms * 1e-3), "ms_per_step": ms,
                        "nn_ms": nn_ms, "nn_tflops": nn_flops_per_launch(spec["K"], n, spec["d"]) / (nn_ms * 1e-3) / 1e12,
                        "propagate_ms": kt["k_propagate"]["ms"] / max(kt["k_propagate"]["launches"], 1),
                        "append_ms": kt["k_append"]["ms"] / max(kt["k_append"]["launches"], 1),
                        "sample_ms": kt["k_sample"]["ms"] / max(kt["k_sample"]["launches"], 1)})
        planner.close()
        out.sort(key=lambda r: (r["workload"], r["n"]))
        del tree
    return out


def grown_tree_expansions(dev, stream, steps=10, warmup=3, max_expansions=600):
    """Expansions/s on a snapshot of a tree from real growth (the other fixed-size trees are
    prefilled uniformly): the benchmark workload's tree grown from the start by plain
    expansions under an infinite bound until it holds N_PREFILL nodes, then expanded from its
    first N_PREFILL nodes (truncated back before every step, L2 flushed before every timed
    step), as in the tree-size sweep."""
    import torch

    from paper_2607_03987_gb300 import pakr
    from paper_2607_03987_gb300 import workloads as W

    spec = W.problem(WORKLOAD, env_seed=0)
    R = spec["K"] * spec["k"]
    planner = pakr.Planner(spec, device=dev, stream=stream)
    try:
        planner.tree_reset(spec["x_init"], spec["x_goal"])
        n, grown = 1, 0
        while n < N_PREFILL and grown < max_expansions:
            planner.expand(np.inf, 70_000 + grown, info=False)
            grown += 1
            n, _ = planner.tree_size()
        if n < N_PREFILL:
            return {"workload": WORKLOAD, "error": f"the tree reached {n} nodes in {grown} expansions"}
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")
        for w in range(warmup):
            planner.tree_truncate(N_PREFILL)
            planner.expand(np.inf, 900 + w, info=False)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for s_, (a, b) in enumerate(ev):
            planner.tree_truncate(N_PREFILL)
            flush.zero_()
            a.record(stream)
            planner.expand(np.inf, s_, info=False)
            b.record(stream)
        torch.cuda.synchronize(dev)
        ms = sum(a.elapsed_time(b) for a, b in ev) / steps
        planner.set_profiling(True)  # per-kernel times: a second pass with per-launch events
        for s_ in range(steps):
            planner.tree_truncate(N_PREFILL)
            flush.zero_()
            planner.expand(np.inf, 500 + s_, info=False)
        kt = planner.kernel_times()
        planner.set_profiling(False)
        nk = "k_nn_tc" if nn_uses_tensor_cores(spec, N_PREFILL) else "k_nn"
        nn_ms = kt[nk]["ms"] / max(kt[nk]["launches"], 1)
        return {"workload": WORKLOAD, "n": N_PREFILL, "grown_in_expansions": grown, "parents": spec["K"],
                "branching": spec["k"], "rollouts_per_s": R / (ms * 1e-3), "ms_per_step": ms, "nn_kernel": nk,
                "nn_ms": nn_ms,
                "nn_tflops": nn_flops_per_launch(spec["K"], N_PREFILL, spec["d"]) / (nn_ms * 1e-3) / 1e12,
                "propagate_ms": kt["k_propagate"]["ms"] / max(kt["k_propagate"]["launches"], 1),
                "append_ms": kt["k_append"]["ms"] / max(kt["k_append"]["launches"], 1),
                "sample_ms": kt["k_sample"]["ms"] / max(kt["k_sample"]["launches"], 1),
                "tree": "the first 1,000,000 nodes of a tree grown from the start by plain expansions under an "
                        "infinite bound (the same problem, 1024 parents x 8 controls per expansion)"}
    finally:
        planner.close()


def batched_vs_sequential(dev, stream, n_queries=256, seed=4242, max_iterations=2000, budget_s=20.0):
    """Queries solved per second: 256 independent 3D double-integrator queries
    (obstacles U{10..200}, tree caps U[64k, 1M], random start / goal pairs),
    each planned to its first solution, as one autotuned persistent launch
    (pakr_batch_plan under a CUDA graph) vs one pakr_plan call per query."""
    import torch

    from paper_2607_03987_gb300 import pakr
    from paper_2607_03987_gb300 import workloads as W

    base, queries = W.batch_queries(n_queries, env_seed=0)
    bp = pakr.BatchPlanner(base, queries, device=dev, stream=stream)
    tuning = bp.autotune(iterations=3, seed=1)
    bp.plan(budget_s=budget_s, max_iterations=max_iterations, seed=seed + 1, stop_at_first=True)  # warm-up
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    rb = bp.plan(budget_s=budget_s, max_iterations=max_iterations, seed=seed, stop_at_first=True)
    t_batch = time.perf_counter() - t0
    bp.close()
    planners = []
    for q in queries:
        spec = W.with_sizes(base, boxes=q["boxes"], spheres=q["spheres"], cap=q["cap"], x_init=q["x_init"],
                            x_goal=q["x_goal"])
        pl = pakr.Planner(spec, device=dev, stream=stream)
        pl.plan(q["x_init"], q["x_goal"], budget_s=budget_s, max_iterations=2, seed=1)  # builds the graph
        planners.append(pl)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    rs = [pl.plan(q["x_init"], q["x_goal"], budget_s=budget_s, max_iterations=max_iterations, seed=seed + i,
                  stop_at_first=True) for i, (pl, q) in enumerate(zip(planners, queries))]
    t_seq = time.perf_counter() - t0
    for pl in planners:
        pl.close()
    solved_b = sum(1 for r in rb if r["n_solutions"] > 0)
    solved_s = sum(1 for r in rs if r["n_solutions"] > 0)
    same = all(a["iterations"] == b["iterations"] and (a["cost"] == b["cost"] or (a["n_solutions"] == 0 and
                                                                                b["n_solutions"] == 0))
               for a, b in zip(rb, rs))
    iters = [r["iterations"] for r in rb]
    return {"queries": n_queries, "batched_queries_per_s": n_queries / t_batch,
            "sequential_queries_per_s": n_queries / t_seq, "speedup": t_seq / t_batch,
            "batched_s": t_batch, "sequential_s": t_seq, "solved_batched": solved_b, "solved_sequential": solved_s,
            "identical_results": bool(same), "iterations_p50": float(np.median(iters)),
            "iterations_max": int(max(iters)), "tuning": tuning,
            "workload": "256 x 3D double integrator, K=1024 x k=8 per query, obstacles U{10..200}, caps "
                        "U[64k,1M], random start/goal pairs, plan to first solution; host wall clock including "
                        "launch and result read-back"}


def adjoint_bench(dev, stream, T=1024, N=200, reps=20):
    """Smooth-cost gradient of 1024 quadrotor control sequences of 200 RK4
    steps over the 100-pillar forest (adjoint RK4, checkpoints every 16
    steps): forward and gradient time, and the largest relative gradient error
    against the FP64 oracle's reverse mode on a sample of sequences."""
    import torch

    from paper_2607_03987_gb300 import pakr, refine
    from paper_2607_03987_gb300 import workloads as W

    spec = W.with_sizes(W.problem("quad12", env_seed=0), K=1, k=1, cap=16)
    planner = pakr.Planner(spec, device=dev, stream=stream)
    rng = np.random.default_rng(0)
    x0 = np.zeros((T, 12), np.float32)
    x0[:, :3] = rng.uniform(0.1, 0.9, (T, 3))
    x0[:, 6:9] = rng.uniform(-0.2, 0.2, (T, 3))
    U = np.concatenate([9.81 + rng.normal(0, 0.5, (T, N, 1)), rng.uniform(-0.002, 0.002, (T, N, 3))],
                       axis=2).astype(np.float32)
    w = dict(refine.DEFAULT_WEIGHTS)
    Ut = torch.tensor(U, device=f"cuda:{dev}")
    xt = torch.tensor(x0, device=f"cuda:{dev}")
    cost = torch.empty(T, device=f"cuda:{dev}")
    dU = torch.empty_like(Ut)
    dx = torch.empty_like(xt)
    nck = pakr.lib().pakr_traj_checkpoint_floats(planner.h, T, N)
    ck = torch.empty(int(nck), device=f"cuda:{dev}")
    prm = refine._params(w)
    g, gp = refine._goal(spec["x_goal"])
    import ctypes as C

    def fwd():
        pakr._check(pakr.lib().pakr_traj_cost(planner.h, C.c_void_p(xt.data_ptr()), C.c_void_p(Ut.data_ptr()), T, N,
                                              gp, C.byref(prm), C.c_void_p(cost.data_ptr()), None), "cost")

    def grad():
        pakr._check(pakr.lib().pakr_traj_grad(planner.h, C.c_void_p(xt.data_ptr()), C.c_void_p(Ut.data_ptr()), T, N,
                                              gp, C.byref(prm), None, C.c_void_p(dU.data_ptr()),
                                              C.c_void_p(dx.data_ptr()), C.c_void_p(ck.data_ptr())), "grad")

    for _ in range(3):
        fwd()
        grad()
    times = {}
    for name, fn in (("cost_ms", fwd), ("grad_ms", grad)):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize(dev)
        times[name] = a.elapsed_time(b) / reps
    dUh = dU.cpu().numpy()
    # sampled sequences for the oracle's check in the CPU leg
    samples = [(x0[t].copy(), U[t].copy(), dUh[t].copy()) for t in range(0, T, T // 8)]
    planner.close()
    pending = {"spec": spec, "samples": samples}
    return {"sequences": T, "steps": N, "checkpoint_every": 16, **times,
            "gradients_per_s": T / (times["grad_ms"] * 1e-3),
            "workload": "12D quadrotor, dt 0.02, 100 pillars, hover thrust + N(0,0.5), torques U[-0.002,0.002]; "
                        "cost = duration + 0.1 |u|^2 + softplus(50 (-sdf)) penalty + goal error"}, pending


def refined_vs_plain(dev, stream, budget_s=0.1, seeds=10, n_boxes=50):
    """AO-x path cost after the same wall-clock budget: plain pakr_plan vs the same AO-x run
    (same seed, same random numbers) with gradient refinement beside it (refine.refined_aox_live:
    the run's best path is read while it runs, refined on a second stream, and a shorter refined
    path is offered to the running loop as its bound).  The paths of both are kept for the
    oracle's re-check in the CPU leg."""
    import torch

    from paper_2607_03987_gb300 import pakr, refine
    from paper_2607_03987_gb300 import workloads as W

    spec = W.problem("di3", env_seed=0, n_boxes=n_boxes)
    # the refinement's stream at high priority: its kernel takes the next free SM slot
    s_plan, s_side = torch.cuda.Stream(dev), torch.cuda.Stream(dev, priority=-1)
    planner = pakr.Planner(spec, device=dev, stream=s_plan)
    ref_planner = pakr.Planner(W.with_sizes(spec, K=1, k=1, cap=16), device=dev, stream=s_side)
    refine.refined_aox_live(planner, ref_planner, spec, 0.05, seed=999)  # warm-up (graphs, torch kernels)
    plain, refined, gains, t_plain, t_ref = [], [], [], [], []
    pending = {"spec": spec, "plain": [], "refined": []}
    for sd in range(seeds):
        t0 = time.perf_counter()
        r = planner.plan(spec["x_init"], spec["x_goal"], budget_s=budget_s, seed=sd)
        t_plain.append(time.perf_counter() - t0)
        plain.append(float(r["cost"]))
        if r["n_solutions"]:
            pending["plain"].append((r["states"][0], r["controls"], r["steps"], float(r["cost"])))
        t0 = time.perf_counter()
        c, gain, best = refine.refined_aox_live(planner, ref_planner, spec, budget_s, seed=sd)
        t_ref.append(time.perf_counter() - t0)
        refined.append(c)
        gains.append(gain)
        if best is not None:
            pending["refined"].append((best["x0"], best["controls"], best["steps"], c))
    planner.close()
    ref_planner.close()
    lb = float(np.linalg.norm(spec["x_goal"][:3] - spec["x_init"][:3]) - spec["goal_r"])
    return {"budget_s": budget_s, "seeds": seeds, "plain_cost_p50": float(np.median(plain)),
            "refined_cost_p50": float(np.median(refined)), "refined_lower_in": int(sum(a < b for a, b in
                                                                                     zip(refined, plain))),
            "plain_costs": plain, "refined_costs": refined, "refinement_gain_p50": float(np.median(gains)),
            "wall_s_p50": {"plain": float(np.median(t_plain)), "refined": float(np.median(t_ref))},
            "straight_line_lower_bound": lb,
            "workload": f"di3 (3D double integrator, {n_boxes} boxes, path-length cost), host wall-clock budget "
                        f"per seed; refinement on a second stream beside the AO-x loop"}, pending


def planning_metrics(dev, stream, name, ttfs_trials, aox_trials, rank=0, aox_budget_s=0.1):
    """Paper Tables 1-2 analogues on one planning workload: p50 time to the first solution
    (device AO-x graph stopped at the first solution; device clock, and host wall clock through
    pakr_plan), and the AO-x best cost after a 100 ms device-time budget with its cost-vs-time
    curve (the median over seeds of the best cost found by each time; Fig. 2 analogue)."""
    from paper_2607_03987_gb300 import pakr
    from paper_2607_03987_gb300 import workloads as W

    spec = W.problem(name, env_seed=0)
    planner = pakr.Planner(spec, device=dev, stream=stream)
    planner.plan(spec["x_init"], spec["x_goal"], budget_s=1.0, seed=12345, stop_at_first=True)  # builds the graph
    ttfs_dev, ttfs_host, iters, solved = [], [], [], 0
    d2h = []
    for sd in range(ttfs_trials):
        t0 = time.perf_counter()
        r = planner.plan(spec["x_init"], spec["x_goal"], budget_s=2.0, seed=sd + 1000 * rank, stop_at_first=True)
        th = time.perf_counter() - t0
        if r["n_solutions"]:
            solved += 1
            ttfs_dev.append(r["t_first_solution_s"] * 1e3)
            ttfs_host.append(th * 1e3)
            iters.append(r["iterations_first_solution"])
            ne = r["n_edges"]
            d2h.append(CTL_BYTES + 20 + (ne + 1) * spec["d"] * 4 + ne * (spec["m"] * 4 + 4))
    grid_ms = [1, 2, 5, 10, 20, 50, 100]
    costs, n_sol, curves = [], [], []
    for sd in range(aox_trials):
        r = planner.plan(spec["x_init"], spec["x_goal"], budget_s=aox_budget_s, seed=sd + 1000 * rank)
        costs.append(float(r["cost"]))
        n_sol.append(r["n_solutions"])
        ht = np.asarray(r["history_time_s"]) * 1e3
        hc = np.asarray(r["history_cost"], np.float64)
        curves.append([float(hc[ht <= t].min()) if np.any(ht <= t) else float("inf") for t in grid_ms])
    planner.close()
    curves = np.asarray(curves)

    def q(v, p):
        return float(np.percentile(v, p)) if len(v) else None

    pd = spec["pdim"]
    lb = float(np.linalg.norm(spec["x_goal"][:pd] - spec["x_init"][:pd]) - spec["goal_r"])
    finite = [c for c in costs if np.isfinite(c)]
    return {
        "workload": f"{name}: {spec['K']} parents x {spec['k']} controls, cap {spec['cap']}, "
                    f"{len(spec['boxes'])} boxes, fresh tree from the start to the goal ball r={spec['goal_r']:.2f}",
        "time_to_first_solution_ms": {"p25": q(ttfs_dev, 25), "p50": q(ttfs_dev, 50), "p75": q(ttfs_dev, 75),
                                      "host_p50": q(ttfs_host, 50), "iterations_p50": q(iters, 50),
                                      "trials": ttfs_trials, "success_rate": solved / max(ttfs_trials, 1)},
        "aox_path_cost_at_100ms": {"p25": q(finite, 25), "p50": float(np.median(costs)) if costs else None,
                                   "p75": q(finite, 75), "solved": len(finite), "trials": aox_trials,
                                   "solutions_p50": q(n_sol, 50), "straight_line_lower_bound": lb},
        "cost_vs_time_ms": {"t_ms": grid_ms, "best_cost_p50": [float(np.median(curves[:, i])) for i in
                                                              range(len(grid_ms))] if len(curves) else None,
                            "solved_fraction": [float(np.mean(np.isfinite(curves[:, i]))) for i in
                                                range(len(grid_ms))] if len(curves) else None},
        "_e2e_plan": {"host_ms_p50": q(ttfs_host, 50), "d2h_bytes_mean": float(np.mean(d2h)) if d2h else None},
    }


def run_reference(args):
    """The FP64 oracle as it stands on the machine's host cores (one process per core, spawn):
    each step is one round in which every process expands 64 parents of the 1,000,000-node
    tree; the step's rate is all rollouts over the round's wall time."""
    ws, rank, local = _dist_env()
    if rank != 0:
        return 0
    from paper_2607_03987_gb300 import workloads as W

    spec = W.problem(WORKLOAD, env_seed=0)
    K_sample = 64
    cores = os.cpu_count() or 1
    pool = oracle_pool(cores, tree_seed=1)
    try:
        for w in range(args.warmup):
            pool.map(_ora_expand, [(K_sample, 1000 + 64 * w + c) for c in range(cores)], chunksize=1)
        times, rollouts = [], 0
        for st in range(args.steps):
            t0 = time.perf_counter()
            res = pool.map(_ora_expand, [(K_sample, 64 * st + c) for c in range(cores)], chunksize=1)
            times.append(time.perf_counter() - t0)
            rollouts += sum(r for r, _ in res)
    finally:
        pool.close()
        pool.join()
    total = sum(times)
    value = rollouts / total
    sample = (f"each step {cores} processes (all host cores), each one expansion with {K_sample} of {spec['K']} "
              f"parents x {spec['k']} controls on the {N_PREFILL}-node tree, FP64")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="pakr", choices=["pakr", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip the CPU leg (oracle timing and checks)")
    ap.add_argument("--ttfs-trials", type=int, default=100)
    ap.add_argument("--aox-trials", type=int, default=100)
    ap.add_argument("--no-planning", action="store_true", help="skip the planning metrics of the three workloads")
    ap.add_argument("--no-sweep", action="store_true", help="skip the tree-size sweep")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-vs-sequential comparison")
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint and refinement measurements")
    ap.add_argument("--table4-trials", type=int, default=3,
                    help="trials per cell of the batch size x branching factor sweep (Table 4); 0 skips it")
    ap.add_argument("--plain-launches", action="store_true",
                    help="launch each kernel of the timed steps separately (per-kernel profilers cannot see "
                         "kernels inside the expansion graph's conditional nodes)")
    ap.add_argument("--only-expand", action="store_true",
                    help="time the expansion steps only (no e2e, planning metrics or CPU leg)")
    ap.add_argument("--workload", default=WORKLOAD, choices=["di2", "di3", "quad12"],
                    help="with --only-expand: the workload whose expansions are timed")
    ap.add_argument("--n-tree", type=int, default=N_PREFILL,
                    help="with --only-expand: the prefilled tree size")
    args = ap.parse_args()
    if not args.only_expand and (args.workload != WORKLOAD or args.n_tree != N_PREFILL):
        ap.error("--workload and --n-tree apply to --only-expand runs; the full line measures "
                 f"{WORKLOAD} at {N_PREFILL} nodes")
    if args.impl == "reference":
        return run_reference(args)
    assert args.warmup >= 3, "at least 3 warm-up steps"

    import torch
    import torch.distributed as dist

    ws, rank, local = _dist_env()
    if ws > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    dev = local
    torch.cuda.set_device(dev)

    from paper_2607_03987_gb300 import _build, pakr
    from paper_2607_03987_gb300 import workloads as W

    _build.build()
    n_tree = args.n_tree
    spec = W.problem(args.workload, env_seed=0)
    if n_tree + spec["K"] * spec["k"] > spec["cap"]:
        spec = W.with_sizes(spec, cap=n_tree + spec["K"] * spec["k"])
    tree = W.prefilled_tree(spec, n_tree, seed=1 + rank)
    stream = torch.cuda.current_stream(dev)
    planner = pakr.Planner(spec, device=dev, stream=stream)
    planner.tree_import(tree, spec["x_goal"])
    del tree
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{dev}")
    R = spec["K"] * spec["k"]

    def one_step(seed, info=False):
        return planner.expand(np.inf, seed, info=info)

    clocks = ClockSampler(dev).start()  # samples span the warm-up and the timed steps
    for w in range(args.warmup):
        planner.tree_truncate(n_tree)
        one_step(10_000 + w)
    torch.cuda.synchronize(dev)

    # ---- device-timed steps (value): each step is one expansion graph (sample, the nearest-
    # neighbour kernel the tree size selects, propagate, append) ----
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if args.plain_launches:
        planner.set_profiling(True)
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    for s in range(args.steps):
        planner.tree_truncate(n_tree)
        flush.zero_()
        starts[s].record(stream)
        one_step(s)
        ends[s].record(stream)
    torch.cuda.synchronize(dev)
    if ws > 1:
        dist.barrier()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in zip(starts, ends)]
    local_s = sum(step_ms) / 1e3
    value, t_max, units = aggregate(R * args.steps, local_s)
    launches = args.steps * 4  # sample, one nearest-neighbour kernel, propagate, append per step

    # ---- per-kernel device times: a separate pass with per-launch CUDA events ----
    planner.set_profiling(False)
    planner.set_profiling(True)
    substeps = []
    for s in range(min(args.steps, 300)):
        planner.tree_truncate(n_tree)
        flush.zero_()
        one_step(20_000 + s)
        if s < 20:
            dbg = planner.debug_last_expand()
            substeps.append(float(np.sum(dbg["steps"][dbg["outcome"] != pakr.ROLLOUT_NO_PARENT])))
    kt = planner.kernel_times()
    planner.set_profiling(False)
    kernel_ms = {k: v["ms"] / max(v["launches"], 1) for k, v in kt.items()}

    if args.only_expand:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
                              "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps,
                              "kernel_ms_per_step": kernel_ms, "gpu_launches": launches,
                              "config": {"workload": args.workload, "n_tree": n_tree, "parents": spec["K"],
                                         "branching": spec["k"]}}), flush=True)
        planner.close()
        if ws > 1:
            dist.destroy_process_group()
        return 0

    # ---- e2e through the C ABI: per-step info read back to the host ----
    e2e_times, appended = [], []
    for s in range(args.steps):
        planner.tree_truncate(N_PREFILL)
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        st, info = one_step(50_000 + s, info=True)
        e2e_times.append(time.perf_counter() - t0)
        appended.append(info["n_appended"])
    e2e_value, _, _ = aggregate(R * args.steps, sum(e2e_times))
    planner.close()

    # ---- rooflines: nearest neighbour (dominant) and propagate-collide ----
    peaks, peak_src = measured_peaks()
    props = torch.cuda.get_device_properties(dev)
    sm_mhz = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak_tflops = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12
    fp32_src = (f"FP32 FFMA: {props.multi_processor_count} SMs x 128 lanes x 2 flop x {sm_mhz:.0f} MHz "
                f"({peak_src} max SM clock)")
    K, d = spec["K"], spec["d"]
    tc = nn_uses_tensor_cores(spec, N_PREFILL)
    nn_ms = kernel_ms["k_nn_tc" if tc else "k_nn"]
    method_tflops = nn_flops_per_launch(K, N_PREFILL, d) / (nn_ms * 1e-3) / 1e12
    if tc:
        fp16_peak = float(peaks["bf16_tflops"]) * FP16_PER_BF16
        kt_cols, mma_steps = tc_shape(d)
        roofline = {"bound": "tensor", "achieved": method_tflops, "peak": fp16_peak, "unit": "TFLOP/s",
                    "frac": method_tflops / fp16_peak, "traffic": NN_DRAM_BYTES_NCU, "kernel": "k_nn_tc",
                    "work": "3 K n d (a subtract, a multiply and an add per coordinate of every query-node pair), "
                            "the method's own count",
                    "peak_source": f"FP16 dense = {peak_src} BF16 GEMM {float(peaks['bf16_tflops']):.0f} TFLOP/s "
                                   f"x nominal FP16/BF16 ratio 1 (of {peak_src}; the MMAs are kind::f16)",
                    "traffic_unit": "DRAM bytes read + written per k_nn_tc launch",
                    "traffic_source": NN_DRAM_SOURCE,
                    "filter_tflops_as_formed": nn_tc_filter_flops_per_launch(K, N_PREFILL, d, kt_cols)
                    / (nn_ms * 1e-3) / 1e12,
                    "mma_issued_tflops": nn_tc_mma_flops_per_launch(K, N_PREFILL, d, kt_cols, mma_steps)
                    / (nn_ms * 1e-3) / 1e12,
                    "fp32_ffma_peak_tflops": fp32_peak_tflops, "nn_ms_per_launch": nn_ms,
                    "nn_dram_gbs_algorithmic": nn_bytes_per_launch(N_PREFILL, d) / (nn_ms * 1e-3) / 1e9,
                    "kernel_ms_per_step": kernel_ms}
    else:
        roofline = {"bound": "alu", "achieved": method_tflops, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                    "frac": method_tflops / fp32_peak_tflops, "traffic": None, "kernel": "k_nn",
                    "peak_source": fp32_src, "nn_ms_per_launch": nn_ms,
                    "nn_dram_gbs_algorithmic": nn_bytes_per_launch(N_PREFILL, d) / (nn_ms * 1e-3) / 1e9,
                    "kernel_ms_per_step": kernel_ms}
    prop_ms = kernel_ms["k_propagate"]
    flops_sub = propagate_flops_per_substep(spec)
    sub_mean = float(np.mean(substeps)) if substeps else R * (spec["s_min"] + spec["s_max"]) / 2
    prop_tflops = sub_mean * flops_sub / (prop_ms * 1e-3) / 1e12
    roofline["propagate"] = {
        "di3": {"bound": "alu", "achieved": prop_tflops, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                "frac": prop_tflops / fp32_peak_tflops, "kernel": "k_propagate", "ms_per_launch": prop_ms,
                "substeps_per_launch": sub_mean, "flops_per_substep": flops_sub,
                "work": "sum over rollouts with a parent of the drawn substeps S x (RK4 + dynamics + state box + "
                        "2 pdim O obstacle compares + path length + heuristic)", "peak_source": fp32_src}}

    line = None
    pending = {}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD_DESC, "n_tree": N_PREFILL, "parents": spec["K"],
                       "branching": spec["k"], "rollouts_per_step": R,
                       "l2": "flushed between timed steps (256 MB write); tree truncated back to n before each step",
                       "parallelism": f"replicas x{ws}"},
            "nodes_appended_per_step": float(np.mean(appended)) if appended else None,
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 12, "d2h_bytes_per_step": CTL_BYTES,
                    "how": "pakr_expand through the C ABI on host arguments, host wall clock per step: the cost "
                           "bound (4 B) and seed (8 B) go to the device as the expansion graph's kernel "
                           "parameters, the 216-byte control block comes back to the host to fill the caller's "
                           "pakr_expand_info, the stream is synchronised; the tree stays resident"},
            "gpu_launches": launches,
            "clocks": clk,
        }
    if not args.no_planning:
        plans = {}
        for name in ("di2", "di3", "quad12"):
            plans[name] = planning_metrics(dev, stream, name, args.ttfs_trials, args.aox_trials, rank)
        if rank == 0:
            e2p = plans["di3"].pop("_e2e_plan")
            for v in plans.values():
                v.pop("_e2e_plan", None)
            line["p50_time_to_first_solution_ms"] = plans["di3"]["time_to_first_solution_ms"]["p50"]
            line["aox_path_cost_at_100ms"] = plans["di3"]["aox_path_cost_at_100ms"]["p50"]
            line["planning"] = plans
            line["e2e_plan"] = {"value": e2p["host_ms_p50"], "unit": "ms (p50 time to first solution, host wall "
                                "clock through pakr_plan, di3)",
                                "h2d_bytes_per_step": 160, "d2h_bytes_per_step": e2p["d2h_bytes_mean"],
                                "how": "pakr_plan with host x_init / x_goal (160-byte parameter block copied to the "
                                       "device), the path, its history and the control block copied back"}
    if rank == 0:
        if not args.no_sweep:
            line["by_tree_size"] = tree_size_sweep(dev, stream)
            q12 = [r for r in line["by_tree_size"] if r["workload"] == "quad12"]
            if q12:
                qspec = W.problem("quad12", env_seed=0)
                qr = qspec["K"] * qspec["k"]
                fq = propagate_flops_per_substep(qspec)
                pm = float(np.median([r["propagate_ms"] for r in q12]))
                ach = qr * (qspec["s_min"] + qspec["s_max"]) / 2 * fq / (pm * 1e-3) / 1e12
                roofline["propagate"]["quad12"] = {
                    "bound": "alu", "achieved": ach, "peak": fp32_peak_tflops, "unit": "TFLOP/s",
                    "frac": ach / fp32_peak_tflops, "kernel": "k_propagate", "ms_per_launch": pm,
                    "substeps_per_launch": qr * (qspec["s_min"] + qspec["s_max"]) / 2, "flops_per_substep": fq,
                    "work": "R x mean drawn substeps x flops per substep (as for di3); median over the tree sizes "
                            "of the sweep", "peak_source": fp32_src}
        if not args.no_batched:
            line["batched_256"] = batched_vs_sequential(dev, stream)
        if not args.no_adjoint:
            line["adjoint_1024x200"], pending["adjoint"] = adjoint_bench(dev, stream)
            line["refined_aox_100ms"], p1 = refined_vs_plain(dev, stream)
            line["refined_aox_100ms_cluttered"], p2 = refined_vs_plain(dev, stream, n_boxes=300)
            pending["paths"] = {"refined_aox_100ms": p1, "refined_aox_100ms_cluttered": p2}
        if args.table4_trials > 0:
            line["table4_quad12"] = table4_sweep(dev, stream, trials=args.table4_trials)
        if not args.no_sweep:
            try:
                line["grown_tree"] = grown_tree_expansions(dev, stream)
            except Exception as e:  # a failed extra measurement leaves the rest of the line intact
                line["grown_tree"] = {"workload": WORKLOAD, "error": f"{type(e).__name__}: {e}"}
        # ---- the CPU leg: the oracle timed on the host cores, and its checks of GPU results ----
        if not args.no_cpu_baseline and ws == 1:
            line["cpu_baseline"] = cpu_baseline(spec, tree_seed=1 + rank, seed=7)
            checks = oracle_checks(pending)
            if "adjoint" in checks:
                line["adjoint_1024x200"].update(checks.pop("adjoint"))
            for key, v in checks.items():
                line[key]["oracle_recheck"] = v
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
