"""Dense FP64 re-check of what the GPU produced: every edge of trees it grew,
every edge of the paths pakr_plan returned, and gradient-refined paths.

The planner checks validity at its integration substeps only (Sec. IV-A).  The
re-check replays each edge in FP64 from the GPU's own parent state: the child
must match, every substep must be valid (or within 1e-5 of a deciding face),
and edges that touch an obstacle between substeps (the double integrator
exactly, other models at dt/16) are counted as misses of the discrete check.
"""
import numpy as np
import pytest

from paper_2607_03987_gb300 import pakr
from paper_2607_03987_gb300 import workloads as W
from recheck import STATE_RTOL, recheck_path, recheck_tree, replay_path

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name,K,k,cap,iters", [("di3", 256, 8, 40000, 4), ("quad12", 256, 4, 20000, 3)])
def test_gpu_grown_tree_edges_recheck(cuda_lib, name, K, k, cap, iters):
    spec = W.with_sizes(W.problem(name, env_seed=3), K=K, k=k, cap=cap)
    planner = pakr.Planner(spec)
    try:
        planner.tree_reset(spec["x_init"], spec["x_goal"])
        for _ in range(iters):
            planner.expand(np.inf, 9)
        tree = planner.tree_export()
    finally:
        planner.close()
    rc = recheck_tree(spec, tree)
    assert rc["edges"] > 200
    assert rc["invalid"] == 0, rc
    assert rc["max_rel_state_err"] <= STATE_RTOL, rc
    # substep-only checking lets a few edges graze an obstacle between substeps; they are
    # counted, and they stay a small fraction
    assert rc["misses"] < 0.05 * rc["edges"], rc


@pytest.mark.parametrize("name,budget,stop", [("di3", 0.05, False), ("di2", 0.05, False), ("quad12", 2.0, True)])
def test_plan_paths_recheck(cuda_lib, name, budget, stop):
    spec = W.problem(name, env_seed=0)
    planner = pakr.Planner(spec)
    checked = 0
    try:
        for seed in range(3):
            r = planner.plan(spec["x_init"], spec["x_goal"], budget_s=budget, seed=seed, stop_at_first=stop)
            if not r["n_solutions"]:
                continue
            rc = recheck_path(spec, r["states"], r["controls"], r["steps"])
            assert rc["invalid"] == 0 and rc["max_rel_state_err"] <= STATE_RTOL, rc
            assert rc["misses"] <= max(1, rc["edges"] // 10), rc
            # the whole control sequence replayed in FP64 from the start reaches the goal ball
            # (drift over many edges stays far below the goal radius) with the reported cost
            assert rc["replay_in_goal"] or rc["replay_exempt"] > 0, rc
            assert abs(rc["replay_length"] - r["cost"]) <= 1e-4 * max(1.0, r["cost"]), (rc, r["cost"])
            checked += 1
    finally:
        planner.close()
    assert checked >= 2


def test_refined_path_recheck(cuda_lib):
    """A path shortened by the adjoint refinement passes the same FP64 re-check as the plain
    path it came from: valid at every substep, in the goal ball, with the length the GPU
    reports, and misses of the discrete check counted for both."""
    import torch

    from paper_2607_03987_gb300 import refine

    spec = W.problem("di3", env_seed=0)
    planner = pakr.Planner(spec)
    verdicts = []
    try:
        for seed in range(4):
            r = planner.plan(spec["x_init"], spec["x_goal"], budget_s=0.03, seed=seed)
            if not r["n_solutions"]:
                continue
            out = refine.refine_path(planner, spec, r, spec["x_goal"], iters=15)
            plain = replay_path(spec, r["states"][0], r["controls"], r["steps"])
            assert plain["replay_valid"] and plain["replay_in_goal"], plain
            if out is None:
                continue
            u_ref, length = out
            ref = replay_path(spec, r["states"][0], u_ref.detach().cpu().numpy(), r["steps"])
            assert ref["replay_valid"] and ref["replay_in_goal"], ref
            assert abs(ref["replay_length"] - length) <= 1e-4 * max(1.0, length), (ref, length)
            assert ref["replay_length"] < plain["replay_length"]
            verdicts.append((plain["replay_misses"], ref["replay_misses"]))
            torch.cuda.synchronize()
    finally:
        planner.close()
    assert verdicts, "no refinement improved a path"
