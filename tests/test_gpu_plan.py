"""AO-x loop on the device (one CUDA graph) vs the oracle's AO-x loop."""
import numpy as np
import pytest

import oracle
from paper_2607_03987_gb300 import pakr
from paper_2607_03987_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def oracle_plan(spec, seed, iters, stop_at_first=False):
    prob = oracle.OracleProblem(spec)
    prob.set_goal(spec["x_goal"])
    t = oracle.OracleTree(spec["d"], spec["m"], spec["cap"])
    return oracle.plan(prob, t, spec["x_init"], seed, iters, stop_at_first=stop_at_first)


def check_path_properties(spec, res):
    """Properties any returned path has: starts at x_init, ends in the goal
    ball, durations / controls in range, c_best strictly decreasing."""
    if res["n_solutions"] == 0:
        return
    s = res["states"]
    assert np.allclose(s[0], spec["x_init"])
    pd = spec["pdim"]
    assert np.linalg.norm(s[-1][:pd] - spec["x_goal"][:pd]) <= spec["goal_r"] * (1 + 1e-5)
    assert np.all((res["steps"] >= spec["s_min"]) & (res["steps"] <= spec["s_max"]))
    assert np.all((res["controls"] >= spec["u_lo"]) & (res["controls"] <= spec["u_hi"]))
    hc = res["history_cost"]
    assert res["iterations_first_solution"] == res["history_iteration"][0] + 1
    assert res["nodes_first_solution"] > 1
    assert np.all(np.diff(hc) < 0), hc
    assert abs(hc[-1] - res["cost"]) <= 1e-6 * max(1, res["cost"])
    # path-length cost is at least the straight-line distance start -> goal ball
    lb = np.linalg.norm(spec["x_goal"][:pd] - spec["x_init"][:pd]) - spec["goal_r"]
    assert res["cost"] >= lb * (1 - 1e-5)


@pytest.mark.parametrize("name,iters", [("di2", 40), ("di3", 12)])
def test_plan_matches_oracle(cuda_lib, name, iters):
    spec = W.problem(name, env_seed=0)
    if name == "di3":
        spec = W.with_sizes(spec, cap=200000)
    planner = pakr.Planner(spec)
    compared = 0
    for seed in range(3):
        g = planner.plan(spec["x_init"], spec["x_goal"], budget_s=60.0, max_iterations=iters, seed=seed)
        o = oracle_plan(spec, seed, iters)
        check_path_properties(spec, g)
        frag = o["fragile_iteration"]
        upto = iters if frag < 0 else frag
        og = [(c, i) for c, i in zip(o["hist_cost"], o["hist_iter"]) if i < upto]
        gg = [(c, i) for c, i in zip(g["history_cost"], g["history_iteration"]) if i < upto]
        assert len(og) == len(gg), (seed, og, gg, frag)
        for (oc, oi), (gc, gi) in zip(og, gg):
            assert oi == gi
            assert abs(gc - oc) <= 1e-5 * max(1, oc)
        compared += len(og)
        if frag < 0:
            assert g["iterations"] == o["iterations"]
            assert g["n_solutions"] == o["n_solutions"]
            if o["n_solutions"]:
                assert len(g["states"]) == len(o["path_states"])
                assert np.allclose(g["states"], o["path_states"], rtol=1e-5, atol=1e-5)
    planner.close()


def test_plan_stop_at_first_and_budget(cuda_lib):
    spec = W.problem("di3", env_seed=1)
    planner = pakr.Planner(spec)
    r = planner.plan(spec["x_init"], spec["x_goal"], budget_s=5.0, seed=3, stop_at_first=True)
    assert r["status"] == pakr.GOAL_REACHED and r["n_solutions"] == 1
    assert 0 < r["t_first_solution_s"] <= r["t_total_s"] < 5.0
    check_path_properties(spec, r)
    r = planner.plan(spec["x_init"], spec["x_goal"], budget_s=0.05, seed=3)
    assert r["t_total_s"] < 0.5
    check_path_properties(spec, r)
    r = planner.plan(spec["x_init"], spec["x_goal"], budget_s=10.0, max_iterations=1, seed=3)
    assert r["iterations"] == 1
    planner.close()


def test_plan_invalid_start(cuda_lib):
    spec = W.problem("di2", env_seed=0)
    planner = pakr.Planner(spec)
    bad = spec["x_init"].copy()
    bad[0] = 2.0  # outside the state box
    with pytest.raises(pakr.PakrError) as e:
        planner.plan(bad, spec["x_goal"], budget_s=1.0, seed=0)
    assert e.value.status == pakr.ERR_INVALID_ARG
    with pytest.raises(pakr.PakrError):
        planner.tree_reset(bad, spec["x_goal"])
    planner.close()


def test_plan_quadrotor_runs(cuda_lib):
    spec = W.problem("quad12", env_seed=0)
    planner = pakr.Planner(spec)
    r = planner.plan(spec["x_init"], spec["x_goal"], budget_s=2.0, seed=0)
    assert r["iterations"] > 0
    check_path_properties(spec, r)
    planner.close()


def test_tree_size_matches_export(cuda_lib):
    spec = W.problem("di2", env_seed=0)
    planner = pakr.Planner(spec)
    planner.plan(spec["x_init"], spec["x_goal"], budget_s=60.0, max_iterations=15, seed=4)
    n, it = planner.tree_size()
    tree = planner.tree_export()
    assert n == len(tree["parents"]) and n >= 1
    assert it == tree["iteration"]
    planner.close()


@pytest.mark.parametrize("B,A", [(4096, 2), (4096, 128)])
def test_quadrotor_table4_shapes(cuda_lib, B, A):
    """The batch size x branching factor shapes of Table 4 (K = B / A parents)
    run on the 12D quadrotor: the tree grows by at most B nodes per expansion
    and any path found has the properties of a solution."""
    spec = W.with_sizes(W.problem("quad12", env_seed=0), K=B // A, k=A, cap=200000)
    planner = pakr.Planner(spec)
    iters = 6
    r = planner.plan(spec["x_init"], spec["x_goal"], budget_s=60.0, max_iterations=iters, seed=1,
                     stop_at_first=True)
    n, _ = planner.tree_size()
    assert 1 < n <= 1 + r["iterations"] * B
    assert r["iterations"] <= iters
    if r["n_solutions"]:
        assert 1 < r["nodes_first_solution"] <= 1 + r["iterations_first_solution"] * B
        assert r["iterations_first_solution"] == r["iterations"]
        pd = spec["pdim"]
        s = r["states"]
        assert np.allclose(s[0], spec["x_init"])
        assert np.linalg.norm(s[-1][:pd] - spec["x_goal"][:pd]) <= spec["goal_r"] * (1 + 1e-5)
    planner.close()


def test_offer_bound_reaches_running_plan(cuda_lib):
    """A bound offered from another stream and host thread while the device AO-x loop runs is
    picked up by the loop: a bound just under the straight-line lower bound can be beaten by no
    path (every node's f = g + h is at least that lower bound), so the loop finds no eligible
    node from then on and the run ends
    long before its 5 s budget; the run's own best path keeps its own cost."""
    import threading
    import time

    import torch

    spec = W.problem("di3", env_seed=0)
    s_plan, s_side = torch.cuda.Stream(), torch.cuda.Stream()
    planner = pakr.Planner(spec, stream=s_plan)
    planner.plan(spec["x_init"], spec["x_goal"], budget_s=0.05, seed=1)  # builds the graph
    pd = spec["pdim"]
    lb = float(np.linalg.norm(spec["x_goal"][:pd] - spec["x_init"][:pd]) - spec["goal_r"])
    offer = float(np.float32(lb * (1 - 1e-4)))  # below every node's f, rounding included
    res = []
    # the offered value is on the device before the plan starts: an allocation, or the first
    # launch of a kernel (its code is loaded lazily), while the plan runs may wait for it
    with torch.cuda.stream(s_side):
        cost = torch.full((1,), offer, dtype=torch.float32, device="cuda")
    s_side.synchronize()
    th = threading.Thread(target=lambda: res.append(planner.plan(spec["x_init"], spec["x_goal"], budget_s=5.0,
                                                                 seed=3)))
    t0 = time.perf_counter()
    th.start()
    time.sleep(0.05)
    planner.offer_bound(cost, s_side)
    s_side.synchronize()
    th.join()
    elapsed = time.perf_counter() - t0
    r = res[0]
    planner.close()
    assert r["t_total_s"] < 1.0 and elapsed < 2.0, (r["t_total_s"], elapsed)
    assert r["n_solutions"] > 0 and r["cost"] > lb
    assert np.all(np.diff(r["history_cost"]) < 0)
    check_path_properties(spec, r)


def test_refined_aox_concurrent_paths_valid(cuda_lib):
    """AO-x with refinement running beside it on a second stream: the returned path passes the
    FP64 re-check (valid at every substep, in the goal ball) with the returned cost, and the
    best cost never rises."""
    import torch

    from paper_2607_03987_gb300 import refine
    from recheck import replay_path

    spec = W.problem("di3", env_seed=0, n_boxes=150)
    planner = pakr.Planner(spec, stream=torch.cuda.Stream())
    ref_planner = pakr.Planner(W.with_sizes(spec, K=1, k=1, cap=16), stream=torch.cuda.Stream())
    try:
        for seed in range(3):
            c, hist, gain, best = refine.refined_aox_concurrent(planner, ref_planner, spec, 0.1, seed=seed)
            if best is None:
                continue
            costs = [h[1] for h in hist]
            assert all(b <= a for a, b in zip(costs, costs[1:])), hist
            rp = replay_path(spec, best["x0"], best["controls"], best["steps"])
            assert rp["replay_valid"] and rp["replay_in_goal"], rp
            assert abs(rp["replay_length"] - c) <= 1e-4 * max(1.0, c), (rp, c)
    finally:
        planner.close()
        ref_planner.close()


def test_plan_snapshot_copies_best_path(cuda_lib):
    """pakr_plan_snapshot on another stream returns the plan's best path: after a plan, the
    copy is whole and equals the path and cost pakr_plan returned."""
    import torch

    spec = W.problem("di3", env_seed=0)
    s_plan, s_side = torch.cuda.Stream(), torch.cuda.Stream()
    planner = pakr.Planner(spec, stream=s_plan)
    try:
        r = planner.plan(spec["x_init"], spec["x_goal"], budget_s=0.03, seed=5)
        assert r["n_solutions"] > 0
        E = 512
        with torch.cuda.stream(s_side):
            st = torch.zeros((E + 1, spec["d"]), dtype=torch.float32, device="cuda")
            ct = torch.zeros((E, spec["m"]), dtype=torch.float32, device="cuda")
            sp = torch.zeros(E, dtype=torch.int32, device="cuda")
            info = torch.zeros(4, dtype=torch.int32, device="cuda")
            planner.plan_snapshot(st, ct, sp, info, s_side)
            inf_h = info.cpu().numpy()
            ne = int(inf_h[1])
            assert inf_h[0] == 1 and ne == r["n_edges"] and inf_h[2] >= 2 and inf_h[2] % 2 == 0
            assert np.array_equal(st[: ne + 1].cpu().numpy(), r["states"])
            assert np.array_equal(ct[:ne].cpu().numpy(), r["controls"])
            assert np.array_equal(sp[:ne].cpu().numpy(), r["steps"])
            assert np.array([inf_h[3]], np.int32).view(np.float32)[0] == np.float32(r["cost"])
    finally:
        planner.close()


def test_refined_aox_live_paths_valid(cuda_lib):
    """AO-x run once, with the refinement polling its best path beside it and offering shorter
    refined paths: the returned path passes the FP64 re-check with the returned cost."""
    import torch

    from paper_2607_03987_gb300 import refine
    from recheck import replay_path

    spec = W.problem("di3", env_seed=0, n_boxes=150)
    planner = pakr.Planner(spec, stream=torch.cuda.Stream())
    ref_planner = pakr.Planner(W.with_sizes(spec, K=1, k=1, cap=16), stream=torch.cuda.Stream())
    try:
        refine.refined_aox_live(planner, ref_planner, spec, 0.05, seed=99)  # warm-up
        for seed in range(3):
            c, gain, best = refine.refined_aox_live(planner, ref_planner, spec, 0.1, seed=seed)
            if best is None:
                continue
            rp = replay_path(spec, best["x0"], best["controls"], best["steps"])
            assert rp["replay_valid"] and rp["replay_in_goal"], rp
            assert abs(rp["replay_length"] - c) <= 1e-4 * max(1.0, c), (rp, c)
    finally:
        planner.close()
        ref_planner.close()
