"""Batched planning (one persistent cooperative launch for many queries) vs
one pakr_plan per query: the batch runs the same device code per query, so
every query's result must be identical to its single-query run."""
import numpy as np
import pytest

from paper_2607_03987_gb300 import pakr
from paper_2607_03987_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def single_spec(base, q):
    return W.with_sizes(base, boxes=q["boxes"], spheres=q["spheres"], cap=q["cap"], x_init=q["x_init"],
                        x_goal=q["x_goal"])


def run_single(base, queries, seed, **kw):
    out = []
    for i, q in enumerate(queries):
        pl = pakr.Planner(single_spec(base, q))
        try:
            out.append(pl.plan(q["x_init"], q["x_goal"], seed=seed + i, **kw))
        finally:
            pl.close()
    return out


def assert_same(batch_res, single_res, bp):
    for q, (r, g) in enumerate(zip(batch_res, single_res)):
        assert r["n_solutions"] == g["n_solutions"], (q, r, g["n_solutions"])
        assert r["iterations"] == g["iterations"], (q, r["iterations"], g["iterations"])
        assert r["n_restarts"] == g["n_restarts"]
        if g["n_solutions"]:
            assert r["cost"] == g["cost"], (q, r["cost"], g["cost"])
            assert r["n_edges"] == g["n_edges"]
            states, controls, steps = bp.path(q)
            ne = r["n_edges"]
            assert np.array_equal(states[: ne + 1], g["states"])
            assert np.array_equal(controls[:ne], g["controls"])
            assert np.array_equal(steps[:ne], g["steps"])


def test_batch_equals_single_query_runs(cuda_lib):
    base, queries = W.batch_queries(7, env_seed=1, cap_range=(8192, 65536))
    bp = pakr.BatchPlanner(base, queries)
    res = bp.plan(budget_s=60.0, max_iterations=25, seed=100)
    single = run_single(base, queries, 100, budget_s=60.0, max_iterations=25)
    assert_same(res, single, bp)
    assert sum(r["n_solutions"] for r in res) > 0
    bp.close()


def test_batch_stop_at_first_and_invalid_query(cuda_lib):
    base, queries = W.batch_queries(9, env_seed=2, cap_range=(16384, 131072))
    bad = dict(queries[3])
    box = bad["boxes"][0]
    bad["x_init"] = W.f32(np.concatenate([(box[:3] + box[3:]) / 2, np.zeros(3)]))  # inside a box
    queries[3] = bad
    bp = pakr.BatchPlanner(base, queries)
    res = bp.plan(budget_s=10.0, max_iterations=400, seed=5, stop_at_first=True)
    assert res[3]["status"] == pakr.ERR_INVALID_ARG and res[3]["iterations"] == 0
    others = [r for i, r in enumerate(res) if i != 3]
    assert all(r["status"] == pakr.GOAL_REACHED and r["n_solutions"] == 1 for r in others), others
    good = [q for i, q in enumerate(queries) if i != 3]
    single = run_single(base, good, 0, budget_s=10.0, max_iterations=400, stop_at_first=True)
    # seeds: the batch gives query q seed 5 + q
    for j, (i, q) in enumerate([(i, q) for i, q in enumerate(queries) if i != 3]):
        pl = pakr.Planner(single_spec(base, q))
        g = pl.plan(q["x_init"], q["x_goal"], budget_s=10.0, max_iterations=400, seed=5 + i, stop_at_first=True)
        pl.close()
        assert res[i]["iterations"] == g["iterations"] and res[i]["cost"] == g["cost"]
    del single
    bp.close()


def test_batch_autotune_keeps_results(cuda_lib):
    base, queries = W.batch_queries(12, env_seed=3, cap_range=(8192, 32768))
    bp = pakr.BatchPlanner(base, queries)
    r0 = bp.plan(budget_s=60.0, max_iterations=15, seed=9)
    t = bp.autotune(iterations=4, seed=1)
    assert t["block_threads"] in (128, 256) and t["nn_chunk"] % 8 == 0 and t["n_tried"] == 10
    r1 = bp.plan(budget_s=60.0, max_iterations=15, seed=9)
    for a, b in zip(r0, r1):
        assert a["cost"] == b["cost"] and a["iterations"] == b["iterations"] or (np.isinf(a["cost"]) and np.isinf(b["cost"]))
    bp.set_tuning(128, 512)
    r2 = bp.plan(budget_s=60.0, max_iterations=15, seed=9)
    assert [a["iterations"] for a in r0] == [b["iterations"] for b in r2]
    with pytest.raises(pakr.PakrError):
        bp.set_tuning(96, 512)
    bp.close()


def test_batch_matches_oracle_per_query(cuda_lib):
    """Each query of one batched launch against the FP64 oracle's own Algorithm 1 run for that
    query (its obstacles, tree cap and seed + q), planned to the first solution.  Twelve short
    queries (start and goal 0.15-0.3 apart) with uneven obstacle counts (10-200 boxes) and tree
    caps: where the oracle's run reached its first solution before any near-tie (an
    exemption-class event: a substep within 1e-5 of a face, a nearest-neighbour gap under
    1e-6), the iteration of the first solution, its cost and the path's states and durations
    must match; every returned path must pass the FP64 re-check (valid at every substep, in the
    goal ball, with the reported cost)."""
    import oracle
    from recheck import recheck_path

    base, queries = W.batch_queries(12, env_seed=5, obs_range=(10, 200), cap_range=(4096, 32768),
                                    sep_range=(0.15, 0.3))
    base = W.with_sizes(base, K=128, k=4)
    seed, iters = 300, 400
    bp = pakr.BatchPlanner(base, queries)
    res = bp.plan(budget_s=60.0, max_iterations=iters, seed=seed, stop_at_first=True)
    compared = 0
    for q, (query, r) in enumerate(zip(queries, res)):
        spec = single_spec(base, query)
        prob = oracle.OracleProblem(spec)
        prob.set_goal(spec["x_goal"])
        tree = oracle.OracleTree(spec["d"], spec["m"], spec["cap"])
        o = oracle.plan(prob, tree, spec["x_init"], seed + q, iters, stop_at_first=True)
        frag = o["fragile_iteration"]
        solved_before_frag = o["n_solutions"] > 0 and (frag < 0 or o["hist_iter"][0] < frag)
        if r["n_solutions"]:
            states, controls, steps = bp.path(q)
            ne = r["n_edges"]
            assert r["iterations_first_solution"] == r["iterations"]
            rc = recheck_path(spec, states[: ne + 1], controls[:ne], steps[:ne])
            assert rc["invalid"] == 0 and (rc["replay_in_goal"] or rc["replay_exempt"] > 0), (q, rc)
            assert abs(rc["replay_length"] - r["cost"]) <= 1e-4 * max(1.0, r["cost"]), (q, rc, r["cost"])
        if solved_before_frag:
            assert r["status"] == pakr.GOAL_REACHED, (q, r)
            assert r["iterations_first_solution"] == o["hist_iter"][0] + 1, (q, r, o["hist_iter"])
            assert abs(r["cost"] - o["best_cost"]) <= 1e-5 * max(1.0, o["best_cost"]), (q, r["cost"], o["best_cost"])
            assert r["n_edges"] + 1 == len(o["path_states"])
            assert np.allclose(states[: ne + 1], o["path_states"], rtol=1e-5, atol=1e-5)
            assert np.array_equal(steps[:ne], o["path_steps"][1:])
            compared += 1
        elif frag < 0:
            # no near-tie in the whole oracle run and no solution within the iteration cap
            assert r["n_solutions"] == 0 and r["iterations"] == o["iterations"], (q, r, o["iterations"])
            compared += 1
    bp.close()
    assert compared >= len(queries) // 2, compared
