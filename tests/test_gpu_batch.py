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
