"""Seeded input generators: deterministic, in range, start and goal kept free."""
import numpy as np
import pytest

from paper_2607_03987_gb300 import workloads as W


@pytest.mark.parametrize("name", ["di2", "di3", "quad12"])
def test_problem_deterministic_and_free_endpoints(name):
    a, b = W.problem(name, env_seed=3), W.problem(name, env_seed=3)
    assert np.array_equal(a["boxes"], b["boxes"])
    c = W.problem(name, env_seed=4)
    assert not np.array_equal(a["boxes"], c["boxes"])
    pd = a["pdim"]
    n_boxes = {"di2": 10, "di3": 50, "quad12": 100}[name]
    assert a["boxes"].shape == (n_boxes, 2 * pd)
    assert np.all(a["boxes"][:, :pd] < a["boxes"][:, pd:])
    for p in (a["x_init"], a["x_goal"]):
        for bx in a["boxes"]:
            inside = np.all(p[:pd] >= bx[:pd] - a["goal_r"]) and np.all(p[:pd] <= bx[pd:] + a["goal_r"])
            assert not inside
    # every real number is a float32 value
    for key in ("x_lo", "x_hi", "u_lo", "u_hi", "boxes", "x_init", "x_goal"):
        v = np.asarray(a[key])
        assert np.array_equal(v, v.astype(np.float32).astype(np.float64))
    assert a["dt"] == float(np.float32(a["dt"]))


def test_quad_pillars_span_full_height():
    q = W.problem("quad12", env_seed=0)
    assert np.all(q["boxes"][:, 2] == 0.0) and np.all(q["boxes"][:, 5] == 1.0)


def test_prefilled_tree_structure():
    spec = W.problem("di3")
    t = W.prefilled_tree(spec, 5000, seed=2, cost_hi=1.0)
    assert t["parents"][0] == -1
    assert np.all(t["parents"][1:] >= 0) and np.all(t["parents"][1:] < np.arange(1, 5000))
    assert np.all(t["states"] >= spec["x_lo"]) and np.all(t["states"] <= spec["x_hi"])
    assert np.array_equal(t["states"][0], spec["x_init"])
    assert np.all((t["costs"] >= 0) & (t["costs"] <= 1.0)) and t["costs"][0] == 0
    t2 = W.prefilled_tree(spec, 5000, seed=2, cost_hi=1.0)
    assert np.array_equal(t["states"], t2["states"])
