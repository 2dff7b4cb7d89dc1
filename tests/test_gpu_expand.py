"""GPU expansion vs the FP64 oracle on identical seeded inputs (through the C ABI).

Trees come from the seeded generators or from the oracle's own growth (never
from the CUDA path); both sides then take one expansion from that tree.
"""
import numpy as np
import pytest

import oracle
from paper_2607_03987_gb300 import pakr
from paper_2607_03987_gb300 import workloads as W
from parity import compare

pytestmark = pytest.mark.gpu


def oracle_grown_tree(spec, iters, seed, bound=np.inf):
    prob = oracle.OracleProblem(spec)
    prob.set_goal(spec["x_goal"])
    t = oracle.OracleTree(spec["d"], spec["m"], spec["cap"])
    oracle.tree_reset(prob, t, spec["x_init"])
    for _ in range(iters):
        oracle.expand(prob, t, bound, seed)
    a = t.arrays()
    # both sides start from the FP32 rounding of the oracle's tree
    for key in ("states", "controls", "costs"):
        a[key] = W.f32(a[key])
    return a


def run_case(cuda_lib, spec, tree, bounds, seeds, **kw):
    planner = pakr.Planner(spec)
    out = []
    try:
        for b in bounds:
            for s in seeds:
                out.append(compare(spec, tree, b, s, planner, **kw))
    finally:
        planner.close()
    return out


@pytest.mark.parametrize("name,K,k,cap,n,iters", [
    ("di2", 64, 4, 20000, None, 12),
    ("di3", 1024, 8, 200000, None, 3),
    ("quad12", 4096, 16, 400000, None, 2),
])
def test_expand_oracle_grown_tree(cuda_lib, name, K, k, cap, n, iters):
    spec = W.with_sizes(W.problem(name, env_seed=11), K=K, k=k, cap=cap)
    tree = oracle_grown_tree(spec, iters, seed=5)
    assert tree["count"] > 256, "tree should span several NN tiles"
    stats = run_case(cuda_lib, spec, tree, [np.inf], [21, 22])
    for s in stats:
        assert s["compared_children"] > 0


@pytest.mark.parametrize("name", ["di2", "di3", "quad12"])
def test_expand_prefilled_ragged(cuda_lib, name):
    # 2,777 nodes: several 256-node tiles and a ragged tail; finite bounds prune part of the tree
    spec = W.with_sizes(W.problem(name, env_seed=2), K=300, k=5, cap=10000)
    tree = W.prefilled_tree(spec, 2777, seed=9, cost_hi=2.0)
    stats = run_case(cuda_lib, spec, tree, [np.inf, 2.5, 1.7], [3])
    assert sum(s["compared_rollouts"] for s in stats) > 1000


def test_expand_ties_lowest_index(cuda_lib):
    # duplicated states: equal distances must resolve to the lowest index
    spec = W.with_sizes(W.problem("di3", env_seed=1), K=257, k=2, cap=5000)
    tree = W.prefilled_tree(spec, 1000, seed=4)
    tree["states"][500:1000] = tree["states"][0:500]
    tree["states"][700:760] = tree["states"][20]
    stats = run_case(cuda_lib, spec, tree, [np.inf], [8])
    near = stats[0]["dbg"]["near"]
    assert np.all(near < 500), "a duplicate at a higher index was chosen"


def test_expand_tree_full_truncates(cuda_lib):
    spec = W.with_sizes(W.problem("di3", env_seed=1), K=512, k=8, cap=1100)
    tree = W.prefilled_tree(spec, 1000, seed=6)
    stats = run_case(cuda_lib, spec, tree, [np.inf], [1])
    s = stats[0]
    assert s["gtree"]["count"] == 1100
    assert s["info"]["n_dropped"] > 0 and s["status"] == pakr.TREE_FULL


def test_expand_no_eligible(cuda_lib):
    spec = W.with_sizes(W.problem("di2", env_seed=1), K=64, k=4, cap=5000)
    tree = W.prefilled_tree(spec, 700, seed=6, cost_hi=1.0)
    tree["costs"][:] = 5.0
    tree["costs"][0] = 0.0
    # the root's f-cost (distance to the goal ball, about 1.08) is above the bound too
    stats = run_case(cuda_lib, spec, tree, [0.5], [2])
    assert stats[0]["status"] == pakr.NO_ELIGIBLE
    assert stats[0]["info"]["n_no_parent"] == 64 * 4


def test_expand_single_node_tree(cuda_lib):
    spec = W.with_sizes(W.problem("di3", env_seed=3), K=100, k=3, cap=1000)
    tree = W.prefilled_tree(spec, 1, seed=1)
    run_case(cuda_lib, spec, tree, [np.inf], [1, 2])


@pytest.mark.parametrize("variant", ["duration", "fullstate", "spheres", "weights", "obstacles_outside"])
def test_expand_variants(cuda_lib, variant):
    base = W.problem("di3", env_seed=4)
    over = dict(K=256, k=4, cap=8000)
    if variant == "duration":
        over["cost"] = W.COST_DURATION
    elif variant == "fullstate":
        over["heuristic"] = W.H_FULLSTATE
    elif variant == "spheres":
        over["spheres"] = W.random_spheres(3, 20, 3)
    elif variant == "weights":
        over["nn_w"] = W.f32([1, 1, 1, 0.25, 0.25, 0.25])
    elif variant == "obstacles_outside":
        # obstacles reaching past the state box and one spanning half of it: the obstacle grid
        # clamps their cell ranges at the box edge
        extra = W.f32([[-0.3, 0.4, 0.2, 0.12, 0.6, 0.5], [0.85, -0.2, 0.3, 1.4, 0.15, 0.45],
                       [0.3, 0.55, -0.5, 0.9, 0.95, 0.35]])
        over["boxes"] = np.concatenate([base["boxes"], extra])
        over["spheres"] = W.f32([[1.02, 0.5, 0.5, 0.1], [0.5, 0.5, 1.05, 0.08], [0.3, 0.7, 0.6, 0.06]])
    spec = W.with_sizes(base, **over)
    tree = W.prefilled_tree(spec, 1500, seed=2, cost_hi=1.0)
    run_case(cuda_lib, spec, tree, [np.inf, 2.2], [5])


@pytest.mark.parametrize("dyn", [W.DUBINS3D, W.UNICYCLE1, W.UNICYCLE2])
def test_expand_other_models(cuda_lib, dyn):
    d, m, pdim = W.DIMS[dyn]
    if dyn == W.DUBINS3D:
        x_lo, x_hi = [0, 0, 0, -np.pi, -1, 0.05], [1, 1, 1, np.pi, 1, 0.5]
        u_lo, u_hi = [-1, -1, -0.5], [1, 1, 0.5]
        start, goal = [0.1, 0.1, 0.1, 0, 0, 0.2], [0.9, 0.9, 0.9, 0, 0, 0.2]
    elif dyn == W.UNICYCLE1:
        x_lo, x_hi = [0, 0, -np.pi], [1, 1, np.pi]
        u_lo, u_hi = [-0.5, -1], [0.5, 1]
        start, goal = [0.1, 0.1, 0], [0.9, 0.9, 0]
    else:
        x_lo, x_hi = [0, 0, -np.pi, -0.5, -1], [1, 1, np.pi, 0.5, 1]
        u_lo, u_hi = [-0.25, -0.5], [0.25, 0.5]
        start, goal = [0.1, 0.1, 0, 0, 0], [0.9, 0.9, 0, 0, 0]
    base = W.problem("di3" if pdim == 3 else "di2", env_seed=5)
    spec = W.with_sizes(base, dyn=dyn, d=d, m=m, pdim=pdim, x_lo=W.f32(x_lo), x_hi=W.f32(x_hi),
                        u_lo=W.f32(u_lo), u_hi=W.f32(u_hi), x_init=W.f32(start), x_goal=W.f32(goal),
                        K=128, k=4, cap=6000, dt=float(W.f32(0.1)))
    tree = W.prefilled_tree(spec, 900, seed=3, cost_hi=0.5)
    run_case(cuda_lib, spec, tree, [np.inf, 2.0], [4])


def test_consecutive_expansions_match_oracle(cuda_lib):
    # several iterations back to back on both sides from the same root
    spec = W.with_sizes(W.problem("di2", env_seed=7), K=64, k=4, cap=20000)
    prob = oracle.OracleProblem(spec)
    prob.set_goal(spec["x_goal"])
    ot = oracle.OracleTree(spec["d"], spec["m"], spec["cap"])
    oracle.tree_reset(prob, ot, spec["x_init"])
    planner = pakr.Planner(spec)
    planner.tree_reset(spec["x_init"], spec["x_goal"])
    diverged = None
    for it in range(10):
        ref = oracle.expand(prob, ot, np.inf, 99)
        st, info = planner.expand(np.inf, 99)
        if info["n_appended"] != ref["n_appended"] or info["n_start"] != ref["n_start"]:
            diverged = it
            break
    g = planner.tree_export()
    planner.close()
    if diverged is None:
        o = ot.arrays()
        assert g["count"] == o["count"]
        assert np.array_equal(g["parents"], o["parents"])
        assert np.array_equal(g["steps"], o["steps"])
        assert np.all(np.abs(g["states"] - o["states"]) <= 1e-5 * np.maximum(1, np.abs(o["states"])))
        assert np.all(np.abs(g["costs"] - o["costs"]) <= 1e-5 * np.maximum(1, np.abs(o["costs"])))
    else:
        pytest.fail(f"free-running trees diverged at iteration {diverged}")


@pytest.mark.parametrize("K,k", [(2048, 2), (32, 128)])
def test_expand_table4_extreme_shapes(cuda_lib, K, k):
    """The two extreme batch shapes of Table 4 on the 12D quadrotor (batch 4096 rollouts as
    K = 2048 parents x A = 2 and K = 32 x A = 128), one expansion each from a tree the oracle
    grew and from a prefilled tree with a finite bound, element by element against the oracle."""
    spec = W.with_sizes(W.problem("quad12", env_seed=0), K=K, k=k, cap=60000)
    tree = oracle_grown_tree(W.with_sizes(spec, K=256, k=16), 3, seed=7)
    stats = run_case(cuda_lib, spec, tree, [np.inf], [31])
    pre = W.prefilled_tree(spec, 20011, seed=8, cost_hi=2.0)
    stats += run_case(cuda_lib, spec, pre, [2.2], [32])
    assert sum(s["compared_rollouts"] for s in stats) > 0.9 * 2 * K * k
