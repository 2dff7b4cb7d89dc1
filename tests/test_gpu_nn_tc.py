"""Tensor-core nearest neighbour (k_nn_tc) against the FP32 kernel and the oracle.

Both kernels define the result the same way (the exact FP32 squared distance,
lowest index on a tie), so on the same tree, samples and bound the chosen
parents must be identical, element by element.  Trees come from the seeded
generators; the planners are forced to one kernel with nn_mode.
"""
import numpy as np
import pytest

from paper_2607_03987_gb300 import pakr
from paper_2607_03987_gb300 import workloads as W
from parity import compare

pytestmark = pytest.mark.gpu


def expand_near(spec, tree, bound, seed, mode):
    planner = pakr.Planner(W.with_sizes(spec, nn_mode=mode))
    try:
        planner.tree_import(tree, spec["x_goal"])
        st, info = planner.expand(bound, seed)
        dbg = planner.debug_last_expand()
    finally:
        planner.close()
    return st, info, dbg


def assert_same_expansion(spec, tree, bound, seed):
    s1, i1, d1 = expand_near(spec, tree, bound, seed, pakr.NN_FP32)
    s2, i2, d2 = expand_near(spec, tree, bound, seed, pakr.NN_TENSOR)
    assert s1 == s2
    assert np.array_equal(d1["samples"], d2["samples"])
    bad = np.nonzero(d1["near"] != d2["near"])[0]
    assert bad.size == 0, f"parents differ at queries {bad[:10]}: fp32 {d1['near'][bad[:10]]} tc {d2['near'][bad[:10]]}"
    # identical parents give identical rollouts and the same appended tree
    assert np.array_equal(d1["outcome"], d2["outcome"])
    assert i1 == i2
    return d1


@pytest.mark.parametrize("name,K,k,n", [
    ("di3", 1024, 8, 300_000),      # several query blocks, many 256-node tiles per chunk
    ("di3", 1000, 4, 123_457),      # ragged query block and ragged last tile
    ("di2", 300, 3, 70_001),
    ("quad12", 512, 4, 100_000),    # d = 12: five MMA k-steps
])
def test_tc_matches_fp32_uniform(cuda_lib, name, K, k, n):
    spec = W.with_sizes(W.problem(name, env_seed=3), K=K, k=k, cap=n + 64)
    tree = W.prefilled_tree(spec, n, seed=9)
    d = assert_same_expansion(spec, tree, np.inf, seed=17)
    assert (d["near"] >= 0).all()


def test_tc_matches_fp32_finite_bound(cuda_lib):
    # costs uniform in [0, 3]: a finite bound leaves part of the tree ineligible
    spec = W.with_sizes(W.problem("di3", env_seed=4), K=1024, k=4, cap=200_064)
    tree = W.prefilled_tree(spec, 200_000, seed=10, cost_hi=3.0)
    for bound in (2.5, 1.4):
        assert_same_expansion(spec, tree, bound, seed=31)


def test_tc_matches_fp32_lattice_ties(cuda_lib):
    # states on a coarse lattice: many exactly equal distances, the lowest index must win
    spec = W.with_sizes(W.problem("di3", env_seed=5), K=512, k=2, cap=80_000)
    tree = W.prefilled_tree(spec, 80_000, seed=12)
    tree["states"] = W.f32(np.round(tree["states"] * 8.0) / 8.0)
    tree["states"][0] = spec["x_init"]
    assert_same_expansion(spec, tree, np.inf, seed=5)


def test_tc_matches_fp32_offset_box(cuda_lib):
    # a state box far from the origin: the filter works on centred coordinates
    spec = W.problem("di3", env_seed=6)
    off = np.array([50.0, 50.0, 50.0, 0, 0, 0])
    spec = W.with_sizes(spec, K=512, k=2, cap=70_000,
                        x_lo=W.f32(spec["x_lo"] + off), x_hi=W.f32(spec["x_hi"] + off),
                        x_init=W.f32(spec["x_init"] + off), x_goal=W.f32(spec["x_goal"] + off),
                        boxes=W.f32(spec["boxes"] + np.concatenate([off[:3], off[:3]])))
    tree = W.prefilled_tree(spec, 70_000, seed=13)
    assert_same_expansion(spec, tree, np.inf, seed=6)


def test_tc_small_and_out_of_box_trees(cuda_lib):
    spec = W.with_sizes(W.problem("di3", env_seed=7), K=256, k=2, cap=4096)
    # a tree smaller than one tile
    tree = W.prefilled_tree(spec, 77, seed=14)
    assert_same_expansion(spec, tree, np.inf, seed=8)
    # states outside the state box (imported, not grown): the tree is flagged and the
    # tensor-core kernel rescans exactly
    tree = W.prefilled_tree(spec, 3000, seed=15)
    tree["states"][1:40, 0] = W.f32(7.5)
    assert_same_expansion(spec, tree, np.inf, seed=9)


def test_tc_against_oracle(cuda_lib):
    # the oracle's parity rules (element by element, exemptions for near-ties) on the tensor-core path
    spec = W.with_sizes(W.problem("di3", env_seed=8), K=1024, k=2, cap=104_096, nn_mode=pakr.NN_TENSOR)
    tree = W.prefilled_tree(spec, 100_000, seed=16)
    planner = pakr.Planner(spec)
    try:
        stats = compare(spec, tree, np.inf, 41, planner)
    finally:
        planner.close()
    assert stats["compared_children"] > 0


def test_tc_plan_matches_fp32(cuda_lib):
    # a whole AO-x run crosses the size threshold and restarts: both modes give the same history
    spec = W.with_sizes(W.problem("di3", env_seed=0), cap=300_000)
    res = []
    for mode in (pakr.NN_FP32, pakr.NN_AUTO):
        planner = pakr.Planner(W.with_sizes(spec, nn_mode=mode))
        try:
            res.append(planner.plan(spec["x_init"], spec["x_goal"], budget_s=60.0, max_iterations=60, seed=3))
        finally:
            planner.close()
    a, b = res
    assert a["iterations"] == b["iterations"]
    assert np.array_equal(a["history_cost"], b["history_cost"])
    assert np.array_equal(a["history_iteration"], b["history_iteration"])


def test_expand_graph_matches_plain_launches(cuda_lib):
    # without profiling pakr_expand launches one graph per nearest-neighbour kernel; with
    # profiling it launches the kernels one by one: same tree, bounds and seeds, same results
    spec = W.with_sizes(W.problem("di3", env_seed=9), K=512, k=4, cap=200_000)
    n0 = 28_500  # just below the automatic switch to the tensor-core kernel (28672 nodes)
    tree = W.prefilled_tree(spec, n0, seed=17, cost_hi=2.0)
    out = []
    for profile in (False, True):
        planner = pakr.Planner(spec)
        try:
            planner.tree_import(tree, spec["x_goal"])
            planner.set_profiling(profile)
            recs, sizes = [], []
            for bound, seed in ((np.inf, 1), (1.8, 2), (np.inf, 3), (1.2, 4)):  # the tree crosses the switch
                st, info = planner.expand(bound, seed)
                recs.append((st, info, planner.debug_last_expand()))
                sizes.append(planner.tree_size()[0])
            out.append((recs, sizes))
        finally:
            planner.close()
    (ra, na), (rb, nb) = out
    assert na == nb
    assert n0 < 28672 < na[0], "the first expansion runs the FP32 kernel, the later ones the tensor cores"
    for (sa, ia, da), (sb, ib, db) in zip(ra, rb):
        assert sa == sb and ia == ib
        for key in ("samples", "near", "outcome", "controls", "steps"):
            assert np.array_equal(da[key], db[key]), key


def test_host_kernel_choice_is_exact_either_way(cuda_lib):
    # the host picks the nearest-neighbour kernel from an upper bound on the tree size (exact only
    # after a read of the control block): expansions that never read it back cross the tensor-core
    # switch with a stale bound, and the planner forced to the FP32 kernel grows the same tree
    spec = W.with_sizes(W.problem("di3", env_seed=9), K=512, k=4, cap=200_000)
    n0 = 27_000
    tree = W.prefilled_tree(spec, n0, seed=17, cost_hi=2.0)
    out = []
    for mode in (pakr.NN_AUTO, pakr.NN_FP32):
        planner = pakr.Planner(W.with_sizes(spec, nn_mode=mode))
        try:
            planner.tree_import(tree, spec["x_goal"])
            for bound, seed in ((np.inf, 1), (1.8, 2), (np.inf, 3), (1.2, 4), (np.inf, 5)):
                planner.expand(bound, seed, info=False)
            out.append(planner.tree_export())
        finally:
            planner.close()
    a, b = out
    assert a["count"] == b["count"] and a["count"] > 28672
    n = a["count"]
    for key in ("states", "controls", "parents", "costs", "steps"):
        assert np.array_equal(np.asarray(a[key])[:n], np.asarray(b[key])[:n]), key


# The benchmarked workloads at their full sizes, in the launch configuration the benchmark times
# (pakr_expand's expansion graph): the 3D double integrator with 1024 parents x 8 controls on a
# 1,000,000-node tree (cap 2^20), and the 12D quadrotor with 4096 parents x 16 controls on a
# 3,934,464-node tree (cap 4,000,000).  Trees are the benchmark's seeded prefills.
BENCH_CASES = [("di3", 1_000_000, 1), ("quad12", 4_000_000 - 65536, 3)]


@pytest.mark.parametrize("name,n,tree_seed", BENCH_CASES)
def test_tc_matches_fp32_at_benchmark_size(cuda_lib, name, n, tree_seed):
    spec = W.problem(name, env_seed=0)
    tree = W.prefilled_tree(spec, n, seed=tree_seed)
    for seed in (0, 1):
        d = assert_same_expansion(spec, tree, np.inf, seed)
        assert (d["near"] >= 0).all()


@pytest.mark.parametrize("name,n,tree_seed,n_sample", [(c[0], c[1], c[2], s) for c, s in zip(BENCH_CASES, (128, 64))])
def test_tc_against_oracle_sampled_at_benchmark_size(cuda_lib, name, n, tree_seed, n_sample):
    """A sample of the queries of one benchmark expansion against the oracle's brute-force
    nearest neighbour (FP64, on the oracle's own Philox samples): the index must match unless
    the oracle's best and second-best distances are within the 1e-6 near-tie margin."""
    import oracle
    from parity import NN_GAP, SAMPLE_RTOL, rel_close

    spec = W.with_sizes(W.problem(name, env_seed=0), nn_mode=pakr.NN_TENSOR)
    tree = W.prefilled_tree(spec, n, seed=tree_seed)
    seed = 5
    _, info, dbg = expand_near(spec, tree, np.inf, seed, pakr.NN_TENSOR)
    assert info["n_start"] == n
    prob = oracle.OracleProblem(spec)
    prob.set_goal(spec["x_goal"])
    ot = oracle.OracleTree.from_arrays(spec["d"], spec["m"], n + 1, tree["states"], tree["controls"],
                                       tree["parents"], tree["costs"], tree["steps"])
    f = oracle.fcosts(prob, ot)
    rng = np.random.default_rng(7)
    picks = np.sort(rng.choice(spec["K"], n_sample, replace=False))
    exempt = 0
    for i in picks:
        q = oracle.sample_state(prob, seed, info["iteration"], int(i))
        assert np.all(rel_close(dbg["samples"][i], q, SAMPLE_RTOL))
        r = oracle.nearest(prob, ot, q, np.inf, f=f)
        if dbg["near"][i] != r["idx"]:
            assert r["d2"] - r["d1"] < NN_GAP, (i, dbg["near"][i], r)
            exempt += 1
    assert exempt <= n_sample // 16


@pytest.mark.parametrize("dyn", [W.UNICYCLE1, W.UNICYCLE2])
def test_tc_matches_fp32_other_dimensions(cuda_lib, dyn):
    # d = 3 and d = 5 use the split packed layout too (as d = 6): forced onto the tensor cores
    d, m, pdim = W.DIMS[dyn]
    if dyn == W.UNICYCLE1:
        x_lo, x_hi, u_lo, u_hi = [0, 0, -np.pi], [1, 1, np.pi], [-0.5, -1], [0.5, 1]
    else:
        x_lo, x_hi, u_lo, u_hi = [0, 0, -np.pi, -0.5, -1], [1, 1, np.pi, 0.5, 1], [-0.25, -0.5], [0.25, 0.5]
    base = W.problem("di2", env_seed=5)
    spec = W.with_sizes(base, dyn=dyn, d=d, m=m, pdim=pdim, x_lo=W.f32(x_lo), x_hi=W.f32(x_hi),
                        u_lo=W.f32(u_lo), u_hi=W.f32(u_hi), x_init=W.f32([0.1, 0.1] + [0.0] * (d - 2)),
                        x_goal=W.f32([0.9, 0.9] + [0.0] * (d - 2)), K=512, k=2, cap=60_000, dt=float(W.f32(0.1)))
    tree = W.prefilled_tree(spec, 50_003, seed=21)
    assert_same_expansion(spec, tree, np.inf, seed=3)
    tree = W.prefilled_tree(spec, 50_003, seed=22, cost_hi=2.0)
    assert_same_expansion(spec, tree, 1.5, seed=4)
