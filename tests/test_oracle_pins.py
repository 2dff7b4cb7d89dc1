"""Pins of the FP64 oracle to facts outside itself (no GPU).

Each test checks the oracle against something the paper or mathematics fixes:
published RNG vectors, closed-form solutions, rigid-body invariants, a k-d tree
library routine, hand-worked validity cases, and invariants of the tree and of
the AO-x bound.  A dropped term, a wrong sign, index or transposed operand in
the oracle fails at least one of them.
"""
import os

import numpy as np
import pytest
from scipy import stats
from scipy.spatial import cKDTree

import oracle
from paper_2607_03987_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def prob_of(spec):
    p = oracle.OracleProblem(spec)
    p.set_goal(spec["x_goal"])
    return p


# ---------------------------------------------------------------- Philox ----
def test_philox_known_answer_vectors():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if not ln.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r if x != "->"]
        ctr, key, want = v[0:4], v[4:6], v[6:10]
        assert oracle.philox4x32_10(ctr, key) == want


def test_u01_exact_endpoints():
    assert oracle.u01(0) == 0.0
    assert oracle.u01(0xFF) == 0.0
    assert oracle.u01(0x100) == 2.0 ** -24
    assert oracle.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24


def test_state_samples_uniform_and_independent():
    spec = W.problem("di3", env_seed=0)
    P = prob_of(spec)
    xs = np.array([oracle.sample_state(P, 42, 3, i) for i in range(20000)])
    lo, hi = spec["x_lo"], spec["x_hi"]
    assert np.all(xs >= lo) and np.all(xs < hi)
    for a in range(spec["d"]):
        u = (xs[:, a] - lo[a]) / (hi[a] - lo[a])
        assert stats.kstest(u, "uniform").pvalue > 1e-3
    c = np.corrcoef(xs.T)
    assert np.all(np.abs(c - np.eye(spec["d"])) < 0.03)
    # distinct iterations and seeds give distinct streams
    assert not np.allclose(oracle.sample_state(P, 42, 3, 0), oracle.sample_state(P, 42, 4, 0))
    assert not np.allclose(oracle.sample_state(P, 42, 3, 0), oracle.sample_state(P, 43, 3, 0))


def test_control_samples_and_durations():
    spec = W.problem("quad12", env_seed=0)
    P = prob_of(spec)
    us, Ss = [], []
    for i in range(200):
        for j in range(50):
            u, S = oracle.sample_control(P, 7, 1, i, j)
            us.append(u)
            Ss.append(S)
    us, Ss = np.array(us), np.array(Ss)
    assert np.all(us >= spec["u_lo"]) and np.all(us < spec["u_hi"])
    counts = np.bincount(Ss - spec["s_min"], minlength=spec["s_max"] - spec["s_min"] + 1)
    assert Ss.min() == spec["s_min"] and Ss.max() == spec["s_max"]
    assert stats.chisquare(counts).pvalue > 1e-3
    for a in range(spec["m"]):
        u = (us[:, a] - spec["u_lo"][a]) / (spec["u_hi"][a] - spec["u_lo"][a])
        assert stats.kstest(u, "uniform").pvalue > 1e-3
    # the duration and control words differ from the state sample words
    P2 = prob_of(W.with_sizes(spec, s_min=5, s_max=5))
    assert all(oracle.sample_control(P2, 7, 1, 3, j)[1] == 5 for j in range(20))


# ---------------------------------------------------- double integrator ----
def open_problem(name):
    spec = W.problem(name, env_seed=0)
    return W.with_sizes(spec, boxes=np.zeros((0, 2 * spec["pdim"])), x_lo=spec["x_lo"] * 0 - 100,
                        x_hi=spec["x_hi"] * 0 + 100)


@pytest.mark.parametrize("name", ["di2", "di3"])
def test_double_integrator_matches_closed_form(name):
    spec = open_problem(name)
    P = prob_of(spec)
    pd, dt = spec["pdim"], spec["dt"]
    rng = np.random.default_rng(0)
    for _ in range(50):
        x0 = rng.uniform(-1, 1, spec["d"])
        u = rng.uniform(-1, 1, spec["m"])
        S = int(rng.integers(1, 21))
        r = oracle.propagate(P, x0, 0.25, u, S)
        t = S * dt
        p = x0[:pd] + x0[pd:] * t + 0.5 * u * t * t
        v = x0[pd:] + u * t
        assert np.allclose(r["x_end"][:pd], p, atol=1e-12)
        assert np.allclose(r["x_end"][pd:], v, atol=1e-12)
        ts = np.arange(S + 1) * dt
        ps = x0[:pd][None] + x0[pd:][None] * ts[:, None] + 0.5 * u[None] * ts[:, None] ** 2
        length = np.sum(np.linalg.norm(np.diff(ps, axis=0), axis=1))
        assert abs(r["cost_end"] - (0.25 + length)) < 1e-12
        assert not r["collided"]


def test_duration_cost():
    spec = W.with_sizes(open_problem("di3"), cost=W.COST_DURATION)
    P = prob_of(spec)
    r = oracle.propagate(P, np.zeros(6), 1.0, np.ones(3) * 0.1, 7)
    assert abs(r["cost_end"] - (1.0 + 7 * spec["dt"])) < 1e-15


# ------------------------------------------------------------ quadrotor ----
def rot(phi, th, psi):
    cx, sx, cy, sy, cz, sz = np.cos(phi), np.sin(phi), np.cos(th), np.sin(th), np.cos(psi), np.sin(psi)
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def skew(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])


@pytest.fixture
def quad():
    spec = W.problem("quad12", env_seed=0)
    spec = W.with_sizes(spec, boxes=np.zeros((0, 6)), x_lo=np.full(12, -1e3), x_hi=np.full(12, 1e3))
    return spec, prob_of(spec)


def test_quad_hover_is_equilibrium(quad):
    spec, P = quad
    m, g = spec["model"][0], spec["model"][4]
    x = np.zeros(12)
    x[:3] = [0.3, 0.4, 0.5]
    x[5] = 0.7  # any yaw
    xd = oracle.dynamics(P, x, [m * g, 0, 0, 0])
    assert np.allclose(xd, 0, atol=1e-12)


def test_quad_free_fall_closed_form(quad):
    spec, P = quad
    g = spec["model"][4]
    x0 = np.zeros(12)
    x0[2] = 0.5
    r = oracle.propagate(P, x0, 0.0, np.zeros(4), 20)
    t = 20 * spec["dt"]
    assert abs(r["x_end"][2] - (0.5 - 0.5 * g * t * t)) < 1e-12
    assert abs(r["x_end"][8] + g * t) < 1e-12
    assert np.allclose(np.delete(r["x_end"], [2, 8]), 0, atol=1e-14)


def test_quad_kinematics_consistent_with_body_rates(quad):
    spec, P = quad
    rng = np.random.default_rng(1)
    for _ in range(20):
        x = np.zeros(12)
        x[3:6] = rng.uniform([-1, -1, -3], [1, 1, 3])
        x[6:9] = rng.uniform(-1, 1, 3)
        x[9:12] = rng.uniform(-2, 2, 3)
        u = np.array([rng.uniform(0, 20), *rng.uniform(-0.5, 0.5, 3)])
        xd = oracle.dynamics(P, x, u)
        R = rot(*x[3:6])
        # position rate is the body velocity rotated to the world frame
        assert np.allclose(xd[:3], R @ x[6:9], atol=1e-12)
        # Euler-angle rates reproduce R' = R [omega]x
        h = 1e-6
        dR = (rot(*(x[3:6] + h * xd[3:6])) - rot(*(x[3:6] - h * xd[3:6]))) / (2 * h)
        assert np.allclose(dR, R @ skew(x[9:12]), atol=1e-7)
        # world-frame acceleration of the body velocity: gravity plus rotated thrust
        m, g = spec["model"][0], spec["model"][4]
        acc_world = R @ skew(x[9:12]) @ x[6:9] + R @ xd[6:9]
        assert np.allclose(acc_world, np.array([0, 0, -g]) + R @ np.array([0, 0, u[0] / m]), atol=1e-10)
        # Euler's rotation equations
        I = np.array(spec["model"][1:4])
        w = x[9:12]
        assert np.allclose(I * xd[9:12] + np.cross(w, I * w), u[1:], atol=1e-10)


def test_quad_torque_free_invariants(quad):
    spec, P = quad
    I = np.array(spec["model"][1:4])
    x = np.zeros(12)
    x[3:6] = [0.2, -0.1, 0.4]
    x[9:12] = [1.5, -0.7, 2.0]
    g = spec["model"][4]
    u = np.array([spec["model"][0] * g, 0, 0, 0])
    L0 = rot(*x[3:6]) @ (I * x[9:12])
    E0 = 0.5 * np.sum(I * x[9:12] ** 2)
    for _ in range(300):
        x = oracle.rk4_step(P, x, u, 1e-3)
    L1 = rot(*x[3:6]) @ (I * x[9:12])
    E1 = 0.5 * np.sum(I * x[9:12] ** 2)
    assert np.allclose(L1, L0, rtol=1e-8, atol=1e-12)
    assert abs(E1 - E0) < 1e-9 * E0


def test_rk4_is_fourth_order(quad):
    spec, P = quad
    x0 = np.zeros(12)
    x0[3:6] = [0.3, -0.2, 0.1]
    x0[6:9] = [0.2, 0.1, -0.3]
    x0[9:12] = [1.0, -2.0, 0.5]
    u = np.array([12.0, 0.01, -0.02, 0.005])
    T = 0.4

    def integrate(n):
        x = x0.copy()
        for _ in range(n):
            x = oracle.rk4_step(P, x, u, T / n)
        return x

    ref = integrate(1024)
    errs = [np.linalg.norm(integrate(n) - ref) for n in (8, 16, 32)]
    ratios = [errs[i] / errs[i + 1] for i in range(2)]
    assert all(12 < r < 20 for r in ratios), ratios


@pytest.mark.parametrize("dyn", [W.DUBINS3D, W.UNICYCLE1, W.UNICYCLE2])
def test_kinematic_models(dyn):
    d, m, pd = W.DIMS[dyn]
    spec = W.with_sizes(W.problem("di3"), dyn=dyn, d=d, m=m, pdim=pd)
    P = prob_of(spec)
    if dyn == W.DUBINS3D:
        xd = oracle.dynamics(P, [0, 0, 0, np.pi / 2, 0, 2.0], [0.1, 0.2, 0.3])
        assert np.allclose(xd, [0, 2.0, 0, 0.1, 0.2, 0.3], atol=1e-15)
        xd = oracle.dynamics(P, [0, 0, 0, 0, np.pi / 6, 2.0], [0, 0, 0])
        assert np.allclose(xd[:3], [2 * np.cos(np.pi / 6), 0, 1.0], atol=1e-15)
    elif dyn == W.UNICYCLE1:
        xd = oracle.dynamics(P, [0, 0, np.pi / 2], [1.5, -0.3])
        assert np.allclose(xd, [0, 1.5, -0.3], atol=1e-15)
    else:
        xd = oracle.dynamics(P, [0, 0, np.pi, 0.5, 0.2], [0.1, -0.1])
        assert np.allclose(xd, [-0.5, 0, 0.2, 0.1, -0.1], atol=1e-15)


# ------------------------------------------------------------- validity ----
def test_validity_hand_cases():
    spec = W.problem("di2", env_seed=0)
    spec = W.with_sizes(spec, boxes=np.array([[0.4, 0.4, 0.6, 0.6]]), spheres=np.array([[0.2, 0.2, 0.1]]))
    P = prob_of(spec)
    V = lambda *x: oracle.state_valid(P, np.array(x, dtype=float))  # noqa: E731
    assert not V(0.5, 0.5, 0, 0)
    assert not V(0.4, 0.5, 0, 0)      # closed box: the face is an obstacle
    assert V(0.39, 0.5, 0, 0)
    assert V(1.0, 0.5, 0, 0)          # closed state box: the bound is valid
    assert not V(1.0001, 0.5, 0, 0)
    assert V(0.9, 0.9, 1.0, -1.0)
    assert not V(0.9, 0.9, 1.01, 0)
    assert not V(0.3, 0.2, 0, 0)      # on the sphere
    assert V(0.31, 0.2, 0, 0)
    assert not V(np.nan, 0.5, 0, 0)
    assert abs(oracle.face_margin(P, np.array([0.39, 0.5, 0, 0])) - 0.01) < 1e-12


def test_heuristic_values():
    spec = W.problem("di3", env_seed=0)
    P = prob_of(spec)
    g = spec["x_goal"]
    assert oracle.heuristic(P, g) == 0.0
    x = g.copy()
    x[0] -= 0.5
    x[4] = 0.9  # velocity does not enter the position heuristic
    assert abs(oracle.heuristic(P, x) - (0.5 - spec["goal_r"])) < 1e-15
    Pd = prob_of(W.with_sizes(spec, cost=W.COST_DURATION))
    assert abs(oracle.heuristic(Pd, x) - (0.5 - spec["goal_r"]) / spec["h_speed"]) < 1e-15
    Pf = prob_of(W.with_sizes(spec, heuristic=W.H_FULLSTATE))
    assert abs(oracle.heuristic(Pf, x) - np.hypot(0.5, 0.9)) < 1e-15


# ------------------------------------------------------ nearest neighbour ----
def eligible_numpy(spec, states, costs, bound):
    pd = spec["pdim"]
    h = np.maximum(0.0, np.linalg.norm(states[:, :pd] - spec["x_goal"][:pd], axis=1) - spec["goal_r"])
    return costs + h < bound


@pytest.mark.parametrize("weights", [None, [1, 1, 1, 0.25, 0.25, 0.25]])
@pytest.mark.parametrize("bound", [np.inf, 1.8])
def test_nearest_matches_kdtree(weights, bound):
    spec = W.with_sizes(W.problem("di3", env_seed=0), nn_w=None if weights is None else W.f32(weights))
    P = prob_of(spec)
    tree = W.prefilled_tree(spec, 700, seed=3, cost_hi=1.5)
    T = oracle.OracleTree.from_arrays(6, 3, 1000, tree["states"], tree["controls"], tree["parents"],
                                      tree["costs"], tree["steps"])
    elig = eligible_numpy(spec, tree["states"], tree["costs"], bound)
    idx = np.nonzero(elig)[0]
    w = np.ones(6) if weights is None else np.asarray(weights)
    kd = cKDTree(tree["states"][idx] * np.sqrt(w))
    rng = np.random.default_rng(5)
    for q in rng.uniform(spec["x_lo"], spec["x_hi"], (200, 6)):
        r = oracle.nearest(P, T, q, bound)
        dist, j = kd.query(q * np.sqrt(w), k=2)
        assert r["idx"] == idx[j[0]]
        assert abs(r["d1"] - dist[0]) < 1e-12 and abs(r["d2"] - dist[1]) < 1e-12


def test_nearest_tie_lowest_index_and_empty():
    spec = W.problem("di2", env_seed=0)
    P = prob_of(spec)
    tree = W.prefilled_tree(spec, 50, seed=1)
    tree["states"][40] = tree["states"][7]
    T = oracle.OracleTree.from_arrays(4, 2, 64, tree["states"], tree["controls"], tree["parents"], tree["costs"],
                                      tree["steps"])
    r = oracle.nearest(P, T, tree["states"][7], np.inf)
    assert r["idx"] == 7 and r["d1"] == 0.0 and r["d2"] == 0.0
    r = oracle.nearest(P, T, tree["states"][7], 0.0)  # nothing has f < 0
    assert r["idx"] == -1


# ------------------------------------------------------- tree invariants ----
def di_replay(spec, x0, u, S):
    pd, dt = spec["pdim"], spec["dt"]
    ts = np.arange(S + 1) * dt
    ps = x0[:pd][None] + x0[pd:][None] * ts[:, None] + 0.5 * u[None] * ts[:, None] ** 2
    vs = x0[pd:][None] + u[None] * ts[:, None]
    return np.concatenate([ps, vs], axis=1)


def numpy_valid(spec, x):
    if np.any(x < spec["x_lo"]) or np.any(x > spec["x_hi"]):
        return False
    pd = spec["pdim"]
    for b in spec["boxes"]:
        if np.all(x[:pd] >= b[:pd]) and np.all(x[:pd] <= b[pd:]):
            return False
    return True


@pytest.mark.parametrize("bound", [np.inf, 1.6])
def test_tree_invariants_after_expansions(bound):
    spec = W.with_sizes(W.problem("di3", env_seed=2), K=128, k=6, cap=30000)
    P = prob_of(spec)
    T = oracle.OracleTree(6, 3, spec["cap"])
    oracle.tree_reset(P, T, spec["x_init"])
    R = spec["K"] * spec["k"]
    for it in range(6):
        n0 = T.count
        e = oracle.expand(P, T, bound, 17)
        # bookkeeping of one batch
        assert e["n_appended"] + e["n_pruned"] + e["n_collided"] + e["n_no_parent"] + e["n_dropped"] == R
        assert T.count == n0 + e["n_appended"] and T.iteration == it + 1
        assert np.all(e["near"] < n0)  # the frozen snapshot: no node of this batch is a parent in it
        app = np.nonzero(e["outcome"] == oracle.OUT_APPENDED)[0]
        assert np.array_equal(e["node"][app], n0 + np.arange(len(app)))  # ascending rollout order
        assert np.all(e["f_end"][app] < bound)
        assert np.all(e["f_end"][e["outcome"] == oracle.OUT_PRUNED] >= bound)
        if e["goal_found"]:
            g = app[e["in_goal"][app] == 1]
            assert e["goal_cost"] == e["cost_end"][g].min()
    a = T.arrays()
    pd = spec["pdim"]
    for c in range(1, T.count):
        par = a["parents"][c]
        assert 0 <= par < c
        S = a["steps"][c]
        assert spec["s_min"] <= S <= spec["s_max"]
        u = a["controls"][c]
        assert np.all(u >= spec["u_lo"]) and np.all(u <= spec["u_hi"])
        traj = di_replay(spec, a["states"][par], u, S)
        assert np.allclose(traj[-1], a["states"][c], atol=1e-12)
        length = np.sum(np.linalg.norm(np.diff(traj[:, :pd], axis=0), axis=1))
        assert abs(a["costs"][c] - (a["costs"][par] + length)) < 1e-12
        assert all(numpy_valid(spec, s) for s in traj[1:])


def test_tree_full_truncates_in_rollout_order():
    spec = W.with_sizes(W.problem("di3", env_seed=1), K=256, k=8, cap=300)
    P = prob_of(spec)
    T = oracle.OracleTree(6, 3, spec["cap"])
    oracle.tree_reset(P, T, spec["x_init"])
    e = oracle.expand(P, T, np.inf, 3)
    assert T.count == 300 and e["n_dropped"] > 0 and e["status"] == oracle.TREE_FULL
    surv = np.nonzero((e["outcome"] == oracle.OUT_APPENDED) | (e["outcome"] == oracle.OUT_DROPPED))[0]
    assert np.all(e["outcome"][surv[:299]] == oracle.OUT_APPENDED)
    assert np.all(e["outcome"][surv[299:]] == oracle.OUT_DROPPED)


# ------------------------------------------------------------------ AO-x ----
@pytest.mark.parametrize("seed", [0, 1])
def test_aox_bound_decreases_and_paths_replay(seed):
    spec = W.problem("di2", env_seed=4)
    P = prob_of(spec)
    T = oracle.OracleTree(4, 2, spec["cap"])
    res = oracle.plan(P, T, spec["x_init"], seed, 80)
    assert res["n_solutions"] >= 1
    assert np.all(np.diff(res["hist_cost"]) < 0)
    # replay the best path from x_init with the closed form
    x = spec["x_init"].astype(float)
    cost = 0.0
    pd = spec["pdim"]
    for t in range(1, len(res["path"])):
        traj = di_replay(spec, x, res["path_controls"][t], res["path_steps"][t])
        assert all(numpy_valid(spec, s) for s in traj[1:])
        cost += np.sum(np.linalg.norm(np.diff(traj[:, :pd], axis=0), axis=1))
        x = traj[-1]
        assert np.allclose(x, res["path_states"][t], atol=1e-12)
    assert abs(cost - res["best_cost"]) < 1e-12
    assert np.linalg.norm(x[:pd] - spec["x_goal"][:pd]) <= spec["goal_r"]
    lb = np.linalg.norm(spec["x_goal"][:pd] - spec["x_init"][:pd]) - spec["goal_r"]
    assert res["best_cost"] >= lb


def test_aox_no_eligible_when_bound_unbeatable():
    spec = W.problem("di2", env_seed=4)
    P = prob_of(spec)
    T = oracle.OracleTree(4, 2, spec["cap"])
    oracle.tree_reset(P, T, spec["x_init"])
    e = oracle.expand(P, T, 0.5, 1)  # root f (about 1.08) is above the bound
    assert e["status"] == oracle.NO_ELIGIBLE and e["n_no_parent"] == spec["K"] * spec["k"]


# ------------------------------------------------------- dense re-check ----
def test_exact_di_segment_check_agrees_with_dense_sampling():
    spec = W.problem("di2", env_seed=6)
    P = prob_of(spec)
    rng = np.random.default_rng(2)
    agree = 0
    for _ in range(300):
        x0 = np.concatenate([rng.uniform(0.05, 0.95, 2), rng.uniform(-1, 1, 2)])
        if not numpy_valid(spec, x0):
            continue
        u = rng.uniform(-1, 1, 2)
        S = int(rng.integers(1, 11))
        ts = np.linspace(0, S * spec["dt"], 20001)[1:]
        ps = x0[:2][None] + x0[2:][None] * ts[:, None] + 0.5 * u[None] * ts[:, None] ** 2
        vs = x0[2:][None] + u[None] * ts[:, None]
        dense = not all(numpy_valid(spec, np.concatenate([p, v])) for p, v in zip(ps[::10], vs[::10]))
        exact = oracle.di_edge_hits_exact(P, x0, u, S)
        if dense:
            assert exact  # anything a dense sample sees, the exact check sees
        agree += dense == exact
    assert agree > 250


def test_discrete_check_misses_are_counted():
    spec = W.with_sizes(W.problem("di3", env_seed=3), K=256, k=8, cap=40000)
    P = prob_of(spec)
    T = oracle.OracleTree(6, 3, spec["cap"])
    oracle.tree_reset(P, T, spec["x_init"])
    for _ in range(4):
        oracle.expand(P, T, np.inf, 9)
    a = T.arrays()
    misses = 0
    for c in range(1, T.count):
        misses += oracle.di_edge_hits_exact(P, a["states"][a["parents"][c]], a["controls"][c], a["steps"][c])
    # the planner checks substeps only (Sec. IV-A); edges that graze an obstacle between substeps exist
    # and are reported, but they are a small fraction
    assert misses < 0.05 * T.count


def test_dense_recheck_at_one_substep_is_the_planners_check():
    # sub = 1 re-integrates at the planner's own step: it must flag exactly the edges that the
    # oracle's propagation marks as collided (Sec. IV-A: validity at every substep)
    spec = W.problem("di3", env_seed=3)
    P = prob_of(spec)
    rng = np.random.default_rng(11)
    flagged = 0
    for _ in range(400):
        x0 = np.concatenate([rng.uniform(0.05, 0.95, 3), rng.uniform(-1, 1, 3)])
        if not numpy_valid(spec, x0):
            continue
        u = rng.uniform(-1, 1, 3)
        S = int(rng.integers(1, 21))
        col = oracle.propagate(P, x0, 0.0, u, S)["collided"]
        assert oracle.recheck_edge_dense(P, x0, u, S, 1) == col
        flagged += col
    assert flagged > 20


def test_dense_recheck_agrees_with_exact_segment_test():
    # boxes only: a fine state the dense check finds invalid lies on the closed-form path, so the
    # exact continuous test must report a hit too; the exact test's hits are found by the dense
    # check at dt/256 except for grazes shorter than that
    spec = W.problem("di3", env_seed=5)
    P = prob_of(spec)
    rng = np.random.default_rng(12)
    n_exact = n_dense = 0
    for _ in range(300):
        x0 = np.concatenate([rng.uniform(0.05, 0.95, 3), rng.uniform(-1, 1, 3)])
        if not numpy_valid(spec, x0):
            continue
        u = rng.uniform(-1, 1, 3)
        S = int(rng.integers(1, 21))
        exact = oracle.di_edge_hits_exact(P, x0, u, S)
        dense = oracle.recheck_edge_dense(P, x0, u, S, 256)
        if dense:
            assert exact
        n_exact += exact
        n_dense += dense
    assert n_exact > 30 and n_dense >= 0.97 * n_exact


def test_dense_recheck_finds_a_sphere_between_substeps():
    # straight flight at constant velocity through a small sphere that lies between two substeps:
    # the substep check misses it, the dense check sees it; moved off the line by 1.5 radii (a
    # closest approach computed in closed form) nothing is hit
    base = W.problem("di3", env_seed=0)
    r = 0.004
    v = np.array([1.0, 0.0, 0.0])
    x0 = np.concatenate([[0.2, 0.5, 0.5], v])
    dt = base["dt"]
    centre = x0[:3] + v * 1.5 * dt  # midway between substeps 1 and 2 (0.05 apart, more than 2r)
    u = np.zeros(3)
    for offset, want in ((0.0, True), (1.5 * r, False)):
        c = centre + np.array([0.0, offset, 0.0])
        # closest approach of the line p(t) = x0 + v t to the centre
        t_star = float(np.dot(c - x0[:3], v) / np.dot(v, v))
        closest = np.linalg.norm(x0[:3] + v * t_star - c)
        assert (closest <= r) == want
        spec = W.with_sizes(base, boxes=np.zeros((0, 6)), spheres=np.array([[*c, r]]))
        P = prob_of(spec)
        assert not oracle.recheck_edge_dense(P, x0, u, 3, 1)
        assert oracle.recheck_edge_dense(P, x0, u, 3, 16) == want
