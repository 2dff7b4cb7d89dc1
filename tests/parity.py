"""Element-by-element comparison of one GPU expansion with the FP64 oracle.

The comparison rules follow the stated margins: nearest-neighbour indices,
validity and goal flags must match exactly unless the oracle shows the case is
too close to call across precisions (distance gap < 1e-6, a substep within 1e-5
of a deciding face, the f-cost within 1e-5*max(1, bound) of the bound, the end
position within 1e-5 of the goal sphere); states, costs and controls must agree
within 1e-5 relative.  Exempt cases are counted and returned, never hidden.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2607_03987_gb300 import pakr

STATE_RTOL = 1e-5
SAMPLE_RTOL = 1e-6
NN_GAP = 1e-6
FACE_TOL = 1e-5
GOAL_TOL = 1e-5


def rel_close(a, b, rtol):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return np.abs(a - b) <= rtol * np.maximum(1.0, np.abs(b))


def oracle_expand(spec, tree, bound, seed):
    prob = oracle.OracleProblem(spec)
    prob.set_goal(spec["x_goal"])
    otree = oracle.OracleTree.from_arrays(spec["d"], spec["m"], spec["cap"], tree["states"], tree["controls"],
                                          tree["parents"], tree["costs"], tree["steps"], tree.get("iteration", 0))
    ref = oracle.expand(prob, otree, bound, seed)
    return ref, otree


def gpu_expand(planner, spec, tree, bound, seed):
    planner.tree_import(tree, spec["x_goal"])
    st, info = planner.expand(bound, seed)
    dbg = planner.debug_last_expand()
    gtree = planner.tree_export()
    return st, info, dbg, gtree


def compare(spec, tree, bound, seed, planner, require_all=False):
    """Run both sides on the same tree; assert the rules; return exemption stats."""
    ref, otree = oracle_expand(spec, tree, bound, seed)
    st, info, dbg, gtree = gpu_expand(planner, spec, tree, bound, seed)
    K, k, d, m = spec["K"], spec["k"], spec["d"], spec["m"]
    R = K * k
    stats = dict(nn_exempt=0, rollout_exempt=0, goal_exempt=0, compared_rollouts=0, compared_children=0)
    # samples and controls: same Philox words, FP32 vs FP64 rounding of lo + (hi-lo) v
    assert np.all(rel_close(dbg["samples"], ref["samples"], SAMPLE_RTOL)), "state samples differ"
    assert np.all(rel_close(dbg["controls"], ref["u"], SAMPLE_RTOL)), "controls differ"
    assert np.array_equal(dbg["steps"], ref["S"]), "durations differ"
    # nearest neighbour
    near_o = ref["near"]
    near_g = dbg["near"].astype(np.int64)
    with np.errstate(invalid="ignore"):  # inf - inf where a query has no second eligible node
        nn_ex = (ref["nn_fragile"] != 0) | (ref["nn_d2"] - ref["nn_d1"] < NN_GAP)
    bad = (near_o != near_g) & ~nn_ex
    assert not bad.any(), f"NN mismatch at queries {np.nonzero(bad)[0][:10]}: gpu {near_g[bad][:10]} ora {near_o[bad][:10]}"
    stats["nn_exempt"] = int(((near_o != near_g) & nn_ex).sum())
    same_parent = np.repeat(near_o == near_g, k)
    # rollouts
    oo = ref["outcome"]
    go = dbg["outcome"].astype(np.int32)
    finite_bound = np.isfinite(bound)
    tol_f = 1e-5 * max(1.0, abs(bound)) if finite_bound else np.inf
    f_ex = np.abs(ref["f_end"] - bound) < tol_f if finite_bound else np.zeros(R, bool)
    f_ex &= np.isfinite(ref["f_end"])
    face_ex = ref["face_margin"] < FACE_TOL
    ex = f_ex | face_ex | ~same_parent
    o_np = oo == oracle.OUT_NO_PARENT
    assert np.array_equal(o_np[same_parent], (go == pakr.ROLLOUT_NO_PARENT)[same_parent]), "no-parent mismatch"
    o_survive = (oo == oracle.OUT_APPENDED) | (oo == oracle.OUT_DROPPED)
    g_survive = (go == pakr.ROLLOUT_APPENDED) | (go == pakr.ROLLOUT_DROPPED)
    bad = (o_survive != g_survive) & ~ex
    assert not bad.any(), (f"survival mismatch at rollouts {np.nonzero(bad)[0][:10]}: gpu {go[bad][:10]} "
                           f"ora {oo[bad][:10]} f {ref['f_end'][bad][:5]} bound {bound}")
    o_col = (oo == oracle.OUT_COLLIDED)
    bad = o_col & (go != pakr.ROLLOUT_COLLIDED) & ~ex
    assert not bad.any(), f"collision mismatch at rollouts {np.nonzero(bad)[0][:10]}"
    o_pr = oo == oracle.OUT_PRUNED
    bad = o_pr & g_survive & ~ex
    assert not bad.any(), f"prune mismatch at rollouts {np.nonzero(bad)[0][:10]}"
    stats["rollout_exempt"] = int((ex & ((o_survive != g_survive) | (o_col != (go == pakr.ROLLOUT_COLLIDED)))).sum())
    stats["compared_rollouts"] = int((~ex).sum())
    # appended children, matched by rollout
    n0 = ref["n_start"]
    g_app = go == pakr.ROLLOUT_APPENDED
    g_node = np.full(R, -1, np.int64)
    g_node[g_app] = n0 + np.arange(int(g_app.sum()))
    o_node = ref["node"]
    both = g_app & (oo == oracle.OUT_APPENDED)
    otr = otree.arrays()
    gi, oi = g_node[both], o_node[both]
    if both.any():
        assert np.all(rel_close(gtree["states"][gi], otr["states"][oi], STATE_RTOL)), "child states differ"
        assert np.all(rel_close(gtree["costs"][gi], otr["costs"][oi], STATE_RTOL)), "child costs differ"
        assert np.all(rel_close(gtree["controls"][gi], otr["controls"][oi], SAMPLE_RTOL)), "child controls differ"
        assert np.array_equal(gtree["parents"][gi], otr["parents"][oi]), "child parents differ"
        assert np.array_equal(gtree["steps"][gi], otr["steps"][oi]), "child durations differ"
    stats["compared_children"] = int(both.sum())
    # the untouched prefix of the tree is unchanged
    assert np.array_equal(gtree["parents"][:n0], np.asarray(tree["parents"])[:n0])
    # goal flag of every surviving child with the same parent, outside the goal band
    goal_ex = (ref["goal_margin"] < GOAL_TOL) & o_survive
    stats["goal_exempt"] = int(goal_ex.sum())
    g_goal = dbg["goal"].astype(bool)
    assert not (g_goal & ~g_survive).any(), "goal flag on a rollout that did not survive"
    cmp_goal = g_survive & same_parent & ~(ref["goal_margin"] < GOAL_TOL)
    bad = cmp_goal & (g_goal != (ref["in_goal"] != 0))
    assert not bad.any(), f"goal flag mismatch at rollouts {np.nonzero(bad)[0][:10]}"
    stats["compared_goal_flags"] = int(cmp_goal.sum())
    check_counts(spec, tree, bound, ref, st, info, dbg, gtree, ex, g_survive, o_survive)
    stats["counts_checked"] = True
    any_exempt = stats["nn_exempt"] + stats["rollout_exempt"] + stats["goal_exempt"] > 0
    if not any_exempt:
        assert info["n_appended"] == ref["n_appended"], (info["n_appended"], ref["n_appended"])
        assert info["n_dropped"] == ref["n_dropped"]
        assert info["n_no_parent"] == ref["n_no_parent"]
        assert gtree["count"] == otree.count
        assert bool(info["goal_found"]) == bool(ref["goal_found"])
        if ref["goal_found"]:
            assert info["goal_idx"] == ref["goal_idx"]
            assert rel_close(info["goal_cost"], ref["goal_cost"], STATE_RTOL)
        assert gtree["iteration"] == otree.iteration
        assert st == ref["status"], (st, ref["status"])
    if require_all:
        assert not any_exempt, stats
    stats.update(status=st, ref=ref, info=info, gtree=gtree, otree=otree, dbg=dbg)
    return stats


def check_counts(spec, tree, bound, ref, st, info, dbg, gtree, ex, g_survive, o_survive):
    """Counts, tree size, goal choice and status of one expansion, element by
    element after exempt rollouts are set aside.

    On an exempt rollout both survival answers are right, so the GPU's answer
    stands there and the oracle's everywhere else; that merged survivor set
    fixes, in ascending rollout order, which children are appended and which
    are dropped at the cap, the node count and the status.  The goal child
    must be the cheapest appended child in the goal ball (costs within the
    state tolerance), and the goal flags on the rest were compared above.
    """
    R = spec["K"] * spec["k"]
    go = dbg["outcome"].astype(np.int32)
    n0 = int(ref["n_start"])
    cap = spec["cap"]
    surv = np.where(ex, g_survive, o_survive)
    n_surv = int(surv.sum())
    n_app = min(n_surv, max(cap - n0, 0))
    assert info["n_start"] == n0
    assert info["n_appended"] == n_app, (info["n_appended"], n_app)
    assert info["n_dropped"] == n_surv - n_app, (info["n_dropped"], n_surv - n_app)
    assert np.array_equal(np.nonzero(go == pakr.ROLLOUT_APPENDED)[0], np.nonzero(surv)[0][:n_app]), \
        "appended rollouts are not the first survivors in rollout order"
    assert np.array_equal(np.nonzero(go == pakr.ROLLOUT_DROPPED)[0], np.nonzero(surv)[0][n_app:])
    # no eligible parent depends on eligibility alone, never on a near-tie
    assert info["n_no_parent"] == ref["n_no_parent"] == int((go == pakr.ROLLOUT_NO_PARENT).sum())
    assert info["n_pruned"] + info["n_collided"] + n_surv + info["n_no_parent"] == R
    assert gtree["count"] == n0 + n_app
    # the goal child: among the appended children flagged in the goal ball, the cheapest
    app = np.nonzero(go == pakr.ROLLOUT_APPENDED)[0]
    flagged = app[dbg["goal"][app] != 0]
    assert bool(info["goal_found"]) == (flagged.size > 0)
    if flagged.size:
        nodes = n0 + np.searchsorted(app, flagged)
        costs = np.asarray(gtree["costs"], np.float64)[nodes]
        assert info["goal_idx"] in set(nodes.tolist())
        c_min = costs.min()
        assert float(gtree["costs"][info["goal_idx"]]) <= c_min + STATE_RTOL * max(1.0, abs(c_min))
        assert rel_close(info["goal_cost"], gtree["costs"][info["goal_idx"]], 0.0)
    # status, in the ABI's order of precedence
    if info["n_no_parent"] == R:
        want = pakr.NO_ELIGIBLE
    elif info["goal_found"]:
        want = pakr.GOAL_REACHED
    elif n_surv > n_app:
        want = pakr.TREE_FULL
    else:
        want = pakr.OK
    assert st == want, (st, want)
