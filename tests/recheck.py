"""FP64 re-check of edges and paths the GPU produced (Sec. IV-A checks validity
at the integration substeps; this also looks between them).

Every edge is re-integrated by the oracle in FP64 from the GPU's own parent
state, control and duration:
* at the planner's substeps: the child state must match the GPU's within the
  state tolerance, and every substep must be valid unless it lies within the
  face tolerance of a deciding face (then it is counted as exempt);
* between the substeps: the double integrator's continuous edge is tested
  exactly (closed-form segment test), other models densely at dt/16; an edge
  valid at every substep that touches an obstacle in between is a "miss" of
  the discrete check, counted and reported, never hidden.
"""
from __future__ import annotations

import numpy as np

import oracle
from paper_2607_03987_gb300 import workloads as W

FACE_TOL = 1e-5
STATE_RTOL = 1e-5
DENSE_SUB = 16


def problem(spec):
    prob = oracle.OracleProblem(spec)
    prob.set_goal(spec["x_goal"])
    return prob


def check_edge(prob, spec, x0, u, S):
    """(replayed end state, substep verdict: 'valid' | 'exempt' | 'invalid', continuous miss)."""
    r = oracle.propagate(prob, x0, 0.0, u, int(S))
    if not r["collided"]:
        verdict = "valid"
    elif r["face_margin"] < FACE_TOL:
        verdict = "exempt"
    else:
        verdict = "invalid"
    if spec["dyn"] in (W.DI2, W.DI3):
        between = oracle.di_edge_hits_exact(prob, x0, u, int(S))
    else:
        between = oracle.recheck_edge_dense(prob, x0, u, int(S), DENSE_SUB)
    return r["x_end"], verdict, bool(between) and verdict == "valid"


def recheck_tree(spec, tree):
    """Re-check every edge of an exported tree (node-major FP32 arrays)."""
    prob = problem(spec)
    out = dict(edges=0, invalid=0, exempt=0, misses=0, max_rel_state_err=0.0)
    states = np.asarray(tree["states"], np.float64)
    for c in range(1, int(tree["count"])):
        p = int(tree["parents"][c])
        x_end, verdict, miss = check_edge(prob, spec, states[p], np.asarray(tree["controls"][c], np.float64),
                                          tree["steps"][c])
        err = np.max(np.abs(x_end - states[c]) / np.maximum(1.0, np.abs(states[c])))
        out["max_rel_state_err"] = max(out["max_rel_state_err"], float(err))
        out["edges"] += 1
        if verdict != "valid":
            out[verdict] += 1
        out["misses"] += int(miss)
    return out


def recheck_path(spec, states, controls, steps):
    """Re-check a path edge by edge from the GPU's states (root first), and replay the
    whole control sequence in FP64 from the start: whether that replay stays valid at
    every substep and ends in the goal ball, and its path length."""
    prob = problem(spec)
    states = np.asarray(states, np.float64)
    controls = np.asarray(controls, np.float64)
    out = dict(edges=len(steps), invalid=0, exempt=0, misses=0, max_rel_state_err=0.0)
    for e in range(len(steps)):
        x_end, verdict, miss = check_edge(prob, spec, states[e], controls[e], steps[e])
        err = np.max(np.abs(x_end - states[e + 1]) / np.maximum(1.0, np.abs(states[e + 1])))
        out["max_rel_state_err"] = max(out["max_rel_state_err"], float(err))
        if verdict != "valid":
            out[verdict] += 1
        out["misses"] += int(miss)
    out.update(replay_path(spec, states[0], controls, steps, prob))
    return out


def replay_path(spec, x_init, controls, steps, prob=None):
    """FP64 replay of a control sequence from x_init: substep validity (with the
    face-tolerance exemption), continuous misses, goal, and path length."""
    prob = problem(spec) if prob is None else prob
    x = np.asarray(x_init, np.float64)
    length, ok, exempt, misses = 0.0, True, 0, 0
    for e in range(len(steps)):
        u = np.asarray(controls[e], np.float64)
        r = oracle.propagate(prob, x, length, u, int(steps[e]))
        if r["collided"]:
            if r["face_margin"] < FACE_TOL:
                exempt += 1
            else:
                ok = False
        elif (oracle.di_edge_hits_exact(prob, x, u, int(steps[e])) if spec["dyn"] in (W.DI2, W.DI3)
              else oracle.recheck_edge_dense(prob, x, u, int(steps[e]), DENSE_SUB)):
            misses += 1
        length = r["cost_end"]
        x = r["x_end"]
    pd = spec["pdim"]
    in_goal = bool(np.linalg.norm(x[:pd] - np.asarray(spec["x_goal"][:pd], np.float64)) <= spec["goal_r"])
    return dict(replay_valid=ok, replay_exempt=exempt, replay_misses=misses, replay_in_goal=in_goal,
                replay_length=float(length))
