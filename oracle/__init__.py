"""FP64 CPU oracle of the PAKR expansion iteration -- TEST INFRASTRUCTURE.

Plain single-threaded C (``pakr_oracle.c``) wrapped with ctypes.  It restates
Algorithm 1 of the paper step by step (SampleStates, NearestNeighbor,
SampleControls, Propagate, cost-bounded pruning, CollisionFree, insert, goal
test, ExtractPath) and the AO-x outer loop.  Only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm may
import this package; the CUDA library never does, and this package never
imports the CUDA library.

Parity of the quadrotor model against the paper is unpinned (the paper prints
no equations); it is pinned to rigid-body invariants in the tests.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pakr_oracle.c")
_LIB = os.path.join(_HERE, "libpakr_oracle.so")

MAX_D = 16
MAX_M = 8

DI2, DI3, QUAD12, DUBINS3D, UNICYCLE1, UNICYCLE2 = range(6)
COST_PATH_LENGTH, COST_DURATION = 0, 1
H_POSITION, H_FULLSTATE = 0, 1
OUT_APPENDED, OUT_PRUNED, OUT_COLLIDED, OUT_NO_PARENT, OUT_DROPPED = range(5)
OK, GOAL_REACHED, TREE_FULL, NO_ELIGIBLE, BUDGET_EXPIRED = range(5)
ERR_INVALID_ARG = -1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (IEEE semantics: no fast-math, no FMA contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "pakr_oracle.h"))
    ):
        return _LIB
    tmp = _LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-std=c99", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class Problem(C.Structure):
    _fields_ = [
        ("dyn", C.c_int), ("d", C.c_int), ("m", C.c_int), ("pdim", C.c_int),
        ("x_lo", C.c_double * MAX_D), ("x_hi", C.c_double * MAX_D),
        ("u_lo", C.c_double * MAX_M), ("u_hi", C.c_double * MAX_M),
        ("dt", C.c_double), ("s_min", C.c_int), ("s_max", C.c_int),
        ("n_boxes", C.c_int), ("boxes", C.POINTER(C.c_double)),
        ("n_spheres", C.c_int), ("spheres", C.POINTER(C.c_double)),
        ("x_goal", C.c_double * MAX_D), ("goal_r", C.c_double),
        ("cost", C.c_int), ("heuristic", C.c_int), ("h_speed", C.c_double),
        ("nn_w", C.c_double * MAX_D), ("model", C.c_double * 8),
        ("K", C.c_int), ("k", C.c_int),
    ]


class Tree(C.Structure):
    _fields_ = [
        ("cap", C.c_int64), ("count", C.c_int64), ("iteration", C.c_uint32),
        ("states", C.POINTER(C.c_double)), ("controls", C.POINTER(C.c_double)),
        ("parents", C.POINTER(C.c_int32)), ("costs", C.POINTER(C.c_double)),
        ("steps", C.POINTER(C.c_int32)),
    ]


class NNResult(C.Structure):
    _fields_ = [("idx", C.c_int64), ("d1", C.c_double), ("d2", C.c_double), ("fragile_elig", C.c_int)]


class Rollout(C.Structure):
    _fields_ = [
        ("x_end", C.c_double * MAX_D), ("cost_end", C.c_double), ("f_end", C.c_double),
        ("collided", C.c_int), ("first_invalid", C.c_int), ("face_margin", C.c_double),
        ("in_goal", C.c_int), ("goal_margin", C.c_double),
    ]


_PD = C.POINTER(C.c_double)
_PI32 = C.POINTER(C.c_int32)
_PI64 = C.POINTER(C.c_int64)


class ExpandOut(C.Structure):
    _fields_ = [
        ("samples", _PD), ("near", _PI64), ("nn_d1", _PD), ("nn_d2", _PD), ("nn_fragile", _PI32),
        ("u", _PD), ("S", _PI32), ("outcome", _PI32), ("x_end", _PD),
        ("cost_end", _PD), ("f_end", _PD), ("face_margin", _PD), ("goal_margin", _PD),
        ("in_goal", _PI32), ("node", _PI64),
        ("n_start", C.c_int64), ("n_appended", C.c_int64), ("n_pruned", C.c_int64),
        ("n_collided", C.c_int64), ("n_no_parent", C.c_int64), ("n_dropped", C.c_int64),
        ("goal_found", C.c_int), ("goal_idx", C.c_int64), ("goal_cost", C.c_double),
        ("iteration", C.c_uint32),
    ]


class PlanOut(C.Structure):
    _fields_ = [
        ("max_iterations", C.c_int64), ("stop_at_first", C.c_int),
        ("iterations", C.c_int64), ("n_solutions", C.c_int), ("n_restarts", C.c_int),
        ("best_cost", C.c_double), ("best_path_len", C.c_int64), ("best_path", _PI64),
        ("path_cap", C.c_int64), ("best_states", _PD), ("best_controls", _PD), ("best_steps", _PI32),
        ("hist_cost", _PD), ("hist_iter", _PI64), ("hist_cap", C.c_int64),
        ("status", C.c_int), ("fragile_iteration", C.c_int64),
    ]


class TrajParams(C.Structure):
    _fields_ = [("w_dur", C.c_double), ("w_u", C.c_double), ("w_obs", C.c_double), ("beta", C.c_double),
                ("margin", C.c_double), ("w_goal", C.c_double), ("w_len", C.c_double), ("len_eps", C.c_double)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        L.ora_philox4x32_10.argtypes = [C.POINTER(C.c_uint32)] * 3
        L.ora_u01.argtypes = [C.c_uint32]
        L.ora_u01.restype = C.c_double
        L.ora_sample_state.argtypes = [C.POINTER(Problem), C.c_uint64, C.c_uint32, C.c_uint32, _PD]
        L.ora_sample_control.argtypes = [C.POINTER(Problem), C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32,
                                         _PD, C.POINTER(C.c_int)]
        L.ora_dynamics.argtypes = [C.POINTER(Problem), _PD, _PD, _PD]
        L.ora_rk4_step.argtypes = [C.POINTER(Problem), _PD, _PD, C.c_double, _PD]
        L.ora_state_valid.argtypes = [C.POINTER(Problem), _PD]
        L.ora_face_margin.argtypes = [C.POINTER(Problem), _PD]
        L.ora_face_margin.restype = C.c_double
        L.ora_heuristic.argtypes = [C.POINTER(Problem), _PD]
        L.ora_heuristic.restype = C.c_double
        L.ora_fcosts.argtypes = [C.POINTER(Problem), C.POINTER(Tree), C.c_int64, _PD]
        L.ora_nearest.argtypes = [C.POINTER(Problem), C.POINTER(Tree), C.c_int64, _PD, _PD, C.c_double,
                                  C.c_double, C.POINTER(NNResult)]
        L.ora_propagate.argtypes = [C.POINTER(Problem), _PD, C.c_double, _PD, C.c_int, C.c_double,
                                    C.POINTER(Rollout)]
        L.ora_tree_reset.argtypes = [C.POINTER(Problem), C.POINTER(Tree), _PD]
        L.ora_expand.argtypes = [C.POINTER(Problem), C.POINTER(Tree), C.c_double, C.c_uint64,
                                 C.POINTER(ExpandOut)]
        L.ora_extract_path.argtypes = [C.POINTER(Tree), C.c_int64, _PI64, C.c_int64]
        L.ora_extract_path.restype = C.c_int64
        L.ora_plan.argtypes = [C.POINTER(Problem), C.POINTER(Tree), _PD, C.c_uint64, C.POINTER(PlanOut)]
        L.ora_traj_cost.argtypes = [C.POINTER(Problem), _PD, _PD, C.c_int, C.POINTER(TrajParams), _PD]
        L.ora_traj_cost.restype = C.c_double
        L.ora_traj_grad.argtypes = [C.POINTER(Problem), _PD, _PD, C.c_int, C.POINTER(TrajParams), _PD, _PD]
        L.ora_traj_grad.restype = C.c_double
        L.ora_dynamics_vjp.argtypes = [C.POINTER(Problem), _PD, _PD, _PD, _PD, _PD]
        L.ora_recheck_edge_dense.argtypes = [C.POINTER(Problem), _PD, _PD, C.c_int, C.c_int]
        L.ora_di_edge_hits_exact.argtypes = [C.POINTER(Problem), _PD, _PD, C.c_int]
        _lib = L
    return _lib


def _pd(a):
    return a.ctypes.data_as(_PD)


def _f64(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a if n is None else a.reshape(n)


class OracleProblem:
    """Owns the ctypes problem struct and the obstacle buffers it points to."""

    def __init__(self, spec):
        s = spec
        P = Problem()
        P.dyn, P.d, P.m, P.pdim = s["dyn"], s["d"], s["m"], s["pdim"]
        for a in range(s["d"]):
            P.x_lo[a], P.x_hi[a] = float(s["x_lo"][a]), float(s["x_hi"][a])
            P.nn_w[a] = float(s["nn_w"][a]) if s.get("nn_w") is not None else 1.0
        for a in range(s["m"]):
            P.u_lo[a], P.u_hi[a] = float(s["u_lo"][a]), float(s["u_hi"][a])
        P.dt = float(s["dt"])
        P.s_min, P.s_max = int(s["s_min"]), int(s["s_max"])
        self._boxes = _f64(s["boxes"]).reshape(-1)
        self._spheres = _f64(s["spheres"]).reshape(-1)
        P.n_boxes = int(np.asarray(s["boxes"]).shape[0])
        P.n_spheres = int(np.asarray(s["spheres"]).shape[0])
        P.boxes = _pd(self._boxes)
        P.spheres = _pd(self._spheres)
        goal = s.get("x_goal")
        if goal is not None:
            for a in range(s["d"]):
                P.x_goal[a] = float(goal[a])
        P.goal_r = float(s["goal_r"])
        P.cost = int(s.get("cost", COST_PATH_LENGTH))
        P.heuristic = int(s.get("heuristic", H_POSITION))
        P.h_speed = float(s.get("h_speed", 0.0))
        model = s.get("model", [0.0] * 5)
        for a in range(len(model)):
            P.model[a] = float(model[a])
        P.K, P.k = int(s["K"]), int(s["k"])
        self.P = P
        self.spec = s

    def set_goal(self, x_goal):
        for a in range(self.P.d):
            self.P.x_goal[a] = float(x_goal[a])

    @property
    def ref(self):
        return C.byref(self.P)


class OracleTree:
    """Node-major FP64 tree buffers plus the ctypes view of them."""

    def __init__(self, d, m, cap):
        self.d, self.m, self.cap = d, m, int(cap)
        self.states = np.zeros((self.cap, d))
        self.controls = np.zeros((self.cap, m))
        self.parents = np.full(self.cap, -1, dtype=np.int32)
        self.costs = np.zeros(self.cap)
        self.steps = np.zeros(self.cap, dtype=np.int32)
        T = Tree()
        T.cap, T.count, T.iteration = self.cap, 0, 0
        T.states, T.controls, T.costs = _pd(self.states), _pd(self.controls), _pd(self.costs)
        T.parents = self.parents.ctypes.data_as(_PI32)
        T.steps = self.steps.ctypes.data_as(_PI32)
        self.T = T

    @classmethod
    def from_arrays(cls, d, m, cap, states, controls, parents, costs, steps, iteration=0):
        t = cls(d, m, cap)
        n = len(costs)
        t.states[:n] = np.asarray(states, dtype=np.float64).reshape(n, d)
        t.controls[:n] = np.asarray(controls, dtype=np.float64).reshape(n, m)
        t.parents[:n] = parents
        t.costs[:n] = costs
        t.steps[:n] = steps
        t.T.count = n
        t.T.iteration = iteration
        return t

    @property
    def count(self):
        return int(self.T.count)

    @property
    def iteration(self):
        return int(self.T.iteration)

    @property
    def ref(self):
        return C.byref(self.T)

    def arrays(self):
        n = self.count
        return dict(states=self.states[:n].copy(), controls=self.controls[:n].copy(),
                    parents=self.parents[:n].copy(), costs=self.costs[:n].copy(),
                    steps=self.steps[:n].copy(), iteration=self.iteration, count=n)


def philox4x32_10(ctr, key):
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().ora_philox4x32_10(c, k, o)
    return [int(v) for v in o]


def u01(w):
    return lib().ora_u01(int(w) & 0xFFFFFFFF)


def sample_state(prob, seed, it, i):
    x = np.zeros(prob.P.d)
    lib().ora_sample_state(prob.ref, seed, it, i, _pd(x))
    return x


def sample_control(prob, seed, it, i, j):
    u = np.zeros(prob.P.m)
    S = C.c_int()
    lib().ora_sample_control(prob.ref, seed, it, i, j, _pd(u), C.byref(S))
    return u, S.value


def dynamics(prob, x, u):
    x, u = _f64(x), _f64(u)
    out = np.zeros(prob.P.d)
    lib().ora_dynamics(prob.ref, _pd(x), _pd(u), _pd(out))
    return out


def rk4_step(prob, x, u, h):
    x, u = _f64(x), _f64(u)
    out = np.zeros(prob.P.d)
    lib().ora_rk4_step(prob.ref, _pd(x), _pd(u), float(h), _pd(out))
    return out


def state_valid(prob, x):
    x = _f64(x)
    return bool(lib().ora_state_valid(prob.ref, _pd(x)))


def face_margin(prob, x):
    x = _f64(x)
    return lib().ora_face_margin(prob.ref, _pd(x))


def heuristic(prob, x):
    x = _f64(x)
    return lib().ora_heuristic(prob.ref, _pd(x))


def fcosts(prob, tree, n=None):
    n = tree.count if n is None else n
    f = np.zeros(n)
    lib().ora_fcosts(prob.ref, tree.ref, n, _pd(f))
    return f


def nearest(prob, tree, q, bound, f=None, n=None):
    n = tree.count if n is None else n
    f = fcosts(prob, tree, n) if f is None else _f64(f)
    q = _f64(q)
    r = NNResult()
    tol = 1e-5 * max(1.0, abs(bound)) if np.isfinite(bound) else np.inf
    lib().ora_nearest(prob.ref, tree.ref, n, _pd(f), _pd(q), float(bound), float(tol), C.byref(r))
    return dict(idx=r.idx, d1=r.d1, d2=r.d2, fragile=bool(r.fragile_elig))


def propagate(prob, x0, g0, u, S, bound=np.inf):
    x0, u = _f64(x0), _f64(u)
    r = Rollout()
    lib().ora_propagate(prob.ref, _pd(x0), float(g0), _pd(u), int(S), float(bound), C.byref(r))
    return dict(x_end=np.array(r.x_end[: prob.P.d]), cost_end=r.cost_end, f_end=r.f_end,
                collided=bool(r.collided), first_invalid=r.first_invalid, face_margin=r.face_margin,
                in_goal=bool(r.in_goal), goal_margin=r.goal_margin)


def tree_reset(prob, tree, x_init):
    x = _f64(x_init)
    return lib().ora_tree_reset(prob.ref, tree.ref, _pd(x))


def expand(prob, tree, bound, seed):
    """One expansion iteration; returns the status and every per-query / per-rollout record."""
    P = prob.P
    K, k, d, m = P.K, P.k, P.d, P.m
    R = K * k
    o = ExpandOut()
    bufs = dict(
        samples=np.zeros((K, d)), near=np.zeros(K, np.int64), nn_d1=np.zeros(K), nn_d2=np.zeros(K),
        nn_fragile=np.zeros(K, np.int32), u=np.zeros((R, m)), S=np.zeros(R, np.int32),
        outcome=np.zeros(R, np.int32), x_end=np.zeros((R, d)), cost_end=np.zeros(R), f_end=np.zeros(R),
        face_margin=np.zeros(R), goal_margin=np.zeros(R), in_goal=np.zeros(R, np.int32),
        node=np.zeros(R, np.int64),
    )
    for name, arr in bufs.items():
        ptype = dict(o.__class__._fields_)[name]
        setattr(o, name, arr.ctypes.data_as(ptype))
    st = lib().ora_expand(prob.ref, tree.ref, float(bound), int(seed), C.byref(o))
    res = dict(bufs)
    for name in ("n_start", "n_appended", "n_pruned", "n_collided", "n_no_parent", "n_dropped",
                 "goal_found", "goal_idx", "goal_cost", "iteration"):
        res[name] = getattr(o, name)
    res["status"] = st
    res["bound"] = bound
    return res


def extract_path(tree, node):
    out = np.zeros(tree.count + 1, dtype=np.int64)
    n = lib().ora_extract_path(tree.ref, int(node), out.ctypes.data_as(_PI64), len(out))
    return out[:n] if n >= 0 else None


def plan(prob, tree, x_init, seed, max_iterations, stop_at_first=False, path_cap=65536, hist_cap=4096):
    P = prob.P
    o = PlanOut()
    o.max_iterations = int(max_iterations)
    o.stop_at_first = int(bool(stop_at_first))
    path = np.zeros(path_cap, np.int64)
    states = np.zeros((path_cap, P.d))
    controls = np.zeros((path_cap, P.m))
    steps = np.zeros(path_cap, np.int32)
    hc = np.zeros(hist_cap)
    hi = np.zeros(hist_cap, np.int64)
    o.best_path, o.path_cap = path.ctypes.data_as(_PI64), path_cap
    o.best_states, o.best_controls = _pd(states), _pd(controls)
    o.best_steps = steps.ctypes.data_as(_PI32)
    o.hist_cost, o.hist_iter, o.hist_cap = _pd(hc), hi.ctypes.data_as(_PI64), hist_cap
    x = _f64(x_init)
    st = lib().ora_plan(prob.ref, tree.ref, _pd(x), int(seed), C.byref(o))
    L = max(int(o.best_path_len), 0)
    ns = int(o.n_solutions)
    return dict(status=st, iterations=int(o.iterations), n_solutions=ns, n_restarts=int(o.n_restarts),
                best_cost=o.best_cost, path=path[:L].copy(), path_states=states[:L].copy(),
                path_controls=controls[:L].copy(), path_steps=steps[:L].copy(),
                hist_cost=hc[: min(ns, hist_cap)].copy(), hist_iter=hi[: min(ns, hist_cap)].copy(),
                fragile_iteration=int(o.fragile_iteration))


def recheck_edge_dense(prob, x0, u, S, sub=16):
    x0, u = _f64(x0), _f64(u)
    return bool(lib().ora_recheck_edge_dense(prob.ref, _pd(x0), _pd(u), int(S), int(sub)))


def di_edge_hits_exact(prob, x0, u, S):
    x0, u = _f64(x0), _f64(u)
    return bool(lib().ora_di_edge_hits_exact(prob.ref, _pd(x0), _pd(u), int(S)))


TRAJ_DEFAULTS = dict(w_dur=1.0, w_u=0.1, w_obs=1.0, beta=50.0, margin=0.0, w_goal=1.0, w_len=0.0, len_eps=1e-3)


def traj_params(**kw):
    w = dict(TRAJ_DEFAULTS)
    w.update(kw)
    return TrajParams(**w)


def dynamics_vjp(prob, x, u, a):
    x, u, a = _f64(x), _f64(u), _f64(a)
    gx, gu = np.zeros(prob.P.d), np.zeros(prob.P.m)
    lib().ora_dynamics_vjp(prob.ref, _pd(x), _pd(u), _pd(a), _pd(gx), _pd(gu))
    return gx, gu


def traj_cost(prob, x0, U, w=None):
    x0, U = _f64(x0), _f64(U)
    w = traj_params() if w is None else w
    xf = np.zeros(prob.P.d)
    J = lib().ora_traj_cost(prob.ref, _pd(x0), _pd(U), U.shape[0], C.byref(w), _pd(xf))
    return J, xf


def traj_grad(prob, x0, U, w=None):
    x0, U = _f64(x0), _f64(U)
    w = traj_params() if w is None else w
    dU, dx0 = np.zeros_like(U), np.zeros(prob.P.d)
    J = lib().ora_traj_grad(prob.ref, _pd(x0), _pd(U), U.shape[0], C.byref(w), _pd(dU), _pd(dx0))
    return J, dU, dx0
