"""Python binding of the C ABI in include/pakr.h (argument marshalling only).

Every step of the planner runs in libpakr.so's CUDA kernels; this module only
converts numpy / torch arguments to the ABI's plain pointers and sizes.  PyTorch
provides the device memory (the planner's workspace is a torch tensor) and the
stream (the current torch stream at creation).  If libpakr.so is missing or
fails to load, every entry point raises -- there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libpakr.so")

# status codes
OK, GOAL_REACHED, TREE_FULL, NO_ELIGIBLE, BUDGET_EXPIRED = 0, 1, 2, 3, 4
ERR_INVALID_ARG, ERR_CUDA, ERR_OOM, ERR_TIMEOUT, ERR_UNIMPLEMENTED, ERR_DEVICE = -1, -2, -3, -4, -5, -6
STATUS_NAMES = {0: "OK", 1: "GOAL_REACHED", 2: "TREE_FULL", 3: "NO_ELIGIBLE", 4: "BUDGET_EXPIRED",
                -1: "ERR_INVALID_ARG", -2: "ERR_CUDA", -3: "ERR_OOM", -4: "ERR_TIMEOUT",
                -5: "ERR_UNIMPLEMENTED", -6: "ERR_DEVICE"}
# dynamics / cost / heuristic / outcome / flags
DI2, DI3, QUAD12, DUBINS3D, UNICYCLE1, UNICYCLE2 = range(6)
COST_PATH_LENGTH, COST_DURATION = 0, 1
H_POSITION, H_FULLSTATE = 0, 1
ROLLOUT_APPENDED, ROLLOUT_PRUNED, ROLLOUT_COLLIDED, ROLLOUT_NO_PARENT, ROLLOUT_DROPPED = range(5)
PLAN_STOP_AT_FIRST = 1

_PF = C.POINTER(C.c_float)
_PI32 = C.POINTER(C.c_int32)
_PI64 = C.POINTER(C.c_int64)
_PD = C.POINTER(C.c_double)


NN_AUTO, NN_FP32, NN_TENSOR = 0, 1, 2  # pakr_nn_mode


class ProblemDesc(C.Structure):
    _fields_ = [
        ("dynamics", C.c_int32),
        ("x_lo", _PF), ("x_hi", _PF), ("u_lo", _PF), ("u_hi", _PF),
        ("dt", C.c_float), ("steps_min", C.c_int32), ("steps_max", C.c_int32),
        ("n_boxes", C.c_int32), ("boxes", _PF),
        ("n_spheres", C.c_int32), ("spheres", _PF),
        ("goal_radius", C.c_float),
        ("cost", C.c_int32), ("heuristic", C.c_int32), ("heuristic_speed", C.c_float),
        ("nn_weights", _PF), ("model_params", _PF),
        ("n_parents", C.c_int32), ("branching", C.c_int32),
        ("tree_cap", C.c_int64), ("device", C.c_int32), ("cuda_stream", C.c_void_p),
        ("workspace", C.c_void_p), ("workspace_bytes", C.c_uint64),
        ("path_cap", C.c_int32), ("history_cap", C.c_int32), ("nn_mode", C.c_int32),
    ]


class ExpandInfo(C.Structure):
    _fields_ = [
        ("n_start", C.c_int64), ("n_appended", C.c_int64), ("n_pruned", C.c_int64),
        ("n_collided", C.c_int64), ("n_no_parent", C.c_int64), ("n_dropped", C.c_int64),
        ("goal_found", C.c_int32), ("reserved", C.c_int32), ("goal_idx", C.c_int64),
        ("goal_cost", C.c_float), ("iteration", C.c_uint32),
    ]


class TreeHost(C.Structure):
    _fields_ = [
        ("capacity", C.c_int64), ("count", C.c_int64), ("iteration", C.c_uint32),
        ("states", _PF), ("controls", _PF), ("parents", _PI32), ("costs", _PF), ("steps", _PI32),
    ]


class Path(C.Structure):
    _fields_ = [
        ("max_edges", C.c_int32), ("states", _PF), ("controls", _PF), ("steps", _PI32),
        ("max_history", C.c_int32), ("history_time_s", _PD), ("history_cost", _PF),
        ("history_iteration", _PI64),
        ("n_edges", C.c_int32), ("cost", C.c_float), ("n_solutions", C.c_int32), ("n_restarts", C.c_int32),
        ("t_first_solution_s", C.c_double), ("t_total_s", C.c_double), ("iterations", C.c_int64),
        ("nodes_first_solution", C.c_int64), ("iterations_first_solution", C.c_int64),
    ]


class TrajParams(C.Structure):
    _fields_ = [(n, C.c_float) for n in ("w_duration", "w_control", "w_obstacle", "beta", "margin", "w_goal",
                                         "w_length", "length_eps")]


class BatchQuery(C.Structure):
    _fields_ = [
        ("x_init", _PF), ("x_goal", _PF), ("n_boxes", C.c_int32), ("boxes", _PF),
        ("n_spheres", C.c_int32), ("spheres", _PF), ("tree_cap", C.c_int64),
    ]


class BatchTuning(C.Structure):
    _fields_ = [("block_threads", C.c_int32), ("nn_chunk", C.c_int32), ("n_tried", C.c_int32),
                ("best_ms", C.c_double)]


class BatchResult(C.Structure):
    _fields_ = [
        ("status", C.c_int32), ("n_solutions", C.c_int32), ("cost", C.c_float), ("n_edges", C.c_int32),
        ("iterations", C.c_int64), ("t_first_solution_s", C.c_double), ("n_restarts", C.c_int32),
        ("reserved", C.c_int32), ("nodes_first_solution", C.c_int64), ("iterations_first_solution", C.c_int64),
    ]


EXPORTED = [
    "pakr_workspace_size", "pakr_create", "pakr_destroy", "pakr_last_error", "pakr_tree_reset",
    "pakr_expand", "pakr_plan", "pakr_plan_bounded", "pakr_plan_offer_bound", "pakr_plan_snapshot", "pakr_tree_export", "pakr_tree_size", "pakr_tree_import", "pakr_tree_truncate", "pakr_debug_last_expand",
    "pakr_set_profiling", "pakr_kernel_times", "pakr_philox4x32_10", "pakr_nearest_static", "pakr_version",
    "pakr_batch_create", "pakr_batch_destroy", "pakr_batch_plan", "pakr_batch_path", "pakr_batch_autotune",
    "pakr_batch_set_tuning", "pakr_traj_cost", "pakr_traj_grad", "pakr_traj_checkpoint_floats", "pakr_traj_check",
    "pakr_traj_refine", "pakr_traj_refine_scratch_floats",
]

_lib = None


def lib_path() -> str:
    return _LIB_PATH


def lib():
    """Load libpakr.so (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(_LIB_PATH):
        raise RuntimeError(f"{_LIB_PATH} is missing: build it first (python -c 'import __graft_entry__ as g; g.build()')")
    L = C.CDLL(_LIB_PATH)
    L.pakr_workspace_size.argtypes = [C.POINTER(ProblemDesc), C.POINTER(C.c_uint64)]
    L.pakr_create.argtypes = [C.POINTER(ProblemDesc), C.POINTER(C.c_void_p)]
    L.pakr_destroy.argtypes = [C.c_void_p]
    L.pakr_destroy.restype = None
    L.pakr_last_error.argtypes = []
    L.pakr_last_error.restype = C.c_char_p
    L.pakr_version.restype = C.c_char_p
    L.pakr_tree_reset.argtypes = [C.c_void_p, _PF, _PF]
    L.pakr_expand.argtypes = [C.c_void_p, C.c_float, C.c_uint64, C.POINTER(ExpandInfo)]
    L.pakr_plan.argtypes = [C.c_void_p, _PF, _PF, C.c_double, C.c_int64, C.c_uint64, C.c_uint32, C.POINTER(Path)]
    L.pakr_plan_bounded.argtypes = [C.c_void_p, _PF, _PF, C.c_double, C.c_int64, C.c_uint64, C.c_uint32, C.c_float,
                                    C.POINTER(Path)]
    L.pakr_plan_offer_bound.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    L.pakr_plan_snapshot.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                                     C.c_void_p]
    L.pakr_tree_export.argtypes = [C.c_void_p, C.POINTER(TreeHost)]
    L.pakr_tree_import.argtypes = [C.c_void_p, C.POINTER(TreeHost), _PF]
    L.pakr_tree_truncate.argtypes = [C.c_void_p, C.c_int64]
    L.pakr_tree_size.argtypes = [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_uint32)]
    L.pakr_debug_last_expand.argtypes = [C.c_void_p, _PF, _PI32, C.POINTER(C.c_int8), C.POINTER(C.c_int8), _PF,
                                         _PI32]
    L.pakr_set_profiling.argtypes = [C.c_void_p, C.c_int32]
    L.pakr_kernel_times.argtypes = [C.c_void_p, _PD, _PI64, C.POINTER(C.c_char_p), C.c_int32]
    L.pakr_philox4x32_10.argtypes = [C.c_void_p, C.POINTER(C.c_uint32), C.POINTER(C.c_uint32),
                                     C.POINTER(C.c_uint32), C.c_int64]
    L.pakr_nearest_static.argtypes = [C.c_void_p, C.c_int64, C.c_int64, C.c_int32, C.c_void_p, C.c_float,
                                      C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]
    L.pakr_batch_create.argtypes = [C.POINTER(ProblemDesc), C.POINTER(BatchQuery), C.c_int32, C.POINTER(C.c_void_p)]
    L.pakr_batch_destroy.argtypes = [C.c_void_p]
    L.pakr_batch_destroy.restype = None
    L.pakr_batch_plan.argtypes = [C.c_void_p, C.c_double, C.c_int64, C.c_uint64, C.c_uint32, C.POINTER(BatchResult)]
    L.pakr_batch_path.argtypes = [C.c_void_p, C.c_int32, _PF, _PF, _PI32, C.c_int32]
    L.pakr_batch_autotune.argtypes = [C.c_void_p, C.c_int64, C.c_uint64, C.POINTER(BatchTuning)]
    L.pakr_batch_set_tuning.argtypes = [C.c_void_p, C.POINTER(BatchTuning)]
    _vp = C.c_void_p
    L.pakr_traj_cost.argtypes = [_vp, _vp, _vp, C.c_int32, C.c_int32, _PF, C.POINTER(TrajParams), _vp, _vp]
    L.pakr_traj_grad.argtypes = [_vp, _vp, _vp, C.c_int32, C.c_int32, _PF, C.POINTER(TrajParams), _vp, _vp, _vp,
                                 _vp]
    L.pakr_traj_checkpoint_floats.argtypes = [_vp, C.c_int32, C.c_int32]
    L.pakr_traj_check.argtypes = [_vp, _vp, _vp, C.c_int32, C.c_int32, _PF, _vp, _vp, _vp, _vp]
    L.pakr_traj_refine.argtypes = [_vp, _vp, _vp, _vp, C.c_int32, C.c_int32, _PF, C.POINTER(TrajParams), C.c_int32,
                                   C.c_int32, C.c_float, C.c_float, _vp, _vp]
    L.pakr_traj_refine_scratch_floats.argtypes = [_vp, C.c_int32, C.c_int32]
    for name in EXPORTED:
        fn = getattr(L, name)
        if name not in ("pakr_destroy", "pakr_batch_destroy", "pakr_last_error", "pakr_version"):
            fn.restype = C.c_int
    L.pakr_traj_checkpoint_floats.restype = C.c_int64
    L.pakr_traj_refine_scratch_floats.restype = C.c_int64
    _lib = L
    return L


class PakrError(RuntimeError):
    def __init__(self, status, where):
        msg = lib().pakr_last_error().decode(errors="replace")
        super().__init__(f"{where}: {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(st, where):
    if st < 0:
        raise PakrError(st, where)
    return st


def _f32(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float32))


def _pf(a):
    return a.ctypes.data_as(_PF)


def problem_desc(spec, arr):
    """A ProblemDesc for a problem dict; arr() turns a host array into a kept-alive pointer."""
    desc = ProblemDesc()
    desc.dynamics = spec["dyn"]
    desc.x_lo, desc.x_hi = arr(spec["x_lo"]), arr(spec["x_hi"])
    desc.u_lo, desc.u_hi = arr(spec["u_lo"]), arr(spec["u_hi"])
    desc.dt = spec["dt"]
    desc.steps_min, desc.steps_max = spec["s_min"], spec["s_max"]
    boxes = np.asarray(spec["boxes"]).reshape(-1)
    spheres = np.asarray(spec["spheres"]).reshape(-1)
    desc.n_boxes = int(np.asarray(spec["boxes"]).shape[0])
    desc.boxes = arr(boxes) if boxes.size else None
    desc.n_spheres = int(np.asarray(spec["spheres"]).shape[0])
    desc.spheres = arr(spheres) if spheres.size else None
    desc.goal_radius = spec["goal_r"]
    desc.cost = spec.get("cost", COST_PATH_LENGTH)
    desc.heuristic = spec.get("heuristic", H_POSITION)
    desc.heuristic_speed = spec.get("h_speed", 0.0)
    desc.nn_weights = arr(spec["nn_w"]) if spec.get("nn_w") is not None else None
    desc.model_params = arr(spec["model"]) if spec["dyn"] == QUAD12 else None
    desc.n_parents, desc.branching = spec["K"], spec["k"]
    desc.tree_cap = spec["cap"]
    desc.nn_mode = int(spec.get("nn_mode", NN_AUTO))
    return desc


class Planner:
    """One planning problem on one GPU (a pakr_planner handle).

    ``spec`` is a problem dict as produced by ``workloads.problem``.  Device
    memory comes from a torch uint8 tensor sized by pakr_workspace_size; work
    is queued on torch's current stream of the device.
    """

    def __init__(self, spec, device=0, stream=None, path_cap=4096, history_cap=1024, torch_workspace=True):
        import torch

        self.spec = spec
        self.d, self.m = spec["d"], spec["m"]
        self.K, self.k = spec["K"], spec["k"]
        self.cap = spec["cap"]
        self.device = device
        self._keep = []
        keep = self._keep

        def arr(v):
            a = _f32(v).reshape(-1)
            keep.append(a)
            return _pf(a)

        desc = problem_desc(spec, arr)
        desc.n_parents, desc.branching = self.K, self.k
        desc.tree_cap = self.cap
        desc.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        desc.cuda_stream = C.c_void_p(stream.cuda_stream)
        desc.path_cap = path_cap
        desc.history_cap = history_cap
        self.path_cap = path_cap
        self.history_cap = history_cap
        self.workspace = None
        if torch_workspace:
            nbytes = C.c_uint64()
            _check(lib().pakr_workspace_size(C.byref(desc), C.byref(nbytes)), "pakr_workspace_size")
            self.workspace = torch.empty(int(nbytes.value), dtype=torch.uint8, device=f"cuda:{device}")
            desc.workspace = C.c_void_p(self.workspace.data_ptr())
            desc.workspace_bytes = int(nbytes.value)
        self.desc = desc
        h = C.c_void_p()
        _check(lib().pakr_create(C.byref(desc), C.byref(h)), "pakr_create")
        self.h = h

    # -- lifecycle -------------------------------------------------------
    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().pakr_destroy(self.h)
            self.h = None
        self.workspace = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- entry points ----------------------------------------------------
    def tree_reset(self, x_init, x_goal):
        xi, xg = _f32(x_init), _f32(x_goal)
        return _check(lib().pakr_tree_reset(self.h, _pf(xi), _pf(xg)), "pakr_tree_reset")

    def expand(self, bound=np.inf, seed=0, info=True):
        if not info:
            return _check(lib().pakr_expand(self.h, float(bound), int(seed), None), "pakr_expand"), None
        inf = ExpandInfo()
        st = _check(lib().pakr_expand(self.h, float(bound), int(seed), C.byref(inf)), "pakr_expand")
        return st, {f: getattr(inf, f) for f, _ in ExpandInfo._fields_ if f != "reserved"}

    def plan(self, x_init, x_goal, budget_s=1.0, max_iterations=0, seed=0, stop_at_first=False, max_edges=None,
             max_history=None, initial_bound=None):
        max_edges = self.path_cap if max_edges is None else max_edges
        max_history = self.history_cap if max_history is None else max_history
        xi, xg = _f32(x_init), _f32(x_goal)
        p = Path()
        states = np.zeros((max_edges + 1, self.d), np.float32)
        controls = np.zeros((max(max_edges, 1), self.m), np.float32)
        steps = np.zeros(max(max_edges, 1), np.int32)
        ht = np.zeros(max(max_history, 1), np.float64)
        hc = np.zeros(max(max_history, 1), np.float32)
        hi = np.zeros(max(max_history, 1), np.int64)
        p.max_edges = max_edges
        p.states, p.controls, p.steps = _pf(states), _pf(controls), steps.ctypes.data_as(_PI32)
        p.max_history = max_history
        p.history_time_s, p.history_cost = ht.ctypes.data_as(_PD), _pf(hc)
        p.history_iteration = hi.ctypes.data_as(_PI64)
        flags = PLAN_STOP_AT_FIRST if stop_at_first else 0
        if initial_bound is None:
            st = _check(lib().pakr_plan(self.h, _pf(xi), _pf(xg), float(budget_s), int(max_iterations), int(seed),
                                        flags, C.byref(p)), "pakr_plan")
        else:
            st = _check(lib().pakr_plan_bounded(self.h, _pf(xi), _pf(xg), float(budget_s), int(max_iterations),
                                                int(seed), flags, float(initial_bound), C.byref(p)),
                        "pakr_plan_bounded")
        ne = p.n_edges
        ns = min(p.n_solutions, max_history)
        return dict(status=st, cost=p.cost, n_edges=ne, n_solutions=p.n_solutions, n_restarts=p.n_restarts,
                    t_first_solution_s=p.t_first_solution_s, t_total_s=p.t_total_s, iterations=p.iterations,
                    nodes_first_solution=p.nodes_first_solution,
                    iterations_first_solution=p.iterations_first_solution,
                    states=states[: ne + 1].copy() if p.n_solutions else states[:0].copy(),
                    controls=controls[:ne].copy(), steps=steps[:ne].copy(),
                    history_time_s=ht[:ns].copy(), history_cost=hc[:ns].copy(), history_iteration=hi[:ns].copy())

    def offer_bound(self, cost, stream):
        """Lower the bound of a plan running on this planner to the cost held by a one-element
        float32 device tensor, enqueued on another torch stream (pakr_plan_offer_bound)."""
        return _check(lib().pakr_plan_offer_bound(self.h, C.c_void_p(cost.data_ptr()),
                                                  C.c_void_p(stream.cuda_stream)), "pakr_plan_offer_bound")

    def plan_snapshot(self, states, controls, steps, info, stream):
        """Copy the best path of a plan running on this planner into device tensors (states
        [(E+1) x d], controls [E x m], steps [E] int32, info [4] int32), enqueued on another
        torch stream (pakr_plan_snapshot)."""
        max_edges = int(steps.numel())
        return _check(lib().pakr_plan_snapshot(self.h, C.c_void_p(states.data_ptr()), C.c_void_p(controls.data_ptr()),
                                               C.c_void_p(steps.data_ptr()), max_edges, C.c_void_p(info.data_ptr()),
                                               C.c_void_p(stream.cuda_stream)), "pakr_plan_snapshot")

    def tree_export(self):
        t = TreeHost()
        t.capacity = 0
        st = lib().pakr_tree_export(self.h, C.byref(t))
        n = int(t.count)
        if st < 0 and n == 0:
            _check(st, "pakr_tree_export")
        states = np.zeros((max(n, 1), self.d), np.float32)
        controls = np.zeros((max(n, 1), self.m), np.float32)
        parents = np.zeros(max(n, 1), np.int32)
        costs = np.zeros(max(n, 1), np.float32)
        steps = np.zeros(max(n, 1), np.int32)
        t.capacity = n
        t.states, t.controls, t.costs = _pf(states), _pf(controls), _pf(costs)
        t.parents, t.steps = parents.ctypes.data_as(_PI32), steps.ctypes.data_as(_PI32)
        _check(lib().pakr_tree_export(self.h, C.byref(t)), "pakr_tree_export")
        n = int(t.count)
        return dict(states=states[:n], controls=controls[:n], parents=parents[:n], costs=costs[:n],
                    steps=steps[:n], count=n, iteration=int(t.iteration))

    def tree_import(self, tree, x_goal):
        n = int(tree["count"])
        states = _f32(tree["states"]).reshape(n, self.d)
        controls = _f32(tree["controls"]).reshape(n, self.m)
        parents = np.ascontiguousarray(np.asarray(tree["parents"], dtype=np.int32))
        costs = _f32(tree["costs"])
        steps = np.ascontiguousarray(np.asarray(tree["steps"], dtype=np.int32))
        t = TreeHost()
        t.capacity, t.count, t.iteration = n, n, int(tree.get("iteration", 0))
        t.states, t.controls, t.costs = _pf(states), _pf(controls), _pf(costs)
        t.parents, t.steps = parents.ctypes.data_as(_PI32), steps.ctypes.data_as(_PI32)
        xg = _f32(x_goal)
        return _check(lib().pakr_tree_import(self.h, C.byref(t), _pf(xg)), "pakr_tree_import")

    def tree_size(self):
        """(node count, expansion counter) of the tree."""
        n, it = C.c_int64(0), C.c_uint32(0)
        _check(lib().pakr_tree_size(self.h, C.byref(n), C.byref(it)), "pakr_tree_size")
        return int(n.value), int(it.value)

    def tree_truncate(self, count):
        return _check(lib().pakr_tree_truncate(self.h, int(count)), "pakr_tree_truncate")

    def debug_last_expand(self):
        K, R = self.K, self.K * self.k
        samples = np.zeros((K, self.d), np.float32)
        near = np.zeros(K, np.int32)
        outcome = np.zeros(R, np.int8)
        goal = np.zeros(R, np.int8)
        controls = np.zeros((R, self.m), np.float32)
        steps = np.zeros(R, np.int32)
        P8 = C.POINTER(C.c_int8)
        _check(lib().pakr_debug_last_expand(self.h, _pf(samples), near.ctypes.data_as(_PI32),
                                            outcome.ctypes.data_as(P8), goal.ctypes.data_as(P8), _pf(controls),
                                            steps.ctypes.data_as(_PI32)), "pakr_debug_last_expand")
        return dict(samples=samples, near=near, outcome=outcome, goal=goal, controls=controls, steps=steps)

    def set_profiling(self, enable):
        return _check(lib().pakr_set_profiling(self.h, int(bool(enable))), "pakr_set_profiling")

    def kernel_times(self):
        ms = (C.c_double * 5)()
        n = (C.c_int64 * 5)()
        names = (C.c_char_p * 5)()
        _check(lib().pakr_kernel_times(self.h, ms, n, names, 5), "pakr_kernel_times")
        return {names[i].decode(): dict(ms=ms[i], launches=int(n[i])) for i in range(5)}

    def philox(self, ctr, key):
        ctr = np.ascontiguousarray(np.asarray(ctr, dtype=np.uint32).reshape(-1, 4))
        k = np.ascontiguousarray(np.asarray(key, dtype=np.uint32).reshape(2))
        out = np.zeros_like(ctr)
        P32 = C.POINTER(C.c_uint32)
        _check(lib().pakr_philox4x32_10(self.h, ctr.ctypes.data_as(P32), k.ctypes.data_as(P32),
                                        out.ctypes.data_as(P32), ctr.shape[0]), "pakr_philox4x32_10")
        return out


class BatchPlanner:
    """Many independent planning queries advanced by one persistent launch
    (pakr_batch_*).  ``base`` is a problem dict (its obstacles and cap are not
    used); each query is a dict with x_init, x_goal, boxes, spheres and cap."""

    def __init__(self, base, queries, device=0, stream=None, path_cap=1024):
        import torch

        self.d, self.m = base["d"], base["m"]
        self.nq = len(queries)
        self._keep = []
        keep = self._keep

        def arr(v):
            a = _f32(v).reshape(-1)
            keep.append(a)
            return _pf(a)

        desc = problem_desc(base, arr)
        desc.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        desc.cuda_stream = C.c_void_p(stream.cuda_stream)
        desc.path_cap = path_cap
        self.path_cap = path_cap
        qs = (BatchQuery * self.nq)()
        for i, q in enumerate(queries):
            qs[i].x_init, qs[i].x_goal = arr(q["x_init"]), arr(q["x_goal"])
            b = np.asarray(q["boxes"])
            sp = np.asarray(q.get("spheres", np.zeros((0, base["pdim"] + 1))))
            qs[i].n_boxes = int(b.shape[0])
            qs[i].boxes = arr(b) if b.size else None
            qs[i].n_spheres = int(sp.shape[0])
            qs[i].spheres = arr(sp) if sp.size else None
            qs[i].tree_cap = int(q["cap"])
        self._qs = qs
        h = C.c_void_p()
        _check(lib().pakr_batch_create(C.byref(desc), qs, self.nq, C.byref(h)), "pakr_batch_create")
        self.h = h

    def close(self):
        if getattr(self, "h", None) is not None and self.h.value:
            lib().pakr_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def plan(self, budget_s=1.0, max_iterations=0, seed=0, stop_at_first=False):
        res = (BatchResult * self.nq)()
        flags = PLAN_STOP_AT_FIRST if stop_at_first else 0
        _check(lib().pakr_batch_plan(self.h, float(budget_s), int(max_iterations), int(seed), flags, res),
               "pakr_batch_plan")
        return [{f: getattr(r, f) for f, _ in BatchResult._fields_ if f != "reserved"} for r in res]

    def path(self, q, max_edges=None):
        max_edges = self.path_cap if max_edges is None else max_edges
        states = np.zeros((max_edges + 1, self.d), np.float32)
        controls = np.zeros((max(max_edges, 1), self.m), np.float32)
        steps = np.zeros(max(max_edges, 1), np.int32)
        _check(lib().pakr_batch_path(self.h, int(q), _pf(states), _pf(controls), steps.ctypes.data_as(_PI32),
                                     max_edges), "pakr_batch_path")
        return states, controls, steps

    def autotune(self, iterations=3, seed=0):
        t = BatchTuning()
        _check(lib().pakr_batch_autotune(self.h, int(iterations), int(seed), C.byref(t)), "pakr_batch_autotune")
        return dict(block_threads=t.block_threads, nn_chunk=t.nn_chunk, n_tried=t.n_tried, best_ms=t.best_ms)

    def set_tuning(self, block_threads, nn_chunk):
        t = BatchTuning(block_threads, nn_chunk, 0, 0.0)
        return _check(lib().pakr_batch_set_tuning(self.h, C.byref(t)), "pakr_batch_set_tuning")
