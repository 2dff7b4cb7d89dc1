"""Gradient refinement of AO-x solutions through the adjoint RK4 kernels.

``TrajCost`` is a torch.autograd.Function over libpakr.so's pakr_traj_cost /
pakr_traj_grad: its forward returns the smooth trajectory cost of each
control sequence, its backward the gradient with respect to the controls and
the start states (hand-written discrete adjoint of RK4, checkpoints every 16
steps).  ``refine_path`` lowers the cost of a path found by pakr_plan by
projected gradient steps on its per-edge controls and keeps the result only if
the planner's own rules (pakr_traj_check) accept it.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import pakr

DEFAULT_WEIGHTS = dict(w_duration=1.0, w_control=0.1, w_obstacle=1.0, beta=50.0, margin=0.0, w_goal=1.0,
                       w_length=0.0, length_eps=1e-3)


def _params(weights):
    w = dict(DEFAULT_WEIGHTS)
    w.update(weights or {})
    return pakr.TrajParams(**w)


def _goal(x_goal):
    g = np.ascontiguousarray(np.asarray(x_goal, dtype=np.float32).reshape(-1))
    return g, g.ctypes.data_as(C.POINTER(C.c_float))


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


class TrajCost(torch.autograd.Function):
    """J = TrajCost.apply(controls [T,N,m], x0 [T,d], planner, x_goal, weights) -> [T]."""

    @staticmethod
    def forward(ctx, controls, x0, planner, x_goal, weights):
        controls = controls.contiguous().float()
        x0 = x0.contiguous().float()
        T, N = controls.shape[0], controls.shape[1]
        cost = torch.empty(T, dtype=torch.float32, device=controls.device)
        g, gp = _goal(x_goal)
        prm = _params(weights)
        pakr._check(pakr.lib().pakr_traj_cost(planner.h, _ptr(x0), _ptr(controls), T, N, gp, C.byref(prm),
                                              _ptr(cost), None), "pakr_traj_cost")
        ctx.save_for_backward(controls, x0)
        ctx.planner, ctx.x_goal, ctx.weights = planner, g, weights
        return cost

    @staticmethod
    def backward(ctx, grad_cost):
        controls, x0 = ctx.saved_tensors
        T, N = controls.shape[0], controls.shape[1]
        planner = ctx.planner
        grad_cost = grad_cost.contiguous().float()
        dU = torch.empty_like(controls)
        dx0 = torch.empty_like(x0)
        nck = pakr.lib().pakr_traj_checkpoint_floats(planner.h, T, N)
        ckpt = torch.empty(max(int(nck), 1), dtype=torch.float32, device=controls.device)
        prm = _params(ctx.weights)
        gp = ctx.x_goal.ctypes.data_as(C.POINTER(C.c_float))
        pakr._check(pakr.lib().pakr_traj_grad(planner.h, _ptr(x0), _ptr(controls), T, N, gp, C.byref(prm),
                                              _ptr(grad_cost), _ptr(dU), _ptr(dx0), _ptr(ckpt)), "pakr_traj_grad")
        return dU, dx0, None, None, None


def traj_cost(planner, controls, x0, x_goal, **weights):
    return TrajCost.apply(controls, x0, planner, x_goal, weights)


def traj_check(planner, controls, x0, x_goal):
    """(valid, in_goal, path_length, x_final) under the planner's per-substep rules."""
    controls = controls.contiguous().float()
    x0 = x0.contiguous().float()
    T, N = controls.shape[0], controls.shape[1]
    dev = controls.device
    valid = torch.empty(T, dtype=torch.int32, device=dev)
    in_goal = torch.empty(T, dtype=torch.int32, device=dev)
    length = torch.empty(T, dtype=torch.float32, device=dev)
    xf = torch.empty_like(x0)
    g, gp = _goal(x_goal)
    pakr._check(pakr.lib().pakr_traj_check(planner.h, _ptr(x0), _ptr(controls), T, N, gp, _ptr(valid),
                                           _ptr(in_goal), _ptr(length), _ptr(xf)), "pakr_traj_check")
    return valid, in_goal, length, xf


def expand_controls(edge_controls, steps):
    """Per-step controls of a path: edge e's control repeated steps[e] times."""
    reps = torch.as_tensor(np.asarray(steps), dtype=torch.long, device=edge_controls.device)
    return torch.repeat_interleave(edge_controls, reps, dim=0)


def refine_path(planner, spec, path, x_goal, iters=40, lr=0.05, weights=None):
    """Projected gradient descent on a path's per-edge controls.

    Minimises the smooth cost (path length, obstacle penalty, goal error,
    control effort) with the step counts fixed; after every step the controls
    are clamped to the control box.  Returns (controls, length) of the best
    iterate the planner's rules accept (valid at every substep, ending in the
    goal ball), or None if no iterate improves on the input path's length."""
    dev = torch.device(f"cuda:{planner.device}")
    steps = np.asarray(path["steps"])
    if len(steps) == 0:
        return None
    w = dict(w_length=1.0, w_obstacle=0.05, beta=200.0, margin=0.01, w_goal=50.0, w_control=0.0,
             w_duration=0.0, length_eps=1e-4)
    w.update(weights or {})
    x0 = torch.tensor(np.asarray(path["states"][0], np.float32)[None], device=dev)
    u = torch.tensor(np.asarray(path["controls"], np.float32), device=dev, requires_grad=True)
    lo = torch.tensor(np.asarray(spec["u_lo"], np.float32), device=dev)
    hi = torch.tensor(np.asarray(spec["u_hi"], np.float32), device=dev)
    opt = torch.optim.Adam([u], lr=lr)
    best = None
    base_len = None
    for it in range(iters + 1):
        U = expand_controls(u, steps)[None]
        with torch.no_grad():
            valid, in_goal, length, _ = traj_check(planner, U.detach(), x0, x_goal)
            L = float(length[0])
            if base_len is None:
                base_len = L
            if int(valid[0]) and int(in_goal[0]) and L < (best[1] if best else base_len):
                best = (u.detach().clone(), L)
        if it == iters:
            break
        J = traj_cost(planner, U, x0, x_goal, **w).sum()
        opt.zero_grad()
        J.backward()
        opt.step()
        with torch.no_grad():
            u.copy_(torch.max(torch.min(u, hi), lo))
    return best
