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
import time

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
    steps = np.asarray(steps)
    reps = torch.as_tensor(steps, dtype=torch.long, device=edge_controls.device)
    return torch.repeat_interleave(edge_controls, reps, dim=0, output_size=int(steps.sum()))


REFINE_WEIGHTS = dict(w_length=1.0, w_obstacle=0.05, beta=200.0, margin=0.01, w_goal=2.0, w_control=0.0,
                      w_duration=0.0, length_eps=1e-4)


def refine_path(planner, spec, path, x_goal, iters=15, candidates=16, step=0.5, weights=None, goal_margin=1e-3,
                fused=True):
    """Shorten a path found by pakr_plan with its step counts fixed.

    Each iteration takes the gradient of the smooth cost (path length, a
    short-range obstacle penalty, goal error) with respect to the per-edge
    controls, tries `candidates` step sizes step * 2^-i along the normalised
    descent direction at once (clamped to the control box) and keeps the
    shortest candidate that the planner's rules accept (valid after every
    substep, ending in the goal ball, here by a relative margin of goal_margin
    inside it, so that a replay in another precision stays in: 1e-3 of the radius
    covers the FP32 integration drift of a few hundred RK4 steps) if it is shorter
    than the current path.  fused: the whole loop is one pakr_traj_refine launch
    on the planner's stream; otherwise each iteration runs through TrajCost's
    autograd backward and pakr_traj_check (the same rules; the per-edge gradient
    summed in another order).  The host reads the result once.  Returns
    (controls, length), or None if no candidate improved the path."""
    dev = torch.device(f"cuda:{planner.device}")
    steps = np.asarray(path["steps"], dtype=np.int32)
    if len(steps) == 0:
        return None
    w = dict(REFINE_WEIGHTS)
    w.update(weights or {})
    x0v = path["x0"] if "x0" in path else path["states"][0]
    with torch.cuda.stream(planner.stream):
        x0 = torch.tensor(np.asarray(x0v, np.float32)[None], device=dev)
        u = torch.tensor(np.ascontiguousarray(np.asarray(path["controls"], np.float32)), device=dev)
        if fused:
            E, N = len(steps), int(steps.sum())
            st = torch.tensor(steps, device=dev)
            nf = int(pakr.lib().pakr_traj_refine_scratch_floats(planner.h, E, N))
            scratch = torch.empty(max(nf, 1), dtype=torch.float32, device=dev)
            out = torch.empty(2, dtype=torch.float32, device=dev)
            g, gp = _goal(x_goal)
            prm = _params(w)
            pakr._check(pakr.lib().pakr_traj_refine(planner.h, _ptr(x0), _ptr(u), _ptr(st), E, N, gp, C.byref(prm),
                                                    iters, candidates, step, goal_margin, _ptr(scratch), _ptr(out)),
                        "pakr_traj_refine")
            start_f, cur_f = (float(v) for v in out.cpu())
        else:
            u, cur_f, start_f = _refine_path_autograd(planner, spec, x0, u, steps, x_goal, iters, candidates, step,
                                                      w, goal_margin)
    if not np.isfinite(cur_f) or cur_f >= start_f:
        return None
    return u, cur_f


def _refine_path_autograd(planner, spec, x0, u, steps, x_goal, iters, candidates, step, w, goal_margin):
    dev = x0.device
    reps = torch.as_tensor(steps, dtype=torch.long, device=dev)
    lo = torch.tensor(np.asarray(spec["u_lo"], np.float32), device=dev)
    hi = torch.tensor(np.asarray(spec["u_hi"], np.float32), device=dev)
    alphas = step * torch.pow(2.0, -torch.arange(candidates, device=dev, dtype=torch.float32))
    xc = x0.expand(candidates, -1).contiguous()
    inf = torch.tensor(float("inf"), device=dev)
    n_steps = int(steps.sum())  # given to repeat_interleave, which would otherwise read it back from the device

    def per_step(uu):
        return torch.repeat_interleave(uu, reps, dim=-2, output_size=n_steps)

    pd = spec["pdim"]
    g_pos = torch.tensor(np.asarray(x_goal, np.float32)[:pd], device=dev)
    r_in = float(spec["goal_r"]) * (1.0 - goal_margin)

    def inside(xf):
        return torch.linalg.norm(xf[..., :pd] - g_pos, dim=-1) <= r_in

    valid, in_goal, length, xf0 = traj_check(planner, per_step(u)[None], x0, x_goal)
    cur = torch.where((valid[0] == 1) & (in_goal[0] == 1) & inside(xf0[0]), length[0], inf)
    start = cur.clone()
    for _ in range(iters):
        uu = u.clone().requires_grad_(True)
        traj_cost(planner, per_step(uu)[None], x0, x_goal, **w).sum().backward()
        g = uu.grad
        d = g / (g.norm() + 1e-12)
        cand = torch.max(torch.min(u[None] - alphas[:, None, None] * d[None], hi), lo)
        v, ig, L, xf = traj_check(planner, per_step(cand), xc, x_goal)
        L = torch.where((v == 1) & (ig == 1) & inside(xf), L, inf)
        i = torch.argmin(L)
        better = L[i] < cur
        u = torch.where(better, cand[i], u)
        cur = torch.where(better, L[i], cur)
    return u, float(cur), float(start)


def refined_aox(planner, spec, budget_s, seed=0, refine_iters=15, rounds=(0.3, 0.6, 0.85)):
    """AO-x with gradient refinement inside one wall-clock budget.  The device-resident AO-x
    loop runs in slices that end at the given fractions of the budget; after each slice that
    produced a new best path, that path is refined with the adjoint kernels (kept only if the
    planner's own rules accept it and it is shorter), and the next slice continues AO-x from
    the best cost so far as its bound (pakr_plan_bounded), so each refinement tightens the
    bound the search prunes with.  A slice that finds nothing keeps the previous best.
    Returns (best cost, [(elapsed s, cost)], total refinement gain, best path) with the best
    path as dict(x0, controls, steps) (None if nothing was found)."""
    import time

    t0 = time.perf_counter()
    history = []
    best, best_cost, gain = None, float("inf"), 0.0
    fresh = False
    fracs = tuple(rounds) + (1.0,)
    for i, frac in enumerate(fracs):
        left = frac * budget_s - (time.perf_counter() - t0)
        if left <= 0:
            continue
        r = planner.plan(spec["x_init"], spec["x_goal"], budget_s=left, seed=seed + i,
                         initial_bound=None if best is None else best_cost)
        if r["n_solutions"] and float(r["cost"]) < best_cost:
            best_cost = float(r["cost"])
            best = dict(x0=r["states"][0].copy(), controls=r["controls"].copy(), steps=r["steps"].copy(),
                        states=r["states"].copy())
            fresh = True
        history.append((time.perf_counter() - t0, best_cost))
        if i < len(fracs) - 1 and fresh:
            out = refine_path(planner, spec, best, spec["x_goal"], iters=refine_iters)
            fresh = False
            if out is not None and out[1] < best_cost:
                gain += best_cost - out[1]
                best_cost = out[1]
                best = dict(x0=best["x0"], controls=out[0].detach().cpu().numpy(), steps=best["steps"])
            history.append((time.perf_counter() - t0, best_cost))
    return best_cost, history, gain, best


def refined_aox_concurrent(planner, ref_planner, spec, budget_s, seed=0, refine_iters=15,
                           rounds=(0.15, 0.35, 0.55, 0.75)):
    """AO-x with gradient refinement running beside it, within one wall-clock budget.

    The device AO-x loop runs in slices ending at the given fractions of the budget (and the
    last at the whole budget), each continued from the best cost so far.  While a slice runs on
    the planner's stream (driven from a host thread; the C call releases the GIL), the best
    path of the slices before is refined on ref_planner's stream (another planner of the same
    problem, with its own non-default stream), and a shorter refined path is offered to the
    running loop as its new bound (pakr_plan_offer_bound), which picks it up at its next
    iteration.  The refinement therefore takes no time from the search.  planner and ref_planner
    must use different non-blocking streams.  Returns (best cost, [(elapsed s, cost)], total
    refinement gain, best path as dict(x0, controls, steps) or None)."""
    import threading
    import time

    dev = torch.device(f"cuda:{planner.device}")
    # device memory for the offered cost is taken, and the fill kernel run once, before any
    # slice runs: an allocation, or a kernel's first launch (its code is loaded lazily), while the
    # AO-x graph runs may wait for the graph.  Call this once untimed to warm up the refinement's
    # own kernels the same way.
    with torch.cuda.stream(ref_planner.stream):
        cost_dev = torch.empty(1, dtype=torch.float32, device=dev)
        cost_dev.fill_(float("inf"))
    ref_planner.stream.synchronize()
    t0 = time.perf_counter()
    history = []
    best, best_cost, gain = None, float("inf"), 0.0
    fresh = False
    fracs = tuple(rounds) + (1.0,)
    for i, frac in enumerate(fracs):
        left = frac * budget_s - (time.perf_counter() - t0)
        if left <= 0:
            continue
        out_slice = []

        def run_slice(left=left, i=i, bound=None if best is None else best_cost):
            out_slice.append(planner.plan(spec["x_init"], spec["x_goal"], budget_s=left, seed=seed + i,
                                          initial_bound=bound))

        th = threading.Thread(target=run_slice)
        th.start()
        if fresh:
            fresh = False
            with torch.cuda.stream(ref_planner.stream):
                ref = refine_path(ref_planner, spec, best, spec["x_goal"], iters=refine_iters)
                if ref is not None and ref[1] < best_cost:
                    gain += best_cost - ref[1]
                    best_cost = ref[1]
                    best = dict(x0=best["x0"], controls=ref[0].detach().cpu().numpy(), steps=best["steps"])
                    cost_dev.fill_(best_cost)
                    planner.offer_bound(cost_dev, ref_planner.stream)
                    ref_planner.stream.synchronize()
            history.append((time.perf_counter() - t0, best_cost))
        th.join()
        r = out_slice[0]
        if r["n_solutions"] and float(r["cost"]) < best_cost:
            best_cost = float(r["cost"])
            best = dict(x0=r["states"][0].copy(), controls=r["controls"].copy(), steps=r["steps"].copy(),
                        states=r["states"].copy())
            fresh = True
        history.append((time.perf_counter() - t0, best_cost))
    return best_cost, history, gain, best


def refined_aox_live(planner, ref_planner, spec, budget_s, seed=0, refine_iters=15, max_edges=1024,
                     poll_s=0.0005, stats=None):
    """One AO-x run with refinement beside it for its whole budget.

    The device AO-x loop runs once, as pakr_plan with this seed would (the same graph, the same
    random numbers), on the planner's stream, driven from a host thread.  Meanwhile this thread
    polls the run's best path (pakr_plan_snapshot, on ref_planner's stream); each new one is
    refined on ref_planner (another planner of the same problem with its own non-default
    stream) if the last refinement's duration still fits in the budget, and a refined path
    shorter than everything so far is offered to the running loop as its bound
    (pakr_plan_offer_bound).  Until the first offer lands the loop does exactly what
    plain AO-x does; after it, it prunes against the tighter bound.  Returns (best cost,
    total refinement gain, best path as dict(x0, controls, steps) or None).  A dict passed as
    `stats` receives the number of refinements run and improving, their durations and the time
    the first path was seen."""
    import threading

    d, m = spec["d"], spec["m"]
    side = ref_planner.stream
    # every buffer, and every kernel this thread launches, exists or has run once before the
    # plan starts: an allocation, or a kernel's first (lazy) load, while the plan runs may wait
    # for it
    with torch.cuda.stream(side):
        dev = torch.device(f"cuda:{planner.device}")
        st = torch.zeros((max_edges + 1, d), dtype=torch.float32, device=dev)
        ct = torch.zeros((max_edges, m), dtype=torch.float32, device=dev)
        sp = torch.zeros(max_edges, dtype=torch.int32, device=dev)
        info = torch.zeros(4, dtype=torch.int32, device=dev)
        cost_dev = torch.full((1,), float("inf"), dtype=torch.float32, device=dev)
        planner.plan_snapshot(st, ct, sp, info, side)
        info.cpu()
    side.synchronize()
    res, err = [], []

    def run_plan():
        try:
            res.append(planner.plan(spec["x_init"], spec["x_goal"], budget_s=budget_s, seed=seed))
        except BaseException as e:  # re-raised on this thread once the plan has ended
            err.append(e)

    th = threading.Thread(target=run_plan)
    t0 = time.perf_counter()
    th.start()
    seen, best_ref, best_path, gain = 0, float("inf"), None, 0.0
    t_refine = 0.0  # duration of the last refinement: one is started only if that much time is left
    while th.is_alive():
        with torch.cuda.stream(side):
            planner.plan_snapshot(st, ct, sp, info, side)
            inf_h = info.cpu().numpy()
        if inf_h[0] == 1 and int(inf_h[2]) > seen and time.perf_counter() - t0 + t_refine < budget_s:
            t_start = time.perf_counter()
            if stats is not None and "first_path_s" not in stats:
                stats["first_path_s"] = t_start - t0
            seen = int(inf_h[2])
            ne = int(inf_h[1])
            c = float(np.array([inf_h[3]], dtype=np.int32).view(np.float32)[0])
            with torch.cuda.stream(side):
                path = dict(x0=st[0].cpu().numpy(), controls=ct[:ne].cpu().numpy(), steps=sp[:ne].cpu().numpy())
                ref = refine_path(ref_planner, spec, path, spec["x_goal"], iters=refine_iters)
                base = min(c, best_ref)
                if stats is not None:
                    stats["refined"] = stats.get("refined", 0) + 1
                if ref is not None and ref[1] < base:
                    if stats is not None:
                        stats["improved"] = stats.get("improved", 0) + 1
                    gain += base - ref[1]
                    best_ref = ref[1]
                    best_path = dict(x0=path["x0"], controls=ref[0].detach().cpu().numpy(), steps=path["steps"])
                    cost_dev.fill_(best_ref)
                    planner.offer_bound(cost_dev, side)
            side.synchronize()
            t_refine = time.perf_counter() - t_start
            if stats is not None:
                stats.setdefault("refine_s", []).append(t_refine)
        else:
            time.sleep(poll_s)
    th.join()
    if err:
        raise err[0]
    r = res[0]
    own = float(r["cost"]) if r["n_solutions"] else float("inf")
    if best_ref < own:
        return best_ref, gain, best_path
    if r["n_solutions"]:
        return own, gain, dict(x0=r["states"][0].copy(), controls=r["controls"].copy(), steps=r["steps"].copy())
    return own, gain, None
