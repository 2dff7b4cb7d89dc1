"""Adjoint RK4 kernels (pakr_traj_*) vs the FP64 oracle, through the C ABI and
the torch.autograd.Function: cost, gradient (relative error <= 1e-4 against
the oracle's reverse mode and against FP64 central finite differences), the
planner-rule check, and path refinement."""
import numpy as np
import pytest

import oracle
from paper_2607_03987_gb300 import pakr
from paper_2607_03987_gb300 import workloads as W

pytestmark = pytest.mark.gpu

WEIGHTS = dict(w_duration=1.0, w_control=0.1, w_obstacle=1.0, beta=50.0, margin=0.0, w_goal=1.0, w_length=0.3,
               length_eps=1e-2)


def oracle_params(w):
    return oracle.traj_params(w_dur=w["w_duration"], w_u=w["w_control"], w_obs=w["w_obstacle"], beta=w["beta"],
                              margin=w["margin"], w_goal=w["w_goal"], w_len=w["w_length"], len_eps=w["length_eps"])


def sequences(spec, T, N, seed):
    rng = np.random.default_rng(seed)
    d, m = spec["d"], spec["m"]
    x0 = np.zeros((T, d))
    x0[:, :3] = rng.uniform(0.2, 0.8, (T, 3))
    if spec["dyn"] == W.QUAD12:
        U = np.concatenate([9.81 + rng.normal(0, 0.5, (T, N, 1)), rng.uniform(-0.002, 0.002, (T, N, 3))], axis=2)
        x0[:, 6:9] = rng.uniform(-0.2, 0.2, (T, 3))
    else:
        U = rng.uniform(-0.5, 0.5, (T, N, m))
        x0[:, 3:6] = rng.uniform(-0.3, 0.3, (T, 3))
    return W.f32(x0), W.f32(U)


@pytest.mark.parametrize("name", ["di3", "quad12"])
def test_cost_and_gradient_match_oracle(cuda_lib, name):
    import torch

    from paper_2607_03987_gb300 import refine

    spec = W.with_sizes(W.problem(name, env_seed=3), K=1, k=1, cap=16)
    planner = pakr.Planner(spec)
    T, N = 48, 200
    x0, U = sequences(spec, T, N, 11)
    Ut = torch.tensor(U, dtype=torch.float32, device="cuda", requires_grad=True)
    xt = torch.tensor(x0, dtype=torch.float32, device="cuda", requires_grad=True)
    J = refine.traj_cost(planner, Ut, xt, spec["x_goal"], **WEIGHTS)
    gJ = torch.linspace(0.5, 1.5, T, device="cuda")
    (J * gJ).sum().backward()
    Jg, dUg, dxg = J.detach().cpu().numpy(), Ut.grad.cpu().numpy(), xt.grad.cpu().numpy()
    prob = oracle.OracleProblem(spec)
    prob.set_goal(spec["x_goal"])
    w = oracle_params(WEIGHTS)
    worst = 0.0
    for t in range(T):
        Jo, dUo, dxo = oracle.traj_grad(prob, x0[t], U[t], w)
        s = float(gJ[t])
        assert abs(Jg[t] - Jo) <= 1e-4 * max(1.0, abs(Jo)), (t, Jg[t], Jo)
        ref = s * dUo
        err = np.abs(dUg[t] - ref).max() / np.abs(ref).max()
        worst = max(worst, err)
        assert err <= 1e-4, (t, err)
        assert np.linalg.norm(dUg[t] - ref) <= 1e-4 * np.linalg.norm(ref)
        assert np.abs(dxg[t] - s * dxo).max() <= 1e-4 * max(1.0, np.abs(s * dxo).max())
    planner.close()


def test_gradient_matches_fp64_finite_differences(cuda_lib):
    import torch

    from paper_2607_03987_gb300 import refine

    spec = W.with_sizes(W.problem("quad12", env_seed=5), K=1, k=1, cap=16)
    planner = pakr.Planner(spec)
    T, N = 4, 120
    x0, U = sequences(spec, T, N, 3)
    Ut = torch.tensor(U, dtype=torch.float32, device="cuda", requires_grad=True)
    xt = torch.tensor(x0, dtype=torch.float32, device="cuda")
    refine.traj_cost(planner, Ut, xt, spec["x_goal"], **WEIGHTS).sum().backward()
    g = Ut.grad.cpu().numpy()
    prob = oracle.OracleProblem(spec)
    prob.set_goal(spec["x_goal"])
    w = oracle_params(WEIGHTS)
    rng = np.random.default_rng(0)
    h = 1e-6
    for t in range(T):
        scale = np.abs(oracle.traj_grad(prob, x0[t], U[t], w)[1]).max()
        for _ in range(12):
            n, j = int(rng.integers(N)), int(rng.integers(spec["m"]))
            Up, Um = U[t].copy(), U[t].copy()
            Up[n, j] += h
            Um[n, j] -= h
            fd = (oracle.traj_cost(prob, x0[t], Up, w)[0] - oracle.traj_cost(prob, x0[t], Um, w)[0]) / (2 * h)
            assert abs(g[t, n, j] - fd) <= 1e-4 * scale, (t, n, j, g[t, n, j], fd)
    planner.close()


def test_traj_check_matches_oracle_rules(cuda_lib):
    import torch

    from paper_2607_03987_gb300 import refine

    spec = W.with_sizes(W.problem("di3", env_seed=6), K=1, k=1, cap=16)
    planner = pakr.Planner(spec)
    T, N = 200, 40
    x0, U = sequences(spec, T, N, 9)
    valid, in_goal, length, xf = refine.traj_check(planner, torch.tensor(U, device="cuda"),
                                                   torch.tensor(x0, device="cuda", dtype=torch.float32),
                                                   spec["x_goal"])
    valid, length = valid.cpu().numpy(), length.cpu().numpy()
    prob = oracle.OracleProblem(spec)
    prob.set_goal(spec["x_goal"])
    n_valid = 0
    for t in range(T):
        x = x0[t].astype(float)
        ok, margin, L = True, np.inf, 0.0
        for n in range(N):
            xn = oracle.rk4_step(prob, x, U[t, n], spec["dt"])
            L += np.linalg.norm(xn[:3] - x[:3])
            x = xn
            margin = min(margin, oracle.face_margin(prob, x))
            ok = ok and oracle.state_valid(prob, x)
        if margin >= 1e-5:
            assert bool(valid[t]) == ok, t
        assert abs(length[t] - L) <= 1e-5 * max(1.0, L)
        n_valid += ok
    assert 0 < n_valid < T
    planner.close()


def di_replay_valid(spec, x0, u, S):
    pd, dt = 3, spec["dt"]
    x = np.asarray(x0, float)
    L = 0.0
    for _ in range(S):
        p = x[:pd] + x[pd:] * dt + 0.5 * u * dt * dt
        v = x[pd:] + u * dt
        L += np.linalg.norm(p - x[:pd])
        x = np.concatenate([p, v])
        if np.any(x < spec["x_lo"] - 1e-6) or np.any(x > spec["x_hi"] + 1e-6):
            return False, x, L
        for b in spec["boxes"]:
            if np.all(p >= b[:3]) and np.all(p <= b[3:]):
                return False, x, L
    return True, x, L


def test_refine_shortens_a_found_path(cuda_lib):
    from paper_2607_03987_gb300 import refine

    spec = W.problem("di3", env_seed=2)
    planner = pakr.Planner(spec)
    res = planner.plan(spec["x_init"], spec["x_goal"], budget_s=5.0, seed=3, stop_at_first=True)
    assert res["n_solutions"] == 1
    out = refine.refine_path(planner, spec, res, spec["x_goal"], iters=20)
    assert out is not None, "no accepted refinement"
    u, L = out
    assert L < res["cost"]
    # independent replay (closed form, numpy): valid at every substep, ends in the goal ball, same length
    x = res["states"][0].astype(float)
    total = 0.0
    for e in range(len(res["steps"])):
        ok, x, Le = di_replay_valid(spec, x, u[e].cpu().numpy().astype(float), int(res["steps"][e]))
        assert ok, e
        total += Le
    assert np.linalg.norm(x[:3] - spec["x_goal"][:3]) <= spec["goal_r"] * (1 + 1e-5)
    assert abs(total - L) <= 1e-4 * L
    planner.close()


def test_fused_refinement_matches_autograd_loop(cuda_lib):
    """pakr_traj_refine (the whole loop in one launch) against the same loop through TrajCost's
    autograd backward and pakr_traj_check: the same rules and step sizes, the per-edge gradient
    summed in another order, so after one iteration both accept a path of the same length (to
    rounding), and after several both are accepted, valid paths."""
    from paper_2607_03987_gb300 import refine

    spec = W.problem("di3", env_seed=2)
    planner = pakr.Planner(spec)
    res = planner.plan(spec["x_init"], spec["x_goal"], budget_s=5.0, seed=3, stop_at_first=True)
    assert res["n_solutions"] == 1
    a = refine.refine_path(planner, spec, res, spec["x_goal"], iters=1, fused=True)
    b = refine.refine_path(planner, spec, res, spec["x_goal"], iters=1, fused=False)
    assert (a is None) == (b is None)
    if a is not None:
        assert abs(a[1] - b[1]) <= 1e-4 * b[1]
    for fused in (True, False):
        out = refine.refine_path(planner, spec, res, spec["x_goal"], iters=10, fused=fused)
        assert out is not None
        u, L = out
        x = res["states"][0].astype(float)
        total = 0.0
        for e in range(len(res["steps"])):
            ok, x, Le = di_replay_valid(spec, x, u[e].cpu().numpy().astype(float), int(res["steps"][e]))
            assert ok, (fused, e)
            total += Le
        assert np.linalg.norm(x[:3] - spec["x_goal"][:3]) <= spec["goal_r"] * (1 + 1e-5)
        assert abs(total - L) <= 1e-4 * L
    planner.close()


def test_fused_refinement_rejects_bad_step_counts(cuda_lib):
    """Step counts that do not sum to n_steps leave the controls untouched and report NaN."""
    import ctypes as C

    import torch

    from paper_2607_03987_gb300 import refine

    spec = W.problem("di3", env_seed=2)
    planner = pakr.Planner(spec)
    dev = torch.device("cuda:0")
    with torch.cuda.stream(planner.stream):
        x0 = torch.tensor(np.asarray(spec["x_init"], np.float32)[None], device=dev)
        u = torch.zeros((3, spec["m"]), dtype=torch.float32, device=dev)
        u0 = u.clone()
        st = torch.tensor([2, 3, 4], dtype=torch.int32, device=dev)
        nf = int(pakr.lib().pakr_traj_refine_scratch_floats(planner.h, 3, 10))
        scratch = torch.empty(nf, dtype=torch.float32, device=dev)
        out = torch.zeros(2, dtype=torch.float32, device=dev)
        g, gp = refine._goal(spec["x_goal"])
        prm = refine._params(refine.REFINE_WEIGHTS)
        rc = pakr.lib().pakr_traj_refine(planner.h, C.c_void_p(x0.data_ptr()), C.c_void_p(u.data_ptr()),
                                         C.c_void_p(st.data_ptr()), 3, 10, gp, C.byref(prm), 3, 16, 0.5, 1e-4,
                                         C.c_void_p(scratch.data_ptr()), C.c_void_p(out.data_ptr()))
        assert rc == 0
        o = out.cpu().numpy()
        assert np.all(np.isnan(o))
        assert torch.equal(u, u0)
        # out-of-range arguments are refused on the host
        rc = pakr.lib().pakr_traj_refine(planner.h, C.c_void_p(x0.data_ptr()), C.c_void_p(u.data_ptr()),
                                         C.c_void_p(st.data_ptr()), 3, 9, gp, C.byref(prm), 3, 33, 0.5, 1e-4,
                                         C.c_void_p(scratch.data_ptr()), C.c_void_p(out.data_ptr()))
        assert rc != 0
    planner.close()
