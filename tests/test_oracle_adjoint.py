"""Pins of the oracle's smooth trajectory cost and reverse-mode gradient (no GPU):
the hand-written VJPs of every model against central differences of the
dynamics, the adjoint gradient against FP64 central finite differences of the
cost, and a closed-form gradient for the double integrator."""
import numpy as np
import pytest

import oracle
from paper_2607_03987_gb300 import workloads as W


def prob_of(spec):
    p = oracle.OracleProblem(spec)
    p.set_goal(spec["x_goal"])
    return p


def model_spec(dyn):
    d, m, pd = W.DIMS[dyn]
    base = W.problem("quad12" if dyn == W.QUAD12 else ("di3" if pd == 3 else "di2"), env_seed=2)
    return W.with_sizes(base, dyn=dyn, d=d, m=m, pdim=pd, x_lo=np.full(d, -50.0), x_hi=np.full(d, 50.0),
                        u_lo=np.full(m, -50.0), u_hi=np.full(m, 50.0), x_goal=np.full(d, 0.5))


@pytest.mark.parametrize("dyn", [W.DI2, W.DI3, W.QUAD12, W.DUBINS3D, W.UNICYCLE1, W.UNICYCLE2])
def test_vjp_matches_central_differences(dyn):
    spec = model_spec(dyn)
    P = prob_of(spec)
    d, m = spec["d"], spec["m"]
    rng = np.random.default_rng(dyn)
    for _ in range(5):
        x = rng.uniform(-0.8, 0.8, d)
        u = rng.uniform(-0.5, 0.5, m)
        a = rng.normal(size=d)
        gx, gu = oracle.dynamics_vjp(P, x, u, a)
        h = 1e-6
        fx = np.zeros(d)
        for i in range(d):
            e = np.zeros(d)
            e[i] = h
            fx[i] = a @ (oracle.dynamics(P, x + e, u) - oracle.dynamics(P, x - e, u)) / (2 * h)
        fu = np.zeros(m)
        for j in range(m):
            e = np.zeros(m)
            e[j] = h
            fu[j] = a @ (oracle.dynamics(P, x, u + e) - oracle.dynamics(P, x, u - e)) / (2 * h)
        assert np.allclose(gx, fx, rtol=1e-6, atol=1e-7), (gx, fx)
        assert np.allclose(gu, fu, rtol=1e-6, atol=1e-7), (gu, fu)


def fd_grad(P, x0, U, w, h=1e-6):
    g = np.zeros_like(U)
    for idx in np.ndindex(U.shape):
        Up, Um = U.copy(), U.copy()
        Up[idx] += h
        Um[idx] -= h
        g[idx] = (oracle.traj_cost(P, x0, Up, w)[0] - oracle.traj_cost(P, x0, Um, w)[0]) / (2 * h)
    return g


def grazing_start(spec):
    # a start near the first box so the softplus penalty is active along the path
    b = spec["boxes"][0]
    pd = spec["pdim"]
    x0 = np.zeros(spec["d"])
    x0[:pd] = (b[:pd] + b[pd:]) / 2 + 0.3 * (b[pd:] - b[:pd]) / 2  # off the centre lines, where the box SDF has kinks
    x0[0] = b[0] - 0.03
    return x0


@pytest.mark.parametrize("name,dyn,N", [("di3", W.DI3, 30), ("quad12", W.QUAD12, 30), ("di2", W.UNICYCLE2, 25)])
def test_adjoint_gradient_matches_finite_differences(name, dyn, N):
    spec = model_spec(dyn)
    P = prob_of(spec)
    rng = np.random.default_rng(4)
    x0 = grazing_start(spec)
    if dyn == W.QUAD12:
        U = np.column_stack([9.81 + rng.normal(0, 0.5, N), rng.uniform(-0.003, 0.003, (N, 3))])
        x0[6] = 0.5  # moving towards the box
    else:
        U = rng.uniform(-0.5, 0.5, (N, spec["m"]))
        if dyn == W.DI3:
            x0[3] = 0.6
    w = oracle.traj_params(w_len=0.7, len_eps=1e-2)
    J, dU, dx0 = oracle.traj_grad(P, x0, U, w)
    J2, _ = oracle.traj_cost(P, x0, U, w)
    assert J == J2
    g = fd_grad(P, x0, U, w)
    scale = np.max(np.abs(g))
    assert scale > 0
    assert np.max(np.abs(dU - g)) <= 1e-6 * max(1.0, scale), np.max(np.abs(dU - g))
    # gradient in the start state
    h = 1e-6
    for i in range(spec["d"]):
        e = np.zeros(spec["d"])
        e[i] = h
        fd = (oracle.traj_cost(P, x0 + e, U, w)[0] - oracle.traj_cost(P, x0 - e, U, w)[0]) / (2 * h)
        assert abs(dx0[i] - fd) <= 1e-6 * max(1.0, abs(fd))


def test_double_integrator_gradient_closed_form():
    # no obstacles, no length term: J = w_u sum |u|^2 h + w_goal |p_N - g|^2 + w_dur N h, and
    # p_N = p0 + v0 N h + sum_n u_n h^2 (N - n - 1/2) exactly (RK4 is exact on the double integrator)
    spec = W.with_sizes(W.problem("di3", env_seed=0), boxes=np.zeros((0, 6)))
    P = prob_of(spec)
    rng = np.random.default_rng(7)
    N, h = 20, spec["dt"]
    x0 = np.concatenate([rng.uniform(0.2, 0.8, 3), rng.uniform(-0.3, 0.3, 3)])
    U = rng.uniform(-1, 1, (N, 3))
    w = oracle.traj_params(w_obs=0.0, w_len=0.0, w_u=0.1, w_goal=2.0)
    J, dU, dx0 = oracle.traj_grad(P, x0, U, w)
    coef = h * h * (N - np.arange(N) - 0.5)
    pN = x0[:3] + x0[3:] * N * h + (coef[:, None] * U).sum(0)
    g = spec["x_goal"][:3]
    J_cf = 1.0 * N * h + 0.1 * np.sum(U ** 2) * h + 2.0 * np.sum((pN - g) ** 2)
    dU_cf = 2 * 0.1 * h * U + 2 * 2.0 * (pN - g)[None, :] * coef[:, None]
    assert abs(J - J_cf) < 1e-12
    assert np.allclose(dU, dU_cf, atol=1e-12)
    assert np.allclose(dx0[:3], 4.0 * (pN - g), atol=1e-12)
    assert np.allclose(dx0[3:], 4.0 * (pN - g) * N * h, atol=1e-12)
