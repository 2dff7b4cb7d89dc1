"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

The paper's environments (the Kino-PAX Tree / Narrow / House scenes and the
DynoBench problems, Sec. V) are not available; these generators stand in for
them with the shapes, sizes and value ranges of the planning workloads:

* ``di2``    -- planar double integrator, 4D state, 10 random boxes, 64 parents x 4 controls, cap 20k
* ``di3``    -- 3D double integrator (Sec. V-A item 1), 50 random boxes, 1024 parents x 8 controls, cap 2^20
* ``quad12`` -- 12D quadcopter (Sec. V-A item 3), 100-pillar forest, 4096 parents x 16 controls, cap 4M

This module holds no arithmetic of the method: it only draws obstacle sets,
start / goal pairs and pre-filled trees from ``numpy.random.Generator(Philox)``.
Every real number is rounded to float32 so that the FP32 device path and the
FP64 oracle start from identical values.
"""
from __future__ import annotations

import copy

import numpy as np

DI2, DI3, QUAD12, DUBINS3D, UNICYCLE1, UNICYCLE2 = range(6)
COST_PATH_LENGTH, COST_DURATION = 0, 1
H_POSITION, H_FULLSTATE = 0, 1

DIMS = {DI2: (4, 2, 2), DI3: (6, 3, 3), QUAD12: (12, 4, 3), DUBINS3D: (6, 3, 3),
        UNICYCLE1: (3, 2, 2), UNICYCLE2: (5, 2, 2)}


def f32(x):
    """Round to float32 and return float64 carrying exactly that value."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def _boxes(rng, n, pdim, side_lo, side_hi, keep_free, free_r, pillar=False):
    """Axis-aligned boxes with centres uniform in the unit cube and sides
    uniform in [side_lo, side_hi]; boxes touching a keep-free ball are redrawn.
    Pillars span the full height z in [0, 1]."""
    out = []
    while len(out) < n:
        c = rng.uniform(0.0, 1.0, pdim)
        side = rng.uniform(side_lo, side_hi, pdim)
        lo, hi = c - side / 2, c + side / 2
        if pillar:
            lo[2], hi[2] = 0.0, 1.0
        ok = True
        for p in keep_free:
            q = np.clip(p[:pdim], lo, hi)
            if pillar:
                dist = np.linalg.norm((p[:2] - q[:2]))
            else:
                dist = np.linalg.norm(p[:pdim] - q)
            if dist <= free_r:
                ok = False
                break
        if ok:
            out.append(np.concatenate([lo, hi]))
    return f32(np.array(out).reshape(n, 2 * pdim))


def problem(name, env_seed=0, **overrides):
    """The problem description (a plain dict) of a named workload."""
    if name == "di2":
        d, m, pdim = DIMS[DI2]
        start = f32([0.1, 0.1, 0.0, 0.0])
        goal = f32([0.9, 0.9, 0.0, 0.0])
        spec = dict(dyn=DI2, x_lo=[0, 0, -1, -1], x_hi=[1, 1, 1, 1], u_lo=[-1, -1], u_hi=[1, 1],
                    dt=0.05, s_min=1, s_max=10, n_boxes=10, side=(0.05, 0.2), goal_r=0.05,
                    K=64, k=4, cap=20000, start=start, goal=goal, pillar=False, model=[0.0] * 5,
                    h_speed=float(np.sqrt(2.0)))
    elif name == "di3":
        d, m, pdim = DIMS[DI3]
        start = f32([0.1, 0.1, 0.1, 0, 0, 0])
        goal = f32([0.9, 0.9, 0.9, 0, 0, 0])
        spec = dict(dyn=DI3, x_lo=[0, 0, 0, -1, -1, -1], x_hi=[1, 1, 1, 1, 1, 1], u_lo=[-1] * 3,
                    u_hi=[1] * 3, dt=0.05, s_min=1, s_max=20, n_boxes=50, side=(0.05, 0.2), goal_r=0.05,
                    K=1024, k=8, cap=1 << 20, start=start, goal=goal, pillar=False, model=[0.0] * 5,
                    h_speed=float(np.sqrt(3.0)))
    elif name == "quad12":
        d, m, pdim = DIMS[QUAD12]
        start = f32([0.1, 0.1, 0.5] + [0.0] * 9)
        goal = f32([0.9, 0.9, 0.5] + [0.0] * 9)
        pi = float(np.float32(np.pi))
        spec = dict(dyn=QUAD12,
                    x_lo=[0, 0, 0, -1, -1, -pi, -1, -1, -1, -3, -3, -3],
                    x_hi=[1, 1, 1, 1, 1, pi, 1, 1, 1, 3, 3, 3],
                    u_lo=[0, -0.5, -0.5, -0.5], u_hi=[20, 0.5, 0.5, 0.5],
                    dt=0.02, s_min=1, s_max=20, n_boxes=100, side=(0.02, 0.06), goal_r=0.05,
                    K=4096, k=16, cap=4_000_000, start=start, goal=goal, pillar=True,
                    model=[1.0, 0.01, 0.01, 0.02, 9.81], h_speed=float(np.sqrt(3.0)))
    else:
        raise ValueError(f"unknown workload {name!r}")
    spec.update(overrides)
    d, m, pdim = DIMS[spec["dyn"]]
    rng = np.random.Generator(np.random.Philox(int(env_seed)))
    n_boxes = spec.pop("n_boxes")
    side = spec.pop("side")
    pillar = spec.pop("pillar")
    boxes = spec.pop("boxes", None)
    if boxes is None:
        boxes = _boxes(rng, n_boxes, pdim, side[0], side[1], [spec["start"], spec["goal"]],
                       spec["goal_r"] + 0.02, pillar=pillar) if n_boxes > 0 else np.zeros((0, 2 * pdim))
    spheres = spec.pop("spheres", np.zeros((0, pdim + 1)))
    out = dict(
        name=name, dyn=spec["dyn"], d=d, m=m, pdim=pdim,
        x_lo=f32(spec["x_lo"]), x_hi=f32(spec["x_hi"]), u_lo=f32(spec["u_lo"]), u_hi=f32(spec["u_hi"]),
        dt=float(f32(spec["dt"])), s_min=int(spec["s_min"]), s_max=int(spec["s_max"]),
        boxes=f32(boxes).reshape(-1, 2 * pdim), spheres=f32(spheres).reshape(-1, pdim + 1),
        goal_r=float(f32(spec["goal_r"])), cost=int(spec.get("cost", COST_PATH_LENGTH)),
        heuristic=int(spec.get("heuristic", H_POSITION)), h_speed=float(f32(spec["h_speed"])),
        nn_w=None if spec.get("nn_w") is None else f32(spec["nn_w"]),
        model=[float(v) for v in f32(spec["model"])], K=int(spec["K"]), k=int(spec["k"]),
        cap=int(spec["cap"]), x_init=f32(spec["start"]), x_goal=f32(spec["goal"]),
    )
    return out


def with_sizes(spec, **kw):
    """A copy of a problem dict with some fields replaced (K, k, cap, ...)."""
    s = copy.deepcopy(spec)
    s.update(kw)
    return s


def random_spheres(seed, n, pdim, r_lo=0.03, r_hi=0.08):
    rng = np.random.Generator(np.random.Philox(int(seed)))
    c = rng.uniform(0, 1, (n, pdim))
    r = rng.uniform(r_lo, r_hi, (n, 1))
    return f32(np.concatenate([c, r], axis=1))


def prefilled_tree(spec, n, seed, cost_hi=0.0):
    """A synthetic tree of n nodes: states uniform in the state box, controls
    uniform in the control box, each parent a uniformly drawn earlier node,
    costs uniform in [0, cost_hi] (all zero by default), durations uniform."""
    rng = np.random.Generator(np.random.Philox(int(seed)))
    d, m = spec["d"], spec["m"]
    lo, hi = spec["x_lo"], spec["x_hi"]
    states = f32(lo + (hi - lo) * rng.random((n, d)))
    states[0] = spec["x_init"]
    controls = f32(spec["u_lo"] + (spec["u_hi"] - spec["u_lo"]) * rng.random((n, m)))
    controls[0] = 0.0
    parents = np.empty(n, dtype=np.int32)
    parents[0] = -1
    if n > 1:
        parents[1:] = (rng.random(n - 1) * np.arange(1, n)).astype(np.int32)
    costs = f32(rng.random(n) * cost_hi) if cost_hi > 0 else np.zeros(n)
    costs[0] = 0.0
    steps = rng.integers(spec["s_min"], spec["s_max"] + 1, n).astype(np.int32)
    steps[0] = 0
    return dict(states=states, controls=controls, parents=parents, costs=costs, steps=steps, count=n,
                iteration=0)


def batch_queries(n_queries=256, env_seed=0, obs_range=(10, 200), cap_range=(64 * 1024, 1 << 20), min_sep=0.6,
                  sep_range=None):
    """Independent 3D double-integrator queries: per query an obstacle count
    uniform in obs_range, a tree cap uniform in cap_range (a multiple of
    1024), and a random start / goal pair at rest, at least min_sep apart,
    kept free of that query's boxes.  With sep_range = (lo, hi) the goal is
    instead the start moved a distance uniform in [lo, hi] in a uniformly
    random direction (short queries, solved in a few expansions)."""
    rng = np.random.Generator(np.random.Philox(int(env_seed) + 7919))
    base = problem("di3", env_seed=env_seed)
    out = []
    for _ in range(n_queries):
        while True:
            s = rng.uniform(0.08, 0.92, 3)
            if sep_range is None:
                g = rng.uniform(0.08, 0.92, 3)
                if np.linalg.norm(s - g) >= min_sep:
                    break
            else:
                direction = rng.normal(size=3)
                g = s + direction / np.linalg.norm(direction) * rng.uniform(sep_range[0], sep_range[1])
                if np.all((g >= 0.08) & (g <= 0.92)):
                    break
        start = f32(np.concatenate([s, np.zeros(3)]))
        goal = f32(np.concatenate([g, np.zeros(3)]))
        n_obs = int(rng.integers(obs_range[0], obs_range[1] + 1))
        boxes = _boxes(rng, n_obs, 3, 0.05, 0.2, [start, goal], base["goal_r"] + 0.02)
        cap = int(rng.integers(cap_range[0] // 1024, cap_range[1] // 1024 + 1)) * 1024
        out.append(dict(x_init=start, x_goal=goal, boxes=boxes, spheres=np.zeros((0, 4)), cap=cap))
    return base, out
