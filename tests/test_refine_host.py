"""Host logic of refined_aox_live (AO-x with gradient refinement beside it), on CPU.

The planners are fakes: the AO-x run is a host thread that publishes a new best path every few
milliseconds through the snapshot call, and refine_path is replaced by a stand-in that takes a
fixed time and returns a shorter path.  What is checked is the scheduler around them: every
offered bound is a refined cost that beat everything before it, no refinement starts when the
last one's duration no longer fits in the budget, the better of the run's own path and the best
refined one is returned, and an error raised by the run reaches the caller."""
import contextlib
import threading
import time

import numpy as np
import pytest
import torch

from paper_2607_03987_gb300 import refine

D, M = 6, 3


@pytest.fixture
def cpu_torch(monkeypatch):
    """Device tensors of the scheduler on the host; stream contexts as no-ops."""
    zeros, full = torch.zeros, torch.full
    monkeypatch.setattr(torch, "zeros", lambda *a, device=None, **k: zeros(*a, **k))
    monkeypatch.setattr(torch, "full", lambda *a, device=None, **k: full(*a, **k))
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())


class _Stream:
    def synchronize(self):
        pass


class FakeRun:
    """An AO-x run that publishes path k (cost costs[k - 1]) k `period`s after it starts."""

    def __init__(self, costs, period=0.004, fail=False):
        self.costs, self.period, self.fail = list(costs), period, fail
        self.device, self.stream = 0, _Stream()
        self.t0 = None
        self.offers = []
        self.lock = threading.Lock()

    def _published(self):
        if self.t0 is None:
            return 0
        return min(len(self.costs), int((time.perf_counter() - self.t0) / self.period))

    def plan(self, x0, xg, budget_s, seed):
        self.t0 = time.perf_counter()
        time.sleep(budget_s)
        if self.fail:
            raise RuntimeError("device error flags 0x4")
        k = self._published()
        if k == 0:
            return dict(cost=float("inf"), n_solutions=0)
        return dict(cost=self.costs[k - 1], n_solutions=k, states=np.zeros((3, D), np.float32),
                    controls=np.zeros((2, M), np.float32), steps=np.ones(2, np.int32))

    def plan_snapshot(self, st, ct, sp, info, stream):
        k = self._published()
        if k == 0:
            info.zero_()
            return
        bits = int(np.array([self.costs[k - 1]], np.float32).view(np.int32)[0])
        info.copy_(torch.tensor([1, 2, k, bits], dtype=torch.int32))
        ct.fill_(float(k))  # the path's number, for the refinement stand-ins

    def offer_bound(self, cost_dev, stream):
        with self.lock:
            self.offers.append(float(cost_dev[0]))


SPEC = dict(d=D, m=M, x_init=np.zeros(D, np.float32), x_goal=np.ones(D, np.float32))


def _stand_in(duration, calls, next_cost):
    """refine_path's stand-in: takes `duration` seconds and returns the next of `next_cost` (None:
    the refinement found no accepted path)."""
    def refine_path(planner, spec, path, x_goal, iters=15):
        t = time.perf_counter()
        time.sleep(duration)
        calls.append((t, time.perf_counter()))
        c = next_cost.pop(0) if next_cost else None
        return None if c is None else (torch.zeros((len(path["steps"]), M)), c)
    return refine_path


def test_offers_only_improving_refinements(cpu_torch, monkeypatch):
    costs = [2.0, 1.9, 1.8, 1.7, 1.6]
    run = FakeRun(costs=costs, period=0.01)
    seen = []

    def refine_path(planner, spec, path, x_goal, iters=15):
        # path k (numbered from 1) refined to 0.06 below its cost when k is odd, to 0.06 above
        # when k is even (then the run's own path is better: no offer)
        k = int(path["controls"][0, 0])
        seen.append(k)
        time.sleep(0.002)
        c = costs[k - 1] + (-0.06 if k % 2 else 0.06)
        return torch.zeros((len(path["steps"]), M)), c

    monkeypatch.setattr(refine, "refine_path", refine_path)
    stats = {}
    cost, gain, path = refine.refined_aox_live(run, FakeRun([]), SPEC, budget_s=0.08, stats=stats)
    assert stats["refined"] == len(seen) >= 3
    assert seen == sorted(set(seen)), seen  # each new path once, in order
    # an offer for every refinement that beat the run's path and every earlier offer, no other
    expect, best = [], float("inf")
    for k in seen:
        c = costs[k - 1] + (-0.06 if k % 2 else 0.06)
        if c < min(costs[k - 1], best):
            expect.append(c)
            best = c
    assert run.offers == pytest.approx(expect)
    assert stats.get("improved", 0) == len(expect)
    assert gain == pytest.approx(0.06 * len(expect))
    own = costs[run._published() - 1]
    assert cost == pytest.approx(min([own] + expect))
    assert path is not None and path["controls"].shape == (2, M)


def test_no_refinement_starts_past_the_deadline(cpu_torch, monkeypatch):
    budget, duration = 0.06, 0.025
    run = FakeRun(costs=[2.0 - 0.01 * i for i in range(50)], period=0.002)
    calls = []
    # never better than the run's own path: nothing is offered
    monkeypatch.setattr(refine, "refine_path", _stand_in(duration, calls, [3.0] * 50))
    stats = {}
    t0 = time.perf_counter()
    refine.refined_aox_live(run, FakeRun([]), SPEC, budget_s=budget, stats=stats)
    assert run.offers == []
    assert stats.get("improved", 0) == 0
    # the first refinement starts as soon as a path exists; a later one only while the previous
    # refinement's duration still fits before the budget ends
    starts = [s - t0 for s, _ in calls]
    assert len(starts) >= 1
    for k in range(1, len(starts)):
        last = calls[k - 1][1] - calls[k - 1][0]
        assert starts[k] + last < budget + 0.01, (starts, last)
    assert len(starts) <= int(budget / duration) + 1


def test_run_error_reaches_the_caller(cpu_torch):
    run = FakeRun(costs=[], fail=True)
    with pytest.raises(RuntimeError, match="device error"):
        refine.refined_aox_live(run, FakeRun([]), SPEC, budget_s=0.02)


def test_returns_the_runs_own_path_without_refinement(cpu_torch, monkeypatch):
    run = FakeRun(costs=[1.8], period=0.001)
    calls = []
    # the refinement finds no accepted path
    monkeypatch.setattr(refine, "refine_path", _stand_in(0.001, calls, [None]))
    cost, gain, path = refine.refined_aox_live(run, FakeRun([]), SPEC, budget_s=0.02)
    assert run.offers == [] and gain == 0.0
    assert cost == pytest.approx(1.8)
    assert path is not None and path["steps"].tolist() == [1, 1]
