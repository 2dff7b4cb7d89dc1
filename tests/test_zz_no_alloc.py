"""pakr_nearest_static, the nearest-neighbour entry point that allocates nothing.

Callers that cannot allocate device memory (real-time loops that forbid
allocation after start-up, plugins confined to another framework's memory
pool) pass their own inputs and outputs; the search scratch is a static device
array inside the library.  Its answers must equal the nearest neighbours
pakr_expand chose for the same samples on the same tree, on two calls in a row
(the second call reuses the scratch the first one left behind), within the
near-tie margin the other parity tests use: pakr_expand ranks distances on
coordinates centred on the state box, which round differently, so the two may
differ only where the FP64 distances of their two choices are within 1e-6.
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2607_03987_gb300 import pakr
from paper_2607_03987_gb300 import workloads as W
from parity import NN_GAP

pytestmark = pytest.mark.gpu


def test_nearest_static_matches_expand(cuda_lib):
    import torch

    spec = W.with_sizes(W.problem("di3", env_seed=3), K=1024, k=2, cap=40000)
    n = 30011  # several node chunks and a ragged last tile
    tree = W.prefilled_tree(spec, n, seed=5)
    planner = pakr.Planner(spec)
    planner.tree_import(tree, spec["x_goal"])
    d, K = spec["d"], spec["K"]
    states = torch.tensor(np.ascontiguousarray(tree["states"].T), dtype=torch.float32, device="cuda")  # d x n
    fcost = torch.zeros(n, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    lib = pakr.lib()
    for call in range(2):
        planner.tree_truncate(n)
        planner.expand(np.inf, seed=100 + call)
        dbg = planner.debug_last_expand()
        queries = torch.tensor(np.ascontiguousarray(dbg["samples"].T), dtype=torch.float32, device="cuda")
        nearest = torch.full((K,), -7, dtype=torch.int32, device="cuda")
        dist2 = torch.empty(K, dtype=torch.float32, device="cuda")
        st = lib.pakr_nearest_static(C.c_void_p(states.data_ptr()), n, n, d, C.c_void_p(fcost.data_ptr()),
                                     float("inf"), C.c_void_p(queries.data_ptr()), K,
                                     C.c_void_p(nearest.data_ptr()), C.c_void_p(dist2.data_ptr()),
                                     C.c_void_p(stream))
        assert st == pakr.OK, lib.pakr_last_error()
        torch.cuda.synchronize()
        got = nearest.cpu().numpy()
        diff_q = np.nonzero(got != dbg["near"])[0]
        q64 = dbg["samples"].astype(np.float64)
        for i in diff_q:
            a = np.linalg.norm(q64[i] - tree["states"][got[i]])
            b = np.linalg.norm(q64[i] - tree["states"][dbg["near"][i]])
            assert abs(a - b) < NN_GAP, f"call {call}, query {i}: {got[i]} vs {dbg['near'][i]} ({a} vs {b})"
        assert len(diff_q) <= K // 100
        # the reported squared distance is the FP32 distance to the chosen node
        diff = dbg["samples"].astype(np.float64) - tree["states"][got]
        want = np.sum(diff * diff, axis=1)
        assert np.allclose(dist2.cpu().numpy(), want, rtol=1e-5, atol=1e-7)
    planner.close()


def test_nearest_static_rejects_oversize_and_handles_empty(cuda_lib):
    import torch

    lib = pakr.lib()
    out = torch.empty(4, dtype=torch.int32, device="cuda")
    q = torch.zeros(6 * 4, dtype=torch.float32, device="cuda")
    st = lib.pakr_nearest_static(None, 0, 0, 6, None, float("inf"), C.c_void_p(q.data_ptr()), 70000,
                                 C.c_void_p(out.data_ptr()), None, None)
    assert st == pakr.ERR_INVALID_ARG
    assert b"65536" in lib.pakr_last_error()
    st = lib.pakr_nearest_static(None, 0, 0, 7, None, float("inf"), C.c_void_p(q.data_ptr()), 4,
                                 C.c_void_p(out.data_ptr()), None, None)
    assert st == pakr.ERR_INVALID_ARG
    # an empty tree gives -1 for every query
    st = lib.pakr_nearest_static(None, 0, 0, 6, None, float("inf"), C.c_void_p(q.data_ptr()), 4,
                                 C.c_void_p(out.data_ptr()), None, None)
    assert st == pakr.OK
    torch.cuda.synchronize()
    assert np.all(out.cpu().numpy() == -1)
