"""bench.py's host logic on CPU: multi-rank aggregation over gloo (world size 2)
and the reference arm's JSON line."""
import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r processes 1000*(r+1) units in (r+1) seconds
    value, t_max, units = bench.aggregate(1000.0 * (rank + 1), float(rank + 1))
    q.put((rank, value, t_max, units))
    dist.destroy_process_group()


def test_aggregate_two_ranks_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = sorted(q.get() for _ in range(2))
    for rank, value, t_max, units in res:
        assert t_max == 2.0 and units == 3000.0
        assert value == pytest.approx(1500.0)


def test_reference_arm_prints_one_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [ln for ln in out.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "rollouts/s" and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_other_ranks_do_nothing():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                          "--warmup", "0"], capture_output=True, text=True, timeout=120, cwd=ROOT, env=env)
    assert out.returncode == 0 and out.stdout.strip() == ""


def test_work_counts():
    """The roofline's work and byte counts: 3 K n d flops (a subtract, a multiply and an add
    per coordinate of every query-node pair) and n (d + 1) 4-byte words per pass."""
    sys.path.insert(0, ROOT)
    import bench

    assert bench.nn_flops_per_launch(1024, 1_000_000, 6) == 3 * 1024 * 1_000_000 * 6
    assert bench.nn_bytes_per_launch(1_000_000, 6) == 28_000_000
    # as issued: 1024 queries in 8 blocks of 128, 1,000,000 nodes padded to 3907 tiles of 256,
    # two K = 16 MMAs per 128 x 128 block
    assert bench.nn_tc_mma_flops_per_launch(1024, 1_000_000, 6, 16, 2) == 2.0 * 1024 * 3907 * 256 * 16 * 2
    assert bench.nn_tc_filter_flops_per_launch(1024, 1_000_000, 6, 16) == 2.0 * 1024 * 1_000_000 * 16


def test_tc_shape_matches_the_kernel(tmp_path):
    """bench.tc_shape (packed row width, MMAs per stage) agrees with the kernel's TcShape."""
    nvcc = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not found")
    sys.path.insert(0, ROOT)
    import bench

    dims = (3, 4, 5, 6, 12)
    src = tmp_path / "shape.cu"
    body = "".join(f'    std::printf("%d %d %d\\n", {d}, pakr::TcShape<{d}>::KT, pakr::TcShape<{d}>::MMAS);\n'
                   for d in dims)
    src.write_text('#include <cstdio>\n#include "pakr_tc.cuh"\nint main()\n{\n' + body + "    return 0;\n}\n")
    exe = tmp_path / "shape"
    csrc = os.path.join(ROOT, "paper_2607_03987_gb300", "csrc")
    r = subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", csrc, "-I",
                        os.path.join(ROOT, "include"), str(src), "-o", str(exe)], capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    got = {int(a): (int(b), int(c)) for a, b, c in (ln.split() for ln in out.stdout.split("\n") if ln.strip())}
    assert got == {d: bench.tc_shape(d) for d in dims}


def test_grown_tree_measurement_logic(monkeypatch):
    """bench.grown_tree_expansions on a fake planner and fake CUDA events: the tree is grown by
    plain expansions until it holds the benchmark's node count, every timed step starts from
    that count, and the per-kernel times come from the profiled pass alone."""
    import torch

    sys.path.insert(0, ROOT)
    import bench
    from paper_2607_03987_gb300 import pakr

    log = []

    class FakePlanner:
        def __init__(self, spec, device=0, stream=None):
            self.n, self.prof, self.kt = 0, False, {}

        def tree_reset(self, x_init, x_goal):
            self.n = 1

        def expand(self, bound, seed, info=True):
            assert bound == float("inf")
            log.append(("expand", self.n, self.prof))
            self.n = min(1 << 20, self.n + 6000)
            if self.prof:
                for k in ("k_sample", "k_nn_tc", "k_propagate", "k_append"):
                    e = self.kt.setdefault(k, {"ms": 0.0, "launches": 0})
                    e["ms"] += 0.05
                    e["launches"] += 1
            return 0, None

        def tree_size(self):
            return self.n, 0

        def tree_truncate(self, n):
            self.n = min(self.n, n)

        def set_profiling(self, on):
            self.prof = on
            if on:
                self.kt = {}

        def kernel_times(self):
            return self.kt

        def close(self):
            log.append(("close",))

    class Event:
        def __init__(self, enable_timing=True):
            pass

        def record(self, stream=None):
            pass

        def elapsed_time(self, other):
            return 0.1

    empty = torch.empty
    monkeypatch.setattr(pakr, "Planner", FakePlanner)
    monkeypatch.setattr(torch.cuda, "Event", Event)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda dev=None: None)
    monkeypatch.setattr(torch, "empty", lambda *a, device=None, **k: empty(16))
    r = bench.grown_tree_expansions(0, None, steps=4, warmup=3)
    grow = -(-(bench.N_PREFILL - 1) // 6000)
    assert r["n"] == bench.N_PREFILL and r["grown_in_expansions"] == grow
    timed = [e for e in log[grow:] if e[0] == "expand"]
    assert len(timed) == 3 + 4 + 4 and all(n == bench.N_PREFILL for _, n, _ in timed)
    assert r["ms_per_step"] == pytest.approx(0.1) and r["nn_ms"] == pytest.approx(0.05)
    assert r["rollouts_per_s"] == pytest.approx(1024 * 8 / 0.1e-3)
    assert log[-1] == ("close",)
