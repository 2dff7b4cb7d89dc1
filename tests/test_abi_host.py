"""The C ABI library without a GPU: it builds, loads, exports every function
include/pakr.h declares, and its host-side argument checks answer with
statuses and messages (no compute calls)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from paper_2607_03987_gb300 import _build, pakr
from paper_2607_03987_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    src = open(os.path.join(ROOT, "include", "pakr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pakr_[a-z0-9_]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    _build.build()
    return pakr.lib()


def test_every_declared_function_is_exported(lib):
    names = header_functions()
    assert len(names) >= 15
    raw = C.CDLL(pakr.lib_path())
    for n in names:
        assert hasattr(raw, n), n
    assert sorted(pakr.EXPORTED) == names


def test_version(lib):
    assert b"sm_103a" in lib.pakr_version()


def make_desc(spec, keep):
    planner_like = pakr.Planner.__new__(pakr.Planner)
    desc = pakr.ProblemDesc()

    def arr(v):
        a = np.ascontiguousarray(np.asarray(v, dtype=np.float32).reshape(-1))
        keep.append(a)
        return a.ctypes.data_as(C.POINTER(C.c_float))

    desc.dynamics = spec["dyn"]
    desc.x_lo, desc.x_hi = arr(spec["x_lo"]), arr(spec["x_hi"])
    desc.u_lo, desc.u_hi = arr(spec["u_lo"]), arr(spec["u_hi"])
    desc.dt = spec["dt"]
    desc.steps_min, desc.steps_max = spec["s_min"], spec["s_max"]
    desc.n_boxes = spec["boxes"].shape[0]
    desc.boxes = arr(spec["boxes"])
    desc.goal_radius = spec["goal_r"]
    desc.n_parents, desc.branching = spec["K"], spec["k"]
    desc.tree_cap = spec["cap"]
    del planner_like
    return desc


def test_workspace_size_and_argument_checks(lib):
    keep = []
    spec = W.problem("di3")
    desc = make_desc(spec, keep)
    nbytes = C.c_uint64()
    assert lib.pakr_workspace_size(C.byref(desc), C.byref(nbytes)) == pakr.OK
    # the tree alone is cap x (d + m + 4) words
    assert nbytes.value > spec["cap"] * (6 + 3 + 4) * 4
    bad = [("dt", 0.0), ("steps_min", 0), ("n_parents", 0), ("tree_cap", 0), ("dynamics", 42),
           ("goal_radius", float("nan")), ("n_boxes", 5000)]
    for field, val in bad:
        d2 = make_desc(spec, keep)
        setattr(d2, field, val)
        st = lib.pakr_workspace_size(C.byref(d2), C.byref(nbytes))
        assert st == pakr.ERR_INVALID_ARG, field
        assert lib.pakr_last_error(), field
    d2 = make_desc(spec, keep)
    lo = np.array([0, 0, 0, 2, -1, -1], np.float32)  # lo > hi on one axis
    keep.append(lo)
    d2.x_lo = lo.ctypes.data_as(C.POINTER(C.c_float))
    assert lib.pakr_workspace_size(C.byref(d2), C.byref(nbytes)) == pakr.ERR_INVALID_ARG
    assert b"x_lo" in lib.pakr_last_error()


def test_null_arguments_are_rejected(lib):
    assert lib.pakr_expand(None, 1.0, 0, None) == pakr.ERR_INVALID_ARG
    assert lib.pakr_tree_reset(None, None, None) == pakr.ERR_INVALID_ARG
    assert lib.pakr_create(None, None) == pakr.ERR_INVALID_ARG
    lib.pakr_destroy(None)


def test_create_without_gpu_fails_cleanly(lib):
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    keep = []
    desc = make_desc(W.problem("di2"), keep)
    h = C.c_void_p()
    st = lib.pakr_create(C.byref(desc), C.byref(h))
    assert st < 0 and not h.value
    assert lib.pakr_last_error()


def test_binding_refuses_missing_library(monkeypatch, tmp_path):
    monkeypatch.setattr(pakr, "_lib", None)
    monkeypatch.setattr(pakr, "_LIB_PATH", str(tmp_path / "libpakr.so"))
    with pytest.raises(RuntimeError, match="missing"):
        pakr.lib()


STRUCTS = {"pakr_problem_desc": pakr.ProblemDesc, "pakr_expand_info": pakr.ExpandInfo,
           "pakr_tree_host": pakr.TreeHost, "pakr_path": pakr.Path, "pakr_traj_params": pakr.TrajParams,
           "pakr_batch_query": pakr.BatchQuery, "pakr_batch_tuning": pakr.BatchTuning,
           "pakr_batch_result": pakr.BatchResult}


def test_binding_structs_match_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets the
    C compiler gives the header's struct (a small C program prints them)."""
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "pakr.h"', "int main(void) {"]
    for cname, py in STRUCTS.items():
        lines.append(f'  printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'  printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    exe = tmp_path / "layout"
    src.write_text("\n".join(lines) + "\n")
    import subprocess
    subprocess.run(["gcc", "-std=c99", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {}
    for ln in out:
        if ln:
            c, f, v = ln.split()
            got[(c, f)] = int(v)
    for cname, py in STRUCTS.items():
        assert got[(cname, "size")] == C.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
