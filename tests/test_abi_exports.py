"""The C-ABI library builds, loads, and exports every function that
include/s3bfs.h declares (CPU only: no kernel is launched)."""
import ctypes
import os
import re

import pytest

import paper_2209_08764_gb300 as pkg
from paper_2209_08764_gb300 import binding as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(bfs_\w+)\s*\(", src))
    return names


@pytest.fixture(scope="module")
def lib():
    pkg.build()
    return B.load()


def test_every_declared_symbol_is_exported(lib):
    declared = _declared()
    assert {"bfs_create_csr", "bfs_run", "bfs_run_batch", "bfs_destroy", "bfs_strerror"} <= declared
    for name in sorted(declared):
        assert hasattr(lib, name), f"{name} declared in include/ but not exported"
    assert set(B.EXPORTS) >= declared


def test_host_only_calls(lib):
    assert B.bfs_strerror(0) == "ok"
    assert "timed out" in B.bfs_strerror(B.BFS_E_TIMEOUT)
    assert B.bfs_strerror(12345) == "unknown error"
    # argument checks happen before any CUDA call
    out = ctypes.c_void_p()
    assert lib.bfs_create_csr(0, 0, None, None, 0, None, None, ctypes.byref(out)) == B.BFS_E_INVAL
    assert out.value is None
    assert "n = 0" in B.bfs_last_error()
    assert lib.bfs_run(None, 0, None, None, None) == B.BFS_E_INVAL
    assert lib.bfs_run_batch(None, None, 0, None, None, None) == B.BFS_E_INVAL
    lib.bfs_destroy(None)


def test_struct_layout_matches_header():
    # int32 x 10
    assert ctypes.sizeof(B.bfs_opts) == 40
    # 2 int32, 3 int64, 2 float, pointer, int32 (+ padding), int64
    assert B.bfs_stats.per_level.offset == 40
    assert B.bfs_stats.work_edges.offset == 56
    assert ctypes.sizeof(B.bfs_stats) == 64


def test_server_struct_layout():
    assert ctypes.sizeof(B.bfs_server_opts) == 32
    assert B.bfs_completion.t_submit_us.offset == 40
    assert ctypes.sizeof(B.bfs_completion) == 64
