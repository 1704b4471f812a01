"""ctypes binding of the C ABI in ``include/s3bfs.h`` (argument marshalling only).

Every function keeps the C name and argument order.  Arrays may be given as
numpy arrays (host), torch tensors (host or CUDA) or raw integer addresses; all
must be contiguous int32.  A non-zero status is raised as :class:`BFSError`
carrying the code and the library's message.  Every step of the traversal runs
in the CUDA library; nothing here computes.  The library must have been built
(``__graft_entry__.build()`` or ``paper_2209_08764_gb300._build.build()``); a
missing library raises instead of falling back to anything.
"""
from __future__ import annotations

import ctypes
import os

from . import _build

BFS_OK = 0
BFS_E_INVAL = -1
BFS_E_MULTIGRAPH = -2
BFS_E_NOMEM = -3
BFS_E_CUDA = -4
BFS_E_TIMEOUT = -5
BFS_E_CHECK = -6

BFS_DEVICE_PTRS = 1
BFS_VALIDATE = 2
BFS_DEDUP = 4
BFS_SYMMETRIC = 8

BFS_DEBUG_STALL_BARRIER = 1
BFS_DEBUG_CHECK_INJECT = 2
BFS_LEVEL_FIELDS = 9

EXPORTS = ("bfs_create_csr", "bfs_run", "bfs_run_batch", "bfs_destroy", "bfs_strerror", "bfs_last_error",
           "bfs_graph_info", "bfs_graph_device_bytes", "bfs_run_frontiers", "bfs_run_csr_noalloc", "bfs_server_create", "bfs_server_submit", "bfs_server_poll",
           "bfs_server_pending", "bfs_server_destroy")


class bfs_opts(ctypes.Structure):
    _fields_ = [
        ("chunk_edges", ctypes.c_int32),
        ("ctas", ctypes.c_int32),
        ("persistent", ctypes.c_int32),
        ("work_insensitive", ctypes.c_int32),
        ("spin_limit_ms", ctypes.c_int32),
        ("debug_flags", ctypes.c_int32),
        ("relabel", ctypes.c_int32),
        ("batch_bitmask", ctypes.c_int32),
        ("small_level_edges", ctypes.c_int32),
        ("cta_warps", ctypes.c_int32),
        ("direction", ctypes.c_int32),
        ("do_alpha", ctypes.c_int32),
        ("do_beta", ctypes.c_int32),
        ("do_gamma", ctypes.c_int32),
        ("reserved", ctypes.c_int32),
        ("max_device_bytes", ctypes.c_int64),
    ]


class bfs_stats(ctypes.Structure):
    _fields_ = [
        ("num_levels", ctypes.c_int32),
        ("active_ctas", ctypes.c_int32),
        ("reached", ctypes.c_int64),
        ("edges_scanned", ctypes.c_int64),
        ("candidates", ctypes.c_int64),
        ("ms_level_step", ctypes.c_float),
        ("ms_total", ctypes.c_float),
        ("per_level", ctypes.POINTER(ctypes.c_int32)),
        ("per_level_cap", ctypes.c_int32),
        ("launches", ctypes.c_int32),
        ("work_edges", ctypes.c_int64),
    ]


class bfs_server_opts(ctypes.Structure):
    _fields_ = [
        ("slots", ctypes.c_int32),
        ("levels_per_launch", ctypes.c_int32),
        ("chunk_edges", ctypes.c_int32),
        ("cta_warps", ctypes.c_int32),
        ("spin_limit_ms", ctypes.c_int32),
        ("local_levels", ctypes.c_int32),
        ("arena_bytes", ctypes.c_int64),
    ]


class bfs_completion(ctypes.Structure):
    _fields_ = [
        ("tag", ctypes.c_int64),
        ("graph", ctypes.c_int32),
        ("src", ctypes.c_int32),
        ("status", ctypes.c_int32),
        ("num_levels", ctypes.c_int32),
        ("reached", ctypes.c_int64),
        ("edges_scanned", ctypes.c_int64),
        ("t_submit_us", ctypes.c_double),
        ("t_admit_us", ctypes.c_double),
        ("t_done_us", ctypes.c_double),
    ]


class BFSError(RuntimeError):
    def __init__(self, code: int, message: str):
        super().__init__(f"{message} [code {code}]")
        self.code = code


_lib = None


def library_path() -> str:
    """The library this process loads: libs3bfs.so, or the range-checked debug
    build libs3bfs_checked.so when the environment sets S3BFS_LIBRARY=checked."""
    return _build.LIB_CHECKED if os.environ.get("S3BFS_LIBRARY", "") == "checked" else _build.LIB


def load():
    """Load the library (see library_path); raises if it has not been built."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"CUDA library not built: {path} is missing (run __graft_entry__.build())")
    lib = ctypes.CDLL(path)
    vp, i32, i32p = ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p
    lib.bfs_create_csr.restype = ctypes.c_int
    lib.bfs_create_csr.argtypes = [i32, i32, i32p, i32p, ctypes.c_int, ctypes.POINTER(bfs_opts), vp,
                                   ctypes.POINTER(vp)]
    lib.bfs_run.restype = ctypes.c_int
    lib.bfs_run.argtypes = [vp, i32, i32p, i32p, ctypes.POINTER(bfs_stats)]
    lib.bfs_run_batch.restype = ctypes.c_int
    lib.bfs_run_batch.argtypes = [vp, i32p, i32, i32p, i32p, ctypes.POINTER(bfs_stats)]
    lib.bfs_destroy.restype = None
    lib.bfs_destroy.argtypes = [vp]
    lib.bfs_strerror.restype = ctypes.c_char_p
    lib.bfs_strerror.argtypes = [ctypes.c_int]
    lib.bfs_last_error.restype = ctypes.c_char_p
    lib.bfs_last_error.argtypes = []
    lib.bfs_graph_info.restype = ctypes.c_int
    lib.bfs_graph_info.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32), ctypes.POINTER(i32),
                                   ctypes.POINTER(i32)]
    lib.bfs_graph_device_bytes.restype = ctypes.c_int64
    lib.bfs_graph_device_bytes.argtypes = [vp]
    lib.bfs_run_frontiers.restype = ctypes.c_int
    lib.bfs_run_frontiers.argtypes = [vp, i32, i32p, i32p, ctypes.POINTER(bfs_stats), i32p]
    lib.bfs_run_csr_noalloc.restype = ctypes.c_int
    lib.bfs_run_csr_noalloc.argtypes = [i32, i32, i32p, i32p, i32, i32p, i32p, vp]
    lib.bfs_server_create.restype = ctypes.c_int
    lib.bfs_server_create.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(bfs_server_opts), vp,
                                      ctypes.POINTER(vp)]
    lib.bfs_server_submit.restype = ctypes.c_int
    lib.bfs_server_submit.argtypes = [vp, i32, i32, i32p, i32p, ctypes.c_int64]
    lib.bfs_server_poll.restype = ctypes.c_int
    lib.bfs_server_poll.argtypes = [vp, ctypes.POINTER(bfs_completion), i32, ctypes.POINTER(i32)]
    lib.bfs_server_pending.restype = ctypes.c_int
    lib.bfs_server_pending.argtypes = [vp, ctypes.POINTER(i32), ctypes.POINTER(i32)]
    lib.bfs_server_destroy.restype = None
    lib.bfs_server_destroy.argtypes = [vp]
    _lib = lib
    return lib


def _addr(x, what: str):
    """Address of an int32 contiguous array-like (numpy, torch, int) or None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    mod = type(x).__module__
    if mod.startswith("torch"):
        import torch
        if x.dtype != torch.int32 or not x.is_contiguous():
            raise TypeError(f"{what}: need a contiguous int32 tensor")
        return x.data_ptr()
    if mod.startswith("numpy"):
        import numpy as np
        if x.dtype != np.int32 or not x.flags["C_CONTIGUOUS"]:
            raise TypeError(f"{what}: need a C-contiguous int32 array")
        return x.ctypes.data
    raise TypeError(f"{what}: unsupported array type {type(x)}")


def _check(rc: int):
    if rc != BFS_OK:
        lib = load()
        msg = lib.bfs_last_error().decode() or lib.bfs_strerror(rc).decode()
        raise BFSError(rc, f"{lib.bfs_strerror(rc).decode()}: {msg}")


def bfs_create_csr(n: int, nnz: int, row_ptr, col_idx, flags: int = 0, opts: bfs_opts | None = None,
                   cuda_stream: int | None = None) -> int:
    """Returns the opaque graph handle (an int)."""
    lib = load()
    out = ctypes.c_void_p()
    rc = lib.bfs_create_csr(int(n), int(nnz), _addr(row_ptr, "row_ptr"), _addr(col_idx, "col_idx"), int(flags),
                            ctypes.byref(opts) if opts is not None else None, cuda_stream or None, ctypes.byref(out))
    _check(rc)
    return out.value


def bfs_run(g: int, src: int, level_out, parent_out=None, stats: bfs_stats | None = None) -> None:
    rc = load().bfs_run(g, int(src), _addr(level_out, "level_out"), _addr(parent_out, "parent_out"),
                        ctypes.byref(stats) if stats is not None else None)
    _check(rc)


def bfs_run_batch(g: int, srcs, k: int, levels_out, parents_out=None, stats=None) -> None:
    """``stats``: None or a ctypes array of k bfs_stats."""
    rc = load().bfs_run_batch(g, _addr(srcs, "srcs"), int(k), _addr(levels_out, "levels_out"),
                              _addr(parents_out, "parents_out"), stats)
    _check(rc)


def bfs_destroy(g: int | None) -> None:
    if g:
        load().bfs_destroy(g)


def bfs_strerror(code: int) -> str:
    return load().bfs_strerror(int(code)).decode()


def bfs_last_error() -> str:
    return load().bfs_last_error().decode()


def bfs_run_frontiers(g: int, src: int, level_out, parent_out, stats, frontiers_out) -> None:
    rc = load().bfs_run_frontiers(g, int(src), _addr(level_out, "level_out"), _addr(parent_out, "parent_out"),
                                  ctypes.byref(stats) if stats is not None else None,
                                  _addr(frontiers_out, "frontiers_out"))
    _check(rc)


def bfs_graph_device_bytes(g: int) -> int:
    return int(load().bfs_graph_device_bytes(g))


def bfs_graph_info(g: int) -> dict:
    n, nnz, ctas, warps = (ctypes.c_int32() for _ in range(4))
    _check(load().bfs_graph_info(g, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(ctas), ctypes.byref(warps)))
    return {"n": n.value, "nnz": nnz.value, "ctas": ctas.value, "warps": warps.value}


def bfs_run_csr_noalloc(n: int, nnz: int, row_ptr, col_idx, src: int, level_out, parent_out,
                        cuda_stream: int | None = None) -> None:
    """One traversal with no allocation: device CSR and device outputs from the
    caller, working memory in the library's fixed static device array (for
    callers that must not allocate device memory; sizes are capped)."""
    rc = load().bfs_run_csr_noalloc(int(n), int(nnz), _addr(row_ptr, "row_ptr"), _addr(col_idx, "col_idx"),
                                    int(src), _addr(level_out, "level_out"), _addr(parent_out, "parent_out"),
                                    cuda_stream or None)
    _check(rc)


def bfs_server_create(graphs, opts: bfs_server_opts | None = None, cuda_stream: int | None = None) -> int:
    """``graphs``: handles from bfs_create_csr.  Returns the server handle."""
    lib = load()
    arr = (ctypes.c_void_p * len(graphs))(*graphs)
    out = ctypes.c_void_p()
    rc = lib.bfs_server_create(arr, len(graphs), ctypes.byref(opts) if opts is not None else None,
                               cuda_stream or None, ctypes.byref(out))
    _check(rc)
    return out.value


def bfs_server_submit(s: int, graph: int, src: int, level_out=None, parent_out=None, tag: int = 0) -> None:
    _check(load().bfs_server_submit(s, int(graph), int(src), _addr(level_out, "level_out"),
                                    _addr(parent_out, "parent_out"), int(tag)))


def bfs_server_poll(s: int, cap: int = 256) -> list:
    """One scheduling round; returns the completion records it produced."""
    buf = (bfs_completion * cap)()
    nd = ctypes.c_int32()
    _check(load().bfs_server_poll(s, buf, cap, ctypes.byref(nd)))
    return [buf[i] for i in range(nd.value)]


def bfs_server_pending(s: int) -> tuple[int, int]:
    q, r = ctypes.c_int32(), ctypes.c_int32()
    _check(load().bfs_server_pending(s, ctypes.byref(q), ctypes.byref(r)))
    return q.value, r.value


def bfs_server_destroy(s: int | None) -> None:
    if s:
        load().bfs_server_destroy(s)
