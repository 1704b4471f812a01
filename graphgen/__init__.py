"""Seeded synthetic graph inputs (R-MAT, Erdos-Renyi, 2-D grid) as int32 CSR.

Input preparation only: this package holds none of the BFS method's arithmetic.
Both the CPU oracle tests and the CUDA path's tests and benchmark draw their
graphs and sources from here.  The C generator (``graphgen.c``) uses integer
arithmetic only, so a seed gives byte-identical graphs on every host.

Workload shapes follow the paper's setting of large sparse real-world graphs
(Wikipedia, "real-world and synthetic graphs", Experimental Results): R-MAT is
the usual power-law stand-in; grids stand in for high-diameter meshes.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from fractions import Fraction

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_SO = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


class _CSR(ctypes.Structure):
    _fields_ = [
        ("n", ctypes.c_int32),
        ("nnz", ctypes.c_int64),
        ("row_ptr", ctypes.POINTER(ctypes.c_int32)),
        ("col_idx", ctypes.POINTER(ctypes.c_int32)),
    ]


def build(force: bool = False) -> str:
    """Compile ``libgraphgen.so`` next to its source (gcc, portable flags)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        base = ["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", tmp, _SRC]
        try:  # OpenMP only speeds generation up; results do not depend on it
            subprocess.check_call(base + ["-fopenmp"], stderr=subprocess.DEVNULL)
        except (subprocess.CalledProcessError, OSError):
            subprocess.check_call(base)
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_CSR)
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.gg_rmat.restype = P
            lib.gg_rmat.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint32,
                                    ctypes.c_uint32, ctypes.c_uint64, ctypes.c_int32]
            lib.gg_er.restype = P
            lib.gg_er.argtypes = [ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64]
            lib.gg_grid.restype = P
            lib.gg_grid.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_uint64, ctypes.c_uint64]
            lib.gg_from_edges.restype = P
            lib.gg_from_edges.argtypes = [ctypes.c_int32, ctypes.c_int64, i32p, i32p]
            lib.gg_sample_sources.restype = ctypes.c_int32
            lib.gg_sample_sources.argtypes = [ctypes.c_int32, i32p, ctypes.c_int32, ctypes.c_uint64, i32p]
            lib.gg_free.restype = None
            lib.gg_free.argtypes = [P]
            _lib = lib
    return _lib


def _take(p) -> tuple[np.ndarray, np.ndarray]:
    lib = _load()
    if not p:
        raise MemoryError("graph generator failed (bad arguments or out of memory)")
    g = p.contents
    n, nnz = int(g.n), int(g.nnz)
    row_ptr = np.ctypeslib.as_array(g.row_ptr, shape=(n + 1,)).copy()
    col_idx = np.ctypeslib.as_array(g.col_idx, shape=(max(nnz, 1),))[:nnz].copy()
    lib.gg_free(p)
    return row_ptr, col_idx


def _thresh32(p: float) -> int:
    return min(int(Fraction(p) * (1 << 32)), (1 << 32) - 1)


def rmat(scale: int, edgefactor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1, relabel: bool = True) -> tuple[np.ndarray, np.ndarray]:
    """R-MAT graph: 2^scale vertices, edgefactor*2^scale edge samples, quadrant
    probabilities A/B/C/D (D = 1-A-B-C), seeded vertex relabelling, then
    symmetrised with self-loops and duplicates removed and rows sorted."""
    ta = _thresh32(a)
    tab = _thresh32(a + b)
    tabc = _thresh32(a + b + c)
    p = _load().gg_rmat(scale, edgefactor << scale, ta, tab, tabc, seed, 1 if relabel else 0)
    return _take(p)


def erdos_renyi(n: int, m: int, seed: int = 4) -> tuple[np.ndarray, np.ndarray]:
    """G(n, m): m distinct undirected non-loop edges, symmetrised CSR."""
    return _take(_load().gg_er(n, m, seed))


def grid(rows: int, cols: int, p_delete: float = 0.01, seed: int = 3) -> tuple[np.ndarray, np.ndarray]:
    """rows x cols 4-neighbour grid (id = r*cols + c); every undirected edge is
    deleted independently with probability p_delete."""
    t = min(int(Fraction(p_delete) * (1 << 64)), (1 << 64) - 1)
    return _take(_load().gg_grid(rows, cols, t, seed))


def from_edges(n: int, edges) -> tuple[np.ndarray, np.ndarray]:
    """Symmetric simple CSR of an undirected edge list [(u, v), ...]."""
    e = np.asarray(edges, dtype=np.int32).reshape(-1, 2)
    a = np.ascontiguousarray(e[:, 0])
    b = np.ascontiguousarray(e[:, 1])
    i32p = ctypes.POINTER(ctypes.c_int32)
    p = _load().gg_from_edges(n, len(a), a.ctypes.data_as(i32p), b.ctypes.data_as(i32p))
    return _take(p)


def sample_sources(row_ptr: np.ndarray, k: int, seed: int = 2) -> np.ndarray:
    """k distinct sources drawn uniformly among vertices with degree > 0."""
    rp = np.ascontiguousarray(row_ptr, dtype=np.int32)
    out = np.empty(max(k, 1), dtype=np.int32)
    i32p = ctypes.POINTER(ctypes.c_int32)
    got = _load().gg_sample_sources(len(rp) - 1, rp.ctypes.data_as(i32p), k, seed, out.ctypes.data_as(i32p))
    if got < 0:
        raise MemoryError("source sampling failed")
    return out[:got].copy()


# Named workloads (sizes and seeds of the benchmark configurations).
def rmat_s16():
    return rmat(16, 16, seed=1)


def rmat_s22():
    return rmat(22, 16, seed=1)


def grid_4096():
    return grid(4096, 4096, 0.01, seed=3)


def er_2p20():
    return erdos_renyi(1 << 20, 8 << 20, seed=4)
