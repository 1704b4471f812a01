"""CPU oracle for the S3BFS level step -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  It shares no code with the CUDA library and
never imports it; the only module both sides use is ``graphgen`` (seeded
inputs, none of the method's arithmetic).

Contents
--------
``bfs``              plain definition of the result: sequential FIFO-queue BFS
                     (C, ``bfs_oracle.c``), returning hop distances ``d`` (the
                     array Parallel-BFS returns, Fig. 1 header) and a BFS tree.
``check_bfs_tree``   validity of any parent array against the levels (a parent
                     sits one level up and the tree edge exists).
``level_profile``    per-level frontier size n_l and edge count e_l implied by
                     a level array (Fig. 1's main loop, degree gather and EdgeSum).
``s3bfs_fig1``       Fig. 1 itself, step by step in the paper's order and
                     notation (numpy per step), for per-level quantities:
                     n_l, e_l, P_l, the start points, candidates and Sizes.
``traversed_edges``  Graph500 traversed-edge count of one traversal (half the
                     degree sum of the reached vertices), the numerator of
                     every GTEPS figure.
``start_points_scatter`` / ``start_points_bsearch``
                     Find-StartExpPoint (Fig. 1) in the paper's range-
                     scatter form (Analysis, last paragraph) and in the binary
                     search form it replaces.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bfs_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

INF = -1  # the oracle writes -1 where the paper writes infinity (Fig. 1, initialisation)


def build(force: bool = False) -> str:
    """Compile ``liboracle.so`` (plain C, single-threaded)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.oracle_bfs.restype = ctypes.c_int64
            lib.oracle_bfs.argtypes = [ctypes.c_int32, i32p, i32p, ctypes.c_int32, i32p, i32p, i32p]
            _lib = lib
    return _lib


def _i32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.int32)


class Oracle:
    """Reusable oracle for one CSR graph (keeps scratch buffers)."""

    def __init__(self, row_ptr, col_idx):
        self.row_ptr = _i32(row_ptr)
        self.col_idx = _i32(col_idx) if len(col_idx) else np.zeros(1, np.int32)
        self.n = len(self.row_ptr) - 1
        self._queue = np.empty(max(self.n, 1), np.int32)
        self._p = ctypes.POINTER(ctypes.c_int32)

    def bfs(self, src: int, level: np.ndarray | None = None, parent: np.ndarray | None = None):
        n = self.n
        level = np.empty(n, np.int32) if level is None else level
        parent = np.empty(n, np.int32) if parent is None else parent
        P = self._p
        r = _load().oracle_bfs(n, self.row_ptr.ctypes.data_as(P), self.col_idx.ctypes.data_as(P), int(src),
                               level.ctypes.data_as(P), parent.ctypes.data_as(P), self._queue.ctypes.data_as(P))
        if r < 0:
            raise ValueError(f"oracle_bfs: bad arguments (n={n}, src={src})")
        return level, parent


def bfs(row_ptr, col_idx, src: int):
    """Hop distances from ``src`` (-1 = unreachable) and one BFS tree."""
    return Oracle(row_ptr, col_idx).bfs(src)


def edge_keys(row_ptr, col_idx) -> np.ndarray:
    """Sorted int64 keys u*n+v of all CSR edges (rows sorted ascending)."""
    rp = np.asarray(row_ptr, np.int64)
    n = len(rp) - 1
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    keys = rows * n + np.asarray(col_idx, np.int64)
    if len(keys) > 1 and not np.all(keys[1:] >= keys[:-1]):
        keys = np.sort(keys)
    return keys


def check_bfs_tree(row_ptr, col_idx, src: int, level, parent, keys: np.ndarray | None = None) -> None:
    """Raise AssertionError unless ``parent`` is a BFS tree for ``level``:
    (i) parent[s] == s; (ii) every reached v != s has a reached parent one
    level up; (iii) the edge parent[v] -> v exists in the CSR; (iv) parent is
    -1 exactly where level is -1."""
    level = np.asarray(level)
    parent = np.asarray(parent)
    n = len(row_ptr) - 1
    assert level.shape == (n,) and parent.shape == (n,), "shape"
    assert parent[src] == src, f"parent[src]={parent[src]} != src={src}"
    reached = level >= 0
    assert np.array_equal(parent < 0, ~reached), "parent == -1 must match level == -1"
    v = np.nonzero(reached)[0]
    v = v[v != src]
    if len(v) == 0:
        return
    p = parent[v].astype(np.int64)
    assert np.all((p >= 0) & (p < n)), "parent out of range"
    bad = level[p] != level[v] - 1
    assert not bad.any(), f"{int(bad.sum())} parents not one level up, e.g. v={int(v[bad][0])}"
    keys = edge_keys(row_ptr, col_idx) if keys is None else keys
    want = p * n + v
    pos = np.searchsorted(keys, want)
    ok = (pos < len(keys)) & (keys[np.minimum(pos, len(keys) - 1)] == want)
    assert ok.all(), f"{int((~ok).sum())} tree edges missing from the CSR, e.g. v={int(v[~ok][0])}"


def level_profile(row_ptr, level) -> tuple[np.ndarray, np.ndarray]:
    """(n_l, e_l) for l = 0..L-1: vertices at distance l, and the sum of their
    out-degrees (the edges level l explores: Fig. 1's EdgeSum total e_l)."""
    level = np.asarray(level)
    deg = np.diff(np.asarray(row_ptr, np.int64))
    r = level >= 0
    if not r.any():
        return np.zeros(0, np.int64), np.zeros(0, np.int64)
    L = int(level[r].max()) + 1
    n_l = np.bincount(level[r], minlength=L).astype(np.int64)
    e_l = np.bincount(level[r], weights=deg[r], minlength=L).astype(np.int64)
    return n_l, e_l


def traversed_edges(row_ptr, level) -> int:
    """Graph500 count of traversed (undirected) edges for a symmetric CSR:
    half the summed degree of the reached vertices."""
    deg = np.diff(np.asarray(row_ptr, np.int64))
    return int(deg[np.asarray(level) >= 0].sum() // 2)


# ---------------------------------------------------------------------------
# Fig. 1, step by step
# ---------------------------------------------------------------------------

def start_points_scatter(EdgeSum: np.ndarray, e_l: int, P_l: int, C: int) -> np.ndarray:
    """Find-StartExpPoint as the Analysis section's last paragraph describes:
    for every EdgeSum entry u (inclusive prefix sums of frontier degrees) find
    the range of thread ids t_s..t_e whose start edge t*C falls on one of u's
    edges, and write (u, offset within u's edges) as thread t's start.  Only
    threads with t*C < e_l get a start.  Returns an int64 array (T, 2)."""
    EdgeSum = np.asarray(EdgeSum, np.int64)
    T = min(P_l, -(-e_l // C)) if e_l > 0 else 0
    out = np.full((T, 2), -1, np.int64)
    lo = np.concatenate([[0], EdgeSum[:-1]])           # first edge of entry u
    t_s = -(-lo // C)                                  # ceil(lo / C)
    t_e = -(-EdgeSum // C) - 1                         # ceil(hi / C) - 1
    for u in np.nonzero(t_e >= t_s)[0]:                # non-empty ranges only
        for t in range(int(t_s[u]), int(min(t_e[u], T - 1)) + 1):
            out[t] = (u, t * C - lo[u])
    return out


def start_points_bsearch(ex: np.ndarray, e_l: int, P_l: int, C: int) -> np.ndarray:
    """The same start points found by binary search on the exclusive scan
    ``ex`` (ex[0] = 0, ex[n_l] = e_l): thread t starts in the last entry u
    with ex[u] <= t*C."""
    T = min(P_l, -(-e_l // C)) if e_l > 0 else 0
    starts = np.arange(T, dtype=np.int64) * C
    u = np.searchsorted(np.asarray(ex, np.int64), starts, side="right") - 1
    return np.stack([u, starts - np.asarray(ex, np.int64)[u]], axis=1) if T else np.zeros((0, 2), np.int64)


def s3bfs_fig1(row_ptr, col_idx, s: int, P: int, grain: int = 1, race: str = "max") -> tuple[np.ndarray, list]:
    """Parallel-BFS(s, P) of Fig. 1 with the P_l threads of every step
    simulated.  Returns (d, levels) where ``levels[k]`` describes the k-th pass
    of the main loop (frontier = vertices at distance k).

    ``grain`` is the minimum number of edges per thread: P_l = min(P,
    ceil(e_l / grain)); grain = 1 is Fig. 1's thread count exactly.  Thread i explores edges
    [i*C, min((i+1)*C, e_l)) with C = ceil(e_l / P_l), the near-equal
    division of the Algorithm paragraph.

    EXPLORE-VERTEX's body is not printed; it follows the Algorithm paragraph:
    a thread that meets an unvisited neighbour v sets d[v], claims Owner[v]
    and enqueues v in its private queue Q[i].  A thread sees its own writes.
    ``race`` picks the interleaving of the benign race: "max" lets every
    thread read d before any other thread of the level writes (the most
    duplicate claims a valid execution can produce; the last writer in thread
    order wins Owner), "none" runs threads one after another (no duplicates).
    """
    rp = np.asarray(row_ptr, np.int64)
    ci = np.asarray(col_idx, np.int64)
    n = len(rp) - 1
    Degree = np.diff(rp)
    # initialisation
    d = np.full(n, INF, np.int64)
    Owner = np.full(n, P, np.int64)
    d[s] = 0
    Owner[s] = 0
    CurLevelVertices = np.array([s], np.int64)
    l = 0
    levels = []
    # main loop while the frontier is non-empty
    while len(CurLevelVertices) > 0:
        n_l = len(CurLevelVertices)
        l += 1                                               # next level
        # degree gather; prefix sum (EdgeSum); its last entry e_l
        EdgeSum = np.cumsum(Degree[CurLevelVertices])
        e_l = int(EdgeSum[-1])
        rec = {"n_l": n_l, "e_l": e_l, "frontier": CurLevelVertices.copy()}
        if e_l == 0:
            rec.update(P_l=0, C=0, starts=np.zeros((0, 2), np.int64), candidates=0, undiscovered_edges=0,
                       Sizes=np.zeros(0, np.int64))
            levels.append(rec)
            break
        P_l = min(P, -(-e_l // grain))                       # thread count (grain 1: min(P, e_l))
        C = -(-e_l // P_l)
        # Find-StartExpPoint
        starts = start_points_scatter(EdgeSum, e_l, P_l, C)
        # EXPLORE-VERTEX over every thread's edge segment
        ex = np.concatenate([[0], EdgeSum[:-1]])
        u_idx = np.repeat(np.arange(n_l), Degree[CurLevelVertices])
        u = CurLevelVertices[u_idx]
        e = np.arange(e_l)
        v = ci[rp[u] + (e - ex[u_idx])]
        thread = e // C
        unvisited = d[v] == INF
        if race == "max":
            # every thread reads the level-start d, plus its own writes: its
            # first edge to each unvisited v enqueues v
            cand = np.zeros(e_l, bool)
            idx = np.nonzero(unvisited)[0]
            key = thread[idx] * n + v[idx]
            _, first = np.unique(key, return_index=True)
            cand[idx[first]] = True
        elif race == "none":
            cand = np.zeros(e_l, bool)
            idx = np.nonzero(unvisited)[0]
            _, first = np.unique(v[idx], return_index=True)
            cand[idx[first]] = True
        else:
            raise ValueError(race)
        ce = np.nonzero(cand)[0]
        d[v[ce]] = l
        # Owner[v] <- i by every claiming thread; the last writer in thread
        # order (the largest i) is the one that remains
        Owner[v[ce]] = -1
        np.maximum.at(Owner, v[ce], thread[ce])
        # owner check: each thread keeps the vertices it still owns
        keep = ce[Owner[v[ce]] == thread[ce]]
        Sizes = np.bincount(thread[keep], minlength=P_l)
        # prefix sum of Sizes, then linearisation
        Sizes_incl = np.cumsum(Sizes)
        order = np.argsort(thread[keep], kind="stable")
        CurLevelVertices = v[keep][order]
        assert len(CurLevelVertices) == (Sizes_incl[-1] if P_l else 0)
        rec.update(P_l=P_l, C=C, starts=starts, candidates=int(len(ce)),
                   undiscovered_edges=int(unvisited.sum()), Sizes=Sizes)
        levels.append(rec)
    d[d == INF] = -1
    return d.astype(np.int32), levels
