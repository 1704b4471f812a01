"""Shared helpers for the GPU parity tests (imported by tests only)."""
import ctypes

import numpy as np

import oracle
from paper_2209_08764_gb300 import binding as B


def make_opts(**kw):
    o = B.bfs_opts()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Dev:
    """A graph on the GPU through the C ABI, with torch output buffers."""

    def __init__(self, rp, ci, flags=B.BFS_VALIDATE, **opts):
        import torch
        sl = opts.get("small_level_edges", 0)
        self._small_opt = sl
        self.persistent = opts.get("persistent", 0) >= 0
        # direction-optimising levels (persistent loop only)
        self.direction = opts.get("direction", 0) if self.persistent else 0
        self.alpha = opts.get("do_alpha", 0) or 15
        self.beta = opts.get("do_beta", 0) or 18
        g = opts.get("do_gamma", 0)
        self.gamma = 2 if g == 0 else (0 if g == -1 else g)
        self.torch = torch
        self.rp = np.ascontiguousarray(rp, np.int32)
        self.ci = np.ascontiguousarray(ci, np.int32)
        self.n = len(self.rp) - 1
        self.n_live = int((np.diff(self.rp) > 0).sum())
        self.g = B.bfs_create_csr(self.n, len(self.ci), self.rp, self.ci if len(self.ci) else None, flags,
                                  make_opts(**opts) if opts else None, torch.cuda.current_stream().cuda_stream)
        self.info = B.bfs_graph_info(self.g)
        # levels with at most this many edges run on one CTA (small-level mode)
        wpc = self.info["warps"] // self.info["ctas"]
        self.small = 256 * wpc if self._small_opt == 0 else (0 if self._small_opt < 0 else self._small_opt)
        if opts.get("work_insensitive"):
            self.small = 0          # every level on the whole grid
        self.level = torch.empty(self.n, dtype=torch.int32, device="cuda")
        self.parent = torch.empty(self.n, dtype=torch.int32, device="cuda")

    def run(self, src, per_level_cap=0):
        st = B.bfs_stats()
        buf = None
        if per_level_cap:
            buf = (ctypes.c_int32 * (per_level_cap * B.BFS_LEVEL_FIELDS))()
            st.per_level = ctypes.cast(buf, ctypes.POINTER(ctypes.c_int32))
            st.per_level_cap = per_level_cap
        B.bfs_run(self.g, int(src), self.level, self.parent, st)
        lv = self.level.cpu().numpy()
        par = self.parent.cpu().numpy()
        pl = None
        if buf is not None:
            L = min(st.num_levels, per_level_cap)
            pl = np.frombuffer(buf, dtype=np.int32)[:L * B.BFS_LEVEL_FIELDS].reshape(L, B.BFS_LEVEL_FIELDS).copy()
        return lv, par, st, pl

    def close(self):
        B.bfs_destroy(self.g)
        self.g = None


def expected_directions(n, nnz, n_l, e_l, direction, alpha, beta, gamma=0, n_live=0):
    """Direction of every level (0 top-down, 1 bottom-up) by the switching
    rule of a direction-optimising traversal (Beamer et al., SC 2012), from
    the oracle's level profile: with m_u = nnz - (e summed over the levels up
    to the next one), turn bottom-up when the next frontier's edges exceed
    m_u / alpha and gamma times the unvisited vertices of degree > 0 (n_live
    minus the vertices of the levels up to the next one); turn back when the
    frontier shrinks below n / beta."""
    d = [0]
    cum = int(e_l[0])
    vcum = int(n_l[0])
    for l in range(len(n_l) - 1):
        n_next, e_next = int(n_l[l + 1]), int(e_l[l + 1])
        cum += e_next
        vcum += n_next
        if not direction or n_next <= 0:
            nd = 0
        elif d[-1] == 0:
            nd = 1 if (e_next * alpha > nnz - cum and e_next > gamma * (n_live - vcum)) else 0
        else:
            nd = 0 if (n_next * beta < n and n_next < int(n_l[l])) else 1
        d.append(nd)
    return np.array(d, np.int64)


def check_against_oracle(dev, src, orc=None, keys=None, per_level=True, grain=64):
    """Levels bit-exact, parents a valid BFS tree, per-level statistics
    consistent with the oracle's level profile."""
    orc = orc or oracle.Oracle(dev.rp, dev.ci)
    want, _ = orc.bfs(src)
    cap = 1 << 16
    lv, par, st, pl = dev.run(src, per_level_cap=cap if per_level else 0)
    bad = np.nonzero(lv != want)[0]
    assert len(bad) == 0, f"src {src}: {len(bad)} levels differ, first v={bad[0]} got {lv[bad[0]]} want {want[bad[0]]}"
    oracle.check_bfs_tree(dev.rp, dev.ci, src, lv, par, keys=keys)
    n_l, e_l = oracle.level_profile(dev.rp, want)
    assert st.num_levels == len(n_l)
    assert st.reached == int(n_l.sum())
    assert st.edges_scanned == int(e_l.sum())
    # the GTEPS numerator: the library's count equals the pinned oracle count
    assert st.edges_scanned // 2 == oracle.traversed_edges(dev.rp, want)
    dirs = expected_directions(dev.n, len(dev.ci), n_l, e_l, dev.direction, dev.alpha, dev.beta, dev.gamma,
                               dev.n_live)
    bu = dirs == 1
    if not bu.any():
        assert st.work_edges == st.edges_scanned
    if per_level and pl is not None:
        L = min(len(n_l), cap)
        assert np.array_equal(pl[:L, 0], n_l[:L]), "per-level n_l"
        assert np.array_equal(pl[:L, 1], e_l[:L]), "per-level e_l"
        assert np.array_equal(pl[:L, 7], dirs[:L]), "per-level direction"
        # work: e_l top-down; bottom-up at least one entry per vertex found
        # and at most the degree sum of the unvisited vertices
        td = ~bu[:L]
        assert np.array_equal(pl[:L, 8][td], e_l[:L][td]), "top-down work != e_l"
        nxt_all = np.append(n_l[1:], 0)
        unvisited_deg = len(dev.ci) - np.cumsum(e_l)
        assert np.all(pl[:L, 8][~td] >= nxt_all[:L][~td]), "bottom-up work below the vertices found"
        assert np.all(pl[:L, 8][~td] <= unvisited_deg[:L][~td]), "bottom-up work above the unvisited degree sum"
        assert st.work_edges == int(pl[:L, 8].sum()) or L < len(n_l)
        # candidates: at least the vertices found, at most the edges into the next level
        nxt = np.append(n_l[1:], 0)[:L]
        rows = np.repeat(np.arange(dev.n), np.diff(dev.rp))
        into = (want[rows] >= 0) & (want[dev.ci] == want[rows] + 1)
        e_next = np.bincount(want[rows][into], minlength=len(n_l))[:L]
        assert np.all(pl[:L, 2] >= nxt) and np.all(pl[:L, 2] <= e_next), "candidates out of bounds"
        # a bottom-up level finds every new vertex exactly once
        assert np.array_equal(pl[:L, 2][bu[:L]], nxt[bu[:L]]), "bottom-up candidates != next frontier"
        assert st.candidates == int(pl[:, 2].sum()) or L < len(n_l)
        P = dev.info["warps"]
        W = P // dev.info["ctas"]
        small = (e_l[:L] <= dev.small) & dev.persistent & ~bu[:L]
        want_P = np.where(e_l[:L] > 0, np.minimum(np.where(small, W, P), -(-e_l[:L] // grain)), 0)
        want_P = np.where(bu[:L], P, want_P)
        if "wi" not in dev.__dict__:
            assert np.array_equal(pl[:L, 3], want_P), "active warps != min(P, ceil(e_l/grain))"
    return lv, par, st, pl
