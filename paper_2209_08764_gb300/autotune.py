"""Autotuner of the traversal options per graph class, with a JSON cache.

The level step has a few knobs whose best values depend on the graph: the
CTA shape (8, 16 or 32 warps), the grain (minimum edges per warp chunk), the
small-level threshold (levels run by one CTA), the persistent grid size, the
renumbering with shared-memory visited bits, and direction-optimising levels.
A deep, thin graph (a mesh) spends its time in thousands of tiny levels and
wants small levels on one CTA; a skewed one (R-MAT) wants the renumbering and
bottom-up levels.  The tuner measures a handful of settings on the graph
itself (device time per traversal, CUDA events inside the library) and keeps
the fastest, by coordinate descent from the defaults: one knob at a time,
each knob's values tried with the others fixed.  Results are cached in a
JSON file under a key that names the graph class (size, mean degree,
skew, depth), so a later graph of the same class starts from the cached
options.

Host-side logic only; every traversal runs through the C ABI.
"""
from __future__ import annotations

import json
import math
import os
import time

import numpy as np

# knob -> values tried (0 = the library default); the order is the order of
# the coordinate descent
SPACE = {
    "cta_warps": [0, 8, 16, 32],
    "small_level_edges": [0, -1, 2048, 8192, 32768],
    "chunk_edges": [0, 32, 128, 512],
    "ctas": [0, -1, -2],      # -1: one CTA per SM, -2: half the SMs (resolved by the caller)
    "relabel": [0, -1, 1],
    "direction": [0, 1],      # tried only on symmetric graphs
    "do_alpha": [0, 5, 10, 30],  # bottom-up switch threshold (0 = 15)
    "do_gamma": [0, -1, 8],      # unvisited-vertex test of the switch (0 = 2, -1 = off)
}


def graph_key(rp, ci, depth: int | None = None) -> str:
    """Class of a graph: log2 of n, mean degree, skew (share of edge endpoints
    at the 2^18 highest-degree vertices) and, when known, a depth bucket."""
    n = len(rp) - 1
    nnz = len(ci)
    deg = np.diff(np.asarray(rp, dtype=np.int64))
    top = np.sort(deg)[::-1][: 1 << 18].sum() if n else 0
    skew = "skewed" if nnz and top >= 0.5 * nnz and n > (1 << 18) else "flat"
    key = f"n2^{round(math.log2(max(n, 1)))}-d{round(nnz / max(n, 1))}-{skew}"
    if depth is not None:
        key += "-" + ("shallow" if depth < 32 else "deep" if depth >= 1024 else "medium")
    return key


class Cache:
    """Best options per graph class, in a JSON file ({key: {"opts", "ms", ...}})."""

    def __init__(self, path: str | None):
        self.path = path
        self.data = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.data = json.load(f)

    def get(self, key):
        e = self.data.get(key)
        return dict(e["opts"]) if e else None

    def put(self, key, opts, ms, trials):
        self.data[key] = {"opts": dict(opts), "ms": ms, "trials": trials, "when": time.strftime("%Y-%m-%d %H:%M:%S")}
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.data, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def coordinate_descent(measure, space=None, start=None):
    """Minimise measure(opts) -> ms over the knob space, one knob at a time.
    Returns (best opts, best ms, trials [(opts, ms), ...]).  A setting whose
    measure raises (e.g. an option the graph does not allow) is skipped."""
    space = SPACE if space is None else space
    best = {k: v[0] for k, v in space.items()}
    if start:
        best.update({k: v for k, v in start.items() if k in space})
    memo = {}
    trials = []

    def run(o):
        key = tuple(sorted(o.items()))
        if key not in memo:
            try:
                memo[key] = float(measure(dict(o)))
            except Exception:  # noqa: BLE001 - an invalid combination is simply not a candidate
                memo[key] = math.inf
            trials.append((dict(o), memo[key]))
        return memo[key]

    best_ms = run(best)
    for knob, values in space.items():
        for v in values:
            if v == best[knob]:
                continue
            cand = dict(best)
            cand[knob] = v
            ms = run(cand)
            if ms < best_ms:
                best, best_ms = cand, ms
    return best, best_ms, trials


def resolve(opts: dict, sms: int) -> dict:
    """Options as bfs_opts fields: ctas = -1 (one CTA per SM) becomes the SM
    count, ctas = -2 half of it.  A high-diameter graph whose levels fill a
    few dozen CTAs at most waits at every grid barrier for all of them, so a
    smaller grid can pay (grid 4096^2: 86.0 against 87.9 ms per traversal
    with 76 CTAs instead of 152)."""
    o = {k: int(v) for k, v in opts.items()}
    if o.get("ctas") == -1:
        o["ctas"] = sms
    elif o.get("ctas") == -2:
        o["ctas"] = max(1, sms // 2)
    return o


def make_measure(B, rp, ci, sources, flags, stream, sms: int, reps: int = 2):
    """measure(opts) -> median device time (ms, init + level loop) of one
    traversal over the sources, after one warm-up pass."""
    import torch
    n = len(rp) - 1

    def measure(o):
        o = resolve(o, sms)
        fl = flags
        if o.get("direction"):
            fl |= B.BFS_SYMMETRIC
        opts = B.bfs_opts(**o)
        g = B.bfs_create_csr(n, len(ci), rp, ci, fl, opts, stream)
        try:
            lv = torch.empty(n, dtype=torch.int32, device="cuda")
            st = B.bfs_stats()
            for s in sources:
                B.bfs_run(g, int(s), lv, None, None)
            ms = []
            for _ in range(reps):
                for s in sources:
                    B.bfs_run(g, int(s), lv, None, st)
                    ms.append(st.ms_total)
            return float(np.median(ms))
        finally:
            B.bfs_destroy(g)
    return measure


def tune(B, rp, ci, sources, cache_path=None, symmetric=True, flags=0, space=None, stream=None, reps=2):
    """Options for this graph: from the cache when its class is there, else
    by coordinate descent (and cached).  Returns (opts, key, info)."""
    import torch
    stream = torch.cuda.current_stream().cuda_stream if stream is None else stream
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    # depth from one default traversal
    n = len(rp) - 1
    g = B.bfs_create_csr(n, len(ci), rp, ci, flags, None, stream)
    st = B.bfs_stats()
    lv = torch.empty(n, dtype=torch.int32, device="cuda")
    B.bfs_run(g, int(sources[0]), lv, None, st)
    B.bfs_destroy(g)
    key = graph_key(rp, ci, st.num_levels)
    cache = Cache(cache_path)
    hit = cache.get(key)
    if hit is not None:
        return hit, key, {"cached": True}
    sp = dict(SPACE if space is None else space)
    if not symmetric:
        sp.pop("direction", None)
        sp.pop("do_alpha", None)
        sp.pop("do_gamma", None)
    best, best_ms, trials = coordinate_descent(make_measure(B, rp, ci, sources, flags, stream, sms, reps), sp)
    cache.put(key, best, best_ms, [[o, ms] for o, ms in trials])
    return best, key, {"cached": False, "ms": best_ms, "trials": len(trials)}
