"""Parity suite run against the range-checked debug build (libs3bfs_checked.so).

Started by test_gpu_checked.py in a process of its own with
S3BFS_LIBRARY=checked, so the binding loads the checked library.  Every
traversal runs with every global index of the level step range-checked (a
failed check would stop it with BFS_E_CHECK); levels must equal the oracle's
bit for bit, parents form a valid tree, and every level's frontier, dumped by
bfs_run_frontiers, must be exactly the set {v : level[v] == l} (Fig. 1:
CurLevelVertices after the owner check and linearisation), with no vertex
twice.  Then an injected out-of-range row start must come back as BFS_E_CHECK,
with the handle still usable.
"""
import ctypes
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))
sys.path.insert(0, HERE)

import numpy as np  # noqa: E402

import graphgen  # noqa: E402
import oracle  # noqa: E402
from gpu_helpers import Dev, check_against_oracle, make_opts  # noqa: E402
from paper_2209_08764_gb300 import _build  # noqa: E402
from paper_2209_08764_gb300 import binding as B  # noqa: E402


def frontier_sets(d, src, want):
    """Dump every level's frontier and compare it, as a set, with the oracle's."""
    n = d.n
    cap = 1 << 16
    buf = (ctypes.c_int32 * (cap * B.BFS_LEVEL_FIELDS))()
    st = B.bfs_stats()
    st.per_level = ctypes.cast(buf, ctypes.POINTER(ctypes.c_int32))
    st.per_level_cap = cap
    dump = np.full(n, -7, np.int32)
    B.bfs_run_frontiers(d.g, int(src), d.level, d.parent, st, dump)
    lv = d.level.cpu().numpy()
    assert np.array_equal(lv, want), "levels differ from the oracle (frontier dump run)"
    L = st.num_levels
    n_l = np.frombuffer(buf, dtype=np.int32)[:L * B.BFS_LEVEL_FIELDS].reshape(L, B.BFS_LEVEL_FIELDS)[:, 0]
    assert int(n_l.sum()) == st.reached == int((want >= 0).sum())
    off = 0
    for l in range(L):
        F = dump[off:off + n_l[l]]
        off += n_l[l]
        assert len(np.unique(F)) == len(F), f"level {l}: a vertex appears twice in the frontier"
        assert np.array_equal(np.sort(F), np.nonzero(want == l)[0]), f"level {l}: frontier set differs"
    assert np.all(dump[off:] == -7), "dump wrote past the reached vertices"


def main():
    assert B.library_path() == _build.LIB_CHECKED, "run with S3BFS_LIBRARY=checked"
    B.load()
    cases = [("rmat16", graphgen.rmat(16, 16, seed=1), {}, 6),
             ("rmat16 not renumbered", graphgen.rmat(16, 16, seed=1), {"relabel": -1}, 3),
             ("rmat16 8-warp CTAs, no small levels", graphgen.rmat(16, 16, seed=1),
              {"cta_warps": 8, "small_level_edges": -1}, 3),
             ("rmat16 per phase", graphgen.rmat(16, 16, seed=1), {"persistent": -1}, 2),
             ("rmat16 direction-optimising", graphgen.rmat(16, 16, seed=1), {"direction": 1}, 3),
             ("grid 200x300", graphgen.grid(200, 300, 0.01, seed=3), {}, 2),
             ("er 2^15", graphgen.erdos_renyi(1 << 15, 1 << 18, seed=4), {}, 2)]
    for name, (rp, ci), opts, k in cases:
        d = Dev(rp, ci, flags=B.BFS_VALIDATE | B.BFS_SYMMETRIC, **opts)
        orc = oracle.Oracle(rp, ci)
        keys = oracle.edge_keys(rp, ci)
        for s in graphgen.sample_sources(rp, k, seed=2):
            want, _ = orc.bfs(int(s))
            check_against_oracle(d, int(s), orc=orc, keys=keys)
            frontier_sets(d, int(s), want)
        d.close()
        print("checked:", name, "ok", flush=True)
    # a failed check is an error code, not a fault, and the context survives
    import torch
    rp, ci = graphgen.rmat(12, 16, seed=1)
    n = len(rp) - 1
    stream = torch.cuda.current_stream().cuda_stream
    g = B.bfs_create_csr(n, len(ci), rp, ci, B.BFS_VALIDATE, make_opts(debug_flags=B.BFS_DEBUG_CHECK_INJECT), stream)
    lv = torch.empty(n, dtype=torch.int32, device="cuda")
    src = int(graphgen.sample_sources(rp, 1, seed=3)[0])
    try:
        B.bfs_run(g, src, lv, None, None)
        raise AssertionError("the injected out-of-range row start was not caught")
    except B.BFSError as e:
        assert e.code == B.BFS_E_CHECK and "range check 13" in str(e), str(e)
    B.bfs_destroy(g)
    d = Dev(rp, ci)
    check_against_oracle(d, src)
    d.close()
    print("checked: injected range violation -> BFS_E_CHECK ok", flush=True)


if __name__ == "__main__":
    main()
