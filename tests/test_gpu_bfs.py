"""CUDA path vs the CPU oracle, through the C ABI (GPU only).

Levels must match the oracle bit for bit; parents must form a valid BFS tree
(the tree itself depends on which writer wins the benign race); per-level
frontier sizes and edge counts must equal the oracle's level profile; the
number of active warps per level must be min(P, ceil(e_l / grain)).
"""
import itertools

import numpy as np
import pytest

import graphgen
import oracle
from gpu_helpers import Dev, check_against_oracle, make_opts
from paper_2209_08764_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2209_08764_gb300 as pkg
    pkg.build()
    B.load()
    yield
    torch.cuda.synchronize()


def _named_graphs():
    g = {}
    g["path33"] = graphgen.from_edges(33, [(i, i + 1) for i in range(32)])
    g["cycle20"] = graphgen.from_edges(20, [(i, (i + 1) % 20) for i in range(20)])
    g["star5000"] = graphgen.from_edges(5001, [(0, j) for j in range(1, 5001)])  # hub degree >> chunk
    g["K40"] = graphgen.from_edges(40, list(itertools.combinations(range(40), 2)))
    g["K7_9"] = graphgen.from_edges(16, [(i, 7 + j) for i in range(7) for j in range(9)])
    g["grid45x77"] = graphgen.grid(45, 77, 0.0)
    g["tree"] = graphgen.from_edges(1023, [(i, c) for i in range(1023) for c in (2 * i + 1, 2 * i + 2) if c < 1023])
    g["two_paths"] = graphgen.from_edges(9, [(0, 1), (1, 2), (2, 3), (4, 5), (5, 6), (6, 7), (7, 8)])
    g["single"] = (np.array([0, 0], np.int32), np.zeros(0, np.int32))
    g["isolated_src"] = graphgen.from_edges(4, [(1, 2), (2, 3)])
    return g


@pytest.mark.parametrize("relabel", [0, 1, -1])
@pytest.mark.parametrize("name", sorted(_named_graphs()))
def test_named_graphs(name, relabel):
    rp, ci = _named_graphs()[name]
    d = Dev(rp, ci, relabel=relabel) if relabel else Dev(rp, ci)
    try:
        n = len(rp) - 1
        srcs = sorted({0, n // 2, n - 1})
        for s in srcs:
            check_against_oracle(d, s)
    finally:
        d.close()


def _directed_csr(n, edges):
    edges = sorted(set(edges))
    rp = np.zeros(n + 1, np.int64)
    for u, _ in edges:
        rp[u + 1] += 1
    return np.cumsum(rp).astype(np.int32), np.array([v for _, v in edges], np.int32)


@pytest.mark.parametrize("relabel", [0, 1])
def test_directed_with_zero_outdegree_frontier(relabel):
    rng = np.random.default_rng(5)
    n = 3000
    e = [(int(a), int(b)) for a, b in rng.integers(0, n, size=(9000, 2)) if a != b]
    e += [(0, v) for v in range(1, 200)]           # a hub whose neighbours mostly have out-degree 0
    rp, ci = _directed_csr(n, e)
    d = Dev(rp, ci, relabel=relabel) if relabel else Dev(rp, ci)
    try:
        for s in (0, 1, 17, 2999):
            check_against_oracle(d, s)
    finally:
        d.close()


@pytest.fixture(scope="module")
def rmat16():
    rp, ci = graphgen.rmat_s16()
    return rp, ci, graphgen.sample_sources(rp, 64, seed=2), oracle.edge_keys(rp, ci)


def test_rmat16_64_sources(rmat16):
    rp, ci, srcs, keys = rmat16
    d = Dev(rp, ci)
    orc = oracle.Oracle(rp, ci)
    try:
        for s in srcs:
            check_against_oracle(d, int(s), orc=orc, keys=keys)
    finally:
        d.close()


@pytest.mark.parametrize("opts", [
    dict(chunk_edges=1), dict(chunk_edges=2), dict(chunk_edges=3), dict(chunk_edges=31), dict(chunk_edges=32),
    dict(chunk_edges=33), dict(chunk_edges=4096), dict(ctas=1), dict(ctas=3), dict(ctas=5, chunk_edges=7),
    dict(persistent=-1), dict(persistent=-1, chunk_edges=5), dict(work_insensitive=1),
    dict(work_insensitive=1, ctas=2), dict(relabel=1), dict(relabel=-1), dict(relabel=1, chunk_edges=1, ctas=7),
    dict(relabel=1, persistent=-1), dict(relabel=1, work_insensitive=1),
    dict(small_level_edges=-1), dict(small_level_edges=1 << 22), dict(small_level_edges=3000),
    dict(small_level_edges=1 << 22, relabel=1), dict(small_level_edges=-1, relabel=-1),
    dict(cta_warps=8), dict(cta_warps=8, ctas=3), dict(cta_warps=8, small_level_edges=-1),
    dict(cta_warps=8, persistent=-1), dict(cta_warps=32, relabel=-1), dict(cta_warps=8, relabel=1),
    dict(cta_warps=16), dict(cta_warps=24), dict(cta_warps=16, relabel=-1, ctas=5),
    dict(cta_warps=24, persistent=-1), dict(cta_warps=16, small_level_edges=-1),
], ids=lambda o: ",".join(f"{k}={v}" for k, v in o.items()))
def test_rmat16_launch_configurations(rmat16, opts):
    rp, ci, srcs, keys = rmat16
    d = Dev(rp, ci, **opts)
    if opts.get("work_insensitive"):
        d.wi = True
    orc = oracle.Oracle(rp, ci)
    try:
        for s in srcs[:6]:
            check_against_oracle(d, int(s), orc=orc, keys=keys, grain=opts.get("chunk_edges", 64))
    finally:
        d.close()


def test_work_insensitive_uses_every_warp(rmat16):
    rp, ci, srcs, _ = rmat16
    d = Dev(rp, ci, work_insensitive=1)
    try:
        _, _, st, pl = d.run(int(srcs[0]), per_level_cap=64)
        P = d.info["warps"]
        assert np.all(pl[pl[:, 1] > 0, 3] == P), "a level left warps idle"
    finally:
        d.close()


def test_repeated_runs_race_stress(rmat16):
    """The owner race is benign: 50 runs give identical levels; parents may
    differ between runs but are always valid."""
    rp, ci, srcs, keys = rmat16
    d = Dev(rp, ci, chunk_edges=3)
    try:
        s = int(srcs[1])
        want, _ = oracle.bfs(rp, ci, s)
        parents = set()
        for _ in range(50):
            lv, par, _, _ = d.run(s)
            assert np.array_equal(lv, want)
            oracle.check_bfs_tree(rp, ci, s, lv, par, keys=keys)
            parents.add(hash(par.tobytes()))
    finally:
        d.close()


@pytest.mark.parametrize("relabel", [0, 1])
def test_host_outputs_and_no_parent(rmat16, relabel):
    rp, ci, srcs, keys = rmat16
    d = Dev(rp, ci, relabel=relabel) if relabel else Dev(rp, ci)
    try:
        s = int(srcs[2])
        want, _ = oracle.bfs(rp, ci, s)
        lv = np.empty(d.n, np.int32)
        par = np.empty(d.n, np.int32)
        B.bfs_run(d.g, s, lv, par, None)
        assert np.array_equal(lv, want)
        oracle.check_bfs_tree(rp, ci, s, lv, par, keys=keys)
        lv2 = np.full(d.n, 7, np.int32)
        B.bfs_run(d.g, s, lv2, None, None)
        assert np.array_equal(lv2, want)
        d.level.fill_(5)
        B.bfs_run(d.g, s, d.level, None, None)
        assert np.array_equal(d.level.cpu().numpy(), want)
    finally:
        d.close()


@pytest.mark.parametrize("relabel", [0, 1])
def test_unaligned_device_outputs(rmat16, relabel):
    import torch
    rp, ci, srcs, keys = rmat16
    d = Dev(rp, ci, relabel=relabel) if relabel else Dev(rp, ci)
    try:
        s = int(srcs[3])
        want, _ = oracle.bfs(rp, ci, s)
        big = torch.empty(2 * d.n + 8, dtype=torch.int32, device="cuda")
        lv, par = big[1:1 + d.n], big[d.n + 3:2 * d.n + 3]
        B.bfs_run(d.g, s, lv, par, None)
        assert np.array_equal(lv.cpu().numpy(), want)
        oracle.check_bfs_tree(rp, ci, s, lv.cpu().numpy(), par.cpu().numpy(), keys=keys)
    finally:
        d.close()


@pytest.mark.parametrize("relabel", [0, 1])
def test_run_batch_matches_single_runs(rmat16, relabel):
    import torch
    rp, ci, srcs, keys = rmat16
    d = Dev(rp, ci, relabel=relabel) if relabel else Dev(rp, ci)
    try:
        k = 16
        S = np.ascontiguousarray(srcs[:k])
        L = torch.empty(k * d.n, dtype=torch.int32, device="cuda")
        P = torch.empty(k * d.n, dtype=torch.int32, device="cuda")
        B.bfs_run_batch(d.g, S, k, L, P, None)
        L = L.cpu().numpy().reshape(k, d.n)
        P = P.cpu().numpy().reshape(k, d.n)
        orc = oracle.Oracle(rp, ci)
        for i, s in enumerate(S):
            want, _ = orc.bfs(int(s))
            assert np.array_equal(L[i], want)
            oracle.check_bfs_tree(rp, ci, int(s), L[i], P[i], keys=keys)
        # host outputs, per-run stats
        Lh = np.empty((4, d.n), np.int32)
        st = (B.bfs_stats * 4)()
        B.bfs_run_batch(d.g, S[:4], 4, Lh, None, st)
        for i in range(4):
            want, _ = orc.bfs(int(S[i]))
            assert np.array_equal(Lh[i], want)
            assert st[i].reached == int((want >= 0).sum())
    finally:
        d.close()


@pytest.mark.parametrize("relabel", [-1, 1])
@pytest.mark.parametrize("where", ["pinned", "pageable", "device"])
@pytest.mark.parametrize("parents", [True, False])
def test_run_batch_queued_back_to_back(rmat16, relabel, where, parents):
    """A batch of single-source traversals queued back to back (the host
    checks traversal i - 1 while traversal i runs); host outputs are copied
    from two staging slots on a second stream while the next traversal runs.
    Every source's levels equal the oracle's, its parents form a BFS tree, and
    its stats are its own."""
    import torch
    rp, ci, srcs, keys = rmat16
    d = Dev(rp, ci, relabel=relabel)
    try:
        k = 7  # odd: both slots, the last one used once more
        S = np.ascontiguousarray(srcs[:k])
        if where == "pinned":
            L = torch.full((k * d.n,), -7, dtype=torch.int32, pin_memory=True)
            P = torch.full((k * d.n,), -7, dtype=torch.int32, pin_memory=True) if parents else None
        elif where == "device":
            L = torch.full((k * d.n,), -7, dtype=torch.int32, device="cuda")
            P = torch.full((k * d.n,), -7, dtype=torch.int32, device="cuda") if parents else None
        else:
            L = np.full(k * d.n, -7, np.int32)
            P = np.full(k * d.n, -7, np.int32) if parents else None
        st = (B.bfs_stats * k)()
        B.bfs_run_batch(d.g, S, k, L, P, st)
        if where == "device":
            L, P = L.cpu(), (P.cpu() if parents else None)
        L = np.asarray(L).reshape(k, d.n)
        orc = oracle.Oracle(rp, ci)
        for i, s in enumerate(S):
            want, _ = orc.bfs(int(s))
            assert np.array_equal(L[i], want), f"source {i}"
            if parents:
                oracle.check_bfs_tree(rp, ci, int(s), L[i], np.asarray(P).reshape(k, d.n)[i], keys=keys)
            n_l, e_l = oracle.level_profile(rp, want)
            assert st[i].reached == int(n_l.sum()) and st[i].num_levels == len(n_l)
            assert st[i].edges_scanned == int(e_l.sum())
            assert 0 < st[i].ms_level_step <= st[i].ms_total
            assert st[i].launches >= 2
        # the same handle then serves single runs and a batch without stats
        check_against_oracle(d, int(S[0]))
        Lh = np.empty((2, d.n), np.int32)
        B.bfs_run_batch(d.g, S[:2], 2, Lh, None, None)
        assert np.array_equal(Lh[1], orc.bfs(int(S[1]))[0])
    finally:
        d.close()


def test_run_batch_host_outputs_timeout_names_the_source():
    """An overlapped batch whose traversals time out (test hook: a CTA never
    arrives at the first barrier): the error and the failing source index
    come back, nothing stays in flight, and a new handle works."""
    rp, ci = graphgen.rmat(10, 16, seed=1)
    S = np.ascontiguousarray(graphgen.sample_sources(rp, 3), np.int32)
    d = Dev(rp, ci, debug_flags=B.BFS_DEBUG_STALL_BARRIER, spin_limit_ms=200, ctas=4)
    try:
        L = np.empty(3 * d.n, np.int32)
        with pytest.raises(B.BFSError) as e:
            B.bfs_run_batch(d.g, S, 3, L, None, None)
        assert e.value.code == B.BFS_E_TIMEOUT
        assert "source index 0" in B.bfs_last_error()
    finally:
        d.close()
    d = Dev(rp, ci)
    try:
        L = np.empty(3 * d.n, np.int32)
        B.bfs_run_batch(d.g, S, 3, L, None, None)
        for i, s in enumerate(S):
            assert np.array_equal(L[i * d.n:(i + 1) * d.n], oracle.bfs(rp, ci, int(s))[0])
    finally:
        d.close()


@pytest.mark.parametrize("small", [-1, 0, 1 << 20])
@pytest.mark.parametrize("cw", [8, 16, 32])
def test_long_path_and_grid_small_level_mode(small, cw):
    """Thousands of tiny levels: CTA 0 alone runs them (small-level mode), or
    the whole grid with two grid barriers per level (small = -1)."""
    n = 20000
    rp, ci = graphgen.from_edges(n, [(i, i + 1) for i in range(n - 1)])
    d = Dev(rp, ci, small_level_edges=small, cta_warps=cw)
    try:
        lv, _, st, _ = check_against_oracle(d, 0)
        assert st.num_levels == n
        check_against_oracle(d, n // 3)
    finally:
        d.close()
    rp, ci = graphgen.grid(300, 200, 0.05, seed=7)
    d = Dev(rp, ci, small_level_edges=small, cta_warps=cw)
    try:
        check_against_oracle(d, 0)
        check_against_oracle(d, 30000)
    finally:
        d.close()


def test_er_and_grid_small():
    for rp, ci in (graphgen.erdos_renyi(1 << 14, 1 << 17, seed=4), graphgen.grid(128, 128, 0.01, seed=3)):
        d = Dev(rp, ci)
        orc = oracle.Oracle(rp, ci)
        try:
            for s in graphgen.sample_sources(rp, 4, seed=2):
                check_against_oracle(d, int(s), orc=orc)
            check_against_oracle(d, 0, orc=orc)
        finally:
            d.close()


# ---------------------------------------------------------------------------
# errors (all raised on the host or by a bounded device wait)
# ---------------------------------------------------------------------------

def test_bad_source_and_bad_csr():
    rp, ci = graphgen.from_edges(10, [(i, i + 1) for i in range(9)])
    d = Dev(rp, ci)
    try:
        with pytest.raises(B.BFSError) as e:
            B.bfs_run(d.g, 10, d.level, None, None)
        assert e.value.code == B.BFS_E_INVAL
        with pytest.raises(B.BFSError) as e:
            B.bfs_run(d.g, -1, d.level, None, None)
        assert e.value.code == B.BFS_E_INVAL
        check_against_oracle(d, 3)          # still usable
    finally:
        d.close()
    bad = ci.copy()
    bad[3] = 10
    for flags in (0, B.BFS_VALIDATE):
        with pytest.raises(B.BFSError) as e:
            B.bfs_create_csr(10, len(bad), rp, bad, flags)
        assert e.value.code == B.BFS_E_INVAL
    rp2 = rp.copy()
    rp2[4], rp2[5] = rp2[5], rp2[4]
    with pytest.raises(B.BFSError) as e:
        B.bfs_create_csr(10, len(ci), rp2, ci, 0)
    assert e.value.code == B.BFS_E_INVAL
    with pytest.raises(B.BFSError) as e:
        B.bfs_create_csr(0, 0, np.zeros(1, np.int32), None, 0)
    assert e.value.code == B.BFS_E_INVAL


def test_device_memory_cap_gives_nomem():
    """bfs_opts.max_device_bytes: create-time buffers beyond the cap fail with
    BFS_E_NOMEM; a cap that exactly fits them works, and a later first-use
    allocation beyond it (the bitmask-batch buffers) fails the same way while
    the graph stays usable."""
    import torch
    rp, ci = graphgen.rmat(12, 16, seed=3)
    n = len(rp) - 1
    stream = torch.cuda.current_stream().cuda_stream
    flags = B.BFS_VALIDATE | B.BFS_SYMMETRIC
    g = B.bfs_create_csr(n, len(ci), rp, ci, flags, None, stream)
    need = B.bfs_graph_device_bytes(g)
    B.bfs_destroy(g)
    assert need > 8 * n
    with pytest.raises(B.BFSError) as e:
        B.bfs_create_csr(n, len(ci), rp, ci, flags, make_opts(max_device_bytes=need - 1), stream)
    assert e.value.code == B.BFS_E_NOMEM and "max_device_bytes" in str(e.value)
    g = B.bfs_create_csr(n, len(ci), rp, ci, flags, make_opts(max_device_bytes=need), stream)
    try:
        assert B.bfs_graph_device_bytes(g) == need
        srcs = np.ascontiguousarray(graphgen.sample_sources(rp, 4, seed=1), np.int32)
        L = torch.empty(len(srcs) * n, dtype=torch.int32, device="cuda")
        with pytest.raises(B.BFSError) as e:
            B.bfs_run_batch(g, srcs, len(srcs), L, None, None)
        assert e.value.code == B.BFS_E_NOMEM
        assert B.bfs_graph_device_bytes(g) <= need
        lv = torch.empty(n, dtype=torch.int32, device="cuda")
        B.bfs_run(g, int(srcs[0]), lv, None, None)          # still usable
        assert np.array_equal(lv.cpu().numpy(), oracle.bfs(rp, ci, int(srcs[0]))[0])
    finally:
        B.bfs_destroy(g)
    with pytest.raises(B.BFSError) as e:
        B.bfs_create_csr(n, len(ci), rp, ci, flags, make_opts(max_device_bytes=-5), stream)
    assert e.value.code == B.BFS_E_INVAL


def test_multigraph_rejected_or_deduplicated():
    rp = np.array([0, 3, 5, 6, 7], np.int32)      # row 0 lists 1 twice, row 1 has a self-loop
    ci = np.array([1, 2, 1, 0, 1, 0, 1], np.int32)
    with pytest.raises(B.BFSError) as e:
        B.bfs_create_csr(4, 7, rp, ci, B.BFS_VALIDATE)
    assert e.value.code == B.BFS_E_MULTIGRAPH
    d = Dev(rp, ci, flags=B.BFS_DEDUP)
    try:
        lv, par, st, _ = d.run(0)
        assert lv.tolist() == [0, 1, 1, -1]     # 3 -> 1 only: vertex 3 is not reachable
        lv, par, st, _ = d.run(3)
        assert lv.tolist() == [2, 1, 3, 0]
    finally:
        d.close()


@pytest.mark.parametrize("relabel", [0, 1, -1])
def test_device_pointer_input(relabel):
    import torch
    rp, ci = graphgen.rmat(12, 16, seed=3)
    drp = torch.from_numpy(rp).cuda()
    dci = torch.from_numpy(ci).cuda()
    g = B.bfs_create_csr(len(rp) - 1, len(ci), drp, dci, B.BFS_DEVICE_PTRS,
                         make_opts(relabel=relabel), torch.cuda.current_stream().cuda_stream)
    try:
        del drp, dci
        torch.cuda.synchronize()
        lv = torch.empty(len(rp) - 1, dtype=torch.int32, device="cuda")
        s = int(graphgen.sample_sources(rp, 1)[0])
        B.bfs_run(g, s, lv, None, None)
        want, _ = oracle.bfs(rp, ci, s)
        assert np.array_equal(lv.cpu().numpy(), want)
    finally:
        B.bfs_destroy(g)


def test_barrier_wait_limit_reports_timeout():
    """A CTA that never arrives at the first grid barrier (test hook): the
    bounded wait expires, the kernel returns, bfs_run reports BFS_E_TIMEOUT,
    and the graph and the context stay usable."""
    rp, ci = graphgen.rmat(10, 16, seed=1)
    s = int(graphgen.sample_sources(rp, 1)[0])
    d = Dev(rp, ci, debug_flags=B.BFS_DEBUG_STALL_BARRIER, spin_limit_ms=200, ctas=4)
    try:
        with pytest.raises(B.BFSError) as e:
            B.bfs_run(d.g, s, d.level, d.parent, None)
        assert e.value.code == B.BFS_E_TIMEOUT
    finally:
        d.close()
    d = Dev(rp, ci)
    try:
        check_against_oracle(d, s)
    finally:
        d.close()


# ---------------------------------------------------------------------------
# multi-source batches with bitmask frontiers (BFS_SYMMETRIC graphs)
# ---------------------------------------------------------------------------

def _batch_check(rp, ci, srcs, flags, host=False, parents=True, **opts):
    import torch
    n = len(rp) - 1
    k = len(srcs)
    g = B.bfs_create_csr(n, len(ci), rp, ci, flags, make_opts(**opts) if opts else None,
                         torch.cuda.current_stream().cuda_stream)
    try:
        S = np.ascontiguousarray(srcs, np.int32)
        if host:
            L = np.empty(k * n, np.int32)
            P = np.empty(k * n, np.int32) if parents else None
        else:
            L = torch.empty(k * n, dtype=torch.int32, device="cuda")
            P = torch.empty(k * n, dtype=torch.int32, device="cuda") if parents else None
        st = (B.bfs_stats * k)()
        B.bfs_run_batch(g, S, k, L, P, st)
        L = (L if host else L.cpu().numpy()).reshape(k, n)
        if parents:
            P = (P if host else P.cpu().numpy()).reshape(k, n)
        orc = oracle.Oracle(rp, ci)
        keys = oracle.edge_keys(rp, ci)
        for i, s in enumerate(S):
            want, _ = orc.bfs(int(s))
            assert np.array_equal(L[i], want), f"source {i} ({s}): levels differ"
            if parents:
                oracle.check_bfs_tree(rp, ci, int(s), L[i], P[i], keys=keys)
            n_l, e_l = oracle.level_profile(rp, want)
            assert st[i].reached == int(n_l.sum())
            assert st[i].edges_scanned == int(e_l.sum())
            assert st[i].num_levels == len(n_l)
    finally:
        B.bfs_destroy(g)


@pytest.mark.parametrize("k", [2, 3, 64, 65, 130])
def test_batch_bitmask_rmat16(rmat16, k):
    rp, ci, srcs, _ = rmat16
    S = np.resize(srcs, k)                      # k > 64 repeats sources: duplicates are allowed
    _batch_check(rp, ci, S, B.BFS_VALIDATE | B.BFS_SYMMETRIC)


@pytest.mark.parametrize("variant", ["host", "noparent", "relabel", "host_relabel"])
def test_batch_bitmask_variants(rmat16, variant):
    rp, ci, srcs, _ = rmat16
    kw = {}
    if "relabel" in variant:
        kw["relabel"] = 1
    _batch_check(rp, ci, srcs[:40], B.BFS_VALIDATE | B.BFS_SYMMETRIC, host="host" in variant,
                 parents=variant != "noparent", **kw)


def test_batch_bitmask_er_and_grid():
    for rp, ci in (graphgen.erdos_renyi(1 << 15, 1 << 18, seed=4), graphgen.grid(64, 80, 0.02, seed=3)):
        srcs = graphgen.sample_sources(rp, 64, seed=2)
        _batch_check(rp, ci, srcs, B.BFS_VALIDATE | B.BFS_SYMMETRIC)


@pytest.mark.parametrize("direction", [0, 1])
def test_isolated_vertices_on_renumbered_graph(direction):
    """A symmetric graph renumbered by degree puts its isolated vertices last;
    a traversal then clears and reads only the others' level entries.  Sources
    that are isolated (level 0 alone, its own parent) and ordinary ones, in
    single runs and in a queued batch, must equal the oracle, also after runs
    that left the untouched tail alone."""
    import torch
    rp0, ci0 = graphgen.rmat(12, 8, seed=4)
    n = len(rp0) - 1
    deg = np.diff(rp0)
    iso = np.nonzero(deg == 0)[0]
    assert len(iso) > 10
    d = Dev(rp0, ci0, flags=B.BFS_VALIDATE | B.BFS_SYMMETRIC, relabel=1, direction=direction, batch_bitmask=-1)
    orc = oracle.Oracle(rp0, ci0)
    try:
        live = graphgen.sample_sources(rp0, 3, seed=9)
        order = [int(iso[0]), int(live[0]), int(iso[-1]), int(live[1]), int(iso[len(iso) // 2]), int(live[2])]
        for s in order:
            check_against_oracle(d, s, orc=orc)
        S = np.ascontiguousarray(order, np.int32)
        L = torch.full((len(S) * n,), 77, dtype=torch.int32, device="cuda")
        P = torch.full((len(S) * n,), 77, dtype=torch.int32, device="cuda")
        B.bfs_run_batch(d.g, S, len(S), L, P, None)
        L, P = L.cpu().numpy().reshape(len(S), n), P.cpu().numpy().reshape(len(S), n)
        keys = oracle.edge_keys(rp0, ci0)
        for i, s in enumerate(S):
            want, _ = orc.bfs(int(s))
            assert np.array_equal(L[i], want), f"source {s}"
            oracle.check_bfs_tree(rp0, ci0, int(s), L[i], P[i], keys=keys)
    finally:
        d.close()


@pytest.mark.parametrize("k", [5, 64])
@pytest.mark.parametrize("where", ["device", "host"])
@pytest.mark.parametrize("parents", [True, False])
def test_batch_bitmask_unreached_pairs_written(k, where, parents):
    """A graph with few isolated vertices (here about 1%), whose bitmask
    traversal writes -1 to the (source, vertex) pairs it never reached at the
    end instead of clearing the outputs first: an ER part, a separate path and
    isolated vertices, sources in all three.  Outputs start as a sentinel, so
    an entry left unwritten fails; every row must equal the oracle's levels
    and form a BFS tree."""
    import torch
    rp0, ci0 = graphgen.erdos_renyi(1 << 12, 1 << 14, seed=8)
    n0 = len(rp0) - 1
    rows = np.repeat(np.arange(n0), np.diff(rp0))
    edges = [(int(a), int(b)) for a, b in zip(rows, ci0) if a < b]
    n_path, n_iso = 60, 40
    edges += [(n0 + j, n0 + j + 1) for j in range(n_path - 1)]
    n = n0 + n_path + n_iso
    rp, ci = graphgen.from_edges(n, edges)
    assert (np.diff(rp) == 0).sum() * 16 <= n  # few isolated vertices: the end pass writes the misses
    srcs = list(graphgen.sample_sources(rp0, k - 3, seed=5)) + [n0 + 7, n0 + n_path - 1, n - 1]
    S = np.ascontiguousarray(srcs, np.int32)
    g = B.bfs_create_csr(n, len(ci), rp, ci, B.BFS_VALIDATE | B.BFS_SYMMETRIC, None,
                         torch.cuda.current_stream().cuda_stream)
    try:
        if where == "host":
            L = np.full(k * n, 12345, np.int32)
            P = np.full(k * n, 12345, np.int32) if parents else None
        else:
            L = torch.full((k * n,), 12345, dtype=torch.int32, device="cuda")
            P = torch.full((k * n,), 12345, dtype=torch.int32, device="cuda") if parents else None
        for _ in range(2):  # the second call reuses the staging buffers the first one filled
            B.bfs_run_batch(g, S, k, L, P, None)
        Lh = (L if where == "host" else L.cpu().numpy()).reshape(k, n)
        orc = oracle.Oracle(rp, ci)
        keys = oracle.edge_keys(rp, ci)
        for i, s in enumerate(S):
            want, _ = orc.bfs(int(s))
            assert np.array_equal(Lh[i], want), f"source {i} ({s}): levels differ"
            if parents:
                Ph = (P if where == "host" else P.cpu().numpy()).reshape(k, n)
                oracle.check_bfs_tree(rp, ci, int(s), Lh[i], Ph[i], keys=keys)
    finally:
        B.bfs_destroy(g)


def test_batch_bitmask_off_and_asymmetric_rejected():
    rp, ci = graphgen.rmat(12, 16, seed=3)
    srcs = graphgen.sample_sources(rp, 8, seed=2)
    _batch_check(rp, ci, srcs, B.BFS_VALIDATE | B.BFS_SYMMETRIC, batch_bitmask=-1)
    rp2, ci2 = _directed_csr(5, [(0, 1), (1, 2)])
    with pytest.raises(B.BFSError) as e:
        B.bfs_create_csr(5, len(ci2), rp2, ci2, B.BFS_VALIDATE | B.BFS_SYMMETRIC)
    assert e.value.code == B.BFS_E_INVAL


def test_graphs_of_different_sizes_coexist():
    """Several graphs alive at once, used in an order different from their
    creation (per-kernel launch attributes must suit all of them)."""
    pool = [graphgen.rmat(14, 16, seed=6), graphgen.rmat(10, 16, seed=2), graphgen.grid(40, 40, 0.0),
            graphgen.from_edges(50, [(i, i + 1) for i in range(49)])]
    devs = [Dev(rp, ci, relabel=1 if i == 0 else 0) for i, (rp, ci) in enumerate(pool)]
    try:
        for d in reversed(devs):
            check_against_oracle(d, 0)
        for d in devs:
            check_against_oracle(d, 1)
    finally:
        for d in devs:
            d.close()


def test_batch_edge_sizes(rmat16):
    rp, ci, srcs, keys = rmat16
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    g = B.bfs_create_csr(len(rp) - 1, len(ci), rp, ci, B.BFS_VALIDATE | B.BFS_SYMMETRIC, None, stream)
    try:
        n = len(rp) - 1
        # k = 0 does nothing and succeeds
        B.bfs_run_batch(g, np.zeros(1, np.int32), 0, np.zeros(1, np.int32), None, None)
        # k = 1 through the bitmask path equals a single traversal
        L = np.empty((1, n), np.int32)
        Pm = np.empty((1, n), np.int32)
        s = int(srcs[0])
        B.bfs_run_batch(g, np.array([s], np.int32), 1, L, Pm, None)
        want, _ = oracle.bfs(rp, ci, s)
        assert np.array_equal(L[0], want)
        oracle.check_bfs_tree(rp, ci, s, L[0], Pm[0], keys=keys)
        # the same source twice in one batch: both rows are that source's traversal
        L2 = np.empty((2, n), np.int32)
        B.bfs_run_batch(g, np.array([s, s], np.int32), 2, L2, None, None)
        assert np.array_equal(L2[0], want) and np.array_equal(L2[1], want)
    finally:
        B.bfs_destroy(g)


def test_server_needs_graphs():
    with pytest.raises(B.BFSError):
        B.bfs_server_create([], None, None)
