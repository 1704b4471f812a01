"""Direction-optimising traversal (bottom-up levels) vs the CPU oracle, through
the C ABI (GPU only).

Levels must equal the oracle's bit for bit and parents must form a valid BFS
tree whichever way each level ran.  The helper also checks, level by level,
that the direction the device chose is the one the switching rule gives on
the oracle's level profile, that a bottom-up level emits exactly the next
frontier, and that its examined entries lie between the vertices found and
the degree sum of the unvisited vertices.
"""
import numpy as np
import pytest

import graphgen
import oracle
from gpu_helpers import Dev, check_against_oracle
from paper_2209_08764_gb300 import binding as B

pytestmark = pytest.mark.gpu

SYM = B.BFS_VALIDATE | B.BFS_SYMMETRIC


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2209_08764_gb300 as pkg
    pkg.build()
    B.load()
    yield
    torch.cuda.synchronize()


@pytest.fixture(scope="module")
def rmat16():
    rp, ci = graphgen.rmat(16, 16, seed=1)
    return rp, ci, oracle.Oracle(rp, ci)


@pytest.mark.parametrize("relabel", [0, 1, -1])
def test_rmat16_direction_optimising(rmat16, relabel):
    rp, ci, orc = rmat16
    d = Dev(rp, ci, flags=SYM, direction=1, relabel=relabel)
    try:
        srcs = graphgen.sample_sources(rp, 8, seed=2)
        saw_bu = False
        for s in srcs:
            _, _, st, pl = check_against_oracle(d, int(s), orc)
            saw_bu |= bool((pl[:, 7] == 1).any())
            assert st.work_edges <= st.edges_scanned
        assert saw_bu, "R-MAT should take bottom-up levels with the default alpha / beta"
    finally:
        d.close()


@pytest.mark.parametrize("opts", [
    dict(do_alpha=1 << 20, do_gamma=-1),                    # bottom-up at almost every level
    dict(do_alpha=1 << 20, do_gamma=-1, do_beta=1),         # and never back
    dict(do_alpha=2, do_beta=1 << 20),         # late switch, early switch back
    dict(do_gamma=-1),                         # Beamer's rule alone
    dict(do_gamma=8),
    dict(do_alpha=1 << 20, do_gamma=-1, cta_warps=8),
    dict(do_alpha=1 << 20, do_gamma=-1, cta_warps=16),
    dict(do_alpha=1 << 20, do_gamma=-1, cta_warps=24),
    dict(do_alpha=1 << 20, do_gamma=-1, ctas=3),            # few warps: many words per warp
    dict(do_alpha=1 << 20, do_gamma=-1, ctas=1, cta_warps=8),
    dict(do_alpha=1 << 20, do_gamma=-1, small_level_edges=-1),
    dict(do_alpha=1 << 20, do_gamma=-1, relabel=1),
], ids=lambda o: ",".join(f"{k}={v}" for k, v in o.items()))
def test_rmat16_forced_bottom_up(rmat16, opts):
    rp, ci, orc = rmat16
    d = Dev(rp, ci, flags=SYM, direction=1, **opts)
    try:
        for s in graphgen.sample_sources(rp, 4, seed=9):
            check_against_oracle(d, int(s), orc)
    finally:
        d.close()


def _named():
    g = {}
    g["star3000"] = graphgen.from_edges(3001, [(0, j) for j in range(1, 3001)])
    g["path40"] = graphgen.from_edges(40, [(i, i + 1) for i in range(39)])
    g["grid33x70"] = graphgen.grid(33, 70, 0.05, seed=3)
    g["two_parts"] = graphgen.from_edges(10, [(0, 1), (1, 2), (2, 3), (5, 6), (6, 7), (7, 8), (8, 9)])
    g["er"] = graphgen.erdos_renyi(5000, 40000, seed=4)
    # a heavy vertex (degree > 32) whose only frontier neighbour is its last entry
    hub_edges = [(0, j) for j in range(1, 200)] + [(199, 200), (200, 201)] + [(201, j) for j in range(202, 260)]
    g["late_parent"] = graphgen.from_edges(260, hub_edges)
    return g


@pytest.mark.parametrize("alpha", [0, 1 << 20])
@pytest.mark.parametrize("name", sorted(_named()))
def test_named_graphs_direction_optimising(name, alpha):
    rp, ci = _named()[name]
    d = Dev(rp, ci, flags=SYM, direction=1, do_alpha=alpha, do_gamma=-1 if alpha else 0)
    try:
        n = len(rp) - 1
        for s in sorted({0, n // 2, n - 1}):
            check_against_oracle(d, s)
    finally:
        d.close()


def test_host_outputs_and_batch(rmat16):
    rp, ci, orc = rmat16
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    g = B.bfs_create_csr(len(rp) - 1, len(ci), rp, ci, SYM,
                         B.bfs_opts(direction=1, do_alpha=1 << 20, do_gamma=-1, batch_bitmask=-1),
                         stream)
    try:
        n = len(rp) - 1
        srcs = graphgen.sample_sources(rp, 3, seed=4)
        lv = np.full(n, 7, np.int32)
        pa = np.full(n, 7, np.int32)
        B.bfs_run(g, int(srcs[0]), lv, pa, None)
        want, _ = orc.bfs(int(srcs[0]))
        assert np.array_equal(lv, want)
        oracle.check_bfs_tree(rp, ci, int(srcs[0]), lv, pa)
        # one traversal per source (batch_bitmask = -1) runs the direction-optimising loop
        L = np.empty((3, n), np.int32)
        Pm = np.empty((3, n), np.int32)
        B.bfs_run_batch(g, srcs, 3, L, Pm, None)
        for i, s in enumerate(srcs):
            want, _ = orc.bfs(int(s))
            assert np.array_equal(L[i], want)
            oracle.check_bfs_tree(rp, ci, int(s), L[i], Pm[i])
    finally:
        B.bfs_destroy(g)


def test_requires_symmetric_and_valid_options(rmat16):
    rp, ci, _ = rmat16
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    with pytest.raises(B.BFSError) as e:
        B.bfs_create_csr(len(rp) - 1, len(ci), rp, ci, B.BFS_VALIDATE, B.bfs_opts(direction=1), stream)
    assert e.value.code == B.BFS_E_INVAL
    with pytest.raises(B.BFSError):
        B.bfs_create_csr(len(rp) - 1, len(ci), rp, ci, SYM, B.bfs_opts(direction=2), stream)
    with pytest.raises(B.BFSError):
        B.bfs_create_csr(len(rp) - 1, len(ci), rp, ci, SYM, B.bfs_opts(direction=1, do_alpha=-1), stream)
    with pytest.raises(B.BFSError):
        B.bfs_create_csr(len(rp) - 1, len(ci), rp, ci, SYM, B.bfs_opts(direction=1, do_gamma=-2), stream)


def test_launch_per_phase_stays_top_down(rmat16):
    rp, ci, orc = rmat16
    d = Dev(rp, ci, flags=SYM, direction=1, persistent=-1)
    try:
        for s in graphgen.sample_sources(rp, 2, seed=5):
            _, _, st, pl = check_against_oracle(d, int(s), orc)
            assert (pl[:, 7] == 0).all()
    finally:
        d.close()


@pytest.mark.parametrize("flags", [B.BFS_DEVICE_PTRS | B.BFS_SYMMETRIC,
                                   B.BFS_DEVICE_PTRS | B.BFS_SYMMETRIC | B.BFS_VALIDATE,
                                   B.BFS_SYMMETRIC | B.BFS_DEDUP])
def test_device_csr_and_dedup_inputs(flags):
    # the CSR given as device pointers (the live-vertex count is then read back
    # from the device), or cleaned by BFS_DEDUP on the host
    import torch
    rp, ci = graphgen.rmat(12, 16, seed=3)
    if flags & B.BFS_DEVICE_PTRS:
        a, b = torch.from_numpy(rp).cuda(), torch.from_numpy(ci).cuda()
    else:
        a, b = rp, ci
    g = B.bfs_create_csr(len(rp) - 1, len(ci), a, b, flags, B.bfs_opts(direction=1),
                         torch.cuda.current_stream().cuda_stream)
    try:
        lv = torch.empty(len(rp) - 1, dtype=torch.int32, device="cuda")
        pa = torch.empty_like(lv)
        for s in graphgen.sample_sources(rp, 3, seed=11):
            st = B.bfs_stats()
            B.bfs_run(g, int(s), lv, pa, st)
            want, _ = oracle.bfs(rp, ci, int(s))
            assert np.array_equal(lv.cpu().numpy(), want)
            oracle.check_bfs_tree(rp, ci, int(s), want, pa.cpu().numpy())
            assert st.work_edges <= st.edges_scanned
    finally:
        B.bfs_destroy(g)
