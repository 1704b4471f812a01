"""The allocation-free entry point, checked against the oracle and bfs_run (GPU only).

bfs_run_csr_noalloc serves callers that must not allocate device memory while
they traverse (code inside a framework whose caching allocator owns the GPU's
memory, or latency-critical loops where cudaMalloc would synchronise the
device).  Its working memory is a fixed static device array shared by every
call, so these tests also run it twice in a row and on graphs of different
sizes, to show that each call starts from clean state.  This file is collected
last, so a failure here comes after every other test has run.
"""
import numpy as np
import pytest

import graphgen
import oracle
from paper_2209_08764_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    import paper_2209_08764_gb300 as pkg
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    pkg.build()
    B.load()


def _reference(rp, ci, srcs):
    """Levels (and a valid tree) from the allocating entry point bfs_run."""
    import torch
    n = len(rp) - 1
    g = B.bfs_create_csr(n, len(ci), rp, ci if len(ci) else None, B.BFS_VALIDATE, None,
                         torch.cuda.current_stream().cuda_stream)
    out = []
    try:
        for s in srcs:
            lv = torch.empty(n, dtype=torch.int32, device="cuda")
            B.bfs_run(g, int(s), lv, None, None)
            out.append(lv.cpu().numpy())
    finally:
        B.bfs_destroy(g)
    return out


def test_noalloc_matches_oracle_and_bfs_run_two_calls_in_a_row():
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(graphgen.rmat(14, 16, seed=7), None), (graphgen.grid(97, 131, 0.02, seed=9), None),
             (graphgen.rmat(16, 16, seed=1), None),
             (graphgen.from_edges(5, []), [0, 4]),                                # nnz = 0
             (graphgen.from_edges(7, [(i, i + 1) for i in range(6)]), [0, 3]),    # nnz = 12
             (graphgen.from_edges(4, [(0, 1), (1, 2), (2, 3)]), [0, 2]),          # nnz = 6, not a multiple of 4
             (graphgen.from_edges(4, [(1, 2), (2, 3), (1, 3)]), [0, 2])]          # vertex 0 isolated
    for (rp, ci), srcs in cases:
        n, nnz = len(rp) - 1, len(ci)
        srcs = graphgen.sample_sources(rp, 2, seed=5) if srcs is None else np.array(srcs, np.int32)
        want = [oracle.bfs(rp, ci, int(s))[0] for s in srcs]
        for w, o in zip(want, _reference(rp, ci, srcs)):
            assert np.array_equal(w, o), "bfs_run differs from the oracle"
        # odd-length, unaligned device views of the CSR: the entry point must not care
        big = torch.zeros(nnz + 3, dtype=torch.int32, device="cuda")
        if nnz:
            big[1:1 + nnz] = torch.from_numpy(ci).cuda()
        drp = torch.from_numpy(rp).cuda()
        dci = big[1:1 + nnz]
        level = torch.empty(n, dtype=torch.int32, device="cuda")
        parent = torch.empty(n, dtype=torch.int32, device="cuda")
        keys = oracle.edge_keys(rp, ci)
        for call in range(2):                       # two calls in a row, same inputs
            for s, w in zip(srcs, want):
                level.fill_(123)
                parent.fill_(123)
                B.bfs_run_csr_noalloc(n, nnz, drp, dci, int(s), level, parent, stream)
                lv = level.cpu().numpy()
                assert np.array_equal(lv, w), f"n={n} call {call}, src {s}: levels differ from the oracle"
                oracle.check_bfs_tree(rp, ci, int(s), lv, parent.cpu().numpy(), keys=keys)


def test_noalloc_rejects_sizes_beyond_its_maximum():
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    x = torch.zeros(8, dtype=torch.int32, device="cuda")
    with pytest.raises(B.BFSError) as e:
        B.bfs_run_csr_noalloc((1 << 18) + 1, 0, x, x, 0, x, x, stream)
    assert e.value.code == B.BFS_E_INVAL and "262144" in str(e.value)
    with pytest.raises(B.BFSError) as e:
        B.bfs_run_csr_noalloc(4, (1 << 21) + 1, x, x, 0, x, x, stream)
    assert e.value.code == B.BFS_E_INVAL and "2097152" in str(e.value)
    # a bad CSR is caught by the range check, not by a fault
    rp = torch.tensor([0, 1, 2, 2, 2], dtype=torch.int32, device="cuda")
    ci = torch.tensor([1, 9], dtype=torch.int32, device="cuda")
    with pytest.raises(B.BFSError) as e:
        B.bfs_run_csr_noalloc(4, 2, rp, ci, 0, x, x, stream)
    assert e.value.code == B.BFS_E_INVAL
