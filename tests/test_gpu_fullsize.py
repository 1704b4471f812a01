"""Full-size workloads in the launch configuration the benchmark times
(default options, persistent level loop), checked against the oracle on
sampled sources (GPU only, slow)."""
import numpy as np
import pytest

import graphgen
import oracle
from gpu_helpers import Dev, check_against_oracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2209_08764_gb300 as pkg
    pkg.build()


@pytest.mark.parametrize("name,graph,nsrc", [
    ("rmat22", graphgen.rmat_s22, 3),
    ("grid4096", graphgen.grid_4096, 2),
    ("er2p20", graphgen.er_2p20, 4),
])
def test_fullsize(name, graph, nsrc):
    rp, ci = graph()
    d = Dev(rp, ci)
    orc = oracle.Oracle(rp, ci)
    keys = oracle.edge_keys(rp, ci)
    try:
        srcs = list(graphgen.sample_sources(rp, nsrc, seed=2))
        if name == "grid4096":
            srcs[0] = 0  # the corner: the deepest traversal
        for s in srcs:
            lv, _, st, _ = check_against_oracle(d, int(s), orc=orc, keys=keys)
            assert st.reached == int((lv >= 0).sum())
    finally:
        d.close()


def test_er2p20_batch_64_bitmask():
    """The multi-source workload: ER 2^20, mean degree 16, 64 sources in one
    bitmask launch; every source's levels bit-exact against the oracle."""
    import torch
    from paper_2209_08764_gb300 import binding as B
    rp, ci = graphgen.er_2p20()
    n = len(rp) - 1
    srcs = graphgen.sample_sources(rp, 64, seed=2)
    g = B.bfs_create_csr(n, len(ci), rp, ci, B.BFS_SYMMETRIC, None, torch.cuda.current_stream().cuda_stream)
    try:
        L = torch.empty(64 * n, dtype=torch.int32, device="cuda")
        P = torch.empty(64 * n, dtype=torch.int32, device="cuda")
        B.bfs_run_batch(g, srcs, 64, L, P, None)
        L = L.cpu().numpy().reshape(64, n)
        P = P.cpu().numpy().reshape(64, n)
        orc = oracle.Oracle(rp, ci)
        keys = oracle.edge_keys(rp, ci)
        for i, s in enumerate(srcs):
            want, _ = orc.bfs(int(s))
            assert np.array_equal(L[i], want), f"source {i}"
            if i < 8:
                oracle.check_bfs_tree(rp, ci, int(s), L[i], P[i], keys=keys)
    finally:
        B.bfs_destroy(g)
