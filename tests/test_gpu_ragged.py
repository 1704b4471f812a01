"""Ragged sizes against the oracle (GPU only).

Vertex counts just below, at and above the multiples the kernels tile by (32
lanes, 128-vertex bitmap groups, 4-entry quads, 4096-entry frontier windows of
a CTA), mean degrees from 1 to 17, and the knobs that change how a level is
cut (the grain, the CTA shape, the renumbering).  Every traversal's levels
must equal the oracle's bit for bit, its parents must form a valid tree, and
its per-level statistics must match the oracle's level profile.
"""
import numpy as np
import pytest

import graphgen
import oracle
from gpu_helpers import Dev, check_against_oracle
from paper_2209_08764_gb300 import binding as B

pytestmark = pytest.mark.gpu

SIZES = [1, 2, 31, 32, 33, 127, 128, 129, 4095, 4096, 4097, 65535, 65537]


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2209_08764_gb300 as pkg
    pkg.build()
    B.load()


def _graph(n, mean_deg, seed):
    """Erdős–Rényi with m = n * mean_deg / 2 distinct undirected edges
    (capped at the complete graph); n = 1 has no edge."""
    m = min(n * mean_deg // 2, n * (n - 1) // 2)
    if m == 0:
        return graphgen.from_edges(n, [])
    return graphgen.erdos_renyi(n, m, seed=seed)


@pytest.mark.parametrize("n", SIZES)
@pytest.mark.parametrize("mean_deg", [1, 3, 17])
def test_ragged_sizes_default_options(n, mean_deg):
    rp, ci = _graph(n, mean_deg, seed=n + mean_deg)
    d = Dev(rp, ci, flags=B.BFS_VALIDATE | B.BFS_SYMMETRIC)
    orc = oracle.Oracle(rp, ci)
    try:
        srcs = graphgen.sample_sources(rp, 2, seed=7) if len(ci) else np.array([0, n - 1], np.int32)
        for s in srcs:
            check_against_oracle(d, int(s), orc=orc)
    finally:
        d.close()


@pytest.mark.parametrize("n", [33, 4097, 65537])
@pytest.mark.parametrize("opts", [dict(chunk_edges=1), dict(chunk_edges=7, cta_warps=8), dict(cta_warps=16),
                                  dict(cta_warps=32, relabel=1), dict(relabel=-1, small_level_edges=-1),
                                  dict(direction=1)],
                         ids=lambda o: ",".join(f"{k}={v}" for k, v in o.items()))
def test_ragged_sizes_launch_shapes(n, opts):
    rp, ci = _graph(n, 5, seed=3 * n)
    d = Dev(rp, ci, flags=B.BFS_VALIDATE | B.BFS_SYMMETRIC, **opts)
    orc = oracle.Oracle(rp, ci)
    try:
        for s in graphgen.sample_sources(rp, 2, seed=11):
            check_against_oracle(d, int(s), orc=orc, grain=opts.get("chunk_edges", 64))
    finally:
        d.close()
