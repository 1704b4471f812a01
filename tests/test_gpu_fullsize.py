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
