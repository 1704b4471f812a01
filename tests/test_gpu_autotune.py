"""Autotuner on the GPU: it measures real traversals, caches the winner per
graph class, and the options it picks give oracle-exact levels."""
import pytest

import graphgen
from gpu_helpers import Dev, check_against_oracle
from paper_2209_08764_gb300 import autotune
from paper_2209_08764_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2209_08764_gb300 as pkg
    pkg.build()
    B.load()


@pytest.mark.parametrize("name", ["grid", "rmat"])
def test_tune_caches_and_the_choice_is_exact(name, tmp_path):
    rp, ci = graphgen.grid(96, 80, 0.02, seed=3) if name == "grid" else graphgen.rmat(13, 16, seed=1)
    srcs = graphgen.sample_sources(rp, 2, seed=1)
    space = {"cta_warps": [0, 8, 32], "small_level_edges": [0, -1], "ctas": [0, -1], "direction": [0, 1]}
    path = str(tmp_path / "tune.json")
    opts, key, info = autotune.tune(B, rp, ci, srcs, cache_path=path, space=space, reps=1)
    assert not info["cached"] and info["trials"] >= 4 and info["ms"] > 0
    opts2, key2, info2 = autotune.tune(B, rp, ci, srcs, cache_path=path, space=space, reps=1)
    assert info2["cached"] and opts2 == opts and key2 == key
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    flags = B.BFS_VALIDATE | (B.BFS_SYMMETRIC if opts.get("direction") else 0)
    d = Dev(rp, ci, flags=flags, **{k: v for k, v in autotune.resolve(opts, sms).items() if v})
    try:
        for s in srcs:
            check_against_oracle(d, int(s))
    finally:
        d.close()
