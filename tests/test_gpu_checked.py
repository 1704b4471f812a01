"""The range-checked debug build passes the parity suite (GPU only).

SURVEY's stand-in for a sanitizer: libs3bfs_checked.so range-checks every
global index of the level step and stops with BFS_E_CHECK instead of making
an out-of-range access.  The suite (checked_suite.py) runs in a process of
its own, so that process loads the checked library instead of the product.
"""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


def test_checked_build_parity_and_frontier_sets():
    import paper_2209_08764_gb300 as pkg
    pkg.build()
    env = dict(os.environ, S3BFS_LIBRARY="checked")
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_suite.py")], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, f"checked suite failed:\n{r.stdout[-3000:]}\n{r.stderr[-3000:]}"
    assert "injected range violation -> BFS_E_CHECK ok" in r.stdout
