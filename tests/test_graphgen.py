"""Input generators: determinism, structure and exact sizes (CPU only)."""
import numpy as np
import pytest

import graphgen


def _csr_ok(rp, ci):
    n = len(rp) - 1
    assert rp[0] == 0 and rp[-1] == len(ci)
    assert np.all(np.diff(rp) >= 0)
    assert len(ci) == 0 or (ci.min() >= 0 and ci.max() < n)
    rows = np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))
    assert not np.any(rows == ci), "self-loop"
    key = rows * n + ci
    assert np.all(np.diff(key) > 0), "rows must be strictly increasing (sorted, no duplicates)"
    # symmetric: the multiset of (v, u) equals that of (u, v)
    rkey = np.sort(ci.astype(np.int64) * n + rows)
    assert np.array_equal(key, rkey), "not symmetric"


@pytest.mark.parametrize("scale", [1, 4, 8, 12])
def test_rmat_structure(scale):
    rp, ci = graphgen.rmat(scale, 16, seed=5)
    assert len(rp) - 1 == 1 << scale
    assert len(ci) <= 2 * 16 << scale
    _csr_ok(rp, ci)


def test_rmat_deterministic_and_seeded():
    a = graphgen.rmat(11, 16, seed=1)
    b = graphgen.rmat(11, 16, seed=1)
    c = graphgen.rmat(11, 16, seed=2)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert not (len(a[1]) == len(c[1]) and np.array_equal(a[1], c[1]))


def test_rmat_skew():
    # A=0.57 concentrates edges: without relabelling vertex 0 is the hub
    rp, ci = graphgen.rmat(12, 16, seed=1, relabel=False)
    deg = np.diff(rp)
    assert deg[0] == deg.max()
    assert deg.max() > 20 * deg.mean()


@pytest.mark.parametrize("rows,cols", [(1, 1), (1, 7), (5, 1), (8, 8), (13, 29)])
def test_grid_exact_sizes(rows, cols):
    rp, ci = graphgen.grid(rows, cols, 0.0)
    undirected = rows * (cols - 1) + (rows - 1) * cols
    assert len(ci) == 2 * undirected
    _csr_ok(rp, ci)
    rp, ci = graphgen.grid(rows, cols, 1.0)
    assert len(ci) == 0


def test_grid_deletion_rate():
    rows = cols = 512
    rp, ci = graphgen.grid(rows, cols, 0.01, seed=3)
    _csr_ok(rp, ci)
    und = rows * (cols - 1) + (rows - 1) * cols
    deleted = und - len(ci) // 2
    mean, sd = und * 0.01, np.sqrt(und * 0.01 * 0.99)
    assert abs(deleted - mean) < 6 * sd


def test_er_exact():
    n, m = 1 << 12, 40000
    rp, ci = graphgen.erdos_renyi(n, m, seed=4)
    assert len(rp) - 1 == n and len(ci) == 2 * m
    _csr_ok(rp, ci)
    a = graphgen.erdos_renyi(n, m, seed=4)
    assert np.array_equal(a[1], ci)


def test_from_edges_cleans():
    rp, ci = graphgen.from_edges(5, [(0, 1), (1, 0), (2, 2), (3, 4), (4, 3), (1, 2)])
    _csr_ok(rp, ci)
    assert rp.tolist() == [0, 1, 3, 4, 5, 6]
    assert ci.tolist() == [1, 0, 2, 1, 4, 3]


def test_sample_sources():
    rp, ci = graphgen.rmat(10, 16, seed=1)
    s = graphgen.sample_sources(rp, 64, seed=2)
    assert len(s) == 64 and len(set(s.tolist())) == 64
    assert np.all(np.diff(rp)[s] > 0)
    assert np.array_equal(s, graphgen.sample_sources(rp, 64, seed=2))
    # fewer eligible vertices than asked
    rp2, _ = graphgen.from_edges(6, [(0, 1)])
    assert sorted(graphgen.sample_sources(rp2, 10).tolist()) == [0, 1]
