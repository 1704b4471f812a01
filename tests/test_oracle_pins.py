"""Pins for the CPU oracle (CPU only).

The oracle is checked against things other than itself: closed-form distances
on named graphs, a library shortest-path routine, brute force over every simple
graph on up to 6 vertices, structural invariants on large random graphs, and
hand-worked traces of Fig. 1.  A mutation test then plants plausible mistakes
in copies of the oracle's C source and shows that the pins catch each one.
"""
import ctypes
import itertools
import json
import os
import subprocess

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import connected_components, shortest_path

import graphgen
import oracle

HERE = os.path.dirname(os.path.abspath(__file__))


# ---------------------------------------------------------------------------
# small named graphs
# ---------------------------------------------------------------------------

def path(n):
    return graphgen.from_edges(n, [(i, i + 1) for i in range(n - 1)])


def cycle(n):
    return graphgen.from_edges(n, [(i, (i + 1) % n) for i in range(n)])


def star(k):
    return graphgen.from_edges(k + 1, [(0, j) for j in range(1, k + 1)])


def complete(n):
    return graphgen.from_edges(n, list(itertools.combinations(range(n), 2)))


def complete_bipartite(a, b):
    return graphgen.from_edges(a + b, [(i, a + j) for i in range(a) for j in range(b)])


def binary_tree(h):
    n = (1 << h) - 1
    return graphgen.from_edges(n, [(i, c) for i in range(n) for c in (2 * i + 1, 2 * i + 2) if c < n])


def directed_csr(n, edges):
    edges = sorted(edges)
    rp = np.zeros(n + 1, np.int32)
    for u, _ in edges:
        rp[u + 1] += 1
    rp = np.cumsum(rp).astype(np.int32)
    ci = np.array([v for _, v in edges], np.int32)
    return rp, ci


# ---------------------------------------------------------------------------
# pin suites, parameterised by the BFS under test (returns level, parent)
# ---------------------------------------------------------------------------

def pins_closed_forms(bfs):
    for n in (1, 2, 5, 33):
        rp, ci = path(n)
        for s in {0, n // 2, n - 1}:
            lv, par = bfs(rp, ci, s)
            assert lv.tolist() == [abs(i - s) for i in range(n)], ("path", n, s)
            oracle.check_bfs_tree(rp, ci, s, lv, par)
    for n in (3, 4, 9, 20):
        rp, ci = cycle(n)
        for s in (0, 3 % n):
            lv, par = bfs(rp, ci, s)
            assert lv.tolist() == [min(abs(i - s), n - abs(i - s)) for i in range(n)], ("cycle", n, s)
            oracle.check_bfs_tree(rp, ci, s, lv, par)
    rp, ci = star(9)
    lv, par = bfs(rp, ci, 0)
    assert lv.tolist() == [0] + [1] * 9
    lv, par = bfs(rp, ci, 4)
    assert lv.tolist() == [1, 2, 2, 2, 0, 2, 2, 2, 2, 2]
    oracle.check_bfs_tree(rp, ci, 4, lv, par)
    for n in (2, 6):
        rp, ci = complete(n)
        lv, par = bfs(rp, ci, n - 1)
        assert lv.tolist() == [1] * (n - 1) + [0]
    rp, ci = complete_bipartite(3, 4)
    lv, par = bfs(rp, ci, 1)
    assert lv.tolist() == [2, 0, 2, 1, 1, 1, 1]
    lv, par = bfs(rp, ci, 5)
    assert lv.tolist() == [1, 1, 1, 2, 2, 0, 2]
    rp, ci = graphgen.grid(7, 11, 0.0)
    for s in (0, 7 * 11 - 1, 3 * 11 + 5):
        lv, par = bfs(rp, ci, s)
        r0, c0 = divmod(s, 11)
        want = [abs(r - r0) + abs(c - c0) for r in range(7) for c in range(11)]
        assert lv.tolist() == want, ("grid", s)
        oracle.check_bfs_tree(rp, ci, s, lv, par)
    rp, ci = binary_tree(6)
    lv, par = bfs(rp, ci, 0)
    assert lv.tolist() == [int(np.floor(np.log2(i + 1))) for i in range(63)]
    # disjoint union of two paths: the other component stays unreached
    rp, ci = graphgen.from_edges(9, [(0, 1), (1, 2), (2, 3), (4, 5), (5, 6), (6, 7), (7, 8)])
    lv, par = bfs(rp, ci, 2)
    assert lv.tolist() == [2, 1, 0, 1, -1, -1, -1, -1, -1]
    oracle.check_bfs_tree(rp, ci, 2, lv, par)
    # isolated source
    rp, ci = graphgen.from_edges(4, [(1, 2), (2, 3)])
    lv, par = bfs(rp, ci, 0)
    assert lv.tolist() == [0, -1, -1, -1] and par.tolist() == [0, -1, -1, -1]
    # directed: out-edges only
    rp, ci = directed_csr(5, [(0, 1), (1, 2), (2, 0), (3, 0), (2, 4), (4, 1)])
    lv, par = bfs(rp, ci, 0)
    assert lv.tolist() == [0, 1, 2, -1, 3]
    oracle.check_bfs_tree(rp, ci, 0, lv, par)


def _scipy_levels(rp, ci, srcs, directed):
    n = len(rp) - 1
    A = sp.csr_matrix((np.ones(len(ci)), ci, rp), shape=(n, n))
    D = shortest_path(A, method="D", directed=directed, unweighted=True, indices=srcs)
    return np.where(np.isinf(D), -1, D).astype(np.int64)


def pins_library(bfs):
    graphs = [graphgen.erdos_renyi(300, 700, seed=11), graphgen.rmat(9, 8, seed=3),
              graphgen.grid(20, 30, 0.2, seed=5)]
    for rp, ci in graphs:
        srcs = np.arange(0, len(rp) - 1, 37)
        D = _scipy_levels(rp, ci, srcs, directed=False)
        for k, s in enumerate(srcs):
            lv, par = bfs(rp, ci, int(s))
            assert np.array_equal(lv, D[k]), ("scipy", int(s))
            oracle.check_bfs_tree(rp, ci, int(s), lv, par)
    # a random directed graph (not symmetric)
    rng = np.random.default_rng(7)
    n = 200
    e = {(int(a), int(b)) for a, b in rng.integers(0, n, size=(600, 2)) if a != b}
    rp, ci = directed_csr(n, list(e))
    srcs = np.arange(0, n, 13)
    D = _scipy_levels(rp, ci, srcs, directed=True)
    for k, s in enumerate(srcs):
        lv, par = bfs(rp, ci, int(s))
        assert np.array_equal(lv, D[k]), ("scipy directed", int(s))
        oracle.check_bfs_tree(rp, ci, int(s), lv, par)


def _all_graphs(n):
    """Adjacency (G, n, n) of every simple undirected graph on n vertices."""
    pairs = list(itertools.combinations(range(n), 2))
    G = 1 << len(pairs)
    bits = (np.arange(G)[:, None] >> np.arange(len(pairs))[None, :]) & 1
    A = np.zeros((G, n, n), np.int64)
    for k, (i, j) in enumerate(pairs):
        A[:, i, j] = bits[:, k]
        A[:, j, i] = bits[:, k]
    return A


def _brute_distances(A):
    """Distances by reachability powers: d(s,v) = least k with (I+A)^k[s,v] > 0."""
    G, n, _ = A.shape
    R = np.broadcast_to(np.eye(n, dtype=np.int64), (G, n, n)).copy()
    D = np.where(R > 0, 0, -1)
    for k in range(1, n):
        R = np.minimum(R + R @ A, 1)
        D = np.where((D < 0) & (R > 0), k, D)
    return D


def _csr_of(Ai):
    n = Ai.shape[0]
    rp = np.concatenate([[0], np.cumsum(Ai.sum(1))]).astype(np.int32)
    ci = np.nonzero(Ai)[1].astype(np.int32)
    return rp, ci


def pins_brute_force(bfs, max_n=6, stride=1):
    for n in range(1, max_n + 1):
        A = _all_graphs(n)[::stride]
        D = _brute_distances(A)
        for g in range(len(A)):
            rp, ci = _csr_of(A[g])
            for s in range(n):
                lv, par = bfs(rp, ci, s)
                if not np.array_equal(lv, D[g, s]):
                    raise AssertionError(f"brute force n={n} graph={g} s={s}: {lv} != {D[g, s]}")
                oracle.check_bfs_tree(rp, ci, s, lv, par)


def pins_invariants(bfs):
    for rp, ci in (graphgen.rmat(12, 16, seed=9), graphgen.erdos_renyi(5000, 9000, seed=2)):
        n = len(rp) - 1
        rows = np.repeat(np.arange(n), np.diff(rp))
        A = sp.csr_matrix((np.ones(len(ci)), ci, rp), shape=(n, n))
        _, comp = connected_components(A, directed=False)
        for s in graphgen.sample_sources(rp, 4, seed=1):
            lv, par = bfs(rp, ci, int(s))
            r = lv >= 0
            assert np.array_equal(r, comp == comp[s]), "reached set != connected component"
            both = r[rows] & r[ci]
            assert np.all(np.abs(lv[rows[both]] - lv[ci[both]]) <= 1)
            big = np.where(r, lv, 1 << 30).astype(np.int64)
            deg = np.diff(rp)
            nz = deg > 0
            mins = np.full(n, 1 << 30, np.int64)
            mins[nz] = np.minimum.reduceat(big[ci], rp[:-1][nz])
            other = r & (np.arange(n) != s)
            assert np.array_equal(lv[other], mins[other] + 1), "level != 1 + min neighbour level"
            n_l, e_l = oracle.level_profile(rp, lv)
            assert n_l.sum() == r.sum() and e_l.sum() == deg[r].sum()
            oracle.check_bfs_tree(rp, ci, int(s), lv, par)


def oracle_bfs(rp, ci, s):
    return oracle.bfs(rp, ci, s)


# ---------------------------------------------------------------------------
# the oracle passes every pin
# ---------------------------------------------------------------------------

def test_closed_forms():
    pins_closed_forms(oracle_bfs)


def test_library_shortest_path():
    pins_library(oracle_bfs)


def test_brute_force_all_graphs_up_to_6():
    pins_brute_force(oracle_bfs, max_n=6)


def test_invariants_large():
    pins_invariants(oracle_bfs)


def test_grid_corner_level_counts():
    R = 16
    rp, ci = graphgen.grid(R, R, 0.0)
    lv, _ = oracle.bfs(rp, ci, 0)
    n_l, e_l = oracle.level_profile(rp, lv)
    assert n_l.tolist() == [l + 1 if l < R else 2 * R - 1 - l for l in range(2 * R - 1)]
    deg = np.diff(rp)
    assert e_l.tolist() == [int(deg[lv == l].sum()) for l in range(2 * R - 1)]


def test_bad_arguments():
    rp, ci = path(3)
    with pytest.raises(ValueError):
        oracle.bfs(rp, ci, 3)
    with pytest.raises(ValueError):
        oracle.bfs(rp, ci, -1)


# ---------------------------------------------------------------------------
# the tree checker rejects each kind of broken tree
# ---------------------------------------------------------------------------

def test_tree_checker_rejects():
    rp, ci = graphgen.grid(6, 6, 0.0)
    s = 14
    lv, par = oracle.bfs(rp, ci, s)
    oracle.check_bfs_tree(rp, ci, s, lv, par)
    bad = []
    p = par.copy(); p[s] = 0; bad.append(p)                       # root not its own parent
    v = int(np.nonzero(lv == 3)[0][0])
    p = par.copy(); p[v] = int(np.nonzero(lv == 3)[0][1]); bad.append(p)   # same level
    cands = np.nonzero(lv == lv[v] - 1)[0]
    nb = set(ci[rp[v]:rp[v + 1]].tolist())
    far = [int(c) for c in cands if int(c) not in nb]
    p = par.copy(); p[v] = far[0]; bad.append(p)                   # right level, no edge
    p = par.copy(); p[v] = -1; bad.append(p)                       # reached but no parent
    rp2, ci2 = graphgen.from_edges(5, [(0, 1), (1, 2), (3, 4)])
    lv2, par2 = oracle.bfs(rp2, ci2, 0)
    p = par2.copy(); p[4] = 3
    with pytest.raises(AssertionError):
        oracle.check_bfs_tree(rp2, ci2, 0, lv2, p)                 # unreached with a parent
    for p in bad:
        with pytest.raises(AssertionError):
            oracle.check_bfs_tree(rp, ci, s, lv, p)


# ---------------------------------------------------------------------------
# planted mistakes in copies of the oracle are caught by the pins
# ---------------------------------------------------------------------------

MUTANTS = {
    "dropped +1": ("level[v] = level[u] + 1;", "level[v] = level[u];"),
    "wrong term": ("level[v] = level[u] + 1;", "level[v] = level[u] + 2;"),
    "missed last neighbour": ("e < row_ptr[u + 1]; ++e", "e < row_ptr[u + 1] - 1; ++e"),
    "skipped first neighbour": ("e = row_ptr[u]; e", "e = row_ptr[u] + 1; e"),
    "enqueued wrong vertex": ("queue[tail++] = v;", "queue[tail++] = u;"),
    "transposed operand": ("const int32_t v = col_idx[e];", "const int32_t v = col_idx[u];"),
    "visited test": ("if (level[v] == -1) {", "if (level[v] <= 0) {"),
    "stack not queue": ("const int32_t u = queue[head++];", "const int32_t u = queue[--tail];"),
    "wrong parent": ("parent[v] = u;", "parent[v] = v;"),
}


def _compile_mutant(tmp_path, name, old, new):
    src = open(os.path.join(os.path.dirname(oracle.__file__), "bfs_oracle.c")).read()
    assert old in src, name
    src = src.replace(old, new)
    c = tmp_path / "mutant.c"
    c.write_text(src)
    so = tmp_path / "mutant.so"
    subprocess.check_call(["gcc", "-O1", "-shared", "-fPIC", "-o", str(so), str(c)])
    lib = ctypes.CDLL(str(so))
    P = ctypes.POINTER(ctypes.c_int32)
    lib.oracle_bfs.restype = ctypes.c_int64
    lib.oracle_bfs.argtypes = [ctypes.c_int32, P, P, ctypes.c_int32, P, P, P]

    def bfs(rp, ci, s):
        rp = np.ascontiguousarray(rp, np.int32)
        ci = np.ascontiguousarray(ci if len(ci) else np.zeros(1), np.int32)
        n = len(rp) - 1
        lv = np.empty(n, np.int32)
        par = np.empty(n, np.int32)
        q = np.empty(4 * n + 4, np.int32)   # roomy: a broken visited test may push more
        lib.oracle_bfs(n, rp.ctypes.data_as(P), ci.ctypes.data_as(P), int(s), lv.ctypes.data_as(P),
                       par.ctypes.data_as(P), q.ctypes.data_as(P))
        return lv, par
    return bfs


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(tmp_path, name):
    old, new = MUTANTS[name]
    bfs = _compile_mutant(tmp_path, name, old, new)
    caught = False
    for suite in (pins_closed_forms, lambda b: pins_brute_force(b, max_n=5)):
        try:
            suite(bfs)
        except (AssertionError, IndexError, ValueError):
            caught = True
            break
    assert caught, f"mutant '{name}' passed every pin"


# ---------------------------------------------------------------------------
# Fig. 1 step by step
# ---------------------------------------------------------------------------

def _golden():
    with open(os.path.join(HERE, "golden", "fig1_worked_examples.json")) as f:
        return json.load(f)["examples"]


@pytest.mark.parametrize("ex", _golden(), ids=lambda e: e["name"])
def test_fig1_hand_worked_traces(ex):
    rp, ci = directed_csr(ex["n"], [tuple(e) for e in ex["directed_edges"]])
    for race in ex["race"]:
        d, levels = oracle.s3bfs_fig1(rp, ci, ex["s"], ex["P"], race=race)
        assert d.tolist() == ex["d"]
        assert len(levels) == len(ex["levels"])
        for got, want in zip(levels, ex["levels"]):
            assert sorted(got["frontier"].tolist()) == sorted(want["frontier"])
            assert got["e_l"] == want["e_l"]
            assert got["P_l"] == want["P_l"]
            if want["e_l"] == 0:
                continue
            assert np.cumsum(np.diff(rp)[got["frontier"]]).tolist() == want["EdgeSum"]
            assert got["C"] == want["C"]
            assert got["starts"].tolist() == want["starts"]
            assert got["candidates"] == want["candidates"][race]
            sizes = want["Sizes"][race] if isinstance(want["Sizes"], dict) else want["Sizes"]
            assert got["Sizes"].tolist() == sizes


def test_fig1_matches_fifo_bfs_brute_force():
    rng = np.random.default_rng(3)
    for n in (1, 2, 3, 4, 5, 6):
        A = _all_graphs(n)
        pick = np.arange(len(A)) if len(A) <= 64 else rng.choice(len(A), 64, replace=False)
        for g in pick:
            rp, ci = _csr_of(A[g])
            for s in range(n):
                want, _ = oracle.bfs(rp, ci, s)
                for P in (1, 2, 5):
                    for race in ("none", "max"):
                        d, _ = oracle.s3bfs_fig1(rp, ci, s, P, race=race)
                        assert np.array_equal(d, want), (n, g, s, P, race)


@pytest.mark.parametrize("P,grain", [(1, 1), (4, 1), (64, 1), (4096, 1), (64, 16), (4864, 256)])
def test_fig1_levels_on_rmat(P, grain):
    rp, ci = graphgen.rmat(10, 16, seed=1)
    for s in graphgen.sample_sources(rp, 3, seed=2):
        want, _ = oracle.bfs(rp, ci, int(s))
        n_l, e_l = oracle.level_profile(rp, want)
        per_race = {}
        for race in ("none", "max"):
            d, levels = oracle.s3bfs_fig1(rp, ci, int(s), P, grain=grain, race=race)
            assert np.array_equal(d, want)
            assert [r["n_l"] for r in levels] == n_l.tolist()
            assert [r["e_l"] for r in levels] == e_l.tolist()
            for k, r in enumerate(levels):
                assert set(r["frontier"].tolist()) == set(np.nonzero(want == k)[0].tolist())
                assert r["P_l"] == (min(P, -(-r["e_l"] // grain)) if r["e_l"] else 0)
                if r["e_l"]:
                    nxt = n_l[k + 1] if k + 1 < len(n_l) else 0
                    assert nxt <= r["candidates"] <= r["undiscovered_edges"]
                    assert r["Sizes"].sum() == nxt
            per_race[race] = levels
        for r in per_race["none"][:-1]:
            assert r["candidates"] == r["Sizes"].sum()


def test_start_points_scatter_equals_binary_search():
    rng = np.random.default_rng(11)
    for trial in range(300):
        n_l = int(rng.integers(1, 60))
        deg = rng.integers(0, 9, size=n_l) * (rng.random(n_l) < 0.7)
        if deg.sum() == 0:
            deg[-1] = 1
        EdgeSum = np.cumsum(deg)
        e_l = int(EdgeSum[-1])
        ex = np.concatenate([[0], EdgeSum])
        P = int(rng.integers(1, 80))
        for grain in (1, 3):
            P_l = min(P, -(-e_l // grain))
            C = -(-e_l // P_l)
            a = oracle.start_points_scatter(EdgeSum, e_l, P_l, C)
            b = oracle.start_points_bsearch(ex, e_l, P_l, C)
            assert np.array_equal(a, b)
            # each start names the edge t*C exactly, inside a vertex with edges
            t = np.arange(len(a))
            assert np.array_equal(ex[a[:, 0]] + a[:, 1], t * C)
            assert np.all((a[:, 1] >= 0) & (a[:, 1] < deg[a[:, 0]]))


def test_fig1_star_closed_form():
    k = 37
    rp, ci = star(k)
    for P in (1, 5, 37, 100):
        d, levels = oracle.s3bfs_fig1(rp, ci, 0, P)
        r = levels[0]
        P_l = min(P, k)
        C = -(-k // P_l)
        assert (r["e_l"], r["P_l"], r["C"]) == (k, P_l, C)
        T = -(-k // C)
        assert r["starts"].tolist() == [[0, t * C] for t in range(T)]
        # second pass: every leaf has one edge back to the centre
        assert levels[1]["e_l"] == k and levels[1]["candidates"] == 0


# ---------------------------------------------------------------------------
# traversed_edges: the Graph500 edge count behind every GTEPS figure
# ---------------------------------------------------------------------------

def _disjoint(a, b):
    """Disjoint union of two CSR graphs; b's vertices follow a's."""
    (ra, ca), (rb, cb) = a, b
    na = len(ra) - 1
    rp = np.concatenate([ra, rb[1:] + ra[-1]]).astype(np.int32)
    ci = np.concatenate([ca, cb + na]).astype(np.int32)
    return rp, ci


def pins_traversed_edges(te):
    """Closed forms for the undirected edges inside the source's component,
    then brute force on every simple graph with n <= 5 (the count of listed
    vertex pairs whose two ends lie in the source's component)."""
    def count(rp, ci, s):
        lv, _ = oracle.bfs(rp, ci, s)
        return te(rp, lv)
    for n in (1, 2, 7, 40):
        rp, ci = path(n)
        for s in {0, n // 2, n - 1}:
            assert count(rp, ci, s) == n - 1, ("path", n, s)
    for k in (1, 3, 12):
        rp, ci = star(k)
        assert count(rp, ci, 0) == k and count(rp, ci, k) == k, ("star", k)
    for n in (2, 5, 9):
        rp, ci = complete(n)
        assert count(rp, ci, n - 1) == n * (n - 1) // 2, ("K_n", n)
    for a, b in ((1, 4), (3, 5)):
        rp, ci = complete_bipartite(a, b)
        assert count(rp, ci, 0) == a * b and count(rp, ci, a) == a * b, ("K_ab", a, b)
    for n in (3, 10):
        rp, ci = cycle(n)
        assert count(rp, ci, 1) == n, ("cycle", n)
    rp, ci = graphgen.grid(6, 9, 0.0)
    assert count(rp, ci, 0) == 6 * 8 + 9 * 5, "grid"
    rp, ci = binary_tree(5)
    assert count(rp, ci, 0) == (1 << 5) - 2, "binary tree"
    # disjoint union: only the source's component counts
    rp, ci = _disjoint(path(4), complete(5))
    assert count(rp, ci, 1) == 3 and count(rp, ci, 6) == 10, "disjoint union"
    # an isolated source traverses nothing
    rp, ci = _disjoint(graphgen.from_edges(1, []), complete(4))
    assert count(rp, ci, 0) == 0, "isolated source"
    for n in range(1, 6):
        A = _all_graphs(n)
        for g in range(len(A)):
            rp, ci = _csr_of(A[g])
            _, comp = connected_components(sp.csr_matrix(A[g]), directed=False)
            iu, ju = np.nonzero(np.triu(A[g], 1))
            for s in range(n):
                want = int(np.sum(comp[iu] == comp[s]))
                got = count(rp, ci, s)
                if got != want:
                    raise AssertionError(f"traversed edges n={n} graph={g} s={s}: {got} != {want}")


def test_traversed_edges_pins():
    pins_traversed_edges(oracle.traversed_edges)


TE_MUTANTS = {
    "no halving": ("].sum() // 2)", "].sum())"),
    "every vertex": ("deg[np.asarray(level) >= 0]", "deg"),
    "source left out": ("np.asarray(level) >= 0", "np.asarray(level) > 0"),
    "row ends, not degrees": ("np.diff(np.asarray(row_ptr, np.int64))", "np.asarray(row_ptr, np.int64)[1:]"),
}


@pytest.mark.parametrize("name", sorted(TE_MUTANTS))
def test_traversed_edges_pins_catch_planted_mistake(name):
    import inspect
    import textwrap

    old, new = TE_MUTANTS[name]
    src = textwrap.dedent(inspect.getsource(oracle.traversed_edges))
    assert old in src, name
    ns = {"np": np}
    exec(compile(src.replace(old, new), f"<mutant {name}>", "exec"), ns)
    with pytest.raises(AssertionError):
        pins_traversed_edges(ns["traversed_edges"])
