"""Autotuner host logic (CPU): coordinate descent, the JSON cache and the
graph-class key.  The GPU side (real measurements) is in test_gpu_autotune."""
import json

import numpy as np

import graphgen
from paper_2209_08764_gb300 import autotune


def test_coordinate_descent_finds_the_separable_minimum():
    space = {"a": [0, 1, 2, 3], "b": [0, 5, 7], "c": [0, -1]}
    want = {"a": 2, "b": 7, "c": -1}
    calls = []

    def cost(o):
        calls.append(o)
        return sum((o[k] - want[k]) ** 2 for k in space) + 1.0

    best, ms, trials = autotune.coordinate_descent(cost, space)
    assert best == want and ms == 1.0
    # one pass: the start plus every other value of every knob, none measured twice
    assert len(trials) == len(calls) <= 1 + sum(len(v) - 1 for v in space.values())
    assert len({tuple(sorted(o.items())) for o, _ in trials}) == len(trials)


def test_coordinate_descent_skips_failing_settings():
    space = {"a": [0, 1, 2], "b": [0, 1]}

    def cost(o):
        if o["a"] == 2:
            raise RuntimeError("not allowed on this graph")
        return 10 - o["a"] - o["b"]

    best, ms, trials = autotune.coordinate_descent(cost, space)
    assert best == {"a": 1, "b": 1} and ms == 8
    assert any(ms == float("inf") for _, ms in trials)


def test_coordinate_descent_starts_from_given_options():
    space = {"a": [0, 1], "b": [0, 1]}
    best, _, trials = autotune.coordinate_descent(lambda o: o["a"] + o["b"], space, start={"a": 1})
    assert trials[0][0] == {"a": 1, "b": 0}
    assert best == {"a": 0, "b": 0}


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    c = autotune.Cache(path)
    assert c.get("k") is None
    c.put("k", {"cta_warps": 8, "chunk_edges": 32}, 1.25, [[{"cta_warps": 0}, 2.0]])
    c2 = autotune.Cache(path)
    assert c2.get("k") == {"cta_warps": 8, "chunk_edges": 32}
    data = json.load(open(path))
    assert data["k"]["ms"] == 1.25 and len(data["k"]["trials"]) == 1


def test_graph_key_classes():
    rp, ci = graphgen.rmat(12, 16, seed=1)
    k1 = autotune.graph_key(rp, ci)
    assert k1 == autotune.graph_key(rp, ci)
    assert k1.startswith("n2^12-") and k1.endswith("flat")  # n <= 2^18: every vertex has a visited bit
    rp2, ci2 = graphgen.grid(64, 64, 0.0)
    assert autotune.graph_key(rp2, ci2, depth=127).endswith("-medium")
    assert autotune.graph_key(rp2, ci2, depth=5000).endswith("-deep")
    assert autotune.graph_key(rp2, ci2, depth=3).endswith("-shallow")
    # the mean degree is part of the class
    assert autotune.graph_key(rp2, ci2) != autotune.graph_key(*graphgen.erdos_renyi(4096, 4096 * 8, seed=1))


def test_skew_needs_a_large_graph():
    # skew is measured on the 2^18 highest-degree vertices; below that every
    # vertex is covered and the class is flat
    deg = np.array([5] * 10)
    rp = np.concatenate([[0], np.cumsum(deg)]).astype(np.int32)
    ci = np.zeros(int(rp[-1]), np.int32)
    assert autotune.graph_key(rp, ci).endswith("flat")


def test_resolve_maps_grid_size_codes():
    """ctas = -1 is one CTA per SM, -2 half the SMs (at least one); other
    values pass through."""
    from paper_2209_08764_gb300 import autotune
    assert autotune.resolve({"ctas": -1}, 152)["ctas"] == 152
    assert autotune.resolve({"ctas": -2}, 152)["ctas"] == 76
    assert autotune.resolve({"ctas": -2}, 1)["ctas"] == 1
    assert autotune.resolve({"ctas": 0, "chunk_edges": 32}, 152) == {"ctas": 0, "chunk_edges": 32}
