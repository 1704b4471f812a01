"""The direction-switching rule of the direction-optimising traversal, as the
tests restate it (CPU): the pattern it gives on known level profiles.  The
GPU tests then check that the device chose, level by level, exactly the
directions this restatement gives on the oracle's profile."""
import numpy as np

import graphgen
import oracle
from gpu_helpers import expected_directions


def _profile(rp, ci, s):
    lv, _ = oracle.bfs(rp, ci, s)
    return oracle.level_profile(rp, lv)


def test_rmat_goes_bottom_up_in_the_middle_and_back():
    rp, ci = graphgen.rmat(16, 16, seed=1)
    s = int(graphgen.sample_sources(rp, 1, seed=2)[0])
    n_l, e_l = _profile(rp, ci, s)
    d = expected_directions(len(rp) - 1, len(ci), n_l, e_l, 1, 15, 18)
    assert d[0] == 0 and d.max() == 1 and d[-1] == 0
    # once bottom-up, a level stays so while its frontier grows
    for l in range(1, len(d)):
        if d[l - 1] == 1 and n_l[l] >= n_l[l - 1]:
            assert d[l] == 1


def test_off_means_top_down_everywhere():
    rp, ci = graphgen.rmat(12, 16, seed=1)
    n_l, e_l = _profile(rp, ci, 0)
    assert not expected_directions(len(rp) - 1, len(ci), n_l, e_l, 0, 15, 18).any()


def test_path_turns_bottom_up_only_at_its_end():
    # a path from one end: the frontier always has 2 edges, so it turns
    # bottom-up only once the unvisited part holds fewer than 2 * alpha = 30
    # edge entries, i.e. for its last 15 or so levels
    rp, ci = graphgen.from_edges(200, [(i, i + 1) for i in range(199)])
    n_l, e_l = _profile(rp, ci, 0)
    d = expected_directions(200, len(ci), n_l, e_l, 1, 15, 18)
    first = int(np.nonzero(d)[0][0])
    unvisited = len(ci) - np.cumsum(e_l)
    assert 2 * 15 > unvisited[first] and 2 * 15 <= unvisited[first - 1]
    assert d[first:].all()


def test_rule_by_hand_on_a_small_profile():
    # n = 100, nnz = 400; profile chosen so each branch of the rule fires once
    n_l = np.array([1, 10, 60, 20, 5])
    e_l = np.array([10, 40, 300, 40, 10])
    d = expected_directions(100, 400, n_l, e_l, 1, alpha=2, beta=10)
    # level 1: 40 * 2 = 80 > 400 - 50 = 350?  no -> 0
    # level 2: 300 * 2 = 600 > 400 - 350 = 50 -> 1
    # level 3: bottom-up; 20 * 10 = 200 < 100?  no -> stays 1
    # level 4: 5 * 10 = 50 < 100 and 5 < 20 -> 0
    assert d.tolist() == [0, 0, 1, 1, 0]


def test_gamma_keeps_a_sparse_frontier_top_down():
    # Erdős–Rényi: a level with a small frontier among many unvisited vertices
    # passes Beamer's alpha test but not the unvisited-vertex test, and stays
    # top-down; the dense middle level still turns bottom-up
    rp, ci = graphgen.erdos_renyi(1 << 14, 1 << 17, seed=4)
    s = int(graphgen.sample_sources(rp, 1, seed=2)[0])
    n_l, e_l = _profile(rp, ci, s)
    n = len(rp) - 1
    live = int((np.diff(rp) > 0).sum())
    beamer = expected_directions(n, len(ci), n_l, e_l, 1, 15, 18, gamma=0, n_live=live)
    gpu = expected_directions(n, len(ci), n_l, e_l, 1, 15, 18, gamma=2, n_live=live)
    assert gpu.sum() <= beamer.sum() and gpu.max() == 1
    first_b, first_g = int(np.argmax(beamer)), int(np.argmax(gpu))
    assert first_g >= first_b
