"""Query server (continuous batching) against the oracle and against the same
queries run alone (GPU only).

Every result must be the same alone and in the mix: levels bit-exact with the
oracle and with bfs_run on the same graph; parents a valid BFS tree.
"""
import numpy as np
import pytest

import graphgen
import oracle
from gpu_helpers import make_opts
from paper_2209_08764_gb300 import binding as B

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    import paper_2209_08764_gb300 as pkg
    pkg.build()
    B.load()


def _pool():
    n_path = 3000
    return [
        ("rmat12", *graphgen.rmat(12, 16, seed=5), 0),
        ("rmat14_relabel", *graphgen.rmat(14, 16, seed=6), 1),
        ("er", *graphgen.erdos_renyi(1 << 13, 1 << 15, seed=4), 0),
        ("grid", *graphgen.grid(64, 48, 0.02, seed=3), 0),
        ("path", *graphgen.from_edges(n_path, [(i, i + 1) for i in range(n_path - 1)]), 0),
        ("star", *graphgen.from_edges(2001, [(0, j) for j in range(1, 2001)]), 0),
    ]


def _make(pool):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    handles = []
    for name, rp, ci, relabel in pool:
        handles.append(B.bfs_create_csr(len(rp) - 1, len(ci), rp, ci, B.BFS_VALIDATE,
                                        make_opts(relabel=relabel) if relabel else None, stream))
    return handles


def _drain(s, expect):
    got = {}
    for _ in range(100000):
        for c in B.bfs_server_poll(s, 64):
            got[c.tag] = c
        q, r = B.bfs_server_pending(s)
        if q == 0 and r == 0 and len(got) >= expect:
            break
    assert len(got) == expect, f"{len(got)} of {expect} completions"
    return got


@pytest.mark.parametrize("opts", [dict(), dict(slots=2), dict(levels_per_launch=1), dict(cta_warps=32), dict(cta_warps=8),
                                  dict(slots=5, levels_per_launch=3, chunk_edges=7), dict(local_levels=8),
                                  dict(local_levels=64), dict(local_levels=3, cta_warps=32, slots=3)],
                         ids=lambda o: ",".join(f"{k}={v}" for k, v in o.items()) or "default")
def test_mix_equals_alone_and_oracle(opts):
    import torch
    pool = _pool()
    handles = _make(pool)
    so = B.bfs_server_opts()
    for k, v in opts.items():
        setattr(so, k, v)
    s = B.bfs_server_create(handles, so, torch.cuda.current_stream().cuda_stream)
    try:
        rng = np.random.default_rng(1)
        queries = []
        done = {}
        for t in range(40):
            gi = int(rng.integers(len(pool)))
            rp = pool[gi][1]
            src = int(graphgen.sample_sources(rp, 1, seed=100 + t)[0])
            n = len(rp) - 1
            lv = torch.empty(n, dtype=torch.int32, device="cuda")
            pa = torch.empty(n, dtype=torch.int32, device="cuda")
            B.bfs_server_submit(s, gi, src, lv, pa, t)
            queries.append((gi, src, lv, pa))
            if t % 7 == 3:  # arrivals interleaved with running work
                for c in B.bfs_server_poll(s, 64):
                    done[c.tag] = c
        done.update(_drain(s, len(queries) - len(done)))
        assert sorted(done) == list(range(len(queries)))
        orcs = [oracle.Oracle(rp, ci) for _, rp, ci, _ in pool]
        for t, (gi, src, lv, pa) in enumerate(queries):
            name, rp, ci, _ = pool[gi]
            assert done[t].status == 0, (t, done[t].status)
            want, _ = orcs[gi].bfs(src)
            L = lv.cpu().numpy()
            assert np.array_equal(L, want), f"query {t} on {name}: levels differ from the oracle"
            oracle.check_bfs_tree(rp, ci, src, L, pa.cpu().numpy())
            # the same query alone through bfs_run
            lv1 = torch.empty_like(lv)
            B.bfs_run(handles[gi], src, lv1, None, None)
            assert torch.equal(lv1, lv), f"query {t}: alone != in the mix"
    finally:
        B.bfs_server_destroy(s)
        for h in handles:
            B.bfs_destroy(h)


def test_completion_records_host_outputs_and_discarded():
    import torch
    pool = _pool()
    handles = _make(pool)
    s = B.bfs_server_create(handles, None, torch.cuda.current_stream().cuda_stream)
    try:
        subs = {}
        for t, gi in enumerate([0, 1, 2, 3, 4, 5, 1, 0]):
            rp, ci = pool[gi][1], pool[gi][2]
            src = int(graphgen.sample_sources(rp, 1, seed=7 + t)[0])
            n = len(rp) - 1
            if t % 2 == 0:
                lv = np.full(n, 9, np.int32)
                pa = np.full(n, 9, np.int32)
                B.bfs_server_submit(s, gi, src, lv, pa, t)
            else:
                lv = pa = None
                B.bfs_server_submit(s, gi, src, None, None, t)
            subs[t] = (gi, src, lv, pa)
        done = _drain(s, len(subs))
        for t, (gi, src, lv, pa) in subs.items():
            name, rp, ci, _ = pool[gi]
            c = done[t]
            assert c.status == 0 and c.graph == gi and c.src == src
            want, _ = oracle.bfs(rp, ci, src)
            n_l, e_l = oracle.level_profile(rp, want)
            assert c.num_levels == len(n_l) and c.reached == int(n_l.sum()) and c.edges_scanned == int(e_l.sum())
            assert c.t_submit_us <= c.t_admit_us <= c.t_done_us
            if lv is not None:
                assert np.array_equal(lv, want)
                oracle.check_bfs_tree(rp, ci, src, lv, pa)
    finally:
        B.bfs_server_destroy(s)
        for h in handles:
            B.bfs_destroy(h)


def test_admission_waits_for_memory_and_rejects_oversize():
    import torch
    pool = _pool()
    handles = _make(pool)
    so = B.bfs_server_opts()
    so.arena_bytes = 3 << 20   # fits one or two small queries at a time, not the 16k-vertex graph
    s = B.bfs_server_create(handles, so, torch.cuda.current_stream().cuda_stream)
    try:
        outs = {}
        for t, gi in enumerate([0, 2, 3, 4, 5, 0, 3, 1]):
            rp = pool[gi][1]
            src = int(graphgen.sample_sources(rp, 1, seed=t)[0])
            lv = torch.empty(len(rp) - 1, dtype=torch.int32, device="cuda")
            B.bfs_server_submit(s, gi, src, lv, None, t)
            outs[t] = (gi, src, lv)
        done = _drain(s, len(outs))
        for t, (gi, src, lv) in outs.items():
            name, rp, ci, _ = pool[gi]
            if name == "rmat14_relabel":
                assert done[t].status == B.BFS_E_NOMEM
                continue
            assert done[t].status == 0
            want, _ = oracle.bfs(rp, ci, src)
            assert np.array_equal(lv.cpu().numpy(), want)
    finally:
        B.bfs_server_destroy(s)
        for h in handles:
            B.bfs_destroy(h)


def test_bad_submissions():
    import torch
    pool = _pool()[:1]
    handles = _make(pool)
    s = B.bfs_server_create(handles, None, torch.cuda.current_stream().cuda_stream)
    try:
        with pytest.raises(B.BFSError):
            B.bfs_server_submit(s, 1, 0)
        with pytest.raises(B.BFSError):
            B.bfs_server_submit(s, 0, len(pool[0][1]))
        assert B.bfs_server_poll(s) == []
    finally:
        B.bfs_server_destroy(s)
        for h in handles:
            B.bfs_destroy(h)


def test_submissions_from_another_thread_while_polling():
    """A client thread submits while this thread polls (the poll holds no lock
    while its launch runs; a submission wakes the launch): every result still
    equals the oracle's."""
    import threading
    import time

    import torch
    pool = _pool()
    handles = _make(pool)
    so = B.bfs_server_opts()
    so.levels_per_launch = 1 << 20  # only completions and wake-ups end a launch
    s = B.bfs_server_create(handles, so, torch.cuda.current_stream().cuda_stream)
    try:
        rng = np.random.default_rng(3)
        subs = []
        for t in range(30):
            gi = int(rng.integers(len(pool)))
            rp = pool[gi][1]
            subs.append((gi, int(graphgen.sample_sources(rp, 1, seed=300 + t)[0])))
        outs = {t: np.full(len(pool[gi][1]) - 1, 5, np.int32) for t, (gi, _) in enumerate(subs)}

        def client():
            for t, (gi, src) in enumerate(subs):
                B.bfs_server_submit(s, gi, src, outs[t], None, t)
                time.sleep(0.0005)

        th = threading.Thread(target=client)
        th.start()
        got = {}
        t_end = time.time() + 120
        while len(got) < len(subs) and time.time() < t_end:
            for c in B.bfs_server_poll(s, 64):
                got[c.tag] = c
            if th.is_alive() or B.bfs_server_pending(s) != (0, 0):
                time.sleep(0.0001)
        th.join()
        assert sorted(got) == list(range(len(subs)))
        for t, (gi, src) in enumerate(subs):
            name, rp, ci, _ = pool[gi]
            assert got[t].status == 0
            want, _ = oracle.bfs(rp, ci, src)
            assert np.array_equal(outs[t], want), f"query {t} on {name}"
    finally:
        B.bfs_server_destroy(s)
        for h in handles:
            B.bfs_destroy(h)
