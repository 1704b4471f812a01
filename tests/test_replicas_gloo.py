"""The N>1 path of the benchmark (independent replicas, max time over ranks,
total work of all ranks), on two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    import graphgen
    from paper_2209_08764_gb300 import replicas
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        ms, units = replicas.aggregate(dist, 10.0 + 5.0 * rank, 100 * (rank + 1))
        rp, _ = graphgen.rmat(10, 16, seed=1)
        srcs = graphgen.sample_sources(rp, 8, seed=replicas.rank_source_seed(2, rank))
        out[rank] = (ms, units, tuple(int(x) for x in srcs))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_aggregate():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0][:2] == (15.0, 300.0) and out[1][:2] == (15.0, 300.0)
    assert out[0][2] != out[1][2]           # each replica has its own sources


def test_single_process_aggregate():
    from paper_2209_08764_gb300 import replicas
    assert replicas.aggregate(None, 3.5, 7) == (3.5, 7.0)
