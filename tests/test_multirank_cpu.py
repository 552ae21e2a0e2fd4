"""The multi-rank path of bench.py (weak scaling: one independent matrix per rank, timing
reduced by max over ranks) on CPU with the gloo backend, world size 2."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    seed = bench.rank_seed(rank)
    t = bench.max_over_ranks(1.0 + rank)
    bench.barrier()
    out[rank] = (seed, t)
    dist.destroy_process_group()


def test_weak_scaling_helpers_gloo():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    seeds = sorted(v[0] for v in out.values())
    assert seeds == [0, 1]  # distinct matrices per rank, no shared work
    assert all(v[1] == 2.0 for v in out.values())  # max over ranks seen by both


def test_single_rank_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert bench.dist_env()[1] >= 1
