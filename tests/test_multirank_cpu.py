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


def _range_worker(rank, world, port, out):
    """Each rank takes its contiguous range of the enumeration (range_bounds), evaluates the
    subset terms there with the CPU oracle, forms its compensated partial, and the partials
    are exchanged over gloo; every rank combines them with the library's host-side sum."""
    import numpy as np
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import lhaf as L
    from paper_2010_15595_gb300 import lib, workloads as W
    A = W.single_lhaf_n16()
    N = A.shape[0]
    n = N // 2
    i0, i1 = lib.range_bounds(N, rank, world)
    idx = np.arange(i0, i1, dtype=np.uint64)
    z = idx ^ (idx >> np.uint64(1))
    pz = L.subset_terms(A, z, nthreads=1)
    sgn = np.where(((n - np.array([bin(int(v)).count("1") for v in z])) & 1) == 1, -1.0, 1.0)
    terms = sgn * pz
    # compensated local partial (TwoSum on the high words)
    hi_r = lo_r = hi_i = lo_i = 0.0
    for t in terms:
        for which in (0, 1):
            x = t.real if which == 0 else t.imag
            hi, lo = (hi_r, lo_r) if which == 0 else (hi_i, lo_i)
            s = hi + x
            bb = s - hi
            e = (hi - (s - bb)) + (x - bb)
            if which == 0:
                hi_r, lo_r = s, lo + e
            else:
                hi_i, lo_i = s, lo + e
    mine = torch.tensor([hi_r, lo_r, hi_i, lo_i, float(np.abs(terms.real).sum() + np.abs(terms.imag).sum())],
                        dtype=torch.float64)
    gathered = [torch.zeros(5, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(gathered, mine)
    comb = lib.combine_partials(np.stack([g.numpy() for g in gathered]))
    out[rank] = (i0, i1, lib.partial_value(comb))
    dist.destroy_process_group()


def test_subset_range_split_gloo():
    """World size 2 on CPU: a loop hafnian split into two enumeration ranges, one per rank,
    combined after one exchange of 5 doubles per rank, equals the single evaluation."""
    from oracle import lhaf as L
    from paper_2010_15595_gb300 import workloads as W
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_range_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=180)
        assert p.exitcode == 0
    bounds = sorted((v[0], v[1]) for v in out.values())
    assert bounds == [(0, 128), (128, 256)]
    ref = L.lhaf_subset(W.single_lhaf_n16())
    for v in out.values():
        assert abs(v[2] - ref) <= 1e-12 * abs(ref)
