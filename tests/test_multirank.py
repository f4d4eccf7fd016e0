"""The multi-rank path on CPU: two gloo ranks each evaluate their contiguous
block of points (with the oracle as the per-rank compute, since the CPU has no
GPU) and the gathered result equals the single-process result bit for bit;
the timing reduction takes the MAX over ranks."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1903_04670_gb300 import distributed as D


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, P, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    from paper_1903_04670_gb300 import workloads as W

    O.set_threads(1)
    pb = W.make_problem("c1_homog_n16", points=P)
    pb["N"], pb["L"] = 16, 8.0
    lo, hi = D.shard_range(P, rank, world)
    prob = O.Problem(pb["N"], pb["L"], pb["M"], 2, pb["masses"], pb["pairs"])
    Q = prob.collide_all(pb["f"], points=list(range(lo, hi)))
    full = D.gather_shards(torch.from_numpy(np.ascontiguousarray(Q)), P, rank, world)
    tmax = D.max_over_ranks(float(rank + 1))
    if rank == 0:
        torch.save({"Q": full, "tmax": tmax}, out_path)
    dist.barrier()
    dist.destroy_process_group()


def test_shard_range_partitions_points():
    for P in (1, 5, 24, 128):
        for world in (1, 2, 3, 8):
            spans = [D.shard_range(P, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == P
            for (a, b), (c, d) in zip(spans, spans[1:]):
                assert b == c
            sizes = [b - a for a, b in spans]
            assert max(sizes) - min(sizes) <= 1


def test_two_gloo_ranks_equal_single_process(tmp_path):
    P, world = 3, 2
    out = str(tmp_path / "q.pt")
    mp.start_processes(_worker, args=(world, _free_port(), P, out), nprocs=world, join=True, start_method="spawn")
    res = torch.load(out)
    import oracle as O
    from paper_1903_04670_gb300 import workloads as W

    pb = W.make_problem("c1_homog_n16", points=P)
    prob = O.Problem(16, 8.0, pb["M"], 2, pb["masses"], pb["pairs"])
    ref = prob.collide_all(pb["f"])
    assert res["tmax"] == 2.0
    assert np.array_equal(res["Q"].numpy(), ref)
