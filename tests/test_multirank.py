"""The multi-rank paths on CPU: gloo ranks each evaluate their contiguous
block of points (with the oracle as the per-rank compute, since the CPU has no
GPU) and the gathered result equals the single-process result bit for bit;
the timing reduction takes the MAX over ranks; the sharded adjoint keeps df per
rank and sums dL/d omega over the ranks; a DG slab split over ranks with the
trace halo exchange steps exactly like the undivided slab."""
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



ADJ = dict(N=8, L=4.0, M=6, Nrho=2, masses=(1.0, 2.0), P=5)


def _adj_inputs():
    from paper_1903_04670_gb300 import workloads as W
    rng = np.random.default_rng(21)
    S, N, P = len(ADJ["masses"]), ADJ["N"], ADJ["P"]
    pairs = W.pair_params([0.72, 0.8], [1.0, 1.0], [1.0, 1.1])
    f = rng.uniform(0.1, 1.0, size=(P, S, N, N, N))
    g = rng.normal(size=(P, S, S, N, N, N))
    return pairs, f, g


def _oracle_backward(prob, S):
    """A backward with the plan's contract, computed by the oracle (the CPU has no GPU)."""
    def run(f, g):
        f, g = f.numpy(), g.numpy()
        df = np.zeros_like(f)
        dom = np.zeros(S * S)
        for pt in range(f.shape[0]):
            for p in range(S):
                for q in range(S):
                    dp, dq, dw = prob.pair(p, q).adjoint(f[pt, p], f[pt, q], g[pt, p, q])
                    df[pt, p] += dp
                    df[pt, q] += dq
                    dom[p * S + q] += dw
        return torch.from_numpy(df), torch.from_numpy(dom)
    return run


def _adj_worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    O.set_threads(1)
    pairs, f, g = _adj_inputs()
    S = len(ADJ["masses"])
    prob = O.Problem(ADJ["N"], ADJ["L"], ADJ["M"], ADJ["Nrho"], ADJ["masses"], pairs)
    lo, hi = D.shard_range(ADJ["P"], rank, world)
    df, dom = D.backward_sharded(_oracle_backward(prob, S), torch.from_numpy(f[lo:hi].copy()),
                                 torch.from_numpy(g[lo:hi].copy()))
    full = D.gather_shards(df, ADJ["P"], rank, world)
    if rank == 0:
        torch.save({"df": full, "dom": dom}, out_path)
    dist.barrier()
    dist.destroy_process_group()


def test_sharded_adjoint_sums_omega_gradient_over_ranks(tmp_path):
    out = str(tmp_path / "adj.pt")
    mp.start_processes(_adj_worker, args=(2, _free_port(), out), nprocs=2, join=True, start_method="spawn")
    res = torch.load(out)
    import oracle as O
    pairs, f, g = _adj_inputs()
    S = len(ADJ["masses"])
    prob = O.Problem(ADJ["N"], ADJ["L"], ADJ["M"], ADJ["Nrho"], ADJ["masses"], pairs)
    df, dom = D.backward_sharded(_oracle_backward(prob, S), torch.from_numpy(f), torch.from_numpy(g))
    # df: the same per-point values, gathered; d omega: the two ranks' partial sums
    assert torch.equal(res["df"], df)
    assert float((res["dom"] - dom).abs().max()) <= 1e-13 * float(dom.abs().max())

class _OracleBlock:
    """The operations dg_step_decomposed needs from a slab, done by the DG
    oracle on this rank's block of elements (CPU stand-in for binding.Slab)."""

    def __init__(self, ref):
        self.ref = ref

    def traces(self, f):
        l, r = self.ref.traces(f.reshape(f.shape[0], f.shape[1], -1).numpy())
        return torch.from_numpy(l), torch.from_numpy(r)

    def stage(self, fin, f0, out, a0, a1, dt, with_collisions, hl, hr):
        g = fin.reshape(fin.shape[0], fin.shape[1], -1).numpy()
        r = self.ref.streaming(g, None if hl is None else hl.numpy(), None if hr is None else hr.numpy())
        new = g + dt * r
        if a0 != 0.0:
            new = a0 * f0.reshape(new.shape).numpy() + a1 * new
        else:
            new = a1 * new
        out.copy_(torch.from_numpy(new).reshape(out.shape))
        return out


WALLS = ((1.0, (0.0, -0.2, 0.0)), (2.0, (0.0, 0.2, 0.0)))
SLAB = dict(Ne=5, K=3, N=6, L=4.0, masses=(1.0, 2.0))


def _slab_f():
    rng = np.random.default_rng(11)
    P = SLAB["Ne"] * SLAB["K"]
    return rng.uniform(0.1, 1.0, size=(P, len(SLAB["masses"]), SLAB["N"], SLAB["N"], SLAB["N"]))


def _dg_worker(rank, world, port, out_path):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from oracle import dg as ODG

    Ne, K = SLAB["Ne"], SLAB["K"]
    e0, e1 = D.element_range(Ne, rank, world)
    he = 1.0 / Ne
    ref = ODG.Slab(e1 - e0, K, e0 * he, e1 * he, SLAB["N"], SLAB["L"], SLAB["masses"], WALLS)
    f = torch.from_numpy(_slab_f()[e0 * K:e1 * K].copy())
    D.dg_step_decomposed(_OracleBlock(ref), f, 0.004, with_collisions=False, rank=rank, world=world)
    parts = [None] * world
    dist.all_gather_object(parts, (e0, f.numpy()))
    if rank == 0:
        torch.save(parts, out_path)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_decomposed_dg_step_equals_single_slab(tmp_path, world):
    """Elements split over gloo ranks, boundary traces exchanged before every
    SSP-RK3 stage: the same result as the undivided slab."""
    from oracle import dg as ODG

    out = str(tmp_path / "dg.pt")
    mp.start_processes(_dg_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
    parts = sorted(torch.load(out, weights_only=False), key=lambda t: t[0])
    got = np.concatenate([p[1] for p in parts])
    ref = ODG.Slab(SLAB["Ne"], SLAB["K"], 0.0, 1.0, SLAB["N"], SLAB["L"], SLAB["masses"], WALLS)
    f = _slab_f()
    want = ref.ssp_rk3(f.reshape(f.shape[0], f.shape[1], -1), 0.004).reshape(f.shape)
    assert np.abs(got - want).max() <= 1e-14 * np.abs(want).max()


def test_element_range_keeps_elements_whole():
    for Ne in (1, 4, 5, 16):
        for world in (1, 2, 3):
            spans = [D.element_range(Ne, r, world) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == Ne
            assert all(b == c for (_, b), (c, _) in zip(spans, spans[1:]))


def _failing_worker(rank, world, port, out_path):
    """Rank 1 raises between two decomposed DG steps (none of its work in
    flight); rank 0 goes on to its next step and must get an error from the
    trace exchange within the process group's short timeout instead of
    waiting forever."""
    import datetime
    import time

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=5))
    from oracle import dg as ODG

    Ne, K = SLAB["Ne"], SLAB["K"]
    e0, e1 = D.element_range(Ne, rank, world)
    he = 1.0 / Ne
    ref = ODG.Slab(e1 - e0, K, e0 * he, e1 * he, SLAB["N"], SLAB["L"], SLAB["masses"], WALLS)
    f = torch.from_numpy(_slab_f()[e0 * K:e1 * K].copy())
    D.dg_step_decomposed(_OracleBlock(ref), f, 0.004, with_collisions=False, rank=rank, world=world)
    if rank == 1:
        raise RuntimeError("injected failure of rank 1 between steps")
    t0 = time.monotonic()
    try:
        D.dg_step_decomposed(_OracleBlock(ref), f, 0.004, with_collisions=False, rank=rank, world=world)
        res = {"error": None}
    except Exception as e:  # the exchange with the dead neighbour fails
        res = {"error": type(e).__name__ + ": " + str(e)[:200]}
    res["seconds"] = time.monotonic() - t0
    torch.save(res, out_path)


def test_rank_failure_between_steps_surfaces_as_an_error(tmp_path):
    import multiprocessing

    out = str(tmp_path / "fail.pt")
    port = _free_port()
    ctx = multiprocessing.get_context("spawn")
    procs = [ctx.Process(target=_failing_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
    alive = [p.is_alive() for p in procs]
    for p in procs:
        if p.is_alive():
            p.kill()
    assert not any(alive), "a rank hung after its neighbour failed"
    assert procs[1].exitcode != 0  # the failing rank
    assert procs[0].exitcode == 0
    res = torch.load(out)
    assert res["error"] is not None, "rank 0 completed a step with a dead neighbour"
    assert res["seconds"] < 30.0, res
