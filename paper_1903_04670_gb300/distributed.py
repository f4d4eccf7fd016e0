"""Point sharding across ranks.

Every (point, pair) evaluation of the collision operator is independent
(the operator acts in velocity space only, Sec. 2.1), so a multi-rank run
splits the spatial points into contiguous blocks, one per rank, with no
collective on the data path; the read-only tables are built on every rank.
This mirrors the paper's linear domain decomposition of spatial elements
(Sec. 3.3.2) without its trace exchange, which belongs to the DG streaming
term, not to the operator.  Collectives are used only for timing (MAX over
ranks), optionally for gathering results, and in the sharded adjoint for the
omega gradient, a sum over all points.
"""
import torch
import torch.distributed as dist


def shard_range(P, rank, world):
    """Contiguous block [lo, hi) of P points for `rank` of `world` (sizes differ by at most 1)."""
    base, extra = divmod(int(P), int(world))
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return lo, hi


def max_over_ranks(value, device=None):
    """MAX of a scalar over all ranks (identity without an initialised process group)."""
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_shards(local, P, rank, world):
    """Reassemble per-rank point blocks (leading dimension = points) into the
    full [P, ...] tensor on every rank."""
    if world == 1:
        return local
    lo, hi = shard_range(P, rank, world)
    assert local.shape[0] == hi - lo
    width = -(-P // world)
    pad = torch.zeros((width,) + tuple(local.shape[1:]), dtype=local.dtype, device=local.device)
    pad[: hi - lo] = local
    parts = [torch.empty_like(pad) for _ in range(world)]
    dist.all_gather(parts, pad)
    out = []
    for r in range(world):
        a, b = shard_range(P, r, world)
        out.append(parts[r][: b - a])
    return torch.cat(out, dim=0)



def backward_sharded(backward, f_local, dQ_local):
    """Adjoint of a point-sharded collision call.

    backward(f, dQ) -> (df, domega) is a plan's backward (binding.Plan.backward)
    or anything with its contract.  Each rank runs it on its own block of
    points: df stays with the rank (it has the rank's points), while
    dL/d omega_pq, a sum over all points of the bilinear map's omega
    derivative, is summed over the ranks (one all_reduce of S*S values, the
    only collective of the sharded adjoint)."""
    df, dom = backward(f_local, dQ_local)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(dom, op=dist.ReduceOp.SUM)
    return df, dom

# ------------------------------------------------- DG slab split over ranks
def element_range(Ne, rank, world):
    """Contiguous block [e0, e1) of the Ne DG elements owned by `rank` (DG
    elements stay whole, so the split is over elements, not points)."""
    return shard_range(Ne, rank, world)


def exchange_traces(left, right, rank, world):
    """Trace halo exchange at the interfaces between neighbouring ranks.

    left / right: this rank's boundary traces (its first element at its left
    face, its last element at its right face), tensors of equal shape.  The
    left trace goes to rank - 1, the right trace to rank + 1.  Returns
    (halo_left, halo_right): the left neighbour's right trace and the right
    neighbour's left trace, None at the ends of the domain (the walls).  This
    is the only exchange of the decomposed DG step: O(S N^3) values per
    interface (the paper's linear domain decomposition, Sec. 3.3)."""
    if world == 1:
        return None, None
    halo_left = torch.empty_like(right) if rank > 0 else None
    halo_right = torch.empty_like(left) if rank < world - 1 else None
    ops = []
    if rank > 0:
        ops.append(dist.P2POp(dist.isend, left.contiguous(), rank - 1))
        ops.append(dist.P2POp(dist.irecv, halo_left, rank - 1))
    if rank < world - 1:
        ops.append(dist.P2POp(dist.isend, right.contiguous(), rank + 1))
        ops.append(dist.P2POp(dist.irecv, halo_right, rank + 1))
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    return halo_left, halo_right


# SSP-RK3 in Shu-Osher form: (input, f0 weight a0, weight a1), stage 0 reads f
SSP_RK3 = ((0, 0.0, 1.0), (1, 0.75, 0.25), (2, 1.0 / 3.0, 2.0 / 3.0))


def dg_step_decomposed(slab, f, dt, with_collisions=True, rank=0, world=1, work=None):
    """One SSP-RK3 step of this rank's block of elements, exchanging boundary
    traces before every stage.  slab: binding.Slab over the rank's own
    elements (walls of the global domain at the global ends); f: its
    [P_local][S][N][N][N] tensor, updated in place.  work: optional pair of
    stage buffers shaped like f."""
    f1, f2 = work if work is not None else (torch.empty_like(f), torch.empty_like(f))
    bufs = (f, f1, f2)
    outs = (f1, f2, f)
    for k, (src, a0, a1) in enumerate(SSP_RK3):
        fin = bufs[src]
        left, right = slab.traces(fin)
        hl, hr = exchange_traces(left, right, rank, world)
        slab.stage(fin, f if a0 != 0.0 else None, outs[k], a0, a1, dt, with_collisions, hl, hr)
    return f
