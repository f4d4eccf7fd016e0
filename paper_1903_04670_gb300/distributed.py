"""Point sharding across ranks.

Every (point, pair) evaluation of the collision operator is independent
(the operator acts in velocity space only, Sec. 2.1), so a multi-rank run
splits the spatial points into contiguous blocks, one per rank, with no
collective on the data path; the read-only tables are built on every rank.
This mirrors the paper's linear domain decomposition of spatial elements
(Sec. 3.3.2) without its trace exchange, which belongs to the DG streaming
term, not to the operator.  Collectives are used only for timing (MAX over
ranks) and, optionally, for gathering results.
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
