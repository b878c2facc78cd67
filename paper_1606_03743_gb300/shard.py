"""Field-point sharding over ranks (one process per GPU).

phi and E at a field point are a sum over all elements that depends on that
point and the mesh alone (Eq. 4.1 summed over the elements, Sec. 5), so the
points split across ranks with no exchange on the data path: every rank holds
the whole mesh and evaluates its own points.  The only collective is the
host-side reduction of step times (the slowest rank sets the job's time).
"""
from __future__ import annotations


def point_range(n: int, rank: int, world: int) -> tuple[int, int]:
    """[start, stop) of rank's contiguous share of n points; shares differ by
    at most one point and cover 0..n exactly once."""
    if world < 1 or not 0 <= rank < world or n < 0:
        raise ValueError(f"bad shard request n={n} rank={rank} world={world}")
    base, extra = divmod(n, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def rank_seed(seed: int, rank: int) -> int:
    """Seed of rank's own batch when every rank generates its own points
    (weak scaling: the per-rank batch stays fixed as ranks are added)."""
    return seed + 1000 * rank


def slowest_rank_ms(ms: float, dist=None, device=None) -> float:
    """Maximum of ms over all ranks of the default process group (ms itself
    when dist is None).  device: where the reduction tensor lives ('cpu' for
    gloo, the rank's CUDA device for nccl)."""
    if dist is None:
        return float(ms)
    import torch

    t = torch.tensor([float(ms)], dtype=torch.float64, device=device or "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_all_ranks: float, slowest_ms: float) -> float:
    """Whole-job throughput: units processed by all ranks / the slowest rank's time."""
    if slowest_ms <= 0:
        raise ValueError("non-positive time")
    return units_all_ranks / (slowest_ms * 1e-3)
