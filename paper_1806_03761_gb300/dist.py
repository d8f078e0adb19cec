"""Host-side logic of the multi-rank run (one process per GPU).

Chains are independent (PEPS++ Sec. "Process-level parallelism"): rank r runs
chains r*B .. r*B+B-1, so the counter-based Philox streams of different ranks
never overlap.  The GO update's one exchange is the sum of the gradient
accumulators (sum_delta, sum_delta_e, sum_e) over ranks; every rank then
applies the identical sign update (its random step lengths come from the same
counter-based generator, so no broadcast is needed)."""


def shard(rank, world, chains_per_rank):
    """(first chain index, number of chains) of a rank."""
    if not (0 <= rank < world) or chains_per_rank < 0:
        raise ValueError("bad rank/world/chains")
    return rank * chains_per_rank, chains_per_rank


def weak_scaling_plan(rank, world, chains_per_rank):
    """The weak-scaling layout of a VMC step: every rank keeps the same
    number of chains B as the world grows.  Returns (chain offset of this
    rank, chains of this rank, M) with M = B * world the number of samples
    the all-reduced gradient sums cover (the Monte Carlo mean of Eq.
    gradients divides by M)."""
    off, n = shard(rank, world, chains_per_rank)
    return off, n, chains_per_rank * world


def allreduce_sums(sums, world):
    """Sum the gradient accumulators over ranks in place (no-op for one rank)."""
    if world == 1:
        return sums
    import torch.distributed as dist
    for t in sums:
        dist.all_reduce(t)
    return sums
