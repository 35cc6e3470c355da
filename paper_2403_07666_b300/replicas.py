"""Replicas across GPUs: one independent coil (or share of a coil batch) per
rank, no collective on the data path (the solve of one coil does not shard:
every PCG iteration would need the whole search vector on every rank).

Only the measurement is combined: the job's time is the slowest rank's, its
work the sum over ranks.  Coil batches are dealt to ranks by element count.
"""


def shard_coils(sizes, world, rank):
    """Indices of the coils of a batch that rank `rank` of `world` steps.

    Greedy longest-first: each coil, largest first (ties by index), goes to the
    rank with the fewest elements so far (ties to the lower rank), so every
    rank gets a share within one coil of the mean; deterministic on every rank.
    """
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank outside the world")
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    load = [0] * world
    mine = []
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        load[r] += int(sizes[i])
        if r == rank:
            mine.append(i)
    return sorted(mine)


def job_throughput(local_secs, local_units, dist=None, device=None):
    """(units per second of the whole job, the job's seconds): the units all
    ranks processed over the slowest rank's time (max over ranks)."""
    if dist is None:
        return local_units / local_secs, local_secs
    import torch
    t = torch.tensor([float(local_secs)], dtype=torch.float64, device=device)
    u = torch.tensor([float(local_units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    secs = float(t.item())
    return float(u.item()) / secs, secs
