"""Replica coordination for runs under torchrun: one process per GPU, each
running a whole independent copy of the workload (the method has no exchange
step between copies).  The job's time is the slowest rank's, and its
throughput counts the work of every rank.  Only host-side arithmetic on
already-measured times happens here."""


def max_over_ranks(dist, x, device="cpu"):
    """The largest x over all ranks (x itself without a process group)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(dist, units_per_rank, seconds, device="cpu"):
    """Units per second of the whole job: world * units_per_rank over the
    slowest rank's time."""
    world = dist.get_world_size() if dist is not None else 1
    return world * units_per_rank / max_over_ranks(dist, seconds, device)
