"""Host logic of multi-GPU runs: one process per GPU, independent replicas.

The evaluation of one tree does not shard across GPUs here (every GPU holds
its own tree, no data-path collective); what is distributed is work made of
independent units: charge sets of a batch, or whole replicas of a workload.
These helpers assign units to ranks and combine per-rank timings, and are
backend-agnostic (tested with gloo on the CPU).
"""
import torch
import torch.distributed as dist


def shard_sets(sizes, rank, world):
    """Indices of the charge sets rank `rank` evaluates: sets sorted by size,
    largest first, each given to the rank with the least work so far (ties:
    lowest rank).  Deterministic, so every rank computes the same assignment."""
    order = sorted(range(len(sizes)), key=lambda i: (-int(sizes[i]), i))
    load = [0] * world
    owner = [0] * len(sizes)
    for i in order:
        r = min(range(world), key=lambda k: (load[k], k))
        owner[i] = r
        load[r] += int(sizes[i])
    return [i for i in range(len(sizes)) if owner[i] == rank]


def max_over_ranks(x, device=None):
    """Maximum of a per-rank float over all ranks (x itself without a group)."""
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, device=None):
    """Sum of a per-rank number over all ranks (x itself without a group)."""
    if not (dist.is_available() and dist.is_initialized()):
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def aggregate_throughput(units, ms, device=None):
    """Whole-job throughput: the units all ranks processed divided by the
    slowest rank's time (per million units per second)."""
    total = sum_over_ranks(units, device)
    slowest = max_over_ranks(ms, device)
    return total / (slowest * 1e-3) / 1e6, total, slowest
