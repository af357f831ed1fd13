"""Multi-GPU runs as independent replicas (host logic only).

The path shards by independent problems: each rank computes its own instance
(seed offset = rank) and writes its own grid, so no collective touches the data.
The only collectives are the barrier around the timed region and the
aggregation of the job's figures: the whole-job throughput is the units all
ranks processed divided by the slowest rank's time.
"""
from __future__ import annotations


def instance_offset(rank: int) -> int:
    """Seed offset of the synthetic instance computed by `rank`."""
    return int(rank)


def job_throughput(dist, local_units: float, local_seconds: float, device=None):
    """(units of all ranks / max seconds over ranks, max seconds, total units).

    ``dist`` is ``torch.distributed`` with an initialised process group, or None
    for a single process; ``device`` is where the reduction tensors live (the
    rank's GPU under NCCL, the CPU under gloo)."""
    if dist is None:
        return local_units / local_seconds, local_seconds, local_units
    import torch

    t = torch.tensor([local_seconds], dtype=torch.float64, device=device)
    u = torch.tensor([local_units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    secs, units = float(t.item()), float(u.item())
    return units / secs, secs, units
