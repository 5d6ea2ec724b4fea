"""Host-side logic of multi-GPU runs: independent replicas, one process per GPU.

A single control problem does not shard (its solve is a chain of dependent
V-cycles), so N GPUs run N independent replicas of the same step; the batch
of independent problems is dealt to the ranks.  There is no collective on
the data path: the only communication is the end-of-run combination of
timings and work counts.
"""
from __future__ import annotations


def deal(n_items: int, rank: int, world: int) -> list[int]:
    """Indices of the items rank `rank` of `world` takes (round robin)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("need 0 <= rank < world")
    return [i for i in range(n_items) if i % world == rank]


def combine(max_values, sum_values, device="cpu"):
    """Whole-job figures: elementwise max over ranks of `max_values` (times)
    and sum over ranks of `sum_values` (work).  Without an initialised process
    group (one process) the inputs come back unchanged."""
    import torch
    import torch.distributed as dist
    mx = [float(v) for v in max_values]
    sm = [float(v) for v in sum_values]
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return mx, sm
    a = torch.tensor(mx, dtype=torch.float64, device=device)
    b = torch.tensor(sm, dtype=torch.float64, device=device)
    if len(mx):
        dist.all_reduce(a, op=dist.ReduceOp.MAX)
    if len(sm):
        dist.all_reduce(b, op=dist.ReduceOp.SUM)
    return a.tolist(), b.tolist()
