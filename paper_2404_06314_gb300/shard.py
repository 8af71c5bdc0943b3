"""Batch sharding across processes (one per GPU).

Samples are independent (Sec. II-B, Eq. (qnn_batched)), so a batch shards
across ranks with no exchange on the data path: rank r takes the contiguous
block given by the paper's partition rule (the first B mod R ranks take one
extra sample).  The only collectives are for bookkeeping: the maximum of the
ranks' timings and, when a caller wants one batch-summed weight gradient, a
single sum of grad_w [P]."""
from __future__ import annotations


def partition(B: int, world: int, rank: int):
    """(start, count) of rank's block of a batch of B samples."""
    base, extra = divmod(B, world)
    count = base + (1 if rank < extra else 0)
    start = rank * base + min(rank, extra)
    return start, count


def max_over_ranks(value: float, group=None) -> float:
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64)
    if dist.get_backend(group) == "nccl":
        t = t.cuda()
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())


def sum_grad_w(gw, group=None):
    """All-reduce (sum) of a batch-summed weight gradient, in place."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized():
        dist.all_reduce(gw, op=dist.ReduceOp.SUM, group=group)
    return gw
