"""Multi-GPU sharding of a quartet list (host logic).

Quartets are independent, so N GPUs share a batch by partitioning its work
units; no collective is needed until a digested quantity (an energy, a
gradient) is summed over ranks.  ``partition`` assigns units to ranks by
longest-processing-time-first on an estimated cost (the FP64 work of a
unit), so every rank gets a near-equal share of the total cost; ``allreduce_sum``
adds per-rank partial digests.
"""
from __future__ import annotations

import numpy as np


def partition(costs, nranks: int) -> list[np.ndarray]:
    """Indices of the units of each rank: the library's longest-processing-
    time-first partition on ``costs`` (eri_partition, host only), the same
    rule eri_plan_set_slice applies to a plan's work items."""
    if nranks < 1:
        raise ValueError("nranks must be >= 1")
    from .binding import partition as lpt
    owner, _ = lpt(costs, nranks)
    return [np.where(owner == r)[0] for r in range(nranks)]


def allreduce_sum(value, dist, device=None):
    """Sum a per-rank float (or 1-D array) over the process group."""
    import torch
    t = torch.as_tensor(np.atleast_1d(np.asarray(value, dtype=np.float64)), device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    out = t.cpu().numpy()
    return float(out[0]) if np.ndim(value) == 0 else out
