"""Host logic of the multi-GPU run: every rank solves its own points and no
data crosses ranks; only the per-rank timings are reduced (maximum).

The method has no exchange step: query points are independent (§I, §III.A),
so N GPUs run N shards with the same system and options.
"""
import numpy as np


def rank_point_seed(rank, base=2):
    """Seed of rank r's query points; rank 0 uses the standard point set."""
    return base + 1000 * int(rank)


def reduce_max(values, dist=None, device=None):
    """Element-wise maximum over ranks of a small float vector (timings)."""
    v = np.asarray(values, dtype=np.float64)
    if dist is None:
        return v
    import torch
    t = torch.tensor(v, device=device) if device is not None else torch.tensor(v)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.cpu().numpy()


def job_throughput(solves_per_rank_step, world, step_time_s):
    """Whole-job solves/s: all ranks' certified solves over the slowest rank's time."""
    return world * float(solves_per_rank_step) / float(step_time_s)
