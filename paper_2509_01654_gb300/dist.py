"""The exchange step of a sharded all-pairs run over several processes.

Every unordered pair belongs to exactly one shard (``nw_all_pairs_topk_shard``);
each rank scores its shard and holds, per word, its k best neighbours among that
shard's pairs plus that shard's score histogram.  The full result is the
k best of the union of all ranks' lists (``nw_topk_merge``, associative and
order-independent because neighbour keys are totally ordered) and the sum of
the histograms.  This module moves the partial results with torch.distributed
(NCCL between GPUs, gloo on CPU) and merges them on the host.
"""
from __future__ import annotations

import numpy as np

from . import nw


def _as_tensor(a):
    import torch
    if isinstance(a, np.ndarray):
        return torch.from_numpy(np.ascontiguousarray(a))
    return a


def gather_merge_topk(idx, score, k: int, group=None):
    """All-gathers every rank's (n, k) partial lists and returns the merged
    (idx uint32, score int16) numpy arrays on every rank."""
    import torch
    import torch.distributed as dist

    ti = _as_tensor(np.asarray(idx).view(np.int32) if isinstance(idx, np.ndarray) else idx)
    # scores travel as int32: gloo has no 16-bit integer collectives
    ts = _as_tensor(np.asarray(score).astype(np.int32) if isinstance(score, np.ndarray) else score.to(torch.int32))
    world = dist.get_world_size(group)
    gi = [torch.empty_like(ti) for _ in range(world)]
    gs = [torch.empty_like(ts) for _ in range(world)]
    dist.all_gather(gi, ti, group=group)
    dist.all_gather(gs, ts, group=group)
    parts = [(a.cpu().numpy().view(np.uint32), b.cpu().numpy().astype(np.int16)) for a, b in zip(gi, gs)]
    return nw.topk_merge(parts, k)


def allreduce_histogram(hist, group=None):
    """Sums every rank's int64 histogram (same bins on every rank)."""
    import torch.distributed as dist

    t = _as_tensor(hist).clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()
