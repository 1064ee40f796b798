"""The exchange step of a sharded all-pairs run over several processes.

Every unordered pair belongs to exactly one shard (``nw_all_pairs_topk_shard``);
each rank scores its shard and holds, per word, its k best neighbours among that
shard's pairs plus that shard's score histogram.  The full result is the
k best of the union of all ranks' lists (``nw_topk_merge``, associative and
order-independent because neighbour keys are totally ordered) and the sum of
the histograms.  This module moves the partial results with torch.distributed:
``exchange`` gathers every rank's lists into one contiguous tensor and merges
them where they live (CUDA tensors over NCCL: on the device by
``nw_topk_merge_device``; CPU tensors over gloo: on the host by
``nw_topk_merge``, the same per-word merge) and sums the histograms;
``gather_merge_topk`` is the older host-side form.  The same
shards make a long exhaustive run resumable: ``topk_with_checkpoints`` saves
each finished shard and, after an interruption, scores only the missing ones.
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


def exchange(idx, score, k: int, hist=None, ctx=None, group=None):
    """The exchange step of a sharded run.  idx (int32 view of the uint32
    indices) and score (int16) are this rank's (n, k) partial lists as torch
    tensors, CUDA (NCCL; ctx: the library context of their device) or CPU
    (gloo); hist (int64, optional) is this rank's histogram and is summed in
    place.  Returns the merged (idx, score) lists, on every rank, on the same
    device as the inputs."""
    import torch
    import torch.distributed as dist

    world = dist.get_world_size(group)
    n = int(idx.shape[0])
    # outputs concatenated along the first dimension (rank r's rows at r * n)
    gi = torch.empty((world * n, k), dtype=torch.int32, device=idx.device)
    dist.all_gather_into_tensor(gi, idx.contiguous(), group=group)
    # int16 scores travel as raw bytes: the collectives have no 16-bit integer type
    gb = torch.empty((world * n, 2 * k), dtype=torch.uint8, device=score.device)
    dist.all_gather_into_tensor(gb, score.contiguous().view(torch.uint8), group=group)
    gi = gi.view(world, n, k)
    gs = gb.view(torch.int16).view(world, n, k)
    if hist is not None:
        dist.all_reduce(hist, op=dist.ReduceOp.SUM, group=group)
    if idx.is_cuda:
        return nw.topk_merge_device(ctx, gi, gs, k)
    mi, ms = nw.topk_merge([(gi[r].numpy().view(np.uint32), gs[r].numpy()) for r in range(world)], k)
    return torch.from_numpy(mi.view(np.int32)), torch.from_numpy(ms)


def allreduce_histogram(hist, group=None):
    """Sums every rank's int64 histogram (same bins on every rank)."""
    import torch.distributed as dist

    t = _as_tensor(hist).clone()
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


# ---------------------------------------------------------------------------
# checkpoint / resume of a long exhaustive run

def _workload_tag(d, k: int, nshards: int, hist: bool, fingerprint: str) -> str:
    i = d.info()
    keys = ("n", "alphabet", "min_len", "max_len", "score_lo", "score_hi", "pairs", "cells")
    return "|".join([f"{key}={i[key]}" for key in keys] + [f"k={k}", f"nshards={nshards}", f"hist={int(hist)}",
                                                          f"fingerprint={fingerprint}"])


def topk_with_checkpoints(d, k: int, nshards: int, ckpt_dir: str, hist: bool = True, fingerprint: str = "",
                          after_shard=None):
    """The exhaustive top-k lists (and histogram) of dictionary `d`, computed as
    `nshards` shards (``nw_all_pairs_topk_shard``) with each finished shard
    saved to `ckpt_dir`.  A run that stops between shards (a crash, a
    preemption) is resumed by calling this again with the same arguments: the
    saved shards are read back and only the missing ones are scored.  The
    result is exactly that of one ``nw_all_pairs_topk`` call: every pair lies
    in one shard, the histograms add up, and the merge of the partial lists is
    exact and order-independent.

    `fingerprint` (e.g. a hash of the word list) is stored with each shard, as
    are the dictionary's size, lengths, score range and pair counts; a shard
    saved for another workload is refused.  `after_shard(g)` is called after
    shard g is saved.  Returns (idx uint32 [n, k], score int16 [n, k], hist
    int64 or None, hist_lo)."""
    import os

    if nshards < 1:
        raise ValueError("nshards must be >= 1")
    os.makedirs(ckpt_dir, exist_ok=True)
    tag = _workload_tag(d, k, nshards, hist, fingerprint)
    parts, total, lo = [], None, 0
    for g in range(nshards):
        path = os.path.join(ckpt_dir, f"shard{g:05d}-of-{nshards:05d}.npz")
        if os.path.exists(path):
            with np.load(path) as z:
                if str(z["tag"]) != tag:
                    raise ValueError(f"{path} was saved for another workload")
                idx, score, lo = z["idx"], z["score"], int(z["hist_lo"])
                h = z["hist"] if hist else None
        else:
            idx, score, h, lo = d.all_pairs_topk(k, hist=hist, shard=(g, nshards))
            tmp = path + ".partial.npz"
            np.savez(tmp, tag=np.array(tag), idx=idx, score=score, hist_lo=np.array(lo),
                     hist=h if hist else np.zeros(0, np.int64))
            os.replace(tmp, path)  # a shard file is complete or absent
            if after_shard is not None:
                after_shard(g)
        parts.append((idx, score))
        if hist:
            total = h.astype(np.int64).copy() if total is None else total + h
    idx, score = nw.topk_merge(parts, k)
    return idx, score, total, lo
