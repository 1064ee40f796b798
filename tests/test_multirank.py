"""Sharded all-pairs over several processes (gloo on CPU, world sizes 2 and 3).

Each rank takes exactly the pairs of its shard from the library's planner
(nw_debug_enumerate_pairs runs the same planner and task-to-pair mapping as the
kernels), scores them with the oracle (there is no GPU here), reduces them to
per-word partial top-k lists and a histogram, and the exchange step
(paper_2509_01654_gb300.dist: all_gather + nw_topk_merge, all_reduce) must give
exactly the oracle's unsharded lists and histogram on every rank."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

K = 8
SC = (1, -1, -1)


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def partial_lists(n, a, b, s, k):
    """Per word, the k best (score desc, index asc) among the given pairs, both directions."""
    words = np.concatenate([a, b]).astype(np.int64)
    nbrs = np.concatenate([b, a]).astype(np.int64)
    sc = np.concatenate([s, s]).astype(np.int64)
    order = np.lexsort((nbrs, -sc, words))
    words, nbrs, sc = words[order], nbrs[order], sc[order]
    idx = np.full((n, k), 0xFFFFFFFF, dtype=np.uint32)
    out = np.full((n, k), -32768, dtype=np.int16)
    starts = np.searchsorted(words, np.arange(n))
    ends = np.searchsorted(words, np.arange(n), side="right")
    for w in range(n):
        m = min(k, ends[w] - starts[w])
        idx[w, :m] = nbrs[starts[w]:starts[w] + m]
        out[w, :m] = sc[starts[w]:starts[w] + m]
    return idx, out


def worker(rank, world, port, n, seed, q, mode="host"):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import oracle
    from paper_2509_01654_gb300 import dist as nwdist
    from paper_2509_01654_gb300 import nw, synth

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        w = synth.make_words(n, 12, 1.0, 6.0, 2.5, 1, 14, seed=seed)
        a, b = nw.debug_enumerate_pairs(w.lengths, rank, world)
        s = oracle.score_pairs(w, a, b, SC, nthreads=2)
        idx, score = partial_lists(w.n, a, b, s, K)
        lo, nb = -40, 80
        hist = np.bincount(s - lo, minlength=nb).astype(np.int64)
        if mode == "exchange":
            # the tensor exchange (all_gather_into_tensor of the lists, scores
            # as raw bytes, merge where the tensors live, in-place all_reduce)
            th = torch.from_numpy(hist.copy())
            ti, ts = nwdist.exchange(torch.from_numpy(idx.view(np.int32).copy()), torch.from_numpy(score.copy()), K,
                                     hist=th)
            mi, ms, mh = ti.numpy().view(np.uint32), ts.numpy(), th.numpy()
        else:
            mi, ms = nwdist.gather_merge_topk(idx, score, K)
            mh = nwdist.allreduce_histogram(hist)
        npairs = torch.tensor([a.size], dtype=torch.int64)
        dist.all_reduce(npairs)
        if rank == 0:
            want_i, want_s = oracle.topk_rows(w, np.arange(w.n), K, SC, nthreads=2)
            want_s = np.where(want_s == oracle.MISSING_SCORE, -32768, want_s).astype(np.int16)
            want_h = oracle.histogram(w, SC, lo, nb, nthreads=2)
            ok = (np.array_equal(mi, want_i) and np.array_equal(ms, want_s) and np.array_equal(mh, want_h)
                  and int(npairs.item()) == w.n * (w.n - 1) // 2)
            q.put(("ok" if ok else "mismatch", int(npairs.item())))
        else:
            # every rank holds the same merged result
            q.put(("rank_ok", int(mi.sum() % 1000003)))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,mode", [(2, "host"), (3, "host"), (2, "exchange"), (3, "exchange")])
def test_sharded_lists_merge_across_ranks(world, mode):
    from paper_2509_01654_gb300 import build
    build.build()  # the planner and merge are host functions of libnw
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=worker, args=(r, world, port, 240, 17 + world, q, mode)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
    codes = [p.exitcode for p in procs]
    results = [q.get(timeout=5) for _ in range(world)]
    assert codes == [0] * world, codes
    assert ("ok", 240 * 239 // 2) in results, results
