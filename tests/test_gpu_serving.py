"""The query server: continuous batching with exact, batch-independent results.

Requests of mixed sizes and lengths are submitted from several threads while
others are on the GPU; every result must equal, bit for bit, what nw_query
returns for that request alone and what the oracle returns."""
import threading

import numpy as np
import pytest

from paper_2509_01654_gb300 import nw, serving, synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2509_01654_gb300 import build
    build.build()
    c = nw.Context(0)
    yield c
    c.close()


def test_server_results_equal_alone_and_in_the_mix(ctx, oracle_mod):
    w = synth.exhaustive_words(30_000)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, synth.PAPER_SCORING)
    pool = synth.serving_queries(3000)
    sizes = [1, 3, 700, 17, 1200, 5, 250, 64, 1, 400]
    reqs, start = [], 0
    for s in sizes:
        reqs.append(pool.subset(np.arange(start, start + s)))
        start += s
    with nw.Server(d, k=10, max_batch_queries=1500, max_inflight=3) as srv:
        ids = [None] * len(reqs)

        def submit(lo, hi):
            for r in range(lo, hi):
                ids[r] = srv.submit(reqs[r].codes, reqs[r].offsets)

        ths = [threading.Thread(target=submit, args=(0, 5)), threading.Thread(target=submit, args=(5, 10))]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
        out = [srv.wait(i) for i in ids]
    shared = 0
    for r, (idx, sc, info) in zip(reqs, out):
        alone_i, alone_s = d.query(r.codes, r.offsets, 10)
        assert np.array_equal(idx, alone_i) and np.array_equal(sc, alone_s)
        assert info["nq"] == r.n and info["done_s"] >= info["start_s"] >= info["submit_s"]
        shared += info["batch_requests"] > 1
    assert shared > 0, "no two requests ever shared a batch"
    # and the oracle agrees on a sample of queries
    q = reqs[4].subset(np.arange(0, 1200, 97))
    oi, os_ = oracle_mod.query_topk(q, w, 10, synth.PAPER_SCORING)
    si, ss = d.query(q.codes, q.offsets, 10)
    assert np.array_equal(si, oi) and np.array_equal(ss.astype(np.int32), os_)


def test_batches_overlap_on_the_device_and_results_stay_exact(ctx):
    """Requests submitted back to back, each filling a batch, are admitted
    while earlier batches are still on the GPU (their start sees another batch
    in flight), and each result equals the call made alone."""
    w = synth.exhaustive_words(200_000)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, synth.PAPER_SCORING)
    pool = synth.serving_queries(12_000)
    reqs = [pool.subset(np.arange(i * 2000, (i + 1) * 2000)) for i in range(6)]
    with nw.Server(d, k=10, max_batch_queries=2000, max_inflight=3) as srv:
        ids = [srv.submit(r.codes, r.offsets) for r in reqs]
        out = [srv.wait(i) for i in ids]
    overlapped = [info["inflight_at_start"] for _, _, info in out]
    assert max(overlapped) >= 1, overlapped
    assert all(info["batch_requests"] == 1 for _, _, info in out)
    for r, (idx, sc, info) in zip(reqs, out):
        alone_i, alone_s = d.query(r.codes, r.offsets, 10)
        assert np.array_equal(idx, alone_i) and np.array_equal(sc, alone_s)


def test_server_load_reports_latency(ctx):
    w = synth.exhaustive_words(20_000)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, synth.PAPER_SCORING)
    pool = synth.serving_queries(20_000)
    with nw.Server(d, k=10, max_batch_queries=4096, max_inflight=4) as srv:
        res = serving.run_load(srv, pool, n_requests=60, rate_hz=200.0, max_batch=512)
    assert res["requests"] == 60 and res["p99_ms"] >= res["p50_ms"] > 0
    assert res["queries_per_s"] > 0


def test_server_admission_by_memory_and_errors(ctx):
    w = synth.exhaustive_words(5_000)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, synth.PAPER_SCORING)
    with pytest.raises(nw.NwError) as e:
        nw.Server(d, k=10, max_batch_queries=4096, max_inflight=4, mem_budget_bytes=1 << 16)
    assert e.value.status == nw.NW_ENOMEM
    # a budget below eight slots' worth caps the slot count; the server still answers
    with nw.Server(d, k=10, max_batch_queries=256, max_inflight=8, mem_budget_bytes=600_000) as srv:
        q = synth.serving_queries(10)
        rid = srv.submit(q.codes, q.offsets)
        idx, sc, info = srv.wait(rid)
        assert np.array_equal(idx, d.query(q.codes, q.offsets, 10)[0])
        with pytest.raises(nw.NwError):
            big = synth.serving_queries(300)
            srv.submit(big.codes, big.offsets)  # larger than max_batch_queries
        bad = q.codes.copy()
        bad[0] = 99
        with pytest.raises(nw.NwError):
            srv.submit(bad, q.offsets)
