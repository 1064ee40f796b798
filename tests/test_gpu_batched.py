"""Batches of independent dictionaries and query sets in one CUDA-graph launch.

Each dictionary has its own size, length range (up to 40), alphabet (40..120)
and scoring, and may bring a query set of its own size and lengths; the
batched lists must equal, bit for bit, the lists of each dictionary reduced
alone (nw_all_pairs_topk), of each query set answered alone (nw_query) and the
oracle's, whatever tile shapes the autotuner picked, on every replay of the
graph."""
import numpy as np
import pytest

from paper_2509_01654_gb300 import nw, synth

pytestmark = pytest.mark.gpu

K = 10


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2509_01654_gb300 import build
    build.build()
    c = nw.Context(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def dicts():
    return synth.batched_dictionaries(count=10, size_lo=60, size_hi=2500, seed=30)


def test_batch_equals_each_dictionary_alone(ctx, dicts, oracle_mod):
    batch = nw.Batch(ctx, [(d.words.codes, d.words.offsets, d.words.alphabet, d.scoring) for d in dicts], k=K)
    info = batch.info()
    assert info["ndicts"] == len(dicts)
    assert info["pairs"] == sum(d.words.n * (d.words.n - 1) // 2 for d in dicts)
    chosen = [t for t in info["words_per_task"] if t]
    assert chosen and all(t in (64, 128, 256) for t in chosen)
    first = batch.run()
    second = batch.run()
    for d, (idx, sc), (idx2, sc2) in zip(dicts, first, second):
        alone = ctx.load_dictionary(d.words.codes, d.words.offsets, d.words.alphabet, d.scoring)
        ai, asc, _, _ = alone.all_pairs_topk(K, hist=None)
        assert np.array_equal(idx, ai) and np.array_equal(sc, asc), d.scoring
        assert np.array_equal(idx, idx2) and np.array_equal(sc, sc2)
    # the oracle on every row of the three smallest dictionaries
    order = np.argsort([d.words.n for d in dicts])[:3]
    for i in order:
        d = dicts[i]
        oi, os_ = oracle_mod.topk_rows(d.words, np.arange(d.words.n), K, d.scoring)
        os_ = np.where(os_ == oracle_mod.MISSING_SCORE, nw.MISSING_SCORE, os_)
        assert np.array_equal(first[i][0], oi) and np.array_equal(first[i][1].astype(np.int32), os_)
    batch.free()


def test_autotuner_choices_are_cached_per_batch_shape(ctx, dicts):
    """A second batch of the same shape reuses the first one's tile shapes
    (chunk sizes and blocks per SM) without timing, and gives the same lists;
    a batch of another shape is tuned afresh."""
    entries = [(d.words.codes, d.words.offsets, d.words.alphabet, d.scoring) for d in dicts[:5]]
    b1 = nw.Batch(ctx, entries, k=K)
    i1 = b1.info()
    b2 = nw.Batch(ctx, entries, k=K)
    i2 = b2.info()
    assert i2["tune_cached"] == 1 and i2["tune_ms"] == 0
    assert i2["words_per_task"] == i1["words_per_task"] and i2["blocks_per_sm"] == i1["blocks_per_sm"]
    assert all(b in (0, 2, 3) for b in i1["blocks_per_sm"])
    for (a1, s1), (a2, s2) in zip(b1.run(), b2.run()):
        assert np.array_equal(a1, a2) and np.array_equal(s1, s2)
    b3 = nw.Batch(ctx, entries[:4], k=K)
    assert b3.info()["tune_cached"] == 0
    for b in (b1, b2, b3):
        b.free()


def test_batch_device_outputs_and_fixed_tiles(ctx, dicts):
    import torch
    sub = dicts[:4]
    b1 = nw.Batch(ctx, [(d.words.codes, d.words.offsets, d.words.alphabet, d.scoring) for d in sub], k=7,
                  autotune=False)
    assert all(t in (0, 256) for t in b1.info()["words_per_task"])
    host = b1.run()
    dev = [(torch.empty((d.words.n, 7), dtype=torch.int32, device="cuda"),
            torch.empty((d.words.n, 7), dtype=torch.int16, device="cuda")) for d in sub]
    b1.run(dev)
    for (hi, hs), (di, ds) in zip(host, dev):
        assert np.array_equal(hi, di.cpu().numpy().view(np.uint32)) and np.array_equal(hs, ds.cpu().numpy())
    b1.free()


def test_batch_with_query_sets_equals_each_call_alone(ctx, dicts, oracle_mod):
    import torch
    qsets = synth.batched_query_sets(dicts, size_lo=1, size_hi=700, seed=30)
    # dictionary 2 brings no queries; dictionary 5 asks only for its queries
    entries = []
    for i, (d, q) in enumerate(zip(dicts, qsets)):
        e = (d.words.codes, d.words.offsets, d.words.alphabet, d.scoring)
        if i == 2:
            entries.append(e)
        else:
            entries.append(e + ((q.codes, q.offsets), i == 5))
    batch = nw.Batch(ctx, entries, k=K)
    info = batch.info()
    nq = [0 if i == 2 else q.n for i, q in enumerate(qsets)]
    assert info["query_words"] == sum(nq)
    assert info["query_pairs"] == sum(a * d.words.n for a, d in zip(nq, dicts))
    own = sum(d.words.n * (d.words.n - 1) // 2 for i, d in enumerate(dicts) if i != 5)
    assert info["pairs"] == own + info["query_pairs"]
    first, qfirst = batch.run_queries()
    second, qsecond = batch.run_queries()
    for i, (d, q) in enumerate(zip(dicts, qsets)):
        alone = ctx.load_dictionary(d.words.codes, d.words.offsets, d.words.alphabet, d.scoring)
        if i != 5:
            ai, asc, _, _ = alone.all_pairs_topk(K, hist=None)
            assert np.array_equal(first[i][0], ai) and np.array_equal(first[i][1], asc), i
            assert np.array_equal(second[i][0], ai) and np.array_equal(second[i][1], asc), i
        if i != 2:
            qi, qs = alone.query(q.codes, q.offsets, K)
            assert qfirst[i][0].shape == (q.n, K)
            assert np.array_equal(qfirst[i][0], qi) and np.array_equal(qfirst[i][1], qs), i
            assert np.array_equal(qsecond[i][0], qi) and np.array_equal(qsecond[i][1], qs), i
        alone.free()
    # the oracle on the three smallest query sets
    for i in [j for j in np.argsort(nq) if nq[j]][:3]:
        oi, os_ = oracle_mod.query_topk(qsets[i], dicts[i].words, K, dicts[i].scoring)
        assert np.array_equal(qfirst[i][0], oi) and np.array_equal(qfirst[i][1].astype(np.int32), os_), i
    # device buffers give the same lists
    dev = [(torch.empty((d.words.n, K), dtype=torch.int32, device="cuda"),
            torch.empty((d.words.n, K), dtype=torch.int16, device="cuda")) for d in dicts]
    qdev = [(torch.empty((n, K), dtype=torch.int32, device="cuda"),
             torch.empty((n, K), dtype=torch.int16, device="cuda")) for n in nq]
    batch.run_queries(dev, qdev)
    for i in range(len(dicts)):
        if i != 5:
            assert np.array_equal(dev[i][0].cpu().numpy().view(np.uint32), first[i][0])
        assert np.array_equal(qdev[i][0].cpu().numpy().view(np.uint32), qfirst[i][0])
        assert np.array_equal(qdev[i][1].cpu().numpy(), qfirst[i][1])
    # the plain run still gives the dictionaries' lists
    plain = batch.run()
    assert all(np.array_equal(plain[i][0], first[i][0]) for i in range(len(dicts)) if i != 5)
    batch.free()


def test_batch_query_set_refusals(ctx, dicts):
    import ctypes
    d = dicts[0]
    q = synth.batched_query_sets(dicts[:1], size_lo=5, size_hi=6, seed=30)[0]
    bad = q.codes.copy()
    bad[0] = d.words.alphabet  # a code outside the dictionary's alphabet
    with pytest.raises(nw.NwError) as e:
        nw.Batch(ctx, [(d.words.codes, d.words.offsets, d.words.alphabet, d.scoring, (bad, q.offsets))], k=K)
    assert e.value.status == nw.NW_EINVAL
    # a queries-only batch needs no dictionary outputs; its query outputs are required
    b = nw.Batch(ctx, [(d.words.codes, d.words.offsets, d.words.alphabet, d.scoring, (q.codes, q.offsets), True)],
                 k=K, autotune=False)
    L = nw.load_library()
    qi = np.empty((q.n, K), np.uint32)
    qs = np.empty((q.n, K), np.int16)
    P = ctypes.c_void_p * 1
    st = L.nw_batch_run_queries(b.handle, None, None, P(qi.ctypes.data), P(qs.ctypes.data), 0)
    assert st == nw.NW_OK
    alone = ctx.load_dictionary(d.words.codes, d.words.offsets, d.words.alphabet, d.scoring)
    ai, asc = alone.query(q.codes, q.offsets, K)
    assert np.array_equal(qi, ai) and np.array_equal(qs, asc)
    st = L.nw_batch_run_queries(b.handle, None, None, P(None), P(None), 0)
    assert st == nw.NW_EINVAL
    b.free()


def test_benchmarked_64_dictionary_batch_against_oracle_sampled_rows(ctx, oracle_mod):
    """The benchmarked batched workload itself: 64 dictionaries of 1k..50k
    words, lengths 1..40, alphabets 40..120 and per-dictionary scoring, in one
    autotuned batch.  64 seeded sampled rows of every dictionary (its first and
    last words included) equal the oracle's top-10 with that dictionary's
    scoring, bit for bit, on two replays of the graph."""
    dicts = synth.batched_dictionaries(64)
    batch = nw.Batch(ctx, [(d.words.codes, d.words.offsets, d.words.alphabet, d.scoring) for d in dicts], k=K)
    first = batch.run()
    second = batch.run()
    assert len(first) == 64
    for di, (d, (idx, sc), (idx2, sc2)) in enumerate(zip(dicts, first, second)):
        n = d.words.n
        assert idx.shape == (n, K)
        assert np.array_equal(idx, idx2) and np.array_equal(sc, sc2)
        rows = np.unique(np.concatenate([synth.sample_rows(n, 64, seed=100 + di), [0, n - 1]])).astype(np.uint32)
        oi, os_ = oracle_mod.topk_rows(d.words, rows, K, d.scoring)
        assert np.array_equal(idx[rows], oi), (di, d.scoring)
        assert np.array_equal(sc[rows].astype(np.int32), os_), (di, d.scoring)
    batch.free()
