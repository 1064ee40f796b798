"""Batches of independent dictionaries in one CUDA-graph launch.

Each dictionary has its own size, length range (up to 40), alphabet (40..120)
and scoring; the batched lists must equal, bit for bit, the lists of each
dictionary reduced alone and the oracle's, whatever tile shapes the autotuner
picked, on every replay of the graph."""
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
