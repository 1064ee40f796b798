"""Checkpoint and resume of a sharded exhaustive run, on the CPU.

dist.topk_with_checkpoints is driven here by a stand-in dictionary whose
shard results come from the product planner's pair enumeration
(nw_debug_enumerate_pairs, the same task-to-pair mapping as the kernels) and
the oracle's scores; the merge is the library's host-side nw_topk_merge.  The
merged result must equal the oracle's lists and histogram over all pairs,
whether the run goes through at once or stops between shards and resumes."""
import numpy as np
import pytest

from paper_2509_01654_gb300 import dist, nw, synth

SC = (1, -1, -1)
K = 5


class OracleShards:
    """Answers all_pairs_topk(k, shard=(g, G)) the way the library does: the k
    best neighbours of every word among shard g's pairs, and their histogram."""

    def __init__(self, w, oracle_mod, lo):
        self.w, self.o, self.lo = w, oracle_mod, lo
        self.calls = []

    def info(self):
        L = self.w.lengths
        return {"n": self.w.n, "alphabet": 40, "min_len": int(L.min()), "max_len": int(L.max()),
                "score_lo": self.lo, "score_hi": int(L.max()), "pairs": self.w.n * (self.w.n - 1) // 2,
                "cells": int(((L.sum()) ** 2 - (L ** 2).sum()) // 2)}

    def all_pairs_topk(self, k, hist=True, shard=(0, 1)):
        self.calls.append(shard)
        a, b = nw.debug_enumerate_pairs(self.w.lengths, *shard)
        s = self.o.score_pairs(self.w, a, b, SC).astype(np.int64)
        word = np.concatenate([a, b]).astype(np.int64)
        other = np.concatenate([b, a]).astype(np.int64)
        sc = np.concatenate([s, s])
        order = np.lexsort((other, -sc, word))  # by word, then score desc, then partner asc
        word, other, sc = word[order], other[order], sc[order]
        idx = np.full((self.w.n, k), nw.MISSING_IDX, dtype=np.uint32)
        score = np.full((self.w.n, k), nw.MISSING_SCORE, dtype=np.int16)
        start = np.searchsorted(word, np.arange(self.w.n))
        end = np.searchsorted(word, np.arange(self.w.n), side="right")
        for i in range(self.w.n):
            m = min(k, end[i] - start[i])
            idx[i, :m] = other[start[i]:start[i] + m]
            score[i, :m] = sc[start[i]:start[i] + m]
        h = np.bincount(s - self.lo, minlength=2 * int(self.w.lengths.max()) * 2 + 1).astype(np.int64) if hist else None
        return idx, score, h, self.lo


@pytest.fixture(scope="module")
def words():
    return synth.make_words(160, 40, 1.1, 6.0, 2.5, 1, 12, seed=31)


def expected(oracle_mod, w, lo, nbins):
    oi, os_ = oracle_mod.topk_rows(w, np.arange(w.n), K, SC)
    os_ = np.where(os_ == oracle_mod.MISSING_SCORE, nw.MISSING_SCORE, os_).astype(np.int16)
    return oi, os_, oracle_mod.histogram(w, SC, lo, nbins)


def test_checkpointed_run_equals_the_oracle(oracle_mod, words, tmp_path):
    lo = -2 * int(words.lengths.max())
    d = OracleShards(words, oracle_mod, lo)
    idx, score, hist, got_lo = dist.topk_with_checkpoints(d, K, 4, str(tmp_path / "a"))
    oi, os_, oh = expected(oracle_mod, words, lo, hist.size)
    assert got_lo == lo
    assert np.array_equal(idx, oi) and np.array_equal(score, os_)
    assert np.array_equal(hist, oh) and hist.sum() == words.n * (words.n - 1) // 2
    assert d.calls == [(g, 4) for g in range(4)]


def test_resume_after_interruption_scores_only_missing_shards(oracle_mod, words, tmp_path):
    lo = -2 * int(words.lengths.max())
    d = OracleShards(words, oracle_mod, lo)
    ck = str(tmp_path / "b")

    def crash_after(g):
        if g == 1:
            raise KeyboardInterrupt  # the run stops between shards

    with pytest.raises(KeyboardInterrupt):
        dist.topk_with_checkpoints(d, K, 5, ck, fingerprint="w31", after_shard=crash_after)
    assert d.calls == [(0, 5), (1, 5)]
    d.calls.clear()
    idx, score, hist, _ = dist.topk_with_checkpoints(d, K, 5, ck, fingerprint="w31")
    assert d.calls == [(2, 5), (3, 5), (4, 5)]
    oi, os_, oh = expected(oracle_mod, words, lo, hist.size)
    assert np.array_equal(idx, oi) and np.array_equal(score, os_) and np.array_equal(hist, oh)
    # a different fingerprint, k or shard count does not reuse these files
    with pytest.raises(ValueError):
        dist.topk_with_checkpoints(d, K, 5, ck, fingerprint="other")
    with pytest.raises(ValueError):
        dist.topk_with_checkpoints(d, K + 1, 5, ck, fingerprint="w31")
    # a file left half-written is never read: only complete shards are renamed into place
    assert not [p for p in (tmp_path / "b").iterdir() if "partial" in p.name]
