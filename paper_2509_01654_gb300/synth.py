"""Seeded synthetic word lists that stand in for the paper's French IPA dictionary.

The paper scores words encoded as integer phoneme codes (Section 3, the encoding
table) drawn from a frequency-sorted dictionary capped at n words (Section 5).
That dataset is not available, so every workload here is synthetic:

* a word is a sequence of uint8 codes in ``[0, alphabet)``;
* code ``c`` is drawn with probability proportional to ``(c + 1) ** -s``
  (Zipf-like phoneme usage, code 0 the most frequent);
* a word's length is ``round(N(mu, sigma))`` re-drawn until it lies in
  ``[len_lo, len_hi]``; that truncated-and-rounded law is sampled exactly by
  inverse CDF over its discrete probabilities;
* the word index is its frequency rank (rank 0 = most frequent), as in the
  paper's frequency-sorted cap; ``rank_weights`` gives the Zipf weight of each
  rank for samplers that need it.

Randomness is counter based: draw ``k`` of stream ``s`` under seed ``S`` is the
SplitMix64 output function (Steele, Lea and Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) applied to the state
``mix(S, s) + (k + 1) * 0x9E3779B97F4A7C15``.  Discrete draws compare the
64-bit output with integer thresholds, so a sample depends only on integers
once the threshold tables are fixed.

This module holds no alignment arithmetic.  It is shared by the CUDA path's
tests and benchmarks and by the oracle's tests; nothing else is.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_MASK64 = (1 << 64) - 1

# stream ids: one per kind of draw so that changing one count never shifts another
STREAM_LENGTH = 1
STREAM_CODE = 2
STREAM_ROWS = 3
STREAM_QUERY_LENGTH = 4
STREAM_QUERY_CODE = 5
STREAM_MISC = 6


def _splitmix_out(z: np.ndarray) -> np.ndarray:
    z = z.astype(np.uint64, copy=True)
    with np.errstate(over="ignore"):
        z ^= z >> np.uint64(30)
        z *= _M1
        z ^= z >> np.uint64(27)
        z *= _M2
        z ^= z >> np.uint64(31)
    return z


def _stream_base(seed: int, stream: int) -> np.uint64:
    # scalar SplitMix64 of (seed, stream) so that distinct streams start far apart
    x = (seed * 0x9E3779B97F4A7C15 + stream * 0xD1B54A32D192ED03 + 0x632BE59BD9B4E019) & _MASK64
    return _splitmix_out(np.array([x], dtype=np.uint64))[0]


def u64(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Draws ``start .. start+count-1`` of one stream as uint64."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        state = _stream_base(seed, stream) + k * _GOLDEN
    return _splitmix_out(state)


def uniform01(seed: int, stream: int, count: int, start: int = 0) -> np.ndarray:
    """Uniform doubles in [0, 1) from the top 53 bits of each draw."""
    return (u64(seed, stream, count, start) >> np.uint64(11)).astype(np.float64) * (1.0 / (1 << 53))


def thresholds(probs) -> np.ndarray:
    """Integer inverse-CDF table: value k is drawn when T[k-1] <= u < T[k]."""
    p = np.asarray(probs, dtype=np.float64)
    c = np.cumsum(p / p.sum())
    t = [min(int(ci * 2.0 ** 64), _MASK64) for ci in c[:-1]]
    return np.array(t, dtype=np.uint64)


def draw_discrete(table: np.ndarray, u: np.ndarray) -> np.ndarray:
    return np.searchsorted(table, u, side="right").astype(np.int64)


def zipf_probs(k: int, s: float) -> np.ndarray:
    r = np.arange(1, k + 1, dtype=np.float64)
    w = r ** (-s)
    return w / w.sum()


def rounded_normal_probs(mu: float, sigma: float, lo: int, hi: int) -> np.ndarray:
    """P(round(X) = l | lo <= round(X) <= hi) for X ~ N(mu, sigma)."""
    def cdf(x):
        return 0.5 * (1.0 + math.erf((x - mu) / (sigma * math.sqrt(2.0))))
    p = np.array([cdf(l + 0.5) - cdf(l - 0.5) for l in range(lo, hi + 1)], dtype=np.float64)
    return p / p.sum()


@dataclass
class WordList:
    """Words in CSR form: word i is ``codes[offsets[i]:offsets[i+1]]``."""
    codes: np.ndarray    # uint8
    offsets: np.ndarray  # uint32, n + 1 entries, offsets[0] == 0
    alphabet: int

    @property
    def n(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def lengths(self) -> np.ndarray:
        return np.diff(self.offsets.astype(np.int64))

    def word(self, i: int) -> np.ndarray:
        return self.codes[int(self.offsets[i]):int(self.offsets[i + 1])]

    @classmethod
    def from_lists(cls, words, alphabet: int = 0) -> "WordList":
        """Words given as lists of codes; alphabet defaults to the largest code + 1."""
        lens = [len(w) for w in words]
        offs = np.zeros(len(words) + 1, dtype=np.int64)
        np.cumsum(lens, out=offs[1:])
        flat = [int(c) for w in words for c in w]
        codes = np.array(flat, dtype=np.uint8)
        alphabet = alphabet or (max(flat) + 1 if flat else 1)
        return cls(codes, offs.astype(np.uint32), alphabet)

    def subset(self, idx) -> "WordList":
        idx = np.asarray(idx, dtype=np.int64)
        lens = self.lengths[idx]
        offs = np.zeros(idx.shape[0] + 1, dtype=np.int64)
        np.cumsum(lens, out=offs[1:])
        codes = np.concatenate([self.word(int(i)) for i in idx]) if idx.size else np.zeros(0, np.uint8)
        return WordList(codes.astype(np.uint8), offs.astype(np.uint32), self.alphabet)


def make_words(n: int, alphabet: int, zipf_s: float, len_mu: float, len_sigma: float,
               len_lo: int, len_hi: int, seed: int,
               length_stream: int = STREAM_LENGTH, code_stream: int = STREAM_CODE) -> WordList:
    if not (1 <= alphabet <= 256):
        raise ValueError("alphabet must be in [1, 256]")
    lt = thresholds(rounded_normal_probs(len_mu, len_sigma, len_lo, len_hi))
    lengths = draw_discrete(lt, u64(seed, length_stream, n)) + len_lo
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    total = int(offsets[-1])
    ct = thresholds(zipf_probs(alphabet, zipf_s))
    codes = draw_discrete(ct, u64(seed, code_stream, total)).astype(np.uint8)
    return WordList(codes, offsets.astype(np.uint32), alphabet)


def make_uniform_length_words(n: int, alphabet: int, zipf_s: float, len_lo: int, len_hi: int,
                              seed: int, length_stream: int = STREAM_QUERY_LENGTH,
                              code_stream: int = STREAM_QUERY_CODE) -> WordList:
    lt = thresholds(np.ones(len_hi - len_lo + 1))
    lengths = draw_discrete(lt, u64(seed, length_stream, n)) + len_lo
    offsets = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(lengths, out=offsets[1:])
    ct = thresholds(zipf_probs(alphabet, zipf_s))
    codes = draw_discrete(ct, u64(seed, code_stream, int(offsets[-1]))).astype(np.uint8)
    return WordList(codes, offsets.astype(np.uint32), alphabet)


def rank_weights(n: int, s: float) -> np.ndarray:
    """Zipf weight of each frequency rank (rank 0 = most frequent word)."""
    return zipf_probs(n, s)


def sample_rows(n: int, count: int, seed: int = 6) -> np.ndarray:
    """``count`` distinct word indices in [0, n), sorted, drawn by a seeded shuffle."""
    count = min(count, n)
    keys = u64(seed, STREAM_ROWS, n)
    return np.sort(np.argsort(keys, kind="stable")[:count]).astype(np.uint32)


# ---------------------------------------------------------------------------
# The workloads.  Scoring triples are (match, mismatch, gap) with the gap added
# per gap column; the paper fixes (+1, -1, -1) from Section 4 on.

PAPER_SCORING = (1, -1, -1)


def pr1_words(n: int = 2000) -> WordList:
    """2,000 words, 40 codes, Zipf(1.0) codes, lengths N(7, 2.5) on [2, 16]."""
    return make_words(n, 40, 1.0, 7.0, 2.5, 2, 16, seed=1)


def exhaustive_words(n: int = 600_000) -> WordList:
    """600,000 words, 40 codes, Zipf(1.1) codes, lengths N(8, 3) on [1, 25]."""
    return make_words(n, 40, 1.1, 8.0, 3.0, 1, 25, seed=2)


def serving_queries(nq: int, seed: int = 5) -> WordList:
    """Query words: lengths uniform on [1, 30], same 40-code Zipf(1.1) alphabet."""
    return make_uniform_length_words(nq, 40, 1.1, 1, 30, seed=seed)


@dataclass
class BatchedDict:
    words: WordList
    scoring: tuple


def batched_dictionaries(count: int = 64, size_lo: int = 1000, size_hi: int = 50_000,
                         seed: int = 3) -> list:
    """Dictionaries of uneven size: sizes floor(exp U(ln lo, ln hi)), lengths
    uniform on [1, 40], alphabet uniform on {40..120}, Zipf(1.0) codes, and a
    scoring triple drawn from {1,2,3} x {-1,-2,-3} x {-1..-4} per dictionary."""
    out = []
    for d in range(count):
        sd = seed + d
        u = uniform01(sd, STREAM_MISC, 5)
        size = int(math.floor(math.exp(math.log(size_lo) + u[0] * (math.log(size_hi) - math.log(size_lo)))))
        alpha = 40 + int(u[1] * 81)
        match = 1 + int(u[2] * 3)
        mismatch = -1 - int(u[3] * 3)
        gap = -1 - int(u[4] * 4)
        w = make_uniform_length_words(size, alpha, 1.0, 1, 40, seed=sd,
                                      length_stream=STREAM_LENGTH, code_stream=STREAM_CODE)
        out.append(BatchedDict(w, (match, mismatch, gap)))
    return out


def batched_query_sets(dicts: list, size_lo: int = 1, size_hi: int = 4096, seed: int = 3) -> list:
    """One query set per dictionary of `batched_dictionaries(seed=seed)`: sizes
    floor(exp U(ln lo, ln hi)), lengths uniform on [1, 40], the dictionary's
    alphabet with Zipf(1.0) codes (query streams of the dictionary's seed)."""
    out = []
    for d, x in enumerate(dicts):
        sd = seed + d
        u = uniform01(sd, STREAM_MISC, 1, start=5)  # after the dictionary's five draws
        size = int(math.floor(math.exp(math.log(size_lo) + u[0] * (math.log(size_hi) - math.log(size_lo)))))
        out.append(make_uniform_length_words(size, x.words.alphabet, 1.0, 1, 40, seed=sd))
    return out
