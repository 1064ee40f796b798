"""CPU oracle for all-pairs Needleman-Wunsch scoring (arxiv 2509.01654).

Test infrastructure only: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the library under
``paper_2509_01654_gb300`` never does.  Every function is a thin ctypes call
into ``nw_oracle.c``, which takes Algorithm 1 literally (full int32 score
matrix per pair) and states which passage each function follows.

Conventions shared with the tests: scoring is ``(match, mismatch, gap)`` with
``gap`` added per gap column (the paper's p, negative); top-k lists rank
higher scores first and lower word indices on equal scores; missing
neighbours are ``idx = 2**32 - 1`` and ``score = INT32_MIN``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

_lib = None

MISSING_IDX = np.uint32(0xFFFFFFFF)
MISSING_SCORE = np.int32(-(2 ** 31))


def default_threads() -> int:
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count() or 1)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        u8p = ctypes.POINTER(ctypes.c_uint8)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        i32p = ctypes.POINTER(ctypes.c_int32)
        i64p = ctypes.POINTER(ctypes.c_int64)
        ci = ctypes.c_int
        L.nwo_score_matrix.argtypes = [u8p, ci, u8p, ci, ci, ci, ci, i32p]
        L.nwo_score_matrix.restype = ci
        L.nwo_score.argtypes = [u8p, ci, u8p, ci, ci, ci, ci]
        L.nwo_score.restype = ctypes.c_int32
        L.nwo_all_pairs.argtypes = [u8p, u32p, ctypes.c_uint32, ci, ci, ci, i32p, ci]
        L.nwo_all_pairs.restype = ci
        L.nwo_topk_rows.argtypes = [u8p, u32p, ctypes.c_uint32, u32p, ctypes.c_uint32, ctypes.c_uint32,
                                    ci, ci, ci, u32p, i32p, ci]
        L.nwo_topk_rows.restype = ci
        L.nwo_topk_rows_normalised.argtypes = L.nwo_topk_rows.argtypes
        L.nwo_topk_rows_normalised.restype = ci
        L.nwo_query_topk.argtypes = [u8p, u32p, ctypes.c_uint32, u8p, u32p, ctypes.c_uint32,
                                     ctypes.c_uint32, ci, ci, ci, u32p, i32p, ci]
        L.nwo_query_topk.restype = ci
        L.nwo_histogram.argtypes = [u8p, u32p, ctypes.c_uint32, ci, ci, ci, ctypes.c_int32,
                                    ctypes.c_uint32, i64p, ci]
        L.nwo_histogram.restype = ctypes.c_int64
        L.nwo_score_pairs.argtypes = [u8p, u32p, ctypes.c_uint32, u32p, u32p, ctypes.c_size_t,
                                      ci, ci, ci, i32p, ci]
        L.nwo_score_pairs.restype = ci
        i32a = ctypes.POINTER(ctypes.c_int32)
        L.nwo_score_sim.argtypes = [u8p, ci, u8p, ci, i32a, ci, ci]
        L.nwo_score_sim.restype = ctypes.c_int32
        L.nwo_all_pairs_sim.argtypes = [u8p, u32p, ctypes.c_uint32, i32a, ci, ci, i32p, ci]
        L.nwo_all_pairs_sim.restype = ci
        L.nwo_topk_rows_sim.argtypes = [u8p, u32p, ctypes.c_uint32, u32p, ctypes.c_uint32, ctypes.c_uint32,
                                        i32a, ci, ci, u32p, i32p, ci]
        L.nwo_topk_rows_sim.restype = ci
        L.nwo_histogram_sim.argtypes = [u8p, u32p, ctypes.c_uint32, i32a, ci, ci, ctypes.c_int32,
                                        ctypes.c_uint32, i64p, ci]
        L.nwo_histogram_sim.restype = ctypes.c_int64
        L.nwo_score_pairs_sim.argtypes = [u8p, u32p, ctypes.c_uint32, u32p, u32p, ctypes.c_size_t,
                                          i32a, ci, ci, i32p, ci]
        L.nwo_score_pairs_sim.restype = ci
        _lib = L
    return _lib


def _p(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _u8(a):
    a = np.ascontiguousarray(a, dtype=np.uint8)
    return a if a.size else np.zeros(1, np.uint8)


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def score_matrix(A, B, scoring):
    """The full (len(A)+1) x (len(B)+1) matrix of Algorithm 1."""
    A = np.asarray(A, dtype=np.uint8)
    B = np.asarray(B, dtype=np.uint8)
    la, lb = len(A), len(B)
    H = np.zeros((la + 1, lb + 1), dtype=np.int32)
    rc = lib().nwo_score_matrix(_p(_u8(A), ctypes.c_uint8), la, _p(_u8(B), ctypes.c_uint8), lb,
                                *scoring, _p(H, ctypes.c_int32))
    if rc != 0:
        raise RuntimeError(f"nwo_score_matrix failed: {rc}")
    return H


def score(A, B, scoring) -> int:
    A = np.asarray(A, dtype=np.uint8)
    B = np.asarray(B, dtype=np.uint8)
    return int(lib().nwo_score(_p(_u8(A), ctypes.c_uint8), len(A), _p(_u8(B), ctypes.c_uint8), len(B),
                               *scoring))


def all_pairs(words, scoring, nthreads=None) -> np.ndarray:
    """int32 scores of every pair i < j in row-major upper-triangle order."""
    n = words.n
    out = np.zeros(n * (n - 1) // 2, dtype=np.int32)
    rc = lib().nwo_all_pairs(_p(_u8(words.codes), ctypes.c_uint8), _p(_u32(words.offsets), ctypes.c_uint32),
                             n, *scoring, _p(out, ctypes.c_int32) if out.size else _p(np.zeros(1, np.int32), ctypes.c_int32),
                             nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"nwo_all_pairs failed: {rc}")
    return out


def topk_rows(words, rows, k, scoring, nthreads=None):
    """(idx, score) arrays of shape (len(rows), k) for the given words."""
    rows = _u32(rows)
    idx = np.zeros((rows.size, k), dtype=np.uint32)
    sc = np.zeros((rows.size, k), dtype=np.int32)
    if rows.size == 0:
        return idx, sc
    rc = lib().nwo_topk_rows(_p(_u8(words.codes), ctypes.c_uint8), _p(_u32(words.offsets), ctypes.c_uint32),
                             words.n, _p(rows, ctypes.c_uint32), rows.size, k, *scoring,
                             _p(idx, ctypes.c_uint32), _p(sc, ctypes.c_int32), nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"nwo_topk_rows failed: {rc}")
    return idx, sc


def topk_rows_normalised(words, rows, k, scoring, nthreads=None):
    """(idx, raw score) of shape (len(rows), k), ranked by the Section 5 weight
    s / max(len(A), len(B)) compared as exact fractions (lower index first on
    equal weights)."""
    rows = _u32(rows)
    idx = np.zeros((rows.size, k), dtype=np.uint32)
    sc = np.zeros((rows.size, k), dtype=np.int32)
    if rows.size == 0:
        return idx, sc
    rc = lib().nwo_topk_rows_normalised(_p(_u8(words.codes), ctypes.c_uint8),
                                        _p(_u32(words.offsets), ctypes.c_uint32), words.n,
                                        _p(rows, ctypes.c_uint32), rows.size, k, *scoring,
                                        _p(idx, ctypes.c_uint32), _p(sc, ctypes.c_int32),
                                        nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"nwo_topk_rows_normalised failed: {rc}")
    return idx, sc


def query_topk(queries, words, k, scoring, nthreads=None):
    """(idx, score) of shape (nq, k): each query against every dictionary word."""
    nq = queries.n
    idx = np.zeros((nq, k), dtype=np.uint32)
    sc = np.zeros((nq, k), dtype=np.int32)
    if nq == 0:
        return idx, sc
    rc = lib().nwo_query_topk(_p(_u8(queries.codes), ctypes.c_uint8), _p(_u32(queries.offsets), ctypes.c_uint32),
                              nq, _p(_u8(words.codes), ctypes.c_uint8), _p(_u32(words.offsets), ctypes.c_uint32),
                              words.n, k, *scoring, _p(idx, ctypes.c_uint32), _p(sc, ctypes.c_int32),
                              nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"nwo_query_topk failed: {rc}")
    return idx, sc


def histogram(words, scoring, lo, nbins, nthreads=None) -> np.ndarray:
    """int64 counts of scores lo .. lo+nbins-1 over all unordered pairs."""
    h = np.zeros(nbins, dtype=np.int64)
    bad = lib().nwo_histogram(_p(_u8(words.codes), ctypes.c_uint8), _p(_u32(words.offsets), ctypes.c_uint32),
                              words.n, *scoring, lo, nbins, _p(h, ctypes.c_int64), nthreads or default_threads())
    if bad != 0:
        raise RuntimeError(f"nwo_histogram: {bad} scores outside the bins (or error)")
    return h


def score_pairs(words, I, J, scoring, nthreads=None) -> np.ndarray:
    I, J = _u32(I), _u32(J)
    out = np.zeros(I.size, dtype=np.int32)
    if I.size == 0:
        return out
    rc = lib().nwo_score_pairs(_p(_u8(words.codes), ctypes.c_uint8), _p(_u32(words.offsets), ctypes.c_uint32),
                               words.n, _p(I, ctypes.c_uint32), _p(J, ctypes.c_uint32), I.size, *scoring,
                               _p(out, ctypes.c_int32), nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"nwo_score_pairs failed: {rc}")
    return out


def upper_index(i, j, n):
    """Row-major upper-triangle offset of pair (i, j), i < j: S_{i-1} + (j - i - 1)."""
    i = np.asarray(i, dtype=np.int64)
    j = np.asarray(j, dtype=np.int64)
    return i * (2 * n - i - 1) // 2 + (j - i - 1)


# ---------------------------------------------------------------------------
# a full similarity matrix: sim[a][b] replaces match / mismatch (Algorithm 1's
# similarity step); gap as above

def _sim(sim):
    sim = np.ascontiguousarray(sim, dtype=np.int32)
    assert sim.ndim == 2 and sim.shape[0] == sim.shape[1]
    return sim, int(sim.shape[0])


def score_sim(A, B, sim, gap) -> int:
    sim, a = _sim(sim)
    A = np.asarray(A, dtype=np.uint8)
    B = np.asarray(B, dtype=np.uint8)
    return int(lib().nwo_score_sim(_p(_u8(A), ctypes.c_uint8), len(A), _p(_u8(B), ctypes.c_uint8), len(B),
                                   _p(sim, ctypes.c_int32), a, gap))


def all_pairs_sim(words, sim, gap, nthreads=None) -> np.ndarray:
    sim, a = _sim(sim)
    n = words.n
    out = np.zeros(max(1, n * (n - 1) // 2), dtype=np.int32)
    rc = lib().nwo_all_pairs_sim(_p(_u8(words.codes), ctypes.c_uint8), _p(_u32(words.offsets), ctypes.c_uint32),
                                 n, _p(sim, ctypes.c_int32), a, gap, _p(out, ctypes.c_int32),
                                 nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"nwo_all_pairs_sim failed: {rc}")
    return out[:n * (n - 1) // 2]


def topk_rows_sim(words, rows, k, sim, gap, nthreads=None):
    sim, a = _sim(sim)
    rows = _u32(rows)
    idx = np.zeros((rows.size, k), dtype=np.uint32)
    sc = np.zeros((rows.size, k), dtype=np.int32)
    if rows.size == 0:
        return idx, sc
    rc = lib().nwo_topk_rows_sim(_p(_u8(words.codes), ctypes.c_uint8), _p(_u32(words.offsets), ctypes.c_uint32),
                                 words.n, _p(rows, ctypes.c_uint32), rows.size, k, _p(sim, ctypes.c_int32), a, gap,
                                 _p(idx, ctypes.c_uint32), _p(sc, ctypes.c_int32), nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"nwo_topk_rows_sim failed: {rc}")
    return idx, sc


def histogram_sim(words, sim, gap, lo, nbins, nthreads=None) -> np.ndarray:
    sim, a = _sim(sim)
    h = np.zeros(nbins, dtype=np.int64)
    bad = lib().nwo_histogram_sim(_p(_u8(words.codes), ctypes.c_uint8), _p(_u32(words.offsets), ctypes.c_uint32),
                                  words.n, _p(sim, ctypes.c_int32), a, gap, lo, nbins, _p(h, ctypes.c_int64),
                                  nthreads or default_threads())
    if bad != 0:
        raise RuntimeError(f"nwo_histogram_sim: {bad} scores outside the bins (or error)")
    return h


def score_pairs_sim(words, I, J, sim, gap, nthreads=None) -> np.ndarray:
    sim, a = _sim(sim)
    I, J = _u32(I), _u32(J)
    out = np.zeros(max(1, I.size), dtype=np.int32)
    rc = lib().nwo_score_pairs_sim(_p(_u8(words.codes), ctypes.c_uint8), _p(_u32(words.offsets), ctypes.c_uint32),
                                   words.n, _p(I, ctypes.c_uint32), _p(J, ctypes.c_uint32), I.size,
                                   _p(sim, ctypes.c_int32), a, gap, _p(out, ctypes.c_int32),
                                   nthreads or default_threads())
    if rc != 0:
        raise RuntimeError(f"nwo_score_pairs_sim failed: {rc}")
    return out[:I.size]


def match_mismatch_matrix(alphabet, match, mismatch) -> np.ndarray:
    """The matrix of the scalar scoring: match on the diagonal, mismatch elsewhere."""
    m = np.full((alphabet, alphabet), mismatch, dtype=np.int32)
    np.fill_diagonal(m, match)
    return m
