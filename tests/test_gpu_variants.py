"""GPU parity of the method variants against the CPU oracle, bit-exact:

* the length-normalised ranking (Section 5: score / max(len(A), len(B))) of
  the neighbour lists, against the oracle's exact-fraction ranking;
* the int8 matrix produced in host-copied chunks (Section 5's proposal for
  dictionaries whose matrix exceeds device memory), against the oracle's
  matrix and the one-shot device matrix;
* dictionaries scored with a full similarity matrix (Algorithm 1's
  similarity step from a table): lists, histogram, matrix, pairs, queries and
  the normalised ranking against the oracle's matrix variants, the
  match/mismatch matrix against the scalar oracle, and the refusals."""
import numpy as np
import pytest

from paper_2509_01654_gb300 import nw, synth

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


def oracle_norm_lists(oracle_mod, w, rows, k, sc):
    idx, score = oracle_mod.topk_rows_normalised(w, rows, k, sc)
    score = np.where(score == oracle_mod.MISSING_SCORE, nw.MISSING_SCORE, score).astype(np.int16)
    return idx, score


# ---------------------------------------------------------------------------
# normalised ranking

@pytest.mark.parametrize("sc,k", [((1, -1, -1), 10), ((2, -3, -1), 7), ((1, 0, 0), 16), ((3, -2, -2), 1),
                                  ((1, -1, -1), 128)])
def test_normalised_topk_all_rows(ctx, oracle_mod, sc, k):
    # lengths 0..20 (empty words included), several B lengths per launch and
    # ragged buckets; a small alphabet makes equal weights common
    w = synth.make_uniform_length_words(900, 6, 1.0, 0, 20, seed=40 + k)
    d = ctx.load_dictionary(w.codes, w.offsets, 6, sc)
    idx, score, h, lo = d.all_pairs_topk(k, normalised=True)
    oi, os_ = oracle_norm_lists(oracle_mod, w, np.arange(w.n), k, sc)
    assert np.array_equal(score, os_), "neighbour scores differ"
    assert np.array_equal(idx, oi), "neighbour indices differ"
    # the histogram still counts raw scores
    assert np.array_equal(h, oracle_mod.histogram(w, sc, lo, h.size))


def test_normalised_differs_from_raw_and_raw_unchanged(ctx, oracle_mod):
    w = synth.make_words(1500, 40, 1.1, 8.0, 3.0, 1, 25, seed=2)
    sc = synth.PAPER_SCORING
    d = ctx.load_dictionary(w.codes, w.offsets, 40, sc)
    ri, rs, _, _ = d.all_pairs_topk(10)
    ni, ns, _, _ = d.all_pairs_topk(10, normalised=True)
    ri2, rs2, _, _ = d.all_pairs_topk(10)  # the raw mode after a normalised call
    oi, os_ = oracle_norm_lists(oracle_mod, w, np.arange(w.n), 10, sc)
    assert np.array_equal(ns, os_) and np.array_equal(ni, oi)
    assert np.array_equal(ri, ri2) and np.array_equal(rs, rs2)
    assert not np.array_equal(ni, ri)
    # every list is ordered by weight, ties by index
    lens = w.lengths
    for i in range(0, w.n, 97):
        m = np.maximum(np.maximum(lens[i], lens[ni[i].astype(np.int64)]), 1)
        wt = ns[i].astype(np.float64) / m
        assert np.all(np.diff(wt) <= 0)


def test_normalised_exhaustive_sampled_rows(ctx, oracle_mod):
    """200,000 words of the exhaustive workload's length mix: 300 sampled
    rows against the oracle."""
    w = synth.exhaustive_words(200_000)
    sc = synth.PAPER_SCORING
    d = ctx.load_dictionary(w.codes, w.offsets, 40, sc)
    idx, score, _, _ = d.all_pairs_topk(10, hist=None, normalised=True)
    rows = synth.sample_rows(w.n, 300)
    oi, os_ = oracle_norm_lists(oracle_mod, w, rows, 10, sc)
    assert np.array_equal(score[rows], os_)
    assert np.array_equal(idx[rows], oi)


def test_normalised_refused_where_unsupported(ctx):
    w = synth.make_words(50, 10, 1.0, 5.0, 2.0, 1, 9, seed=4)
    d = ctx.load_dictionary(w.codes, w.offsets, 10, (1, -1, -1))
    with pytest.raises(nw.NwError) as e:
        d.all_pairs_topk(5, shard=(0, 2), normalised=True)
    assert e.value.status == nw.NW_EINVAL
    L = nw.load_library()
    q = synth.make_words(3, 10, 1.0, 5.0, 2.0, 1, 9, seed=5)
    qi = np.zeros((3, 5), np.uint32)
    qs = np.zeros((3, 5), np.int16)
    st = L.nw_query(d.handle, q.codes.ctypes.data, q.offsets.ctypes.data, 3, 5, qi.ctypes.data, qs.ctypes.data,
                    nw.NW_RANK_NORMALISED)
    assert st == nw.NW_EINVAL


# ---------------------------------------------------------------------------
# chunked matrix

@pytest.mark.parametrize("chunk", [1, 4096, 65_537, 187_000, 10 ** 9])
def test_matrix_chunked_equals_oracle(ctx, oracle_mod, chunk):
    # 613 words: 187,578 entries, so the chunk sizes give 187,578 / 46 / 3 / 2 / 1 chunks
    w = synth.make_uniform_length_words(613, 7, 1.0, 0, 20, seed=11)
    sc = (1, -1, -1)
    d = ctx.load_dictionary(w.codes, w.offsets, 7, sc)
    want = oracle_mod.all_pairs(w, sc)
    if chunk == 1:
        # one entry per chunk: a prefix of rows is enough to check, so use a small dictionary
        ws = w.subset(np.arange(40))
        ds = ctx.load_dictionary(ws.codes, ws.offsets, 7, sc)
        got = ds.all_pairs_matrix_chunked(1)
        assert np.array_equal(got.astype(np.int32), oracle_mod.all_pairs(ws, sc))
        return
    got = d.all_pairs_matrix_chunked(chunk)
    assert np.array_equal(got.astype(np.int32), want)
    assert np.array_equal(got, d.all_pairs_matrix())


def test_matrix_chunked_pr1(ctx, oracle_mod):
    # the 2,000-word matrix (1,999,000 entries) in 7 uneven chunks
    w = synth.pr1_words()
    d = ctx.load_dictionary(w.codes, w.offsets, 40, synth.PAPER_SCORING)
    got = d.all_pairs_matrix_chunked(300_001)
    assert np.array_equal(got.astype(np.int32), oracle_mod.all_pairs(w, synth.PAPER_SCORING))


def test_matrix_chunked_refuses_device_output(ctx):
    import torch
    w = synth.make_uniform_length_words(100, 7, 1.0, 1, 10, seed=2)
    d = ctx.load_dictionary(w.codes, w.offsets, 7, (1, -1, -1))
    out = torch.empty(100 * 99 // 2, dtype=torch.int8, device="cuda")
    L = nw.load_library()
    assert L.nw_all_pairs_matrix_chunked(d.handle, out.data_ptr(), 1000, nw.NW_DEVICE_PTRS) == nw.NW_EINVAL
    assert L.nw_all_pairs_matrix_chunked(d.handle, out.data_ptr(), 0, nw.NW_DEVICE_PTRS) == nw.NW_EINVAL


# ---------------------------------------------------------------------------
# full similarity matrix (nw_load_dictionary_sim)

def sym_matrix(alphabet, lo, hi, seed):
    g = np.random.default_rng(seed)
    S = g.integers(lo, hi + 1, (alphabet, alphabet))
    S = np.triu(S) + np.triu(S, 1).T
    return S.astype(np.int32)


@pytest.mark.parametrize("alphabet,lo,hi,gap,lens", [(20, -3, 4, -2, (0, 16)), (7, -2, 2, -1, (0, 9)),
                                                     (64, -5, 9, -3, (1, 12)), (12, 0, 3, -1, (25, 40))])
def test_sim_topk_histogram_matrix_pairs(ctx, oracle_mod, alphabet, lo, hi, gap, lens):
    S = sym_matrix(alphabet, lo, hi, seed=alphabet)
    np.fill_diagonal(S, hi + 2)  # identical symbols score highest, as in a phoneme similarity
    w = synth.make_uniform_length_words(700, alphabet, 1.0, lens[0], lens[1], seed=alphabet + 1)
    d = ctx.load_dictionary_sim(w.codes, w.offsets, alphabet, S, gap)
    idx, score, h, hlo = d.all_pairs_topk(10)
    oi, os_ = oracle_mod.topk_rows_sim(w, np.arange(w.n), 10, S, gap)
    os_ = np.where(os_ == oracle_mod.MISSING_SCORE, nw.MISSING_SCORE, os_).astype(np.int16)
    assert np.array_equal(score, os_) and np.array_equal(idx, oi)
    assert np.array_equal(h, oracle_mod.histogram_sim(w, S, gap, hlo, h.size))
    info = d.info()
    if info["score_lo"] >= -128 and info["score_hi"] <= 127:
        assert np.array_equal(d.all_pairs_matrix().astype(np.int32), oracle_mod.all_pairs_sim(w, S, gap))
    g = np.random.default_rng(5)
    I, J = g.integers(0, w.n, 3000), g.integers(0, w.n, 3000)
    assert np.array_equal(d.score_pairs(I, J).astype(np.int32), oracle_mod.score_pairs_sim(w, I, J, S, gap))


def test_sim_match_mismatch_matrix_equals_scalar_scoring(ctx, oracle_mod):
    w = synth.make_words(1500, 40, 1.1, 8.0, 3.0, 1, 25, seed=2)
    S = oracle_mod.match_mismatch_matrix(40, 1, -1)
    d = ctx.load_dictionary_sim(w.codes, w.offsets, 40, S, -1)
    idx, score, h, hlo = d.all_pairs_topk(10)
    oi, os_ = oracle_mod.topk_rows(w, np.arange(w.n), 10, (1, -1, -1))
    assert np.array_equal(score, os_.astype(np.int16)) and np.array_equal(idx, oi)
    assert np.array_equal(h, oracle_mod.histogram(w, (1, -1, -1), hlo, h.size))


def test_sim_query_and_normalised(ctx, oracle_mod):
    alphabet, gap = 30, -2
    S = sym_matrix(alphabet, -2, 3, seed=7)
    np.fill_diagonal(S, 5)
    w = synth.make_uniform_length_words(900, alphabet, 1.0, 1, 14, seed=8)
    q = synth.make_uniform_length_words(40, alphabet, 1.0, 0, 14, seed=9)
    d = ctx.load_dictionary_sim(w.codes, w.offsets, alphabet, S, gap)
    qi, qs = d.query(q.codes, q.offsets, 10)
    for a in range(q.n):
        row = np.array([oracle_mod.score_sim(q.word(a), w.word(j), S, gap) for j in range(w.n)])
        order = np.lexsort((np.arange(w.n), -row))[:10]
        assert np.array_equal(qi[a], order) and np.array_equal(qs[a].astype(np.int64), row[order])
    # the normalised ranking over matrix scores: lists ordered by s / max(len), ties by index
    ni, ns, _, _ = d.all_pairs_topk(10, hist=None, normalised=True)
    lens = w.lengths
    M = np.zeros((w.n, w.n), dtype=np.int64)
    iu = np.triu_indices(w.n, 1)
    M[iu] = oracle_mod.all_pairs_sim(w, S, gap)
    M = M + M.T
    from fractions import Fraction
    for i in range(0, w.n, 61):
        cand = [j for j in range(w.n) if j != i]
        best = sorted(cand, key=lambda j: (-Fraction(int(M[i, j]), max(lens[i], lens[j], 1)), j))[:10]
        assert ni[i].tolist() == best and ns[i].tolist() == [int(M[i, j]) for j in best]


def test_sim_dictionary_refusals(ctx):
    w = synth.make_uniform_length_words(50, 10, 1.0, 1, 8, seed=3)
    S = sym_matrix(10, -2, 3, seed=1)
    bad = S.copy()
    bad[0, 1] += 1  # not symmetric
    for args in [(w.codes, w.offsets, 10, bad, -1), (w.codes, w.offsets, 65, np.zeros((65, 65), np.int32), -1),
                 (w.codes, w.offsets, 10, S * 400, -1)]:
        with pytest.raises(nw.NwError) as e:
            ctx.load_dictionary_sim(*args)
        assert e.value.status in (nw.NW_EINVAL, nw.NW_ERANGE)
    d = ctx.load_dictionary_sim(w.codes, w.offsets, 10, S, -1)
    with pytest.raises(nw.NwError) as e:
        nw.Server(d, k=5, max_batch_queries=64, max_inflight=1)
    assert e.value.status == nw.NW_EINVAL
    import torch
    ti = torch.empty((w.n, 5), dtype=torch.int32, device="cuda")
    ts = torch.empty((w.n, 5), dtype=torch.int16, device="cuda")
    with pytest.raises(nw.NwError) as e:
        d.all_pairs_topk_noalloc(5, ti, ts)
    assert e.value.status == nw.NW_EINVAL


def test_sim_large_sampled_rows(ctx, oracle_mod):
    # 60,000 words of the exhaustive mix under a phoneme-like matrix: near
    # codes (adjacent in the code order) are similar
    alphabet = 40
    a = np.arange(alphabet)
    S = np.where(a[:, None] == a[None, :], 3, np.where(np.abs(a[:, None] - a[None, :]) <= 2, 1, -2)).astype(np.int32)
    w = synth.exhaustive_words(60_000)
    d = ctx.load_dictionary_sim(w.codes, w.offsets, alphabet, S, -2)
    idx, score, h, hlo = d.all_pairs_topk(10)
    assert h.sum() == w.n * (w.n - 1) // 2
    rows = synth.sample_rows(w.n, 200)
    oi, os_ = oracle_mod.topk_rows_sim(w, rows, 10, S, -2)
    assert np.array_equal(score[rows], os_.astype(np.int16)) and np.array_equal(idx[rows], oi)
