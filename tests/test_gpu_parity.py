"""GPU parity: every libnw entry point against the CPU oracle, element by
element, through the C ABI.  Scores are integers, so the bar is bit-exact:
the full int8 matrix, every (index, score) of every neighbour list, every
histogram bin."""
import os

import numpy as np
import pytest

from paper_2509_01654_gb300 import nw, synth

pytestmark = pytest.mark.gpu

SCORINGS = [(1, -1, -1), (1, -1, -2), (2, -1, -2), (3, -3, -4), (1, -3, -1), (2, 1, -1), (0, -1, -1), (1, 0, 0)]


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2509_01654_gb300 import build
    build.build()
    c = nw.Context(0)
    yield c
    c.close()


def oracle_lists(oracle_mod, w, rows, k, sc):
    idx, score = oracle_mod.topk_rows(w, rows, k, sc)
    score = np.where(score == oracle_mod.MISSING_SCORE, nw.MISSING_SCORE, score).astype(np.int16)
    return idx, score


def check_topk(oracle_mod, d, w, sc, k, rows=None, hist=True):
    idx, score, h, lo = d.all_pairs_topk(k, hist=hist)
    if rows is None:
        rows = np.arange(w.n)
    oi, os_ = oracle_lists(oracle_mod, w, rows, k, sc)
    assert np.array_equal(score[rows], os_), "neighbour scores differ"
    assert np.array_equal(idx[rows], oi), "neighbour indices differ"
    return idx, score, h, lo


# ---------------------------------------------------------------------------
# the int8 matrix (row-major upper triangle)

def test_pr1_matrix_bit_exact(ctx, oracle_mod):
    w = synth.pr1_words()
    d = ctx.load_dictionary(w.codes, w.offsets, 40, synth.PAPER_SCORING)
    got = d.all_pairs_matrix()
    want = oracle_mod.all_pairs(w, synth.PAPER_SCORING)
    assert got.size == 1_999_000
    assert np.array_equal(got.astype(np.int32), want)


@pytest.mark.parametrize("sc", SCORINGS)
def test_matrix_scorings_and_lengths(ctx, oracle_mod, sc):
    # lengths 0..20 so every B length up to 20 and empty words appear; ragged buckets
    w = synth.make_uniform_length_words(613, 7, 1.0, 0, 20, seed=7 + SCORINGS.index(sc))
    d = ctx.load_dictionary(w.codes, w.offsets, 7, sc)
    info = d.info()
    if info["score_lo"] < -128 or info["score_hi"] > 127:
        with pytest.raises(nw.NwError) as e:
            d.all_pairs_matrix()
        assert e.value.status == nw.NW_ERANGE
        return
    got = d.all_pairs_matrix()
    assert np.array_equal(got.astype(np.int32), oracle_mod.all_pairs(w, sc))


def test_matrix_long_words(ctx, oracle_mod):
    w = synth.make_uniform_length_words(300, 60, 1.0, 1, 40, seed=99)
    d = ctx.load_dictionary(w.codes, w.offsets, 60, (1, -1, -1))
    assert np.array_equal(d.all_pairs_matrix().astype(np.int32), oracle_mod.all_pairs(w, (1, -1, -1)))


def test_matrix_alphabet_256(ctx, oracle_mod):
    # the XOR encoding with codes up to 255 (match - mismatch = 1 keeps the shift at 0)
    w = synth.make_uniform_length_words(200, 256, 0.3, 1, 12, seed=3)
    d = ctx.load_dictionary(w.codes, w.offsets, 256, (1, 0, -1))
    assert np.array_equal(d.all_pairs_matrix().astype(np.int32), oracle_mod.all_pairs(w, (1, 0, -1)))


# ---------------------------------------------------------------------------
# top-k lists and histogram

def test_topk_and_histogram_all_rows(ctx, oracle_mod):
    w = synth.make_words(1500, 40, 1.1, 8.0, 3.0, 1, 25, seed=2)
    sc = synth.PAPER_SCORING
    d = ctx.load_dictionary(w.codes, w.offsets, 40, sc)
    _, _, h, lo = check_topk(oracle_mod, d, w, sc, 10)
    want = oracle_mod.histogram(w, sc, lo, h.size)
    assert np.array_equal(h, want)
    assert h.sum() == w.n * (w.n - 1) // 2


@pytest.mark.parametrize("sc,k", [((2, -1, -2), 1), ((3, -3, -4), 7), ((1, -1, -1), 33), ((1, -3, -1), 128),
                                  ((0, -1, -1), 10), ((1, 0, 0), 16)])
def test_topk_scorings_and_k(ctx, oracle_mod, sc, k):
    w = synth.make_uniform_length_words(700, 12, 1.0, 1, 18, seed=k)
    d = ctx.load_dictionary(w.codes, w.offsets, 12, sc)
    _, _, h, lo = check_topk(oracle_mod, d, w, sc, k)
    assert np.array_equal(h, oracle_mod.histogram(w, sc, lo, h.size))


def test_topk_fewer_words_than_k(ctx, oracle_mod):
    w = synth.make_words(5, 40, 1.0, 7.0, 2.5, 2, 16, seed=1)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, (1, -1, -1))
    idx, score, _, _ = check_topk(oracle_mod, d, w, (1, -1, -1), 10)
    assert np.all(idx[:, 4:] == nw.MISSING_IDX) and np.all(score[:, 4:] == nw.MISSING_SCORE)


def test_topk_heavy_ties(ctx, oracle_mod):
    # two codes and lengths 1..3: almost every word has hundreds of equal-score
    # neighbours, so the lower-index tie-break decides every list
    w = synth.make_uniform_length_words(2000, 2, 0.5, 1, 3, seed=4)
    d = ctx.load_dictionary(w.codes, w.offsets, 2, (1, -1, -1))
    check_topk(oracle_mod, d, w, (1, -1, -1), 10)


def test_all_equal_words(ctx, oracle_mod):
    # one bucket, every pair identical: every score is len * match, each list
    # is the lowest other indices, the histogram has one non-empty bin
    word = [3, 1, 4, 1, 5, 9, 2, 6, 5]
    w = synth.WordList.from_lists([word] * 300, alphabet=10)
    sc = (1, -1, -1)
    d = ctx.load_dictionary(w.codes, w.offsets, 10, sc)
    idx, score, h, lo = check_topk(oracle_mod, d, w, sc, 10)
    assert np.all(score == len(word))
    for i in (0, 5, 299):
        assert list(idx[i]) == [j for j in range(11) if j != i][:10]
    assert h[len(word) - lo] == w.n * (w.n - 1) // 2 and h.sum() == h[len(word) - lo]
    assert np.all(d.all_pairs_matrix() == len(word))


def test_single_length_bucket(ctx, oracle_mod):
    # every word of one length: one bucket, only same-length (triangular) tasks
    w = synth.make_uniform_length_words(900, 6, 1.0, 12, 12, seed=12)
    sc = (2, -1, -2)
    d = ctx.load_dictionary(w.codes, w.offsets, 6, sc)
    _, _, h, lo = check_topk(oracle_mod, d, w, sc, 10)
    assert np.array_equal(h, oracle_mod.histogram(w, sc, lo, h.size))
    assert np.array_equal(d.all_pairs_matrix().astype(np.int32), oracle_mod.all_pairs(w, sc))


def test_topk_empty_words(ctx, oracle_mod):
    w = synth.make_uniform_length_words(400, 5, 1.0, 0, 6, seed=8)
    assert (w.lengths == 0).sum() > 10
    d = ctx.load_dictionary(w.codes, w.offsets, 5, (1, -1, -1))
    _, _, h, lo = check_topk(oracle_mod, d, w, (1, -1, -1), 12)
    assert np.array_equal(h, oracle_mod.histogram(w, (1, -1, -1), lo, h.size))


def test_topk_repeatable_and_histogram_optional(ctx, oracle_mod):
    w = synth.make_words(900, 40, 1.1, 8.0, 3.0, 1, 25, seed=5)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, (1, -1, -1))
    a = d.all_pairs_topk(10)
    b = d.all_pairs_topk(10, hist=None)
    assert b[2] is None
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_exhaustive_600k_sampled_rows(ctx, oracle_mod):
    """The full 600,000-word workload: top-10 of 10,000 sampled words against
    the oracle, the histogram's total, and sampled list scores re-scored."""
    w = synth.exhaustive_words()
    sc = synth.PAPER_SCORING
    d = ctx.load_dictionary(w.codes, w.offsets, 40, sc)
    idx, score, h, lo = d.all_pairs_topk(10)
    assert h.sum() == 179_999_700_000
    assert lo == d.info()["score_lo"]
    rows = synth.sample_rows(w.n, int(os.environ.get("NW_SAMPLED_ROWS", "10000")))
    oi, os_ = oracle_lists(oracle_mod, w, rows, 10, sc)
    assert np.array_equal(score[rows], os_)
    assert np.array_equal(idx[rows], oi)
    # every list is sorted, excludes its word and carries true scores
    r = rows[:2000]
    assert np.all(np.diff(score[r].astype(np.int32), axis=1) <= 0)
    assert not np.any(idx[r] == r[:, None])
    I = np.repeat(r, 10)
    J = idx[r].reshape(-1)
    assert np.array_equal(oracle_mod.score_pairs(w, I, J, sc), score[r].reshape(-1))


def test_histogram_50k_in_full(ctx, oracle_mod):
    w = synth.exhaustive_words(50_000)
    sc = synth.PAPER_SCORING
    d = ctx.load_dictionary(w.codes, w.offsets, 40, sc)
    _, _, h, lo = d.all_pairs_topk(10)
    assert np.array_equal(h, oracle_mod.histogram(w, sc, lo, h.size))


# ---------------------------------------------------------------------------
# shards, explicit pairs, queries, device buffers

@pytest.mark.parametrize("G", [2, 3])
def test_shards_merge_to_full_result(ctx, oracle_mod, G):
    w = synth.make_words(1200, 40, 1.1, 8.0, 3.0, 1, 25, seed=6)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, (1, -1, -1))
    full = d.all_pairs_topk(10)
    parts, hsum = [], 0
    for g in range(G):
        i, s, h, _ = d.all_pairs_topk(10, shard=(g, G))
        parts.append((i, s))
        hsum = hsum + h
    mi, ms = nw.topk_merge(parts, 10)
    assert np.array_equal(mi, full[0]) and np.array_equal(ms, full[1])
    assert np.array_equal(hsum, full[2])


@pytest.mark.parametrize("G", [1, 3, 8])
def test_shards_merge_on_the_device(ctx, G):
    """Shards scored into device buffers, stacked as an all-gather would
    leave them, and merged by nw_topk_merge_device give the one-call lists;
    the host merge of the same parts agrees."""
    import torch
    w = synth.make_words(3000, 40, 1.1, 8.0, 3.0, 1, 25, seed=9)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, (1, -1, -1))
    k = 10
    full_i, full_s, full_h, _ = d.all_pairs_topk(k)
    gi = torch.empty((G, w.n, k), dtype=torch.int32, device="cuda")
    gs = torch.empty((G, w.n, k), dtype=torch.int16, device="cuda")
    hs = torch.zeros(d.info()["nbins"], dtype=torch.int64, device="cuda")
    for g in range(G):
        h = torch.empty_like(hs)
        d.all_pairs_topk(k, nbr_idx=gi[g], nbr_score=gs[g], hist=h, shard=(g, G))
        hs += h
    mi, ms = nw.topk_merge_device(ctx, gi, gs, k)
    assert np.array_equal(mi.cpu().numpy().view(np.uint32), full_i)
    assert np.array_equal(ms.cpu().numpy(), full_s)
    assert np.array_equal(hs.cpu().numpy(), full_h)
    hi, hsc = nw.topk_merge([(gi[g].cpu().numpy().view(np.uint32), gs[g].cpu().numpy()) for g in range(G)], k)
    assert np.array_equal(hi, full_i) and np.array_equal(hsc, full_s)


def test_exchange_over_nccl_on_one_rank(ctx):
    """dist.exchange over a one-rank NCCL group: the gather, the raw-byte
    score transfer and the device merge leave the lists unchanged."""
    import os
    import torch
    import torch.distributed as tdist
    from paper_2509_01654_gb300 import dist as nwdist
    w = synth.make_words(1500, 40, 1.1, 8.0, 3.0, 1, 25, seed=10)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, (1, -1, -1))
    k = 10
    full_i, full_s, full_h, _ = d.all_pairs_topk(k)
    ti = torch.empty((w.n, k), dtype=torch.int32, device="cuda")
    ts = torch.empty((w.n, k), dtype=torch.int16, device="cuda")
    th = torch.empty(d.info()["nbins"], dtype=torch.int64, device="cuda")
    d.all_pairs_topk(k, nbr_idx=ti, nbr_score=ts, hist=th, shard=(0, 1))
    os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
    os.environ.setdefault("MASTER_PORT", "29561")
    tdist.init_process_group("nccl", rank=0, world_size=1)
    try:
        mi, ms = nwdist.exchange(ti, ts, k, hist=th, ctx=ctx)
        torch.cuda.synchronize()
    finally:
        tdist.destroy_process_group()
    assert np.array_equal(mi.cpu().numpy().view(np.uint32), full_i)
    assert np.array_equal(ms.cpu().numpy(), full_s)
    assert np.array_equal(th.cpu().numpy(), full_h)


def test_interrupted_run_resumes_from_checkpoints(ctx, oracle_mod, tmp_path):
    # a run that stops after its third shard (an exception raised on the host
    # between shards) resumes from the saved shards and scores only the rest
    from paper_2509_01654_gb300 import dist
    w = synth.make_words(1500, 40, 1.1, 8.0, 3.0, 1, 25, seed=8)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, (1, -1, -1))
    full = d.all_pairs_topk(10)
    done = []

    def stop_after_third(g):
        done.append(g)
        if g == 2:
            raise RuntimeError("interrupted")

    ck = str(tmp_path / "ck")
    with pytest.raises(RuntimeError):
        dist.topk_with_checkpoints(d, 10, 5, ck, fingerprint="seed8", after_shard=stop_after_third)
    assert done == [0, 1, 2]
    done.clear()
    idx, score, hist, lo = dist.topk_with_checkpoints(d, 10, 5, ck, fingerprint="seed8", after_shard=done.append)
    assert done == [3, 4]
    assert np.array_equal(idx, full[0]) and np.array_equal(score, full[1])
    assert np.array_equal(hist, full[2]) and lo == full[3]
    # everything saved: a third call scores nothing and gives the same result
    done.clear()
    again = dist.topk_with_checkpoints(d, 10, 5, ck, fingerprint="seed8", after_shard=done.append)
    assert done == [] and np.array_equal(again[0], idx) and np.array_equal(again[2], hist)
    # shards saved for another workload are refused
    with pytest.raises(ValueError):
        dist.topk_with_checkpoints(d, 10, 5, ck, fingerprint="other words")
    oi, os_ = oracle_mod.topk_rows(w, np.arange(0, w.n, 7), 10, (1, -1, -1))
    assert np.array_equal(idx[::7], oi) and np.array_equal(score[::7].astype(np.int32), os_)


def test_score_pairs(ctx, oracle_mod):
    w = synth.make_uniform_length_words(500, 30, 1.0, 0, 40, seed=10)
    sc = (2, -1, -2)
    d = ctx.load_dictionary(w.codes, w.offsets, 30, sc)
    rng = np.random.default_rng(0)
    I = rng.integers(0, w.n, 20_000).astype(np.uint32)
    J = rng.integers(0, w.n, 20_000).astype(np.uint32)
    I[:50] = J[:50]  # self pairs are allowed here
    got = d.score_pairs(I, J)
    assert np.array_equal(got.astype(np.int32), oracle_mod.score_pairs(w, I, J, sc))


def test_query_against_dictionary(ctx, oracle_mod):
    w = synth.exhaustive_words(20_000)
    q = synth.serving_queries(300)
    sc = synth.PAPER_SCORING
    d = ctx.load_dictionary(w.codes, w.offsets, 40, sc)
    idx, score = d.query(q.codes, q.offsets, 10)
    oi, os_ = oracle_mod.query_topk(q, w, 10, sc)
    assert np.array_equal(score.astype(np.int32), os_)
    assert np.array_equal(idx, oi)


def test_query_result_independent_of_batch(ctx, oracle_mod):
    w = synth.exhaustive_words(8_000)
    q = synth.serving_queries(64)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, (1, -1, -1))
    bi, bs = d.query(q.codes, q.offsets, 10)
    for a in (0, 17, 63):
        one = q.subset([a])
        si, ss = d.query(one.codes, one.offsets, 10)
        assert np.array_equal(si[0], bi[a]) and np.array_equal(ss[0], bs[a])


def test_device_pointer_calls_match_host_calls(ctx, oracle_mod):
    import torch
    w = synth.make_words(1000, 40, 1.0, 7.0, 2.5, 2, 16, seed=1)
    sc = synth.PAPER_SCORING
    dh = ctx.load_dictionary(w.codes, w.offsets, 40, sc)
    codes = torch.from_numpy(w.codes).cuda()
    offs = torch.from_numpy(w.offsets.astype(np.int32)).cuda()
    dd = ctx.load_dictionary(codes, offs, 40, sc)
    E = w.n * (w.n - 1) // 2
    mat = torch.empty(E, dtype=torch.int8, device="cuda")
    dd.all_pairs_matrix(out=mat)
    assert np.array_equal(mat.cpu().numpy(), dh.all_pairs_matrix())
    ti = torch.empty((w.n, 10), dtype=torch.int32, device="cuda")
    ts = torch.empty((w.n, 10), dtype=torch.int16, device="cuda")
    th = torch.empty(dd.info()["nbins"], dtype=torch.int64, device="cuda")
    dd.all_pairs_topk(10, nbr_idx=ti, nbr_score=ts, hist=th)
    hi, hs, hh, _ = dh.all_pairs_topk(10)
    assert np.array_equal(ti.cpu().numpy().view(np.uint32), hi)
    assert np.array_equal(ts.cpu().numpy(), hs)
    assert np.array_equal(th.cpu().numpy(), hh)


# ---------------------------------------------------------------------------
# errors: status codes, messages, and a context that stays usable

def test_invalid_inputs(ctx):
    w = synth.pr1_words(50)
    bad = w.codes.copy()
    bad[3] = 40
    with pytest.raises(nw.NwError) as e:
        ctx.load_dictionary(bad, w.offsets, 40, (1, -1, -1))
    assert e.value.status == nw.NW_EINVAL and "alphabet" in str(e.value)
    long_off = np.array([0, 41], dtype=np.uint32)
    with pytest.raises(nw.NwError) as e:
        ctx.load_dictionary(np.zeros(41, np.uint8), long_off, 40, (1, -1, -1))
    assert e.value.status == nw.NW_EINVAL
    with pytest.raises(nw.NwError) as e:
        ctx.load_dictionary(w.codes, w.offsets, 40, (-1, 1, -1))  # mismatch > match
    assert e.value.status == nw.NW_EINVAL
    d = ctx.load_dictionary(w.codes, w.offsets, 40, (1, -1, -1))
    for k in (0, 129):
        with pytest.raises(nw.NwError) as e:
            d.all_pairs_topk(k)
        assert e.value.status == nw.NW_EINVAL
    with pytest.raises(nw.NwError) as e:
        d.all_pairs_topk(10, hist=np.zeros(3, np.int64))
    assert e.value.status == nw.NW_ERANGE
    with pytest.raises(nw.NwError) as e:
        d.score_pairs(np.array([0, 50], np.uint32), np.array([1, 2], np.uint32))
    assert e.value.status == nw.NW_EINVAL
    w0 = w.word(0).copy()
    one = ctx.load_dictionary(w0, np.array([0, w0.size], np.uint32), 40, (1, -1, -1))
    with pytest.raises(nw.NwError):
        one.all_pairs_topk(10)
    # the context still works
    idx, score, h, lo = d.all_pairs_topk(5)
    assert h.sum() == 50 * 49 // 2


def test_matrix_range_error(ctx):
    w = synth.make_uniform_length_words(20, 4, 1.0, 30, 40, seed=1)
    d = ctx.load_dictionary(w.codes, w.offsets, 4, (3, -3, -4))
    with pytest.raises(nw.NwError) as e:
        d.all_pairs_matrix()
    assert e.value.status == nw.NW_ERANGE


def test_memory_budget_and_injected_failure():
    w = synth.pr1_words(500)
    with nw.Context(0, mem_budget_bytes=8 * 1024) as c:
        with pytest.raises(nw.NwError) as e:
            c.load_dictionary(w.codes, w.offsets, 40, (1, -1, -1))
        assert e.value.status == nw.NW_ENOMEM and "budget" in str(e.value)
    with nw.Context(0) as c:
        for countdown in (1, 3, 6):
            c.debug_fail_alloc(countdown)
            with pytest.raises(nw.NwError) as e:
                c.load_dictionary(w.codes, w.offsets, 40, (1, -1, -1))
            assert e.value.status == nw.NW_ENOMEM
        c.debug_fail_alloc(0)
        d = c.load_dictionary(w.codes, w.offsets, 40, (1, -1, -1))
        c.debug_fail_alloc(1)
        with pytest.raises(nw.NwError) as e:
            d.all_pairs_topk(10)
        assert e.value.status == nw.NW_ENOMEM
        idx, score, h, _ = d.all_pairs_topk(10)
        assert h.sum() == 500 * 499 // 2


def test_profile_and_rates(ctx):
    w = synth.pr1_words()
    d = ctx.load_dictionary(w.codes, w.offsets, 40, (1, -1, -1))
    ctx.set_profiling(True)
    d.all_pairs_topk(10)
    p = ctx.last_profile()
    ctx.set_profiling(False)
    assert p["pairs"] == 1_999_000 and p["cells"] == d.info()["cells"]
    assert p["dp_ms"] > 0 and p["dp_launches"] >= 1 and p["list_inserts"] > 0
    r = ctx.measure_int_rates(20)
    assert r["sm_count"] > 0 and r["sm_clock_mhz"] > 100
    assert all(r[key] > 1e9 for key in ("viaddmax_s16x2", "vimax3_s16x2", "iadd3", "lop3", "nw_cell_mix"))
