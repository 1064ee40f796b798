"""GPU parity of the learned candidate proposal (include/nw_proposal.h)
against the CPU oracle (oracle/proposal.py):

* forward embeddings and the loss gradient: the bf16 tensor-core products
  against the oracle's bf16 mode (the same operands rounded the same way,
  exact products), relative tolerance 1e-3: float32 accumulation of at most
  384 products per output, float32 atomics in the weight gradients, and the
  rare operand that float32 and float64 round to different bf16 neighbours;
  and against the float64 definition within the rounding's few percent;
* quantisation: bit-exact (both sides divide and round in float32);
* the dot-product top-C: bit-exact (integer dot products, exact in the
  tensor cores' float32 accumulation), with ties, ragged tails, fewer rows
  than C, and rows far beyond the append buffer so that compaction runs;
* rescoring of given candidate lists: bit-exact against Algorithm 1;
* training: Adam's first step has size lr per coordinate, and the loss falls;
* what training gains: at the same candidate budget the trained network's
  lists reach the exact neighbours far more often than the untrained
  network's or than candidates taken without a network (a length window);
* the whole path: lists sorted, scores equal to Algorithm 1's, and every
  listed neighbour among the exact top list or tied with it in score when
  the candidates cover everything.
"""
import numpy as np
import pytest

from oracle import proposal as PR
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


def small_dict(ctx, n=300, alphabet=9, seed=5, lo=0, hi=12):
    w = synth.make_uniform_length_words(n, alphabet, 1.0, lo, hi, seed=seed)
    return w, ctx.load_dictionary(w.codes, w.offsets, alphabet, (1, -1, -1))


def rand_params(alphabet, seed, scale=0.2):
    return np.random.default_rng(seed).normal(0.0, scale, PR.param_count(alphabet)).astype(np.float32)


# ---------------------------------------------------------------------------
# network

def test_param_count(ctx):
    m = nw.Model(ctx, 40, seed=1)
    assert m.param_count == PR.param_count(40)
    p = m.get_params()
    assert np.isfinite(p).all() and np.abs(p).max() <= np.sqrt(3.0) + 1e-6
    P = PR.unflatten(p.astype(np.float64), 40)
    assert np.all(P["b1"] == 0) and np.all(P["bl"] == 0)


@pytest.mark.parametrize("seed", [1, 2])
def test_forward_matches_oracle(ctx, seed):
    w, d = small_dict(ctx, n=700, seed=seed)  # lengths 0..12 incl. empty words; > one 128-row tile of words
    m = nw.Model(ctx, 9, seed=seed)
    flat = rand_params(9, seed)
    m.set_params(flat)
    assert np.array_equal(m.get_params(), flat)
    got = m.embed(d)
    want = PR.forward(flat.astype(np.float64), w, 9, bf16=True)
    err = np.abs(got - want).max() / max(1e-6, np.abs(want).max())
    assert err < 1e-3, err
    exact = PR.forward(flat.astype(np.float64), w, 9)
    assert np.abs(got - exact).max() / np.abs(exact).max() < 3e-2


def test_gradient_matches_oracle(ctx):
    w, d = small_dict(ctx, n=200, seed=7)
    m = nw.Model(ctx, 9, seed=3)
    flat = rand_params(9, 11, scale=0.15)
    m.set_params(flat)
    g = np.random.default_rng(8)
    M = 300
    pi = g.integers(0, w.n, M)
    pj = g.integers(0, w.n, M)
    pj[:5] = pi[:5]  # self pairs
    y = g.uniform(-1, 1, M)
    loss, grad = m.loss_grad(d, pi, pj, y.astype(np.float32))
    want_loss, want_grad = PR.loss_and_grad(flat.astype(np.float64), w, 9, pi, pj, y.astype(np.float32), bf16=True)
    assert abs(loss - want_loss) <= 1e-3 * abs(want_loss)
    _, exact_grad = PR.loss_and_grad(flat.astype(np.float64), w, 9, pi, pj, y.astype(np.float32))
    o = 0
    for name, shape in PR.param_shapes(9):
        n = int(np.prod(shape))
        a, b = grad[o:o + n].astype(np.float64), want_grad[o:o + n]
        rel = np.linalg.norm(a - b) / max(1e-12, np.linalg.norm(b))
        assert rel < 1e-3, (name, rel)
        c = exact_grad[o:o + n]
        assert np.linalg.norm(a - c) / max(1e-12, np.linalg.norm(c)) < 5e-2, name
        o += n


# Element-wise tolerance against the oracle's bf16 mode.  Both sides round
# the same operands to bf16 and multiply them exactly; they differ in the
# float32 accumulation of each product, whose error is at most K * 2^-24 of
# the sum of the terms' magnitudes for a sum of K terms: K <= 384 (3 taps x 128
# channels) for activations and input gradients, K = the batch's packed
# positions (thousands) for weight and bias gradients.  Either is far below
# one bf16 unit (2^-8..2^-7 relative), but when an intermediate value (a ReLU
# activation, a pooled feature, a back-propagated gradient) sits within it of
# a bf16 rounding boundary the two sides round it to neighbouring bf16 values,
# and every later product sees operands one bf16 unit apart.  An output is a
# sum of many terms, a few of them moved by one unit, so its error is bounded
# by a few units of 2^-8 of its largest terms: RTOL = 2^-6 of the element,
# and an absolute floor of 2^-6 x the tensor's rms for elements that are
# small because their terms cancel (which the deep weight-gradient sums do
# most).  A wrong element (a bad conv tap, a bias row, a missing position) is
# off by far more than either.
RTOL = 2.0 ** -6


def assert_elementwise(got, want, what):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    atol = RTOL * float(np.sqrt(np.mean(want * want)))
    bad = np.abs(got - want) > atol + RTOL * np.abs(want)
    assert not bad.any(), (what, int(bad.sum()), bad.size, float(np.abs(got - want).max()), atol)


@pytest.mark.parametrize("seed", [3, 4])
def test_forward_elementwise_product_shapes(ctx, seed):
    """Alphabet 40 and lengths 0..25, the exhaustive workload's shapes."""
    w = synth.make_uniform_length_words(1500, 40, 1.1, 0, 25, seed=seed)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, (1, -1, -1))
    m = nw.Model(ctx, 40, seed=seed)
    flat = rand_params(40, seed, scale=0.15)
    m.set_params(flat)
    got = m.embed(d)
    want = PR.forward(flat.astype(np.float64), w, 40, bf16=True)
    for c in range(64):
        assert_elementwise(got[:, c], want[:, c], f"output {c}")
    assert_elementwise(got, want, "all outputs")


def test_forward_across_a_chunk_boundary(ctx):
    """Embedding passes take at most 2^20 packed positions; words on both
    sides of the first chunk boundary (sorted by length, then index) match the
    oracle element by element."""
    n = 120_000
    w = synth.make_uniform_length_words(n, 40, 1.1, 0, 25, seed=21)
    assert int(w.lengths.sum()) > (1 << 20)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, (1, -1, -1))
    m = nw.Model(ctx, 40, seed=2)
    flat = rand_params(40, 5, scale=0.15)
    m.set_params(flat)
    got = m.embed(d)
    order = np.lexsort((np.arange(n), w.lengths))  # sorted positions
    rows = np.cumsum(w.lengths[order])
    p = int(np.searchsorted(rows, 1 << 20, side="right"))  # first word of the second chunk
    near = order[max(0, p - 150):p + 150]
    pick = np.unique(np.concatenate([near, synth.sample_rows(n, 300, seed=6)]))
    sub = w.subset(pick)
    want = PR.forward(flat.astype(np.float64), sub, 40, bf16=True)
    assert_elementwise(got[pick], want, "embeddings near the chunk boundary")


def test_gradient_elementwise_product_shapes(ctx):
    w = synth.make_uniform_length_words(600, 40, 1.1, 0, 25, seed=13)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, (1, -1, -1))
    m = nw.Model(ctx, 40, seed=5)
    flat = rand_params(40, 17, scale=0.15)
    m.set_params(flat)
    g = np.random.default_rng(19)
    M = 700
    pi = g.integers(0, w.n, M)
    pj = g.integers(0, w.n, M)
    pj[:7] = pi[:7]  # self pairs
    y = g.uniform(-1, 1, M).astype(np.float32)
    loss, grad = m.loss_grad(d, pi, pj, y)
    want_loss, want_grad = PR.loss_and_grad(flat.astype(np.float64), w, 40, pi, pj, y, bf16=True)
    assert abs(loss - want_loss) <= RTOL * abs(want_loss)
    o = 0
    for name, shape in PR.param_shapes(40):
        size = int(np.prod(shape))
        a, b = grad[o:o + size].reshape(shape), want_grad[o:o + size].reshape(shape)
        assert_elementwise(a, b, name)
        o += size


def test_invalid_pair_index_is_reported(ctx):
    w, d = small_dict(ctx, n=50)
    m = nw.Model(ctx, 9)
    with pytest.raises(nw.NwError) as e:
        m.loss_grad(d, [0, 50], [1, 2], [0.0, 0.0])
    assert e.value.status == nw.NW_EINVAL
    # the model stays usable
    m.loss_grad(d, [0, 1], [1, 2], [0.0, 0.0])


def test_dictionary_alphabet_above_model_refused(ctx):
    w, d = small_dict(ctx, n=50, alphabet=9)
    m = nw.Model(ctx, 5)
    with pytest.raises(nw.NwError) as e:
        m.embed(d)
    assert e.value.status == nw.NW_EINVAL


def test_first_adam_step_and_training_lowers_loss(ctx):
    w, d = small_dict(ctx, n=2000, alphabet=12, seed=9, lo=1, hi=14)
    m = nw.Model(ctx, 12, seed=4)
    p0 = m.get_params()
    lr = 1e-3
    m.train(d, steps=1, batch_pairs=512, lr=lr, seed=3)
    p1 = m.get_params()
    delta = np.abs(p1.astype(np.float64) - p0)
    # first Adam step: |delta| = lr * |g| / (|g| + eps) <= lr, and = lr (to float32) where |g| >> eps
    assert delta.max() <= lr * (1 + 1e-3)
    assert np.mean(delta > 0.9 * lr) > 0.5
    # a fixed evaluation batch scored by the oracle's definition of the target
    g = np.random.default_rng(2)
    pi = g.integers(0, w.n, 2000)
    pj = (pi + 1 + g.integers(0, w.n - 1, 2000)) % w.n
    import oracle
    s = oracle.score_pairs(w, pi, pj, (1, -1, -1))
    y = (s / np.maximum(np.maximum(w.lengths[pi], w.lengths[pj]), 1)).astype(np.float32)
    before, _ = m.loss_grad(d, pi, pj, y, grad=False)
    losses = m.train(d, steps=300, batch_pairs=1024, lr=2e-3, seed=4)
    after, _ = m.loss_grad(d, pi, pj, y, grad=False)
    assert np.isfinite(losses).all()
    assert after < 0.5 * before, (before, after)
    assert losses[-20:].mean() < losses[:20].mean()


# ---------------------------------------------------------------------------
# quantisation and candidates

def test_quantize_matches_oracle(ctx):
    g = np.random.default_rng(1)
    E = (g.normal(0, 1, (5000, 64)) * g.uniform(0.1, 3.0, (5000, 1))).astype(np.float32)
    E[:, 63] = g.normal(-10, 5, 5000).astype(np.float32)  # biases on their own scale
    E[17, 63] = 1e9  # saturates at 2^23
    q, b, s = nw.quantize_embeddings(ctx, E)
    wq, wb, ws = PR.quantize(E)
    assert s == ws
    assert np.array_equal(q, wq)
    assert np.array_equal(b, wb)
    assert int(b[17]) == 1 << 23 and not q[:, 63].any()
    z, zb, s0 = nw.quantize_embeddings(ctx, np.zeros((3, 64), np.float32))
    assert s0 == 0 and not z.any() and not zb.any()


@pytest.mark.parametrize("n,C,levels,bias_range", [(1000, 64, 127, 0), (777, 32, 2, 0), (20, 64, 5, 0),
                                                   (1, 4, 3, 0), (300, 512, 127, 0), (4100, 256, 127, 0),
                                                   (1000, 64, 127, 300_000), (777, 32, 2, 40), (301, 64, 127, -1)])
def test_dot_topk_matches_oracle(ctx, n, C, levels, bias_range):
    g = np.random.default_rng(n + C)
    q = g.integers(-levels, levels + 1, (n, 64)).astype(np.int8)
    if n > 10:
        q[n // 3] = q[1]  # duplicate rows
    bias = None
    if bias_range > 0:
        bias = g.integers(-bias_range, bias_range + 1, n).astype(np.int32)
    elif bias_range < 0:  # the extremes: sums near 2^24 must stay exact
        bias = g.choice(np.array([-(1 << 23), (1 << 23), 0, 1], np.int32), n)
    idx, dot = nw.dot_topk(ctx, q, C, bias=bias)
    wi, wd = PR.dot_topk(q, C, bias=bias)
    assert np.array_equal(dot, wd)
    assert np.array_equal(idx, wi)


def test_dot_topk_device_buffers_and_unaligned_bias(ctx):
    import torch
    n, C = 700, 48
    g = np.random.default_rng(3)
    q = g.integers(-60, 61, (n, 64)).astype(np.int8)
    bias = g.integers(-5000, 5001, n + 1).astype(np.int32)
    wi, wd = PR.dot_topk(q, C, bias=bias[1:])
    tq = torch.from_numpy(q).cuda()
    tb = torch.from_numpy(bias).cuda()[1:]  # 4 bytes past an aligned start
    assert tb.data_ptr() % 16 != 0
    idx, dot = nw.dot_topk(ctx, tq, C, bias=tb)
    assert np.array_equal(dot.cpu().numpy(), wd)
    assert np.array_equal(idx.cpu().numpy().view(np.uint32), wi)


def test_dot_topk_large_sampled_rows(ctx):
    # 40,000 rows: each row's buffer is compacted many times during the sweep
    n, C = 40_000, 256
    g = np.random.default_rng(77)
    q = g.integers(-20, 21, (n, 64)).astype(np.int8)
    idx, dot = nw.dot_topk(ctx, q, C)
    rows = synth.sample_rows(n, 64)
    wi, wd = PR.dot_topk(q, C, rows=rows)
    assert np.array_equal(dot[rows], wd)
    assert np.array_equal(idx[rows], wi)
    # every row: sorted, distinct, no self
    assert np.all(np.diff(dot.astype(np.int64), axis=1) <= 0)
    assert not np.any(idx == np.arange(n, dtype=np.uint32)[:, None])


@pytest.mark.parametrize("kind", ["constant", "two_values", "narrow", "wide"])
def test_dot_topk_compaction_value_spreads(ctx, kind):
    # C = 16 compacts every 64 keys.  Constant values put every key in one
    # histogram bin (the exact select runs); two values, a narrow and a wide
    # spread exercise the histogram threshold with few and many keys per bin.
    n, C = 3000, 16
    g = np.random.default_rng(5)
    q = np.zeros((n, 64), np.int8)
    bias = None
    if kind == "two_values":
        q[:, 0] = g.integers(0, 2, n)
        q[:, 1] = 1
    elif kind == "narrow":
        q[:, :4] = g.integers(-3, 4, (n, 4))
    elif kind == "wide":
        q = g.integers(-127, 128, (n, 64)).astype(np.int8)
        bias = g.integers(-(1 << 22), 1 << 22, n).astype(np.int32)
    idx, dot = nw.dot_topk(ctx, q, C, bias=bias)
    rows = np.unique(np.concatenate([synth.sample_rows(n, 96), [0, 1, n - 2, n - 1]])).astype(np.int64)
    wi, wd = PR.dot_topk(q, C, rows=rows, bias=bias)
    assert np.array_equal(dot[rows], wd)
    assert np.array_equal(idx[rows], wi)


# n = 700: one column split; 3000 and 20,000: several splits (their lists are
# merged into the original rows); 60,000: one split again, rows written by
# the candidate kernel itself.  Few levels give many equal values, so the
# lower-original-index tie rule decides which columns make the list.
@pytest.mark.parametrize("n,C,levels,bias_range", [(700, 64, 1, 0), (3000, 16, 2, 40), (20_000, 64, 1, 0),
                                                   (20_000, 256, 127, 300_000), (60_000, 128, 3, 0),
                                                   (3000, 64, 127, -1)])
def test_dot_topk_locality_order_matches_oracle(ctx, n, C, levels, bias_range):
    """NW_LOCALITY_ORDER sweeps the rows sorted by their principal components;
    the lists must equal the oracle's for the rows in their own order."""
    g = np.random.default_rng(n + C + levels)
    q = g.integers(-levels, levels + 1, (n, 64)).astype(np.int8)
    q[n // 3] = q[1]  # duplicate rows
    bias = None
    if bias_range > 0:
        bias = g.integers(-bias_range, bias_range + 1, n).astype(np.int32)
    elif bias_range < 0:
        bias = g.choice(np.array([-(1 << 23), (1 << 23), 0, 1], np.int32), n)
    idx, dot = nw.dot_topk(ctx, q, C, bias=bias, locality=True)
    pi, pd = nw.dot_topk(ctx, q, C, bias=bias)
    assert np.array_equal(dot, pd)
    assert np.array_equal(idx, pi)
    rows = np.arange(n) if n <= 3000 else np.unique(np.concatenate([synth.sample_rows(n, 200), [0, 1, n - 1]]))
    wi, wd = PR.dot_topk(q, C, rows=rows, bias=bias)
    assert np.array_equal(dot[rows], wd)
    assert np.array_equal(idx[rows], wi)


def test_proposal_sweep_order_does_not_change_results(ctx):
    w = synth.make_words(20000, 40, 1.1, 8.0, 3.0, 1, 25, seed=31)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, (1, -1, -1))
    m = nw.Model(ctx, 40, seed=4)
    ex_i, _, _, _ = d.all_pairs_topk(10, hist=None)
    m.train(d, steps=300, batch_pairs=2048, lr=2e-3, seed=5, nbr=ex_i, nbr_fraction=0.5)
    try:
        for C in (32, 256):
            m.set_sweep_order(True)
            li, ls, prof = m.proposal_topk(d, C=C, k=10)
            assert prof["candidates_ms"] > 0
            m.set_sweep_order(False)
            di, ds, _ = m.proposal_topk(d, C=C, k=10)
            assert np.array_equal(li, di)
            assert np.array_equal(ls, ds)
    finally:
        m.set_sweep_order(True)
        m.free()


def test_dot_topk_rejects_bad_C(ctx):
    q = np.zeros((10, 64), np.int8)
    for C in (0, nw.MAX_CANDIDATES + 1):
        with pytest.raises(nw.NwError) as e:
            nw.dot_topk(ctx, q, C)
        assert e.value.status == nw.NW_EINVAL


# ---------------------------------------------------------------------------
# rescoring

@pytest.mark.parametrize("k,C", [(10, 64), (1, 7), (33, 40)])
def test_rescore_matches_oracle(ctx, oracle_mod, k, C):
    w = synth.make_words(1500, 40, 1.1, 8.0, 3.0, 1, 25, seed=12)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, (1, -1, -1))
    g = np.random.default_rng(k * 100 + C)
    cand = np.empty((w.n, C), dtype=np.uint32)
    for i in range(w.n):
        pool = g.choice(w.n - 1, C, replace=False)
        cand[i] = np.where(pool >= i, pool + 1, pool)  # distinct, never i
    cand[::7, C // 2:] = PR.MISSING_IDX  # some rows with missing candidates
    idx, sc = nw.rescore_topk(d, cand, k)
    wi, ws = PR.rescore_topk(oracle_mod, w, cand, k, (1, -1, -1))
    ws = np.where(ws == PR.MISSING_SCORE, nw.MISSING_SCORE, ws).astype(np.int16)
    assert np.array_equal(sc, ws)
    assert np.array_equal(idx, wi)


@pytest.mark.parametrize("C", [7, 32, 129])
def test_rescore_with_a_similarity_matrix(ctx, oracle_mod, C):
    # the paired rescoring's table variant: scores from a full similarity
    # matrix, candidates of mixed lengths, odd C (one unpaired entry per row)
    alphabet, gap, k = 24, -2, 6
    g = np.random.default_rng(C)
    S = g.integers(-3, 4, (alphabet, alphabet))
    S = (np.triu(S) + np.triu(S, 1).T).astype(np.int32)
    np.fill_diagonal(S, 6)
    w = synth.make_uniform_length_words(900, alphabet, 1.0, 0, 20, seed=C + 3)
    d = ctx.load_dictionary_sim(w.codes, w.offsets, alphabet, S, gap)
    cand = np.empty((w.n, C), dtype=np.uint32)
    for i in range(w.n):
        pool = g.choice(w.n - 1, C, replace=False)
        cand[i] = np.where(pool >= i, pool + 1, pool)
    cand[::5, C // 3:] = PR.MISSING_IDX
    idx, sc = nw.rescore_topk(d, cand, k)
    I = np.repeat(np.arange(w.n), C)
    J = cand.reshape(-1).astype(np.int64)
    ok = J != PR.MISSING_IDX
    full = np.full(I.size, np.iinfo(np.int64).min, dtype=np.int64)
    full[ok] = oracle_mod.score_pairs_sim(w, I[ok], J[ok], S, gap)
    full = full.reshape(w.n, C)
    for i in range(w.n):
        v = cand[i] != PR.MISSING_IDX
        j, s_ = cand[i][v].astype(np.int64), full[i][v]
        order = np.lexsort((j, -s_))[:k]
        assert np.array_equal(idx[i, :order.size], j[order])
        assert np.array_equal(sc[i, :order.size].astype(np.int64), s_[order])
        assert np.all(idx[i, order.size:] == PR.MISSING_IDX)


def test_proposal_query_with_a_similarity_matrix(ctx):
    # cross rescoring's table variant: with every word a candidate the lists
    # equal the exhaustive query's over matrix scores
    alphabet, gap = 30, -2
    g = np.random.default_rng(9)
    S = g.integers(-2, 4, (alphabet, alphabet))
    S = (np.triu(S) + np.triu(S, 1).T).astype(np.int32)
    np.fill_diagonal(S, 5)
    w = synth.make_uniform_length_words(400, alphabet, 1.0, 1, 14, seed=10)
    q = query_set(60, alphabet, seed=11, lo=0, hi=16)
    d = ctx.load_dictionary_sim(w.codes, w.offsets, alphabet, S, gap)
    m = nw.Model(ctx, alphabet, seed=3)
    idx, sc = m.query(d, q.codes, q.offsets, C=400, k=8)
    wi, ws = d.query(q.codes, q.offsets, 8)
    assert np.array_equal(idx, wi) and np.array_equal(sc, ws)


def test_rescore_reports_self_candidate(ctx):
    w = synth.make_words(100, 10, 1.0, 5.0, 2.0, 1, 9, seed=1)
    d = ctx.load_dictionary(w.codes, w.offsets, 10, (1, -1, -1))
    cand = np.tile(np.arange(5, dtype=np.uint32), (w.n, 1))
    with pytest.raises(nw.NwError) as e:
        nw.rescore_topk(d, cand, 3)
    assert e.value.status == nw.NW_EINVAL


# ---------------------------------------------------------------------------
# the whole path

def test_proposal_path_properties(ctx, oracle_mod):
    w = synth.make_words(6000, 40, 1.1, 8.0, 3.0, 1, 25, seed=21)
    sc = (1, -1, -1)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, sc)
    m = nw.Model(ctx, 40, seed=2)
    ex_i, ex_s, _, _ = d.all_pairs_topk(10, hist=None)
    m.train(d, steps=200, batch_pairs=2048, lr=2e-3, seed=5, nbr=ex_i, nbr_fraction=0.5)
    idx, score, prof = m.proposal_topk(d, C=128, k=10)
    assert prof["total_ms"] > 0
    ok = idx != nw.MISSING_IDX
    assert ok.all()  # 128 candidates always give 10 neighbours
    assert np.all(np.diff(score.astype(np.int32), axis=1) <= 0)
    rows = synth.sample_rows(w.n, 300)
    I = np.repeat(rows, 10)
    J = idx[rows].reshape(-1)
    assert np.array_equal(oracle_mod.score_pairs(w, I, J, sc), score[rows].reshape(-1))
    # the approximate lists never beat the exact ones
    assert np.all(score[:, 0] <= ex_s[:, 0])
    strict, tie = PR.recall_at_k(ex_i, ex_s, idx, score)
    assert 0.0 < strict <= tie <= 1.0


def test_exact_length_gives_long_words_their_exhaustive_lists(ctx):
    """With nw_proposal_set_exact_length(L), words of at least L symbols get
    exactly the exhaustive lists (themselves excluded), and every shorter
    word keeps its proposal list."""
    import torch
    w = synth.make_words(5000, 40, 1.1, 8.0, 3.0, 1, 25, seed=23)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, synth.PAPER_SCORING)
    ex_i, ex_s, _, _ = d.all_pairs_topk(10, hist=None)
    m = nw.Model(ctx, 40, seed=3)
    m.train(d, steps=100, batch_pairs=2048, lr=2e-3, seed=6, nbr=ex_i)
    base_i, base_s, _ = m.proposal_topk(d, C=64, k=10)
    L = 13
    long_rows = w.lengths >= L
    assert 0 < long_rows.sum() < w.n
    m.set_exact_length(L)
    try:
        idx, score, prof = m.proposal_topk(d, C=64, k=10)
        assert prof["exact_ms"] > 0 and prof["total_ms"] >= prof["exact_ms"]
        assert np.array_equal(idx[long_rows], ex_i[long_rows])
        assert np.array_equal(score[long_rows], ex_s[long_rows])
        assert np.array_equal(idx[~long_rows], base_i[~long_rows])
        assert np.array_equal(score[~long_rows], base_s[~long_rows])
        # device outputs
        ti = torch.empty((w.n, 10), dtype=torch.int32, device="cuda")
        ts = torch.empty((w.n, 10), dtype=torch.int16, device="cuda")
        m.proposal_topk(d, C=64, k=10, nbr_idx=ti, nbr_score=ts)
        assert np.array_equal(ti.cpu().numpy().view(np.uint32), idx)
        # every word long: the whole graph is the exhaustive one
        m.set_exact_length(1)
        i1, s1, _ = m.proposal_topk(d, C=64, k=10)
        assert np.array_equal(i1[w.lengths >= 1], ex_i[w.lengths >= 1])
    finally:
        m.set_exact_length(0)
    with pytest.raises(nw.NwError):
        m.set_exact_length(nw.MAX_WORD_LEN + 1)


def test_exact_length_routes_long_queries_to_the_exhaustive_kernel(ctx):
    import torch
    w = synth.make_words(4000, 40, 1.1, 8.0, 3.0, 1, 25, seed=24)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, synth.PAPER_SCORING)
    m = nw.Model(ctx, 40, seed=4)
    m.train(d, steps=50, batch_pairs=1024, lr=2e-3, seed=7)
    q = synth.serving_queries(700, seed=12)  # lengths 1..30
    base_i, base_s = m.query(d, q.codes, q.offsets, 64, 10)
    ex_i, ex_s = d.query(q.codes, q.offsets, 10)
    L = 15
    lng = q.lengths >= L
    assert 0 < lng.sum() < q.n
    m.set_exact_length(L)
    try:
        i, s_ = m.query(d, q.codes, q.offsets, 64, 10)
        assert np.array_equal(i[lng], ex_i[lng]) and np.array_equal(s_[lng], ex_s[lng])
        assert np.array_equal(i[~lng], base_i[~lng]) and np.array_equal(s_[~lng], base_s[~lng])
        # device buffers both ways
        tc = torch.from_numpy(q.codes).cuda()
        to = torch.from_numpy(q.offsets.astype(np.int32)).cuda()
        ti, tsc = m.query(d, tc, to, 64, 10)
        assert np.array_equal(ti.cpu().numpy().view(np.uint32), i)
        assert np.array_equal(tsc.cpu().numpy(), s_)
        # only long queries, and a single short one
        sub = np.where(lng)[0][:5]
        li, ls = m.query(d, q.subset(sub).codes, q.subset(sub).offsets, 64, 10)
        assert np.array_equal(li, ex_i[sub]) and np.array_equal(ls, ex_s[sub])
        one = q.subset([int(np.argmin(q.lengths))])
        oi, os_ = m.query(d, one.codes, one.offsets, 64, 10)
        assert np.array_equal(oi, base_i[[int(np.argmin(q.lengths))]])
    finally:
        m.set_exact_length(0)


def test_trained_network_beats_the_proposal_without_it(ctx):
    # The same candidate budget three ways, each rescored exactly: the trained
    # network, the same network untrained, and no network at all (the C words
    # nearest in length order). Only the trained network finds the neighbours.
    w = synth.make_words(20000, 40, 1.1, 8.0, 3.0, 1, 25, seed=23)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, (1, -1, -1))
    ex_i, ex_s, _, _ = d.all_pairs_topk(10, hist=None)
    C = 128
    untrained = nw.Model(ctx, 40, seed=6)
    ui, us, _ = untrained.proposal_topk(d, C=C, k=10)
    untrained.free()
    order = np.argsort(w.lengths, kind="stable")
    pos = np.empty(w.n, dtype=np.int64)
    pos[order] = np.arange(w.n)
    lo = np.clip(pos - C // 2, 0, w.n - C - 1)
    win = lo[:, None] + np.arange(C + 1)[None, :]
    win = win[win != pos[:, None]].reshape(w.n, C)
    li, ls = nw.rescore_topk(d, order[win].astype(np.uint32), 10)
    m = nw.Model(ctx, 40, seed=6)
    m.train(d, steps=1000, batch_pairs=2048, lr=2e-3, lr_final=2e-4, clip_norm=1.0, seed=7, nbr=ex_i,
            nbr_fraction=0.5)
    ti, ts, _ = m.proposal_topk(d, C=C, k=10)
    m.free()
    _, r_untrained = PR.recall_at_k(ex_i, ex_s, ui, us)
    _, r_window = PR.recall_at_k(ex_i, ex_s, li, ls)
    _, r_trained = PR.recall_at_k(ex_i, ex_s, ti, ts)
    print(f"tie-aware recall@10 at C={C}: trained {r_trained:.3f}, untrained {r_untrained:.3f}, "
          f"length window {r_window:.3f}")
    assert r_trained >= 0.5
    assert r_trained >= max(r_untrained, r_window) + 0.3


def test_proposal_with_all_candidates_is_exact(ctx):
    # with C >= n - 1 every pair is a candidate: the lists equal the exhaustive ones
    w = synth.make_words(400, 40, 1.1, 8.0, 3.0, 1, 25, seed=22)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, (1, -1, -1))
    m = nw.Model(ctx, 40, seed=3)
    ex_i, ex_s, _, _ = d.all_pairs_topk(10, hist=None)
    idx, score, _ = m.proposal_topk(d, C=nw.MAX_CANDIDATES, k=10)
    assert np.array_equal(score, ex_s)
    assert np.array_equal(idx, ex_i)


# ---------------------------------------------------------------------------
# queries through the proposal (rectangular candidates, cross rescoring)

@pytest.mark.parametrize("na,nb,C,levels,bias_range", [(300, 1000, 64, 127, 0), (257, 777, 32, 2, 40),
                                                       (5, 40, 64, 5, 0), (70, 130, 16, 127, 300_000),
                                                       (1000, 20_000, 128, 20, 0)])
def test_dot_topk_cross_matches_oracle(ctx, na, nb, C, levels, bias_range):
    # ragged row and column tails, ties (duplicate columns, few levels),
    # fewer columns than C, and 20,000 columns (compaction) on sampled rows
    g = np.random.default_rng(na + nb + C)
    qa = g.integers(-levels, levels + 1, (na, 64)).astype(np.int8)
    qb = g.integers(-levels, levels + 1, (nb, 64)).astype(np.int8)
    if nb > 10:
        qb[nb // 2] = qb[1]
    bias = g.integers(-bias_range, bias_range + 1, nb).astype(np.int32) if bias_range else None
    idx, val = nw.dot_topk_cross(ctx, qa, qb, C, bias=bias)
    rows = np.arange(na) if na * nb <= 2_000_000 else synth.sample_rows(na, 64).astype(np.int64)
    wi, wv = PR.dot_topk_cross(qa, qb, C, bias=bias, rows=rows)
    assert np.array_equal(val[rows], wv)
    assert np.array_equal(idx[rows], wi)


def test_dot_topk_cross_without_columns(ctx):
    qa = np.ones((3, 64), np.int8)
    idx, val = nw.dot_topk_cross(ctx, qa, np.zeros((0, 64), np.int8), 4)
    assert np.all(idx == 0xFFFFFFFF) and np.all(val == np.iinfo(np.int32).min)


def query_set(n, alphabet, seed, lo=0, hi=14):
    return synth.make_uniform_length_words(n, alphabet, 1.0, lo, hi, seed=seed)


def test_proposal_query_with_every_candidate_equals_exhaustive(ctx):
    # C >= the dictionary's size: every word is rescored, so the lists are
    # the exhaustive query lists, ties included
    w, d = small_dict(ctx, n=300, seed=21, lo=0, hi=12)
    q = query_set(70, 9, seed=22)
    m = nw.Model(ctx, 9, seed=2)
    idx, sc = m.query(d, q.codes, q.offsets, C=300, k=10)
    wi, ws = d.query(q.codes, q.offsets, 10)
    assert np.array_equal(idx, wi) and np.array_equal(sc, ws)
    import oracle
    oi, osc = oracle.query_topk(q, w, 10, (1, -1, -1))
    assert np.array_equal(idx, oi) and np.array_equal(sc.astype(np.int32), osc)


def test_proposal_query_scores_exact_and_sorted(ctx):
    import oracle
    w, d = small_dict(ctx, n=3000, alphabet=12, seed=23, lo=1, hi=14)
    m = nw.Model(ctx, 12, seed=3)
    m.train(d, steps=150, batch_pairs=2048, lr=2e-3, seed=5)
    q = query_set(200, 12, seed=24, lo=1, hi=16)
    idx, sc = m.query(d, q.codes, q.offsets, C=64, k=10)
    assert idx.shape == (200, 10) and not np.any(idx == 0xFFFFFFFF)
    for r in range(q.n):
        assert len(set(idx[r].tolist())) == 10
        want = [oracle.score(q.word(r), w.word(int(j)), (1, -1, -1)) for j in idx[r]]
        assert sc[r].astype(np.int64).tolist() == want
        key = [(-int(s), int(j)) for s, j in zip(sc[r], idx[r])]
        assert key == sorted(key)
    # the exact top-10 score is an upper bound of every listed score
    oi, osc = oracle.query_topk(q, w, 10, (1, -1, -1))
    assert np.all(sc.astype(np.int32) <= osc)


def test_proposal_query_cache_follows_parameters_and_dictionary(ctx):
    w1, d1 = small_dict(ctx, n=400, seed=31, lo=1, hi=12)
    w2, d2 = small_dict(ctx, n=500, seed=32, lo=1, hi=12)
    q = query_set(50, 9, seed=33, lo=1, hi=12)
    a = nw.Model(ctx, 9, seed=4)
    b = nw.Model(ctx, 9, seed=5)
    ra = a.query(d1, q.codes, q.offsets, C=16, k=5)
    rb = b.query(d1, q.codes, q.offsets, C=16, k=5)
    # new parameters: the cached dictionary rows are rebuilt
    a.set_params(b.get_params())
    ra2 = a.query(d1, q.codes, q.offsets, C=16, k=5)
    assert np.array_equal(ra2[0], rb[0]) and np.array_equal(ra2[1], rb[1])
    # another dictionary: the same as a fresh model's
    r2 = a.query(d2, q.codes, q.offsets, C=16, k=5)
    c = nw.Model(ctx, 9, seed=5)
    r2c = c.query(d2, q.codes, q.offsets, C=16, k=5)
    assert np.array_equal(r2[0], r2c[0]) and np.array_equal(r2[1], r2c[1])
    assert ra[0].shape == (50, 5)


def test_proposal_query_refusals(ctx):
    w, d = small_dict(ctx, n=50)
    q = query_set(4, 9, seed=1, lo=1, hi=5)
    m = nw.Model(ctx, 9)
    for C, k in ((0, 5), (nw.MAX_CANDIDATES + 1, 5), (16, 0)):
        with pytest.raises(nw.NwError) as e:
            m.query(d, q.codes, q.offsets, C=C, k=k)
        assert e.value.status == nw.NW_EINVAL
    bad = q.codes.copy()
    bad[0] = 9  # a code past the alphabet
    with pytest.raises(nw.NwError) as e:
        m.query(d, bad, q.offsets, C=8, k=3)
    assert e.value.status == nw.NW_EINVAL
    m.query(d, q.codes, q.offsets, C=8, k=3)  # still usable


def test_proposal_server_results_equal_the_call_alone(ctx):
    # requests of mixed sizes batched by the proposal server: each request's
    # lists equal the proposal query of its words alone (bit for bit)
    w, d = small_dict(ctx, n=2000, alphabet=12, seed=41, lo=1, hi=14)
    m = nw.Model(ctx, 12, seed=6)
    m.train(d, steps=100, batch_pairs=2048, lr=2e-3, seed=2)
    g = np.random.default_rng(7)
    reqs = [query_set(int(g.integers(1, 60)), 12, seed=100 + i, lo=0, hi=16) for i in range(16)]
    alone = [m.query(d, q.codes, q.offsets, C=32, k=7) for q in reqs]
    # one slot: requests that arrive while it runs share the next batch
    with nw.Server(d, k=7, max_batch_queries=160, max_inflight=1, proposal=(m, 32)) as srv:
        ids = [srv.submit(q.codes, q.offsets) for q in reqs]
        shared = 0
        for rid, (wi, ws) in zip(ids, alone):
            idx, sc, info = srv.wait(rid)
            assert np.array_equal(idx, wi) and np.array_equal(sc, ws)
            shared += info["batch_requests"] > 1
        assert shared > 0  # some batches carried several requests


def test_proposal_server_batches_overlap_on_the_device(ctx):
    """Requests submitted back to back, each filling a batch, run on several
    slots at once (a batch starts while others are on the device), and each
    result equals the proposal query of its words alone."""
    w = synth.exhaustive_words(100_000)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, synth.PAPER_SCORING)
    m = nw.Model(ctx, 40, seed=3)
    m.train(d, steps=100, batch_pairs=2048, lr=2e-3, seed=4)
    pool = synth.serving_queries(12_000)
    reqs = [pool.subset(np.arange(i * 2000, (i + 1) * 2000)) for i in range(6)]
    alone = [m.query(d, q.codes, q.offsets, C=128, k=10) for q in reqs]
    with nw.Server(d, k=10, max_batch_queries=2000, max_inflight=3, proposal=(m, 128)) as srv:
        ids = [srv.submit(q.codes, q.offsets) for q in reqs]
        out = [srv.wait(i) for i in ids]
    assert max(info["inflight_at_start"] for _, _, info in out) >= 1
    for (idx, sc, info), (wi, ws) in zip(out, alone):
        assert info["batch_requests"] == 1
        assert np.array_equal(idx, wi) and np.array_equal(sc, ws)


def test_proposal_server_refusals(ctx):
    w, d = small_dict(ctx, n=100)
    m = nw.Model(ctx, 9)
    for C in (0, nw.MAX_CANDIDATES + 1):
        with pytest.raises(nw.NwError) as e:
            nw.Server(d, k=5, proposal=(m, C))
        assert e.value.status == nw.NW_EINVAL
    other = nw.Context(0)
    try:
        m2 = nw.Model(other, 9)
        with pytest.raises(nw.NwError) as e:
            nw.Server(d, k=5, proposal=(m2, 8))
        assert e.value.status == nw.NW_EINVAL
        m2.free()
    finally:
        other.close()

