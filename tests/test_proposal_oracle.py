"""Pins the proposal oracle (oracle/proposal.py) to things other than itself:

* the forward pass against an explicit per-position loop and against closed
  forms for weights that make the network a (shifted) mean of embeddings;
* the autograd gradient against central finite differences of the forward;
* Adam's first step against its closed form -lr * g / (|g| + eps');
* quantisation against hand-worked values, and the quantised ranking value
  against the float prediction;
* the dot-product top-C against brute force on tiny inputs with ties;
* rescoring against sorting by hand-listed scores; recall against hand cases.
"""
import numpy as np
import pytest

from oracle import proposal as PR
from paper_2509_01654_gb300 import synth

torch = pytest.importorskip("torch")


def rand_params(alphabet, seed, scale=0.3):
    g = np.random.default_rng(seed)
    return g.normal(0.0, scale, PR.param_count(alphabet))


def loop_forward(flat, words, alphabet):
    """The network evaluated position by position with Python loops."""
    P = PR.unflatten(np.asarray(flat, dtype=np.float64), alphabet)
    out = np.zeros((words.n, PR.OUT))
    for i in range(words.n):
        w = words.word(i).astype(np.int64)
        L = len(w)
        x = [P["emb"][c] for c in w]
        for W, b in ((P["W1"], P["b1"]), (P["W2"], P["b2"]), (P["W3"], P["b3"])):
            y = []
            for t in range(L):
                acc = b.copy()
                for tap in range(3):
                    s = t + tap - 1
                    if 0 <= s < L:
                        acc = acc + W[:, tap, :] @ x[s]
                y.append(np.maximum(acc, 0.0))
            x = y
        pooled = np.sum(x, axis=0) / L if L else np.zeros(PR.CH)
        out[i] = P["Wl"] @ pooled + P["bl"]
    return out


def test_param_count_and_layout():
    A = 40
    assert PR.param_count(A) == A * 32 + 128 * 3 * 32 + 128 + 2 * (128 * 3 * 128 + 128) + 64 * 128 + 64
    flat = np.arange(PR.param_count(A), dtype=np.float64)
    P = PR.unflatten(flat, A)
    assert P["emb"][0, 0] == 0 and P["W1"][0, 0, 0] == A * 32
    assert P["bl"][-1] == flat[-1]


def test_forward_matches_position_loop():
    base = synth.make_uniform_length_words(25, 9, 1.0, 0, 7, seed=5)
    w = synth.WordList.from_lists([base.word(i).tolist() for i in range(base.n)] + [[], [4], [8, 8]], alphabet=9)
    assert (w.lengths == 0).any() and (w.lengths == 1).any()
    flat = rand_params(9, 1)
    assert np.allclose(PR.forward(flat, w, 9), loop_forward(flat, w, 9), rtol=1e-12, atol=1e-12)


def identity_params(alphabet, shift_tap=1):
    """Each convolution copies channel c < 32 from tap `shift_tap`; Wl reads channels 0..31."""
    P = {name: np.zeros(shape) for name, shape in PR.param_shapes(alphabet)}
    g = np.random.default_rng(3)
    P["emb"][:] = g.uniform(0.0, 1.0, P["emb"].shape)  # non-negative: ReLU passes it
    for W, cin in (("W1", 32), ("W2", 128), ("W3", 128)):
        for c in range(32):
            P[W][c, shift_tap, c] = 1.0
    for c in range(32):
        P["Wl"][c, c] = 1.0
    return np.concatenate([P[name].reshape(-1) for name, _ in PR.param_shapes(alphabet)]), P


def test_forward_closed_form_mean_of_embeddings():
    w = synth.make_words(30, 6, 1.0, 5.0, 2.0, 0, 9, seed=9)
    flat, P = identity_params(6, shift_tap=1)
    E = PR.forward(flat, w, 6)
    for i in range(w.n):
        c = w.word(i).astype(np.int64)
        want = P["emb"][c].mean(axis=0) if len(c) else np.zeros(32)
        assert np.allclose(E[i, :32], want) and np.allclose(E[i, 32:], 0.0)


def test_forward_closed_form_shift_and_zero_padding():
    # tap 0 reads x[t-1]: three layers shift the word right by 3 positions,
    # zero-filled, so the mean keeps the first L-3 embeddings over L
    w = synth.make_words(30, 6, 1.0, 6.0, 2.0, 1, 10, seed=10)
    flat, P = identity_params(6, shift_tap=0)
    E = PR.forward(flat, w, 6)
    for i in range(w.n):
        c = w.word(i).astype(np.int64)
        L = len(c)
        want = P["emb"][c[:max(L - 3, 0)]].sum(axis=0) / L
        assert np.allclose(E[i, :32], want)
    # tap 2 reads x[t+1]: the last L-3 embeddings
    flat2, P2 = identity_params(6, shift_tap=2)
    E2 = PR.forward(flat2, w, 6)
    for i in range(w.n):
        c = w.word(i).astype(np.int64)
        L = len(c)
        assert np.allclose(E2[i, :32], P2["emb"][c[3:]].sum(axis=0) / L)


def test_gradient_against_finite_differences():
    w = synth.make_words(12, 5, 1.0, 4.0, 2.0, 0, 6, seed=12)
    A = 5
    flat = rand_params(A, 2, scale=0.1)  # a loss of order 1: finite differences stay above roundoff
    g = np.random.default_rng(4)
    pi = g.integers(0, w.n, 10)
    pj = g.integers(0, w.n, 10)
    pj[0] = pi[0]  # a self pair
    y = g.uniform(-1, 1, 10)
    loss, grad = PR.loss_and_grad(flat, w, A, pi, pj, y)

    def loss_at(theta):
        E = PR.forward(theta, w, A)
        pred = np.array([E[a, :63] @ E[b, :63] + E[a, 63] + E[b, 63] for a, b in zip(pi, pj)])
        return np.mean((pred - y) ** 2)

    assert abs(loss - loss_at(flat)) < 1e-12 * max(1.0, loss)
    # every parameter block, a few coordinates each (coordinates with a
    # non-zero derivative included)
    h = 1e-6
    o = 0
    checked = 0
    for name, shape in PR.param_shapes(A):
        n = int(np.prod(shape))
        cand = np.nonzero(np.abs(grad[o:o + n]) > 1e-6)[0]
        pick = list(cand[:3]) + [0]
        for c in pick:
            e = np.zeros_like(flat)
            e[o + c] = h
            fd = (loss_at(flat + e) - loss_at(flat - e)) / (2 * h)
            assert abs(fd - grad[o + c]) <= 1e-6 + 1e-5 * abs(fd), (name, c, fd, grad[o + c])
            checked += 1
        o += n
    assert checked >= 18


def test_bf16_rounding_is_nearest_even():
    import torch
    u = 2.0 ** -8  # half the spacing of bfloat16 just above 1
    # ties go to the even neighbour; 65,280 = 255 * 2^8 has 8 significant bits
    x = torch.tensor([1 + u, 1 + 3 * u, -(1 + u), 1 + 1.5 * u, 3.0, 65280.0, 65408.0], dtype=torch.float64)
    want = [1.0, 1 + 4 * u, -1.0, 1 + 2 * u, 3.0, 65280.0, 65536.0]
    assert PR._bf16(x).tolist() == want


def test_bf16_products_match_autograd_on_representable_operands():
    # On operands bfloat16 holds exactly the rounding is the identity, so
    # the bf16 functions' forward and hand-written gradients must equal the
    # plain operations and their autograd gradients.
    import torch
    F = torch.nn.functional
    Conv, Lin = PR._bf16_funcs()
    g = np.random.default_rng(4)

    def rep(*shape):  # multiples of 1/16 in [-2, 2]: exact in bfloat16
        return torch.tensor(g.integers(-32, 33, shape) / 16.0, dtype=torch.float64)

    x, W, b = rep(3, 5, 7), rep(4, 3, 5), rep(4)
    gy = rep(3, 4, 7)
    args = [t.clone().requires_grad_(True) for t in (x, W, b)]
    Conv.apply(*args).backward(gy)
    ref = [t.clone().requires_grad_(True) for t in (x, W, b)]
    F.conv1d(ref[0], ref[1].permute(0, 2, 1), ref[2], padding=1).backward(gy)
    assert torch.equal(Conv.apply(x, W, b), F.conv1d(x, W.permute(0, 2, 1), b, padding=1))
    for a, r in zip(args, ref):
        assert torch.allclose(a.grad, r.grad, rtol=0, atol=1e-12)

    p, Wl, bl, ge = rep(6, 5), rep(3, 5), rep(3), rep(6, 3)
    args = [t.clone().requires_grad_(True) for t in (p, Wl, bl)]
    Lin.apply(*args).backward(ge)
    ref = [t.clone().requires_grad_(True) for t in (p, Wl, bl)]
    (ref[0] @ ref[1].T + ref[2]).backward(ge)
    for a, r in zip(args, ref):
        assert torch.allclose(a.grad, r.grad, rtol=0, atol=1e-12)


def test_bf16_forward_within_rounding_of_float64():
    # each product's operands carry a relative error of at most 2^-8 after
    # rounding; through three convolutions and the linear map the outputs
    # stay within a few percent of the float64 definition
    w = synth.make_uniform_length_words(60, 9, 1.0, 0, 12, seed=8)
    flat = np.random.default_rng(9).normal(0.0, 0.2, PR.param_count(9))
    a = PR.forward(flat, w, 9)
    b = PR.forward(flat, w, 9, bf16=True)
    rel = np.abs(a - b).max() / np.abs(a).max()
    assert 0 < rel < 3e-2, rel


def test_adam_first_step_closed_form():
    g = np.array([0.5, -2.0, 1e-3, 0.0])
    th = np.array([1.0, 1.0, 1.0, 1.0])
    t2, m, v = PR.adam_update(th, g, np.zeros(4), np.zeros(4), 1, lr=0.01)
    # m_hat = g, v_hat = g^2  ->  step = -lr * g / (|g| + eps)
    assert np.allclose(t2, th - 0.01 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)
    # second step with the same gradient: m_hat = g, v_hat = g^2 again
    t3, _, _ = PR.adam_update(t2, g, m, v, 2, lr=0.01)
    assert np.allclose(t3, t2 - 0.01 * g / (np.abs(g) + 1e-8), atol=1e-15)


def test_quantize_hand_values():
    # max |phi| = 2.54 -> scale 0.02; -1.0 / 0.02 = -50, 0.011 / 0.02 = 0.55 -> 1, 1.9 / 0.02 = 95;
    # the bias column (63) is left out of the scale and counted in units of scale^2 = 0.0004
    E = np.zeros((2, 64), dtype=np.float32)
    E[0, :4] = [2.54, -1.0, 0.011, 0.0]
    E[1, :4] = [-2.54, 1.9, -0.009, 0.3]
    E[:, 63] = [1000.0, -0.002]  # far above max |phi|: does not move the scale
    q, b, s = PR.quantize(E)
    assert abs(float(s) - 0.02) < 1e-9
    assert q[:, :4].tolist() == [[127, -50, 1, 0], [-127, 95, 0, 15]]
    assert not q[:, 4:].any()
    assert abs(int(b[0]) - 2_500_000) <= 1 and int(b[1]) == -5
    z, zb, s0 = PR.quantize(np.zeros((3, 64), np.float32))
    assert s0 == 0 and not z.any() and not zb.any()
    # the bias saturates at 2^23
    E[0, 63] = 1e6
    assert int(PR.quantize(E)[1][0]) == 1 << 23


def test_quantize_round_half_even():
    # max 127 -> scale exactly 1, so phi / scale is phi itself and scale^2 = 1
    E = np.zeros((1, 64), dtype=np.float32)
    E[0, :8] = [127.0, 0.5, 1.5, 2.5, -0.5, -1.5, 3.49, -126.51]
    E[0, 63] = 2.5
    q, b, s = PR.quantize(E)
    assert s == 1.0
    assert q[0, :8].tolist() == [127, 0, 2, 2, 0, -2, 3, -127]
    assert int(b[0]) == 2


def test_predict_matches_quantised_ranking_value():
    # q_a . q_b + bias_b approximates (pred(a, b) - beta_a) / scale^2
    g = np.random.default_rng(5)
    E = g.normal(0, 1, (50, 64)).astype(np.float32)
    q, b, s = PR.quantize(E)
    s2 = float(s) ** 2
    for a in range(5):
        for c in range(5, 10):
            exact = PR.predict(E[[a]], E[[c]])[0] - float(E[a, 63])
            approx = (int(q[a].astype(np.int64) @ q[c].astype(np.int64)) + int(b[c])) * s2
            # each quantised value is within scale/2 of its feature, the bias within scale^2/2
            pa, pc = np.abs(E[a, :63].astype(np.float64)), np.abs(E[c, :63].astype(np.float64))
            bound = np.sum(pa * s / 2 + pc * s / 2 + s2 / 4) + s2 / 2
            assert abs(exact - approx) <= bound * (1 + 1e-6)


def brute_dot_topk(q, C, bias=None):
    n = q.shape[0]
    bias = np.zeros(n, np.int64) if bias is None else bias
    out_i, out_d = [], []
    for i in range(n):
        lst = []
        for j in range(n):
            if j != i:
                lst.append((-(int(np.dot(q[i].astype(np.int64), q[j].astype(np.int64))) + int(bias[j])), j))
        lst.sort()
        lst = lst[:C]
        out_i.append([j for _, j in lst] + [0xFFFFFFFF] * (C - len(lst)))
        out_d.append([-d for d, _ in lst] + [-(2 ** 31)] * (C - len(lst)))
    return np.array(out_i, dtype=np.uint32), np.array(out_d, dtype=np.int32)


@pytest.mark.parametrize("n,C,levels", [(17, 5, 3), (9, 12, 2), (40, 8, 127), (2, 1, 5)])
def test_dot_topk_brute_force(n, C, levels):
    g = np.random.default_rng(n * 100 + C)
    q = g.integers(-levels, levels + 1, (n, 64)).astype(np.int8)
    q[n // 2] = q[0]  # duplicate rows: equal dot products
    idx, dot = PR.dot_topk(q, C)
    bi, bd = brute_dot_topk(q, C)
    assert np.array_equal(idx, bi) and np.array_equal(dot, bd)
    # sampled rows give the same lists
    r = np.array([0, n - 1])
    i2, d2 = PR.dot_topk(q, C, rows=r)
    assert np.array_equal(i2, bi[r]) and np.array_equal(d2, bd[r])
    # with per-column biases (ties between bias and dot product included)
    bias = g.integers(-3 * levels, 3 * levels + 1, n)
    bi3, bd3 = brute_dot_topk(q, C, bias)
    i3, d3 = PR.dot_topk(q, C, bias=bias)
    assert np.array_equal(i3, bi3) and np.array_equal(d3, bd3)


def test_dot_topk_cross_hand_case():
    # values qa_i . qb_j + bias_j worked by hand
    qa = np.zeros((2, 64), np.int8)
    qb = np.zeros((4, 64), np.int8)
    qa[0, :2] = (1, 0)
    qa[1, :2] = (0, 1)
    qb[:, :2] = [(2, 0), (1, 1), (0, 3), (1, 1)]
    bias = np.array([0, 1, -1, 1], np.int32)
    # row 0: (2, 2, -1, 2) -> j 0, 1, 3 tie at 2 (lower j first), then 2
    # row 1: (0, 2, 2, 2) -> j 1, 2, 3 tie at 2, then 0
    idx, val = PR.dot_topk_cross(qa, qb, 3, bias=bias)
    assert idx.tolist() == [[0, 1, 3], [1, 2, 3]]
    assert val.tolist() == [[2, 2, 2], [2, 2, 2]]
    idx, val = PR.dot_topk_cross(qa, qb, 6, bias=bias)  # more than nb: missing tail
    assert idx[0, 4:].tolist() == [PR.MISSING_IDX] * 2 and val[1, 4:].tolist() == [PR.MISSING_DOT] * 2
    assert idx[0, :4].tolist() == [0, 1, 3, 2] and val[1, :4].tolist() == [2, 2, 2, 0]


@pytest.mark.parametrize("n,C", [(40, 5), (33, 31), (9, 12)])
def test_dot_topk_cross_with_itself_is_dot_topk_plus_self(n, C):
    # rows against their own set: dropping column i from the C + 1 best
    # gives the C best other rows
    g = np.random.default_rng(n)
    q = g.integers(-2, 3, (n, 64)).astype(np.int8)
    bias = g.integers(-3, 4, n).astype(np.int32)
    ci, cv = PR.dot_topk_cross(q, q, C + 1, bias=bias)
    wi, wv = PR.dot_topk(q, C, bias=bias)
    for i in range(n):
        keep = ci[i] != i
        got_i, got_v = ci[i][keep][:C], cv[i][keep][:C]
        assert np.array_equal(got_i, wi[i]) and np.array_equal(got_v, wv[i])


def test_rescore_topk_hand_case(oracle_mod):
    w = synth.WordList.from_lists([[1, 2, 3], [1, 2, 3], [1, 2], [4, 5, 6], [1, 2, 4]])
    sc = (1, -1, -1)
    # scores against word 0: w1 3, w2 1 (2 matches, 1 gap), w3 -3, w4 1 (2 matches, 1 mismatch)
    cand = np.array([[3, 4, 2, 1], [0, PR.MISSING_IDX, 3, PR.MISSING_IDX],
                     [0, 1, 3, 4], [0, 1, 2, 4], [0, 1, 2, 3]], dtype=np.uint32)
    idx, s = PR.rescore_topk(oracle_mod, w, cand, 3, sc)
    assert idx[0].tolist() == [1, 2, 4] and s[0].tolist() == [3, 1, 1]
    assert idx[1].tolist() == [0, 3, 0xFFFFFFFF] and s[1].tolist() == [3, -3, -(2 ** 31)]


def test_recall_hand_cases():
    ex_i = np.array([[1, 2, 3], [0, 2, 3]], dtype=np.uint32)
    ex_s = np.array([[5, 4, 4], [9, 8, 7]], dtype=np.int32)
    ap_i = np.array([[1, 3, 7], [0, 2, 3]], dtype=np.uint32)
    ap_s = np.array([[5, 4, 4], [9, 8, 7]], dtype=np.int32)  # 7 ties the 3rd exact score
    strict, tie = PR.recall_at_k(ex_i, ex_s, ap_i, ap_s)
    assert abs(strict - (2 / 3 + 1) / 2) < 1e-12
    assert tie == 1.0
