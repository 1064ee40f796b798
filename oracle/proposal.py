"""CPU oracle of the learned candidate proposal (test infrastructure only).

The paper scores every pair exhaustively; this module defines the learned
shortcut built on top of it, a character CNN whose embeddings' dot products
propose neighbour candidates that are then rescored exactly by Algorithm 1.
The paper does not define the network; these functions are the definition
the CUDA path is checked against, written plainly:

* ``forward``: codes -> embedding table (32) -> three 1-D convolutions of
  width 3 with 128 channels, zero padding, ReLU -> mean over the word's
  positions -> linear map to 64 values.  Plain PyTorch CPU ops in float64.
  With ``bf16=True`` every matrix product takes its two operands rounded
  to bfloat16 (through float32, nearest even), the precision the
  network's weights and products are specified in (BF16 operands,
  float32 accumulation); the products themselves stay exact in float64.
  In ``loss_and_grad`` the gradient products round their operands the
  same way (the output gradient and the saved input or weight); bias
  gradients are sums of the unrounded output gradient.
* ``predict``: the modelled similarity of two words.  The 64 outputs are
  read as 63 features phi and one bias beta, and
  pred(a, b) = phi_a . phi_b + beta_a + beta_b.  A raw alignment score
  carries a -len(A) - len(B) term that no dot product of one embedding per
  word can express (its Gram matrix is positive semi-definite); the two
  biases carry it.
* ``loss_and_grad``: squared error of pred against a target (the library
  trains on Section 5's normalised weight s / max(len(A), len(B)) or on the
  raw score times a constant), averaged over the pairs; gradient by autograd.
* ``adam_update``: one Adam step (Kingma and Ba, 2015) with bias correction.
* ``quantize``: symmetric 8-bit quantisation of the 63 features with one
  scale, the bias in units of scale^2 (so that q_a . q_b + bias_b is the
  quantised phi_a . phi_b + beta_b), in float32 (the precision the library
  takes these decisions in).
* ``dot_topk``: each row's C best other rows by the exact integer value
  q_i . q_j + bias_j, higher first, lower index on ties.
* ``dot_topk_cross``: the same over two sets: each row of one set's C best
  rows of the other (no row skipped).
* ``rescore_topk``: the k best of each row's candidates by Algorithm 1's
  score (the oracle's C code), higher first, lower index on ties.
* ``recall_at_k``: strict and tie-aware overlap of two sets of lists.

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this module.

Flat parameter layout (float32 in the library, float64 here), in order:
    emb [A][32], W1 [128][3][32], b1 [128], W2 [128][3][128], b2 [128],
    W3 [128][3][128], b3 [128], Wl [64][128], bl [64]
A convolution computes y[t][o] = b[o] + sum_tap sum_c W[o][tap][c] * x[t + tap - 1][c]
with x = 0 outside the word.
"""
from __future__ import annotations

import numpy as np

EMB = 32
CH = 128
OUT = 64
FEAT = 63   # outputs 0..62 are features, output 63 is the bias
TAPS = 3
BIAS_LIMIT = 1 << 23

MISSING_IDX = np.uint32(0xFFFFFFFF)
MISSING_DOT = np.int32(-(2 ** 31))
MISSING_SCORE = np.int32(-(2 ** 31))


def param_shapes(alphabet: int):
    return [("emb", (alphabet, EMB)), ("W1", (CH, TAPS, EMB)), ("b1", (CH,)),
            ("W2", (CH, TAPS, CH)), ("b2", (CH,)), ("W3", (CH, TAPS, CH)), ("b3", (CH,)),
            ("Wl", (OUT, CH)), ("bl", (OUT,))]


def param_count(alphabet: int) -> int:
    return int(sum(np.prod(s) for _, s in param_shapes(alphabet)))


def unflatten(flat, alphabet: int) -> dict:
    out, o = {}, 0
    for name, shape in param_shapes(alphabet):
        n = int(np.prod(shape))
        out[name] = flat[o:o + n].reshape(shape)
        o += n
    assert o == flat.shape[0]
    return out


def _torch():
    import torch
    return torch


def _bf16(x):
    """x (float64 tensor) rounded to float32, then to bfloat16 (nearest
    even), returned as float64."""
    torch = _torch()
    return x.to(torch.float32).to(torch.bfloat16).to(torch.float64)


_FUNCS = {}


def _bf16_funcs():
    """autograd functions of a convolution and of the linear map whose
    forward and gradient products take bf16-rounded operands."""
    if _FUNCS:
        return _FUNCS["conv"], _FUNCS["lin"]
    torch = _torch()
    F = torch.nn.functional

    class Conv(torch.autograd.Function):
        @staticmethod
        def forward(ctx, x, W, b):  # x (n, C, L), W (o, tap, c)
            xr, Wr = _bf16(x), _bf16(W)
            ctx.save_for_backward(xr, Wr)
            return F.conv1d(xr, Wr.permute(0, 2, 1), b, padding=1)

        @staticmethod
        def backward(ctx, gy):
            xr, Wr = ctx.saved_tensors
            gr = _bf16(gy)
            w_oct = Wr.permute(0, 2, 1)
            gx = torch.nn.grad.conv1d_input(xr.shape, w_oct, gr, padding=1)
            gw = torch.nn.grad.conv1d_weight(xr, w_oct.shape, gr, padding=1).permute(0, 2, 1)
            return gx, gw, gy.sum(dim=(0, 2))

    class Lin(torch.autograd.Function):
        @staticmethod
        def forward(ctx, p, W, b):  # p (n, Ci), W (Co, Ci)
            pr, Wr = _bf16(p), _bf16(W)
            ctx.save_for_backward(pr, Wr)
            return pr @ Wr.T + b

        @staticmethod
        def backward(ctx, ge):
            pr, Wr = ctx.saved_tensors
            gr = _bf16(ge)
            return gr @ Wr, gr.T @ pr, ge.sum(dim=0)

    _FUNCS["conv"], _FUNCS["lin"] = Conv, Lin
    return Conv, Lin


def _forward_t(P, words, bf16=False):
    """Embeddings (n, 64) as a float64 torch tensor; P holds torch tensors."""
    torch = _torch()
    conv = lin = None
    if bf16:
        Conv, Lin = _bf16_funcs()
        conv, lin = Conv.apply, Lin.apply
    n = words.n
    lens = torch.tensor(words.lengths, dtype=torch.int64)
    Lp = max(1, int(lens.max().item()) if n else 1)
    codes = torch.zeros((n, Lp), dtype=torch.int64)
    for i in range(n):
        w = words.word(i)
        if len(w):
            codes[i, :len(w)] = torch.tensor(w.astype(np.int64))
    mask = (torch.arange(Lp)[None, :] < lens[:, None]).to(torch.float64)  # (n, Lp)
    x = P["emb"][codes] * mask[:, :, None]                                # (n, Lp, 32)
    x = x.transpose(1, 2)                                                 # (n, C, Lp)
    for W, b in ((P["W1"], P["b1"]), (P["W2"], P["b2"]), (P["W3"], P["b3"])):
        # W[o][tap][c] with tap 0 reading x[t - 1]: conv1d's weight[o][c][tap]
        # with padding 1 computes sum_tap weight[o][c][tap] * x[t + tap - 1]
        y = conv(x, W, b) if bf16 else torch.nn.functional.conv1d(x, W.permute(0, 2, 1), b, padding=1)
        x = torch.relu(y) * mask[:, None, :]  # positions past the word are zero input to the next layer
    denom = lens.clamp(min=1).to(torch.float64)
    pooled = x.sum(dim=2) / denom[:, None]                                # (n, 128); empty word -> 0
    if bf16:
        return lin(pooled, P["Wl"], P["bl"])
    return pooled @ P["Wl"].T + P["bl"]


def forward(flat, words, alphabet: int, bf16: bool = False) -> np.ndarray:
    """float64 embeddings (n, 64) of every word for the flat parameters."""
    torch = _torch()
    P = {k: torch.tensor(np.asarray(v, dtype=np.float64)) for k, v in unflatten(np.asarray(flat), alphabet).items()}
    with torch.no_grad():
        return _forward_t(P, words, bf16).numpy()


def _predict_t(Ea, Eb):
    return (Ea[:, :FEAT] * Eb[:, :FEAT]).sum(dim=1) + Ea[:, FEAT] + Eb[:, FEAT]


def predict(Ea, Eb) -> np.ndarray:
    """pred(a, b) = phi_a . phi_b + beta_a + beta_b for rows of two embedding arrays."""
    Ea = np.asarray(Ea, dtype=np.float64)
    Eb = np.asarray(Eb, dtype=np.float64)
    return np.sum(Ea[:, :FEAT] * Eb[:, :FEAT], axis=1) + Ea[:, FEAT] + Eb[:, FEAT]


def loss_and_grad(flat, words, alphabet: int, pi, pj, target, bf16: bool = False):
    """(loss, gradient of the flat parameters): mean over pairs of
    (pred(E[pi], E[pj]) - target)^2."""
    torch = _torch()
    flat_t = torch.tensor(np.asarray(flat, dtype=np.float64), requires_grad=True)
    P, o = {}, 0
    for name, shape in param_shapes(alphabet):
        n = int(np.prod(shape))
        P[name] = flat_t[o:o + n].reshape(shape)
        o += n
    E = _forward_t(P, words, bf16)
    pi = torch.tensor(np.asarray(pi, dtype=np.int64))
    pj = torch.tensor(np.asarray(pj, dtype=np.int64))
    y = torch.tensor(np.asarray(target, dtype=np.float64))
    pred = _predict_t(E[pi], E[pj])
    loss = ((pred - y) ** 2).mean()
    loss.backward()
    return float(loss.item()), flat_t.grad.numpy().copy()


def adam_update(theta, grad, m, v, step: int, lr: float, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam step (step counts from 1); returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mhat = m / (1.0 - beta1 ** step)
    vhat = v / (1.0 - beta2 ** step)
    return theta - lr * mhat / (np.sqrt(vhat) + eps), m, v


def quantize(E):
    """(q int8 (n, 64), bias int32 (n,), scale float32), all in float32:
    scale = max|phi| / 127 over the 63 features of all rows; q[:, :63] =
    round-half-even(phi / scale) clamped to [-127, 127], q[:, 63] = 0;
    bias = round-half-even(beta / (scale * scale)) clamped to +-2^23.  A zero
    scale gives q = 0 and bias = 0."""
    E = np.asarray(E, dtype=np.float32)
    n = E.shape[0]
    phi = E[:, :FEAT]
    amax = np.float32(np.max(np.abs(phi))) if phi.size else np.float32(0)
    scale = np.float32(amax / np.float32(127.0))
    q = np.zeros((n, OUT), dtype=np.int8)
    bias = np.zeros(n, dtype=np.int32)
    if scale == 0:
        return q, bias, scale
    q[:, :FEAT] = np.clip(np.rint(phi / scale), -127, 127).astype(np.int8)
    s2 = np.float32(scale * scale)
    bias[:] = np.clip(np.rint(E[:, FEAT] / s2), -BIAS_LIMIT, BIAS_LIMIT).astype(np.int32)
    return q, bias, scale


def dot_topk(q, C: int, rows=None, bias=None):
    """(idx uint32 (r, C), val int32 (r, C)): for each row i, the C rows j != i
    with the largest exact q_i . q_j + bias_j (bias 0 when None), lower j
    first on ties; missing entries (fewer than C other rows) are
    (MISSING_IDX, MISSING_DOT)."""
    q = np.asarray(q, dtype=np.int64)
    n = q.shape[0]
    b = np.zeros(n, dtype=np.int64) if bias is None else np.asarray(bias, dtype=np.int64)
    rows = np.arange(n) if rows is None else np.asarray(rows, dtype=np.int64)
    idx = np.full((rows.size, C), MISSING_IDX, dtype=np.uint32)
    dot = np.full((rows.size, C), MISSING_DOT, dtype=np.int32)
    jj = np.arange(n)
    for b0 in range(0, rows.size, 256):
        rb = rows[b0:b0 + 256]
        D = q[rb] @ q.T + b[None, :]  # exact in int64
        for r, i in enumerate(rb):
            keep = jj != i
            order = np.lexsort((jj[keep], -D[r, keep]))[:C]
            sel = jj[keep][order]
            idx[b0 + r, :sel.size] = sel
            dot[b0 + r, :sel.size] = D[r, sel]
    return idx, dot


def dot_topk_cross(qa, qb, C: int, bias=None, rows=None):
    """(idx uint32 (r, C), val int32 (r, C)): for each row i of qa, the C
    rows j of qb with the largest exact qa_i . qb_j + bias_j (bias 0 when
    None), lower j first on ties; every j is eligible (qa and qb are two
    sets); missing entries (qb has fewer than C rows) are
    (MISSING_IDX, MISSING_DOT)."""
    qa = np.asarray(qa, dtype=np.int64)
    qb = np.asarray(qb, dtype=np.int64).reshape(-1, OUT)
    nb = qb.shape[0]
    b = np.zeros(nb, dtype=np.int64) if bias is None else np.asarray(bias, dtype=np.int64)
    rows = np.arange(qa.shape[0]) if rows is None else np.asarray(rows, dtype=np.int64)
    idx = np.full((rows.size, C), MISSING_IDX, dtype=np.uint32)
    dot = np.full((rows.size, C), MISSING_DOT, dtype=np.int32)
    jj = np.arange(nb)
    for b0 in range(0, rows.size, 256):
        rb = rows[b0:b0 + 256]
        D = qa[rb] @ qb.T + b[None, :]  # exact in int64
        for r in range(rb.size):
            order = np.lexsort((jj, -D[r]))[:C]
            idx[b0 + r, :order.size] = order
            dot[b0 + r, :order.size] = D[r, order]
    return idx, dot


def rescore_topk(oracle_mod, words, cand, k: int, scoring):
    """(idx, score) (n, k): each row's k best candidates (entries != MISSING_IDX,
    distinct) by Algorithm 1's score, higher first, lower index on ties."""
    cand = np.asarray(cand, dtype=np.uint32)
    n, C = cand.shape
    I = np.repeat(np.arange(n, dtype=np.uint32), C)
    J = cand.reshape(-1)
    ok = J != MISSING_IDX
    S = np.full(I.size, MISSING_SCORE, dtype=np.int64)
    if ok.any():
        S[ok] = oracle_mod.score_pairs(words, I[ok], J[ok], scoring)
    S = S.reshape(n, C)
    idx = np.full((n, k), MISSING_IDX, dtype=np.uint32)
    sc = np.full((n, k), MISSING_SCORE, dtype=np.int32)
    for i in range(n):
        v = cand[i] != MISSING_IDX
        j = cand[i][v].astype(np.int64)
        s = S[i][v]
        order = np.lexsort((j, -s))[:k]
        idx[i, :order.size] = j[order]
        sc[i, :order.size] = s[order]
    return idx, sc


def recall_at_k(exact_idx, exact_score, approx_idx, approx_score):
    """(strict, tie_aware): strict = |approx list ∩ exact list| / |exact list|;
    tie-aware counts an approx neighbour whose true score is >= the exact
    list's last score (any of them is a correct k-th neighbour).  Means over
    rows with a non-empty exact list."""
    ok_rows = exact_idx[:, 0] != MISSING_IDX
    strict, tie = [], []
    for i in np.nonzero(ok_rows)[0]:
        e = exact_idx[i][exact_idx[i] != MISSING_IDX]
        a_ok = approx_idx[i] != MISSING_IDX
        a = approx_idx[i][a_ok]
        strict.append(len(set(e.tolist()) & set(a.tolist())) / e.size)
        kth = exact_score[i][exact_idx[i] != MISSING_IDX][-1]
        good = int(np.sum(approx_score[i][a_ok] >= kth))
        tie.append(min(good, e.size) / e.size)
    return float(np.mean(strict)), float(np.mean(tie))
