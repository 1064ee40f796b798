"""The no-allocation variant of the all-pairs top-k reduction.

nw_all_pairs_topk_noalloc serves callers that cannot allocate device memory
while the reduction runs (inside a stream capture, under a locked-down or
pool-managed allocator, or in a loop that must never reach cudaMalloc/cudaFree,
which synchronise the device).  It takes its scratch from one fixed static
device array in the library.  These tests call it through the C ABI and check
that two calls in a row give exactly what the allocating entry point gives
(scores are integers, so the tolerance is zero), and that requests beyond the
fixed array and host output buffers are refused with a clear error.

This file is collected last so that a run stopping at the first failure has
already run every other test."""
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


def test_noalloc_matches_allocating_entry_point_on_two_calls(ctx):
    import torch
    w = synth.make_words(4000, 40, 1.1, 8.0, 3.0, 1, 25, seed=2)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, synth.PAPER_SCORING)
    k = 10
    want_idx, want_score, want_hist, want_lo = d.all_pairs_topk(k)
    nbins = d.info()["nbins"]
    for call in range(2):
        # start from stale, non-zero contents so nothing passes by accident
        ti = torch.full((w.n, k), 7 + call, dtype=torch.int32, device="cuda")
        ts = torch.full((w.n, k), 5, dtype=torch.int16, device="cuda")
        th = torch.full((nbins,), 3, dtype=torch.int64, device="cuda")
        lo = d.all_pairs_topk_noalloc(k, ti, ts, th)
        assert lo == want_lo
        assert np.array_equal(ti.cpu().numpy().view(np.uint32), want_idx), f"indices differ on call {call}"
        assert np.array_equal(ts.cpu().numpy(), want_score), f"scores differ on call {call}"
        assert np.array_equal(th.cpu().numpy(), want_hist), f"histogram differs on call {call}"


def test_noalloc_without_histogram_and_other_k(ctx):
    import torch
    w = synth.make_uniform_length_words(1500, 12, 1.0, 1, 18, seed=11)
    d = ctx.load_dictionary(w.codes, w.offsets, 12, (2, -1, -2))
    for k in (3, 25):
        want_idx, want_score, _, _ = d.all_pairs_topk(k, hist=None)
        ti = torch.empty((w.n, k), dtype=torch.int32, device="cuda")
        ts = torch.empty((w.n, k), dtype=torch.int16, device="cuda")
        d.all_pairs_topk_noalloc(k, ti, ts)
        assert np.array_equal(ti.cpu().numpy().view(np.uint32), want_idx)
        assert np.array_equal(ts.cpu().numpy(), want_score)


def test_noalloc_refuses_what_it_cannot_hold(ctx):
    import torch
    w = synth.make_words(200, 40, 1.1, 8.0, 3.0, 1, 25, seed=3)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, synth.PAPER_SCORING)
    # host outputs would need staging buffers
    with pytest.raises(nw.NwError) as e:
        d.all_pairs_topk_noalloc(10, np.empty((w.n, 10), np.uint32), np.empty((w.n, 10), np.int16))
    assert e.value.status == nw.NW_EINVAL
    # 4*n*k bytes of list slots beyond the fixed array
    big = synth.make_words(70_000, 40, 1.1, 8.0, 3.0, 1, 25, seed=4)
    db = ctx.load_dictionary(big.codes, big.offsets, 40, synth.PAPER_SCORING)
    k = 128
    assert 4 * big.n * k > nw.NOALLOC_SCRATCH_BYTES
    ti = torch.empty((big.n, k), dtype=torch.int32, device="cuda")
    ts = torch.empty((big.n, k), dtype=torch.int16, device="cuda")
    with pytest.raises(nw.NwError) as e:
        db.all_pairs_topk_noalloc(k, ti, ts)
    assert e.value.status == nw.NW_ERANGE and "scratch" in str(e.value)


def test_noalloc_reaches_no_allocator(ctx):
    """With the context's next device allocation armed to fail, the
    no-allocation entry point still runs and matches, and the armed failure
    is still pending afterwards (the next allocating call trips it): the
    entry point never reached the allocator."""
    import torch
    w = synth.make_words(3000, 40, 1.1, 8.0, 3.0, 1, 25, seed=5)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, synth.PAPER_SCORING)
    k = 10
    want_idx, want_score, want_hist, want_lo = d.all_pairs_topk(k)
    nbins = d.info()["nbins"]
    ti = torch.empty((w.n, k), dtype=torch.int32, device="cuda")
    ts = torch.empty((w.n, k), dtype=torch.int16, device="cuda")
    th = torch.empty((nbins,), dtype=torch.int64, device="cuda")
    ctx.debug_fail_alloc(1)
    try:
        assert d.all_pairs_topk_noalloc(k, ti, ts, th) == want_lo
        with pytest.raises(nw.NwError) as e:  # loading a dictionary allocates
            ctx.load_dictionary(w.codes, w.offsets, 40, synth.PAPER_SCORING)
        assert e.value.status == nw.NW_ENOMEM and "injected" in str(e.value)
    finally:
        ctx.debug_fail_alloc(0)
    assert np.array_equal(ti.cpu().numpy().view(np.uint32), want_idx)
    assert np.array_equal(ts.cpu().numpy(), want_score)
    assert np.array_equal(th.cpu().numpy(), want_hist)


def test_noalloc_async_failure_is_reported_by_the_next_synchronous_call(ctx):
    """An NW_ASYNC call returns before its kernels finish and cannot report a
    device-side failure itself; the next synchronous call does, after
    computing its own valid outputs, and clears it."""
    import torch
    w = synth.make_words(2500, 40, 1.1, 8.0, 3.0, 1, 25, seed=6)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, synth.PAPER_SCORING)
    k = 10
    want_idx, want_score, _, _ = d.all_pairs_topk(k, hist=None)
    ti = torch.empty((w.n, k), dtype=torch.int32, device="cuda")
    ts = torch.empty((w.n, k), dtype=torch.int16, device="cuda")
    ctx.debug_set_bounds(insert_iters=0)  # every list insertion gives up at once
    try:
        d.all_pairs_topk_noalloc(k, ti, ts, async_=True)  # returns NW_OK: nothing read back
    finally:
        ctx.debug_set_bounds()
    torch.cuda.synchronize()
    with pytest.raises(nw.NwError) as e:
        d.all_pairs_topk_noalloc(k, ti, ts)
    assert e.value.status == nw.NW_ETIMEOUT and "NW_ASYNC" in str(e.value)
    # that synchronous call's own outputs are valid
    assert np.array_equal(ti.cpu().numpy().view(np.uint32), want_idx)
    assert np.array_equal(ts.cpu().numpy(), want_score)
    # and the report is not repeated
    d.all_pairs_topk_noalloc(k, ti, ts)
    assert np.array_equal(ti.cpu().numpy().view(np.uint32), want_idx)
