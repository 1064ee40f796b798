"""Failure detection on the device, exercised without faulting the GPU.

Every wait or retry loop in the library's kernels is bounded; when a bound
runs out the kernel raises a bit in a device error word, stops the work it
cannot finish, waits (again bounded) for the copies it has in flight and
returns, and the host turns the bit into NW_ETIMEOUT.  These tests make the
bounds run out on purpose through nw_debug_set_bounds:

* the alignment kernel's neighbour-list insertion gives up at its first
  compare-and-swap round (bound 0), so the first list offer fails;
* the candidate kernel's producer never issues one column tile's bulk copy
  and the pipeline waits are cut to about a millisecond, so the waits for that
  tile run out with no copy in flight.

Each test then restores the defaults and checks that the same context gives
the oracle's exact result, i.e. that the failure left the context usable.
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
    c.debug_set_bounds()
    c.close()


def test_list_insertion_bound_reports_timeout_and_context_recovers(ctx, oracle_mod):
    w = synth.make_words(3000, 40, 1.1, 8.0, 3.0, 1, 25, seed=2)
    d = ctx.load_dictionary(w.codes, w.offsets, 40, synth.PAPER_SCORING)
    ctx.debug_set_bounds(insert_iters=0)
    try:
        with pytest.raises(nw.NwError) as e:
            d.all_pairs_topk(10)
        assert e.value.status == nw.NW_ETIMEOUT
        assert "retry bound" in str(e.value)
        # the query path runs the same kernels and bound
        q = synth.serving_queries(50)
        with pytest.raises(nw.NwError) as e:
            d.query(q.codes, q.offsets, 10)
        assert e.value.status == nw.NW_ETIMEOUT
    finally:
        ctx.debug_set_bounds()
    idx, score, hist, lo = d.all_pairs_topk(10)
    rows = synth.sample_rows(w.n, 200, seed=6)
    wi, ws = oracle_mod.topk_rows(w, rows, 10, synth.PAPER_SCORING)
    assert np.array_equal(idx[rows], wi)
    assert np.array_equal(score[rows].astype(np.int32), ws)
    assert int(hist.sum()) == w.n * (w.n - 1) // 2


@pytest.mark.parametrize("withhold", [0, 8])  # issued before the sweep, and by a refill of the ring
def test_candidate_pipeline_wait_reports_timeout_and_context_recovers(ctx, withhold):
    n, C = 20_000, 64  # 157 column tiles of 128, two column splits of 79
    g = np.random.default_rng(11)
    q = g.integers(-127, 128, (n, 64)).astype(np.int8)
    bias = g.integers(-20_000, 20_001, n).astype(np.int32)
    ctx.debug_set_bounds(wait_cycles=2_000_000, withhold_tile=withhold)
    try:
        with pytest.raises(nw.NwError) as e:
            nw.dot_topk(ctx, q, C, bias=bias)
        assert e.value.status == nw.NW_ETIMEOUT
        assert "wait" in str(e.value)
    finally:
        ctx.debug_set_bounds()
    idx, dot = nw.dot_topk(ctx, q, C, bias=bias)
    rows = synth.sample_rows(n, 300, seed=6)
    wi, wd = PR.dot_topk(q, C, rows=rows, bias=bias)
    assert np.array_equal(dot[rows], wd)
    assert np.array_equal(idx[rows], wi)


def test_short_wait_bound_alone_still_completes(ctx):
    """A bound that is short but long enough for every copy to land changes
    nothing: the waits that finish in time are not errors."""
    n, C = 1500, 32
    g = np.random.default_rng(12)
    q = g.integers(-127, 128, (n, 64)).astype(np.int8)
    ctx.debug_set_bounds(wait_cycles=200_000_000)
    try:
        idx, dot = nw.dot_topk(ctx, q, C)
    finally:
        ctx.debug_set_bounds()
    wi, wd = PR.dot_topk(q, C)
    assert np.array_equal(dot, wd)
    assert np.array_equal(idx, wi)
