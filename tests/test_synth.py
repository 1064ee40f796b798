"""The seeded input generator: determinism, CSR validity and the workload shapes."""
import numpy as np

from paper_2509_01654_gb300 import synth


def test_splitmix64_reference_values():
    # SplitMix64 from state 0 (Steele, Lea and Flood 2014): the first outputs
    # of the sequential generator seeded with 0 are published test values.
    state = np.arange(1, 4, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
    out = synth._splitmix_out(state)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def test_deterministic_and_valid_csr():
    a = synth.make_words(5000, 40, 1.1, 8.0, 3.0, 1, 25, seed=2)
    b = synth.make_words(5000, 40, 1.1, 8.0, 3.0, 1, 25, seed=2)
    assert np.array_equal(a.codes, b.codes) and np.array_equal(a.offsets, b.offsets)
    assert a.offsets[0] == 0 and a.offsets.dtype == np.uint32
    assert np.all(np.diff(a.offsets.astype(np.int64)) >= 1)
    assert a.lengths.min() >= 1 and a.lengths.max() <= 25
    assert a.codes.max() < 40
    c = synth.make_words(5000, 40, 1.1, 8.0, 3.0, 1, 25, seed=3)
    assert not np.array_equal(a.codes[:100], c.codes[:100])


def test_workload_distributions():
    w = synth.exhaustive_words(200_000)
    L = w.lengths
    assert abs(L.mean() - 8.0) < 0.1 and abs(L.std() - 3.0) < 0.15
    # Zipf(1.1) over 40 codes: code 0 most frequent, frequencies decrease
    f = np.bincount(w.codes, minlength=40) / w.codes.size
    p = synth.zipf_probs(40, 1.1)
    assert np.allclose(f, p, atol=0.004)
    pr1 = synth.pr1_words()
    assert pr1.n == 2000 and pr1.lengths.min() >= 2 and pr1.lengths.max() <= 16
    assert pr1.n * (pr1.n - 1) // 2 == 1_999_000


def test_rounded_normal_law_matches_rejection_sampling():
    p = synth.rounded_normal_probs(7.0, 2.5, 2, 16)
    rng = np.random.default_rng(0)
    x = np.round(rng.normal(7.0, 2.5, 400_000))
    x = x[(x >= 2) & (x <= 16)].astype(int)
    f = np.bincount(x - 2, minlength=15) / x.size
    assert np.allclose(f, p, atol=0.003)


def test_sample_rows_and_queries():
    r = synth.sample_rows(600_000, 10_000)
    assert r.size == 10_000 and np.unique(r).size == 10_000 and r.max() < 600_000
    assert np.array_equal(r, synth.sample_rows(600_000, 10_000))
    q = synth.serving_queries(1000)
    assert q.lengths.min() >= 1 and q.lengths.max() <= 30


def test_batched_dictionaries_shapes():
    ds = synth.batched_dictionaries(count=6, size_lo=100, size_hi=400)
    for d in ds:
        m, x, g = d.scoring
        assert m in (1, 2, 3) and x in (-1, -2, -3) and g in (-1, -2, -3, -4)
        assert 100 <= d.words.n <= 400
        assert d.words.lengths.min() >= 1 and d.words.lengths.max() <= 40
        assert 40 <= d.words.alphabet <= 120 and d.words.codes.max() < d.words.alphabet


def test_batched_query_sets_shapes():
    ds = synth.batched_dictionaries(count=6, size_lo=100, size_hi=400)
    qs = synth.batched_query_sets(ds, size_lo=1, size_hi=300)
    assert len(qs) == len(ds)
    for d, q in zip(ds, qs):
        assert 1 <= q.n <= 300
        assert q.lengths.min() >= 1 and q.lengths.max() <= 40
        assert q.alphabet == d.words.alphabet and q.codes.max() < q.alphabet
    # deterministic, and not a copy of the dictionaries' own words
    again = synth.batched_query_sets(ds, size_lo=1, size_hi=300)
    assert all(np.array_equal(a.codes, b.codes) and np.array_equal(a.offsets, b.offsets) for a, b in zip(qs, again))
    assert len({q.n for q in qs}) > 1
