"""Pins the CPU oracle to things other than itself (arxiv 2509.01654).

* the paper's printed worked examples (Section 2: puissance/nuance at p = -2,
  the optimal score, single cells along the printed path and the -15
  non-optimal alignment; Section 5: puisant/paysans = 3, puisant/epuisant = 4
  at p = -1 and their normalised weights);
* brute-force enumeration of every alignment of short words, scored as the
  sum over alignment columns of the similarity or the gap value;
* textbook reductions: (0, -1, -1) gives minus the Levenshtein distance,
  (1, 0, 0) gives the length of a longest common subsequence;
* invariants: symmetry, score(a, a) = len * match, the alignment-count bounds;
* layout: the row-major upper triangle against the paper's closed-form
  idx -> (row, col) map of Section 4.2 and the edge count n(n-1)/2;
* selection: top-k lists and histograms against numpy sorts and bincounts.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from conftest import read_golden
from paper_2509_01654_gb300 import synth


def ints(s):
    return [int(t) for t in s.split()]


# ---------------------------------------------------------------------------
# alignment enumeration (independent of any DP)

def alignments(la, lb):
    """Every global alignment as a list of columns (i or None, j or None)."""
    if la == 0 and lb == 0:
        yield []
        return
    if la > 0 and lb > 0:
        for rest in alignments(la - 1, lb - 1):
            yield rest + [(la - 1, lb - 1)]
    if la > 0:
        for rest in alignments(la - 1, lb):
            yield rest + [(la - 1, None)]
    if lb > 0:
        for rest in alignments(la, lb - 1):
            yield rest + [(None, lb - 1)]


def column_score(A, B, cols, scoring):
    m, x, g = scoring
    s = 0
    for i, j in cols:
        if i is None or j is None:
            s += g
        else:
            s += m if A[i] == B[j] else x
    return s


def brute_force(A, B, scoring):
    return max(column_score(A, B, c, scoring) for c in alignments(len(A), len(B)))


def delannoy(m, n):
    return sum(math.comb(m, k) * math.comb(n, k) * 2 ** k for k in range(min(m, n) + 1))


def levenshtein(a, b):
    prev = list(range(len(b) + 1))
    for i in range(1, len(a) + 1):
        cur = [i] + [0] * len(b)
        for j in range(1, len(b) + 1):
            cur[j] = min(prev[j] + 1, cur[j - 1] + 1, prev[j - 1] + (a[i - 1] != b[j - 1]))
        prev = cur
    return prev[-1]


def lcs_length(a, b):
    L = [[0] * (len(b) + 1) for _ in range(len(a) + 1)]
    for i in range(1, len(a) + 1):
        for j in range(1, len(b) + 1):
            L[i][j] = L[i - 1][j - 1] + 1 if a[i - 1] == b[j - 1] else max(L[i - 1][j], L[i][j - 1])
    return L[-1][-1]


def random_word(rng, lo, hi, alphabet):
    return rng.integers(0, alphabet, size=int(rng.integers(lo, hi + 1))).astype(np.uint8)


SCORINGS = [(1, -1, -1), (1, -1, -2), (2, -1, -1), (3, -3, -4), (1, -3, -1), (0, -1, -1),
            (1, 0, 0), (2, 1, -1), (1, 1, 0), (3, -2, 1)]


# ---------------------------------------------------------------------------
# printed worked examples

def test_puissance_nuance_worked_example(oracle_mod):
    g = read_golden("puissance_nuance.txt")
    A, B, sc = ints(g["A"][0]), ints(g["B"][0]), tuple(ints(g["scoring"][0]))
    H = oracle_mod.score_matrix(A, B, sc)
    assert H.shape == (len(A) + 1, len(B) + 1)
    assert int(H[-1, -1]) == int(g["score"][0]) == oracle_mod.score(A, B, sc)
    for c in g["cell"]:
        i, j, v = ints(c)
        assert int(H[i, j]) == v, (i, j)
    # the gap row and column hold p * index (Algorithm 1 initialisation)
    assert list(H[:, 0]) == [sc[2] * i for i in range(len(A) + 1)]
    assert list(H[0, :]) == [sc[2] * j for j in range(len(B) + 1)]


def test_non_optimal_alignment_scores_minus_15(oracle_mod):
    g = read_golden("puissance_nuance.txt")
    A, B, sc = ints(g["A"][0]), ints(g["B"][0]), tuple(ints(g["scoring"][0]))
    cols, ia, ib = [], 0, 0
    for col in g["nonopt"][0].split("|"):
        a, b = col.split()
        assert a == "-" or int(a) == A[ia]
        assert b == "-" or int(b) == B[ib]
        cols.append((None if a == "-" else ia, None if b == "-" else ib))
        ia += a != "-"
        ib += b != "-"
    assert (ia, ib) == (len(A), len(B))
    assert column_score(A, B, cols, sc) == int(g["nonopt_score"][0])
    # the optimum over every alignment is the printed optimal score
    assert brute_force(A, B, sc) == int(g["score"][0]) == oracle_mod.score(A, B, sc)


def test_puisant_paysans_epuisant(oracle_mod):
    g = read_golden("puisant_paysans_epuisant.txt")
    w = {k: ints(g[k][0]) for k in ("puisant", "paysans", "epuisant")}
    sc = tuple(ints(g["scoring"][0]))
    for key, vals in g.items():
        if key.startswith("score "):
            _, a, b = key.split()
            s = oracle_mod.score(w[a], w[b], sc)
            assert s == int(vals[0]) == brute_force(w[a], w[b], sc)
            assert oracle_mod.score(w[b], w[a], sc) == s
    for key, vals in g.items():
        if key.startswith("normalised "):
            _, a, b = key.split()
            s = oracle_mod.score(w[a], w[b], sc)
            assert Fraction(100 * s, max(len(w[a]), len(w[b]))) == Fraction(vals[0])
    assert round(float(Fraction(200, 3)), 1) == 66.7


# ---------------------------------------------------------------------------
# brute force and textbook reductions

def test_delannoy_counts_of_enumerator():
    for la, lb in [(0, 0), (1, 0), (2, 3), (4, 4), (5, 3)]:
        assert sum(1 for _ in alignments(la, lb)) == delannoy(la, lb)
    assert delannoy(7, 7) == 48639


@pytest.mark.parametrize("scoring", SCORINGS)
def test_brute_force_small_words(oracle_mod, scoring):
    rng = np.random.default_rng(1000 + SCORINGS.index(scoring))
    for _ in range(40):
        A = random_word(rng, 0, 5, 4)
        B = random_word(rng, 0, 5, 4)
        assert oracle_mod.score(A, B, scoring) == brute_force(A, B, scoring), (A, B)


def test_brute_force_length_seven(oracle_mod):
    rng = np.random.default_rng(77)
    for scoring in [(1, -1, -1), (2, -3, -1)]:
        for _ in range(3):
            A = random_word(rng, 7, 7, 3)
            B = random_word(rng, 6, 7, 3)
            assert oracle_mod.score(A, B, scoring) == brute_force(A, B, scoring)


def test_levenshtein_and_lcs_reductions(oracle_mod):
    rng = np.random.default_rng(5)
    for _ in range(300):
        A = random_word(rng, 0, 12, 5)
        B = random_word(rng, 0, 12, 5)
        assert oracle_mod.score(A, B, (0, -1, -1)) == -levenshtein(list(A), list(B))
        assert oracle_mod.score(A, B, (1, 0, 0)) == lcs_length(list(A), list(B))


def test_empty_words_score_gap_times_length(oracle_mod):
    for sc in SCORINGS:
        assert oracle_mod.score([], [], sc) == 0
        assert oracle_mod.score([], [1, 2, 3], sc) == 3 * sc[2]
        assert oracle_mod.score([4, 4], [], sc) == 2 * sc[2]


# ---------------------------------------------------------------------------
# invariants

def bounds(la, lb, scoring):
    m, x, g = scoring
    lo_ = max((la + lb) * g, min(la, lb) * min(m, x) + abs(la - lb) * g)
    hi_ = max((la + lb) * g, min(la, lb) * max(m, x) + abs(la - lb) * g)
    return lo_, hi_


def test_invariants_random(oracle_mod):
    rng = np.random.default_rng(9)
    for sc in SCORINGS:
        for _ in range(60):
            A = random_word(rng, 0, 14, 6)
            B = random_word(rng, 0, 14, 6)
            s = oracle_mod.score(A, B, sc)
            assert s == oracle_mod.score(B, A, sc)
            lo_, hi_ = bounds(len(A), len(B), sc)
            assert lo_ <= s <= hi_
            m, x, g = sc
            if m >= x and g <= 0 and m >= 2 * g:
                assert oracle_mod.score(A, A, sc) == len(A) * m


# ---------------------------------------------------------------------------
# layout of the all-pairs output

def paper_row_col(idx, n):
    """Section 4.2: r = floor(z - sqrt(z^2 - 2 idx)), z = n - 1/2, c = r + 1 + idx - S_{r-1},
    in fp64 as the paper does, with an integer fix-up of r for rounding."""
    z = n - 0.5
    r = int(math.floor(z - math.sqrt(z * z - 2.0 * idx)))

    def S_before(r_):  # elements traversed before row r_
        return r_ * (2 * n - r_ - 1) // 2

    while r > 0 and S_before(r) > idx:
        r -= 1
    while S_before(r + 1) <= idx:
        r += 1
    c = 0.5 * r * r + r * (1.5 - n) + (idx + 1)
    return r, int(round(c))


def test_closed_form_row_col_for_n4():
    # Section 4.2, the n = 4 example: idx 0..5 walk (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
    assert [paper_row_col(i, 4) for i in range(6)] == [(0, 1), (0, 2), (0, 3), (1, 2), (1, 3), (2, 3)]


def test_all_pairs_layout_matches_paper_traversal(oracle_mod):
    w = synth.make_words(37, 6, 1.0, 4.0, 2.0, 0, 9, seed=11)
    sc = (1, -1, -1)
    out = oracle_mod.all_pairs(w, sc)
    n = w.n
    assert out.size == n * (n - 1) // 2
    for idx in range(out.size):
        r, c = paper_row_col(idx, n)
        assert 0 <= r < c < n
        assert out[idx] == oracle_mod.score(w.word(r), w.word(c), sc)
        assert oracle_mod.upper_index(r, c, n) == idx


def test_edge_counts():
    assert 600_000 * 599_999 // 2 == 179_999_700_000
    # Section 5: the 100,000-word edge file, one byte per edge, is 4.66 GB
    edges = 100_000 * 99_999 // 2
    assert edges == 4_999_950_000
    assert round(edges / 2 ** 30, 2) == 4.66
    for n in (2, 3, 10, 1000):
        assert sum(n - k - 1 for k in range(n)) == n * (n - 1) // 2


# ---------------------------------------------------------------------------
# top-k, query, histogram and explicit pairs against library sorts

def full_matrix(oracle_mod, w, sc):
    n = w.n
    out = oracle_mod.all_pairs(w, sc)
    M = np.full((n, n), np.iinfo(np.int32).min, dtype=np.int64)
    iu = np.triu_indices(n, 1)
    M[iu] = out
    M[(iu[1], iu[0])] = out
    return M


def lexsort_topk(scores_row, k, exclude=None):
    j = np.arange(scores_row.size)
    keep = np.ones(scores_row.size, bool)
    if exclude is not None:
        keep[exclude] = False
    j = j[keep]
    s = scores_row[keep]
    order = np.lexsort((j, -s))[:k]
    return j[order], s[order]


@pytest.mark.parametrize("sc", [(1, -1, -1), (2, -3, -1), (1, 0, 0)])
def test_topk_rows_against_lexsort(oracle_mod, sc):
    w = synth.make_words(260, 5, 1.0, 5.0, 2.0, 1, 10, seed=21)
    M = full_matrix(oracle_mod, w, sc)
    rows = np.arange(w.n, dtype=np.uint32)
    k = 10
    idx, score = oracle_mod.topk_rows(w, rows, k, sc)
    for i in range(w.n):
        ej, es = lexsort_topk(M[i], k, exclude=i)
        assert np.array_equal(idx[i], ej) and np.array_equal(score[i], es)
        assert i not in set(idx[i].tolist())


def test_topk_missing_neighbours(oracle_mod):
    w = synth.make_words(4, 5, 1.0, 3.0, 1.0, 1, 5, seed=3)
    idx, score = oracle_mod.topk_rows(w, np.arange(4), 6, (1, -1, -1))
    assert np.all(idx[:, 3:] == oracle_mod.MISSING_IDX)
    assert np.all(score[:, 3:] == oracle_mod.MISSING_SCORE)
    assert np.all(idx[:, :3] != oracle_mod.MISSING_IDX)


def test_topk_score_multiset_invariant_under_permutation(oracle_mod):
    w = synth.make_words(150, 4, 1.0, 4.0, 2.0, 1, 8, seed=8)
    sc = (1, -1, -1)
    perm = np.random.default_rng(1).permutation(w.n)
    wp = w.subset(perm)
    _, s1 = oracle_mod.topk_rows(w, np.arange(w.n), 7, sc)
    _, s2 = oracle_mod.topk_rows(wp, np.arange(w.n), 7, sc)
    inv = np.argsort(perm)
    assert np.array_equal(s1, s2[inv])


def normalised_topk_by_fractions(M, lens, i, k):
    """Word i's k best partners by Fraction(s, max(len_i, len_j) or 1), lower index first on ties."""
    cand = [j for j in range(M.shape[0]) if j != i]
    key = lambda j: (-Fraction(int(M[i, j]), max(lens[i], lens[j], 1)), j)
    best = sorted(cand, key=key)[:k]
    return np.array(best, dtype=np.int64), np.array([M[i, j] for j in best], dtype=np.int64)


@pytest.mark.parametrize("sc", [(1, -1, -1), (2, -3, -1)])
def test_topk_rows_normalised_against_fraction_sort(oracle_mod, sc):
    # lengths 0 .. 9 (empty words included) with a small alphabet, so equal
    # weights with different (s, m) -- 2/4 and 3/6 -- occur
    w = synth.make_words(140, 4, 1.0, 4.0, 2.5, 0, 9, seed=23)
    M = full_matrix(oracle_mod, w, sc)
    lens = [len(w.word(i)) for i in range(w.n)]
    k = 9
    idx, score = oracle_mod.topk_rows_normalised(w, np.arange(w.n), k, sc)
    _, raw_score = oracle_mod.topk_rows(w, np.arange(w.n), k, sc)
    for i in range(w.n):
        ej, es = normalised_topk_by_fractions(M, lens, i, k)
        assert np.array_equal(idx[i].astype(np.int64), ej) and np.array_equal(score[i].astype(np.int64), es)
    # the normalised order is not the raw one on this set
    assert not np.array_equal(score, raw_score)


def test_topk_rows_normalised_worked_cases(oracle_mod):
    # Section 5's example: for puisant, epuisant (400/6) ranks above paysans (300/5)
    g = read_golden("puisant_paysans_epuisant.txt")
    names = ("puisant", "paysans", "epuisant")
    w = synth.WordList.from_lists([ints(g[k][0]) for k in names])
    sc = tuple(ints(g["scoring"][0]))
    idx, score = oracle_mod.topk_rows_normalised(w, [0], 2, sc)
    assert idx[0].tolist() == [2, 1] and score[0].tolist() == [4, 3]
    # raw and normalised orders disagree: "ab" against a 12-symbol word that
    # contains it (2 matches, 10 gaps: -8, weight -8/12) and against "cd"
    # (2 mismatches: -2, weight -2/2); by raw score "cd" comes first, by
    # weight the long word does; a length other than the longer one would
    # put "cd" first as well
    w2 = synth.WordList.from_lists([[1, 2], [4, 5], [1, 2] + [3] * 10])
    s = (1, -1, -1)
    assert brute_force([1, 2], [1, 2] + [3] * 10, s) == -8 and brute_force([1, 2], [4, 5], s) == -2
    ri, rs = oracle_mod.topk_rows(w2, [0], 2, s)
    ni, ns = oracle_mod.topk_rows_normalised(w2, [0], 2, s)
    assert ri[0].tolist() == [1, 2] and rs[0].tolist() == [-2, -8]
    assert ni[0].tolist() == [2, 1] and ns[0].tolist() == [-8, -2]
    # two empty words have weight s / 1 = 0: above any negative weight, below any positive one
    w3 = synth.WordList.from_lists([[], [], [7], [1, 2]])
    ni, ns = oracle_mod.topk_rows_normalised(w3, [0], 3, s)
    assert ni[0].tolist() == [1, 2, 3] and ns[0].tolist() == [0, -1, -2]


def test_query_topk_against_lexsort(oracle_mod):
    d = synth.make_words(180, 6, 1.0, 5.0, 2.0, 1, 9, seed=31)
    q = synth.make_uniform_length_words(25, 6, 1.0, 0, 9, seed=32)
    sc = (1, -1, -1)
    idx, score = oracle_mod.query_topk(q, d, 10, sc)
    for a in range(q.n):
        row = np.array([oracle_mod.score(q.word(a), d.word(j), sc) for j in range(d.n)])
        ej, es = lexsort_topk(row, 10)
        assert np.array_equal(idx[a], ej) and np.array_equal(score[a], es)
    # a query equal to a dictionary word finds a neighbour scoring len * match
    q2 = d.subset([5, 17])
    idx2, score2 = oracle_mod.query_topk(q2, d, 3, sc)
    assert score2[0, 0] == len(d.word(5)) and score2[1, 0] == len(d.word(17))


def test_histogram_against_bincount(oracle_mod):
    w = synth.make_words(300, 8, 1.1, 6.0, 2.5, 1, 12, seed=41)
    for sc in [(1, -1, -1), (3, -2, -4)]:
        out = oracle_mod.all_pairs(w, sc)
        lo_ = int(out.min()) - 2
        nb = int(out.max()) - lo_ + 3
        h = oracle_mod.histogram(w, sc, lo_, nb)
        assert np.array_equal(h, np.bincount(out - lo_, minlength=nb))
        assert h.sum() == w.n * (w.n - 1) // 2


def test_histogram_reports_out_of_range(oracle_mod):
    w = synth.make_words(20, 4, 1.0, 4.0, 1.0, 2, 6, seed=2)
    with pytest.raises(RuntimeError):
        oracle_mod.histogram(w, (1, -1, -1), 100, 3)


def test_score_pairs_and_thread_count_independence(oracle_mod):
    w = synth.make_words(120, 7, 1.0, 6.0, 3.0, 0, 14, seed=51)
    sc = (2, -1, -2)
    rng = np.random.default_rng(3)
    I = rng.integers(0, w.n, 500).astype(np.uint32)
    J = rng.integers(0, w.n, 500).astype(np.uint32)
    s = oracle_mod.score_pairs(w, I, J, sc)
    assert all(s[p] == oracle_mod.score(w.word(I[p]), w.word(J[p]), sc) for p in range(0, 500, 7))
    a1 = oracle_mod.all_pairs(w, sc, nthreads=1)
    a4 = oracle_mod.all_pairs(w, sc, nthreads=5)
    assert np.array_equal(a1, a4)


# ---------------------------------------------------------------------------
# a full similarity matrix (Algorithm 1's similarity step read from a table)

def column_score_sim(A, B, cols, sim, gap):
    return sum(gap if (i is None or j is None) else int(sim[A[i]][B[j]]) for i, j in cols)


def test_sim_matrix_hand_case(oracle_mod):
    # two symbols that pay more for being swapped than kept: [0, 1] against [1, 0]
    S = np.array([[1, 5], [5, 1]], dtype=np.int32)
    # diagonal alignment 5 + 5 = 10; keeping one symbol in place costs gaps (e.g. 1 + 4 gaps = -3)
    assert oracle_mod.score_sim([0, 1], [1, 0], S, -1) == 10
    assert oracle_mod.score_sim([0, 1], [1, 0], S, -1) == max(
        column_score_sim([0, 1], [1, 0], c, S, -1) for c in alignments(2, 2))
    # all-gap alignment once every aligned pair costs more than two gaps
    S2 = np.array([[-5, -5], [-5, -5]], dtype=np.int32)
    assert oracle_mod.score_sim([0, 1, 1], [1, 0], S2, -1) == -5


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_sim_matrix_brute_force(oracle_mod, seed):
    rng = np.random.default_rng(seed)
    a = 5
    S = rng.integers(-4, 6, (a, a)).astype(np.int32)
    S = (S + S.T) // 2  # symmetric, entries of both signs
    gap = int(rng.integers(-3, 0))
    for _ in range(25):
        A = random_word(rng, 0, 5, a)
        B = random_word(rng, 0, 5, a)
        want = max(column_score_sim(A, B, c, S, gap) for c in alignments(len(A), len(B)))
        assert oracle_mod.score_sim(A, B, S, gap) == want


def test_sim_matrix_transpose(oracle_mod):
    rng = np.random.default_rng(9)
    S = rng.integers(-3, 4, (6, 6)).astype(np.int32)  # not symmetric
    for _ in range(20):
        A, B = random_word(rng, 0, 7, 6), random_word(rng, 0, 7, 6)
        assert oracle_mod.score_sim(A, B, S, -2) == oracle_mod.score_sim(B, A, S.T, -2)


@pytest.mark.parametrize("sc", [(1, -1, -1), (2, -3, -1), (1, 0, 0)])
def test_sim_matrix_reduces_to_scalar_scoring(oracle_mod, sc):
    w = synth.make_uniform_length_words(120, 7, 1.0, 0, 9, seed=17)
    S = oracle_mod.match_mismatch_matrix(7, sc[0], sc[1])
    assert np.array_equal(oracle_mod.all_pairs_sim(w, S, sc[2]), oracle_mod.all_pairs(w, sc))
    rows = np.arange(w.n)
    i1, s1 = oracle_mod.topk_rows_sim(w, rows, 8, S, sc[2])
    i2, s2 = oracle_mod.topk_rows(w, rows, 8, sc)
    assert np.array_equal(i1, i2) and np.array_equal(s1, s2)
    lo, nb = -40, 120
    assert np.array_equal(oracle_mod.histogram_sim(w, S, sc[2], lo, nb), oracle_mod.histogram(w, sc, lo, nb))
    I, J = rows[:50], rows[::-1][:50]
    assert np.array_equal(oracle_mod.score_pairs_sim(w, I, J, S, sc[2]), oracle_mod.score_pairs(w, I, J, sc))


_ENOMEM_CHILD = r"""
import resource, sys
import numpy as np
sys.path.insert(0, sys.argv[1])
import oracle
from paper_2509_01654_gb300 import synth
oracle.lib()
# one word of 20,000 symbols: each worker's full score matrix needs 1.6 GB,
# more than the address space left to this process
codes = np.zeros(20_000 + 6, np.uint8)
offsets = np.array([0, 20_000, 20_002, 20_004, 20_006], np.uint32)
w = synth.WordList(codes, offsets, 1)
vm = 0
for line in open("/proc/self/status"):
    if line.startswith("VmSize:"):
        vm = int(line.split()[1]) * 1024
resource.setrlimit(resource.RLIMIT_AS, (vm + (384 << 20), vm + (384 << 20)))
sc = (1, -1, -1)
failed = []
for name, call in [
    ("topk_rows", lambda: oracle.topk_rows(w, [0, 1, 2, 3], 2, sc, nthreads=2)),
    ("topk_rows_normalised", lambda: oracle.topk_rows_normalised(w, [0, 1], 2, sc, nthreads=2)),
    ("all_pairs", lambda: oracle.all_pairs(w, sc, nthreads=2)),
    ("histogram", lambda: oracle.histogram(w, sc, -40_000, 80_001, nthreads=2)),
    ("score_pairs", lambda: oracle.score_pairs(w, [0, 1], [1, 2], sc, nthreads=2)),
    ("query_topk", lambda: oracle.query_topk(w, w, 2, sc, nthreads=2)),
]:
    try:
        call()
    except RuntimeError as e:
        if "-2" in str(e) or "error" in str(e):
            failed.append(name)
print(",".join(failed))
"""


def test_worker_allocation_failure_is_reported_not_silent(oracle_mod):
    """A worker that cannot allocate its score matrix must make the call fail
    (NWO_ENOMEM) rather than return with rows unwritten."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    r = subprocess.run([sys.executable, "-c", _ENOMEM_CHILD, root], capture_output=True, text=True, timeout=120,
                       cwd=root)
    assert r.returncode == 0, r.stderr[-2000:]
    got = set(r.stdout.strip().split(","))
    assert got == {"topk_rows", "topk_rows_normalised", "all_pairs", "histogram", "score_pairs", "query_topk"}, (
        r.stdout, r.stderr[-2000:])
