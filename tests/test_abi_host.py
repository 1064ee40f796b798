"""Host-side checks of libnw that need no GPU: the library loads and exports
every entry point of include/nw.h, the pair planner covers every unordered
pair exactly once (in every shard split), the host merge of partial lists is
exact, and calls fail loudly without a GPU."""
import os
import re

import numpy as np
import pytest

from conftest import ROOT
from paper_2509_01654_gb300 import build as nwbuild
from paper_2509_01654_gb300 import nw, synth


@pytest.fixture(scope="module")
def lib():
    nwbuild.build()
    return nw.load_library()


def declared_functions():
    inc = os.path.join(ROOT, "include")
    src = "".join(open(os.path.join(inc, f)).read() for f in sorted(os.listdir(inc)) if f.endswith(".h"))
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nw_[a-z_]+)\s*\(", src)))


def test_header_declarations_are_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(nw.EXPORTED)


def all_unordered(n):
    i, j = np.triu_indices(n, 1)
    return set(zip(i.tolist(), j.tolist()))


def as_set(a, b):
    lo = np.minimum(a, b)
    hi = np.maximum(a, b)
    pairs = list(zip(lo.tolist(), hi.tolist()))
    return pairs, set(pairs)


@pytest.mark.parametrize("case", ["mixed", "single_len", "with_empty", "ragged_big", "long_words"])
def test_planner_covers_each_pair_once(lib, case):
    rng = np.random.default_rng(hash(case) % 1000)
    if case == "mixed":
        L = rng.integers(1, 12, 300)
    elif case == "single_len":
        L = np.full(777, 5)               # one bucket, several A chunks, odd size
    elif case == "with_empty":
        L = rng.integers(0, 4, 150)       # empty words share a bucket
    elif case == "ragged_big":
        L = synth.exhaustive_words(1500).lengths
    else:
        L = rng.integers(30, 41, 200)
    a, b = nw.debug_enumerate_pairs(L)
    pairs, s = as_set(a, b)
    assert len(pairs) == len(s) == L.size * (L.size - 1) // 2
    assert s == all_unordered(L.size)
    assert np.all(a != b)
    # the longer word is always the lane (B) word
    assert np.all(L[b] >= L[a])


@pytest.mark.parametrize("nshards", [2, 3, 7])
def test_planner_shards_partition_pairs(lib, nshards):
    L = synth.pr1_words(400).lengths
    seen = []
    for g in range(nshards):
        a, b = nw.debug_enumerate_pairs(L, g, nshards)
        seen.extend(as_set(a, b)[0])
    assert len(seen) == len(set(seen)) == 400 * 399 // 2


def test_planner_degenerate_sizes(lib):
    for L in ([3], [0], [2, 2], [0, 0], [1, 40], list(range(41))):
        a, b = nw.debug_enumerate_pairs(np.array(L))
        assert as_set(a, b)[1] == all_unordered(len(L))


@pytest.mark.parametrize("case,ta", [("mixed", 0), ("mixed", 64), ("ragged_big", 128), ("long_queries", 256),
                                     ("with_empty", 0), ("no_queries", 0)])
def test_query_planner_covers_each_pair_once(lib, case, ta):
    # nw_query and the batched query sets: every (query, word) pair exactly once
    rng = np.random.default_rng(len(case) + ta)
    if case == "mixed":
        Q, D = rng.integers(1, 12, 70), rng.integers(1, 12, 300)
    elif case == "ragged_big":
        Q, D = synth.serving_queries(257).lengths, synth.exhaustive_words(1100).lengths
    elif case == "long_queries":
        Q, D = rng.integers(26, 41, 90), rng.integers(1, 26, 400)   # queries longer than every word
    elif case == "with_empty":
        Q, D = rng.integers(0, 4, 40), rng.integers(0, 4, 130)
    else:
        Q, D = np.zeros(0, np.int64), rng.integers(1, 9, 50)
    q, d = nw.debug_enumerate_query_pairs(Q, D, ta)
    pairs = list(zip(q.tolist(), d.tolist()))
    assert len(pairs) == len(set(pairs)) == Q.size * D.size
    assert set(pairs) == {(i, j) for i in range(Q.size) for j in range(D.size)}


def test_topk_merge_matches_full_lists(lib, oracle_mod):
    w = synth.make_words(90, 5, 1.0, 4.0, 2.0, 1, 8, seed=12)
    sc = (1, -1, -1)
    k = 6
    full_idx, full_sc = oracle_mod.topk_rows(w, np.arange(w.n), k, sc)
    # split each word's candidates into 3 disjoint parts and rank within each part
    M = np.full((w.n, w.n), -10 ** 6, dtype=np.int64)
    iu = np.triu_indices(w.n, 1)
    vals = oracle_mod.all_pairs(w, sc)
    M[iu] = vals
    M[(iu[1], iu[0])] = vals
    part_of = (np.add.outer(np.arange(w.n), np.arange(w.n)) % 3)
    parts = []
    for p in range(3):
        pi = np.full((w.n, k), nw.MISSING_IDX, dtype=np.uint32)
        ps = np.full((w.n, k), nw.MISSING_SCORE, dtype=np.int16)
        for i in range(w.n):
            js = np.array([j for j in range(w.n) if j != i and part_of[i, j] == p])
            if js.size == 0:
                continue
            order = np.lexsort((js, -M[i, js]))[:k]
            pi[i, :order.size] = js[order]
            ps[i, :order.size] = M[i, js[order]]
        parts.append((pi, ps))
    mi, ms = nw.topk_merge(parts, k)
    assert np.array_equal(mi, full_idx)
    assert np.array_equal(ms, full_sc.astype(np.int16))
    # merging a part with itself changes nothing (duplicates kept once)
    mi2, ms2 = nw.topk_merge([(full_idx, full_sc.astype(np.int16))] * 2, k)
    assert np.array_equal(mi2, full_idx)


def test_calls_fail_loudly_without_gpu(lib):
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(nw.NwError) as e:
        nw.Context(0)
    assert e.value.status in (nw.NW_ECUDA, nw.NW_EINVAL)
    assert str(e.value)


def _reach(sc, m):
    """Score interval a pair whose longer word has m symbols can reach: between
    the all-gap alignment and the diagonal alignments of the shorter word."""
    match, mismatch, gap = sc
    lo, hi = None, None
    for la in range(0, m + 1):
        allgap = (la + m) * gap
        a = max(allgap, la * min(match, mismatch) + (m - la) * gap)
        b = max(allgap, la * max(match, mismatch) + (m - la) * gap)
        lo = a if lo is None else min(lo, a)
        hi = b if hi is None else max(hi, b)
    return lo, hi


@pytest.mark.parametrize("sc,lo,hi", [((1, -1, -1), -40, 40), ((2, -3, -1), -80, 80), ((1, 0, 0), 0, 40),
                                      ((3, -2, -2), -80, 120)])
def test_normalised_rank_tables(lib, sc, lo, hi):
    from fractions import Fraction
    rank, smin, frac = nw.debug_norm_tables(sc, lo, hi)
    R = frac.shape[0]
    vals = [Fraction(int(frac[r, 0]), int(frac[r, 1])) for r in range(R)]
    assert all(int(frac[r, 1]) > 0 for r in range(R))
    assert all(vals[r] < vals[r + 1] for r in range(R - 1))  # strictly ascending, one rank per value
    seen = set()
    for m in range(nw.MAX_WORD_LEN + 1):
        a, b = _reach(sc, m)
        a, b = max(a, lo), min(b, hi)
        for s in range(a, b + 1):
            r = int(rank[s - lo, m])
            assert vals[r] == Fraction(s, max(m, 1))
            # stored in lowest terms
            assert Fraction(int(frac[r, 0]), int(frac[r, 1])).denominator == int(frac[r, 1])
            seen.add(r)
        for r in range(R):
            reach = [s for s in range(a, b + 1) if int(rank[s - lo, m]) >= r]
            assert int(smin[r, m]) == (min(reach) if reach else 32767)
    assert seen == set(range(R))  # every rank is some reachable weight


C_PROGRAM = r"""
#include <stdio.h>
#include "nw.h"
#include "nw_proposal.h"
int main(void) {
  nw_ctx *ctx = NULL;
  nw_status st = nw_create(&ctx, 0, 0, NULL);
  if (st == NW_OK) { nw_destroy(ctx); return 0; }
  const char *msg = nw_last_error(NULL);
  printf("%d %s\n", (int)st, msg ? msg : "");
  return msg && msg[0] ? 3 : 4;
}
"""


def test_headers_are_plain_c_and_link(lib, tmp_path):
    # the boundary is a C ABI: both headers compile as strict C99 and a C
    # program links against libnw and calls it (no GPU: a clean error status)
    import shutil
    import subprocess
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "t.c"
    src.write_text(C_PROGRAM)
    libdir = os.path.dirname(nw.LIB_PATH)
    exe = tmp_path / "t"
    inc = os.path.join(ROOT, "include")
    r = subprocess.run([gcc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", inc,
                        str(src), "-L", libdir, "-lnw", f"-Wl,-rpath,{libdir}", "-o", str(exe)],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    run = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert run.returncode in (0, 3), run.stdout + run.stderr
