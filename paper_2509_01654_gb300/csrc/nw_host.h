// nw_host.h -- host-side internals of libnw shared by its translation units:
// the context and dictionary objects, device buffers with budget accounting,
// the pair planner, kernel launching and error handling.  Everything except
// the two object definitions sits in an anonymous namespace (one copy per
// translation unit).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <set>
#include <string>
#include <utility>
#include <vector>

#include "nw.h"
#include "nw_proposal.h"
#include "nw_internal.cuh"
#include "nw_launch.h"

using namespace nw;

namespace {

thread_local std::string g_create_error;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  template <class T>
  T* as() const { return static_cast<T*>(p); }
};

// A word set on the device (see nw_internal.cuh for the layout).
struct WordSet {
  uint32_t n = 0;
  uint32_t min_len = 0, max_len = 0;
  Buckets bk{};
  DevBuf perm, rank, slen, aoff, brec_w, a_enc, b_rec;
};

struct LaunchPlan {
  int LB = 0;
  int role = 0;  // 0: A and B from one set; 1: A = queries, B = dictionary; 2: A = dictionary, B = queries
  uint32_t ta = 0;  // A words per task of this launch (0: the launch parameters' TA)
  uint32_t bps = 0; // resident blocks per SM at most (0: as many as fit)
  uint32_t seg_first = 0, nsegs = 0;
  uint64_t ntasks = 0;
  uint64_t pairs = 0, cells = 0;
};

struct Plan {
  std::vector<Seg> segs;
  std::vector<LaunchPlan> launches;
  uint64_t pairs = 0, cells = 0;
};

}  // namespace

struct nw_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0, used = 0;
  uint32_t fail_countdown = 0;
  // debug bounds (nw_debug_set_bounds): list-insertion retries (-1 = the
  // kernel's own bound), pipeline wait cycles (-1 = the kernel's own bound),
  // and a column tile the candidate kernel's producer never issues (UINT32_MAX
  // = none)
  int32_t dbg_insert_iters = -1;
  int64_t dbg_wait_cycles = -1;
  uint32_t dbg_withhold_tile = UINT32_MAX;
  std::string err;
  bool profiling = false;
  nw_profile prof{};
  int sm_count = 0;
  std::set<nw_dict*> dicts;
  std::set<nw_model*> models;
  std::atomic<int> busy{0};
  // grow-only workspace
  DevBuf ws_slots, ws_thr, ws_hist, ws_small, ws_out_idx, ws_out_score, ws_mat, ws_pairs, ws_segs, ws_norm;
  std::vector<cudaEvent_t> events;
};

struct nw_dict {
  nw_ctx* ctx = nullptr;
  WordSet ws;
  nw_scoring sc{};
  ShiftedScoring ss{};
  uint32_t alphabet = 0;
  int32_t score_lo = 0, score_hi = 0;
  Plan plan;
  DevBuf d_segs;
  bool subst = false;  // scored with a full similarity matrix (d_tab)
  DevBuf d_tab;        // kTabDim x kTabDim s'+ table
  uint64_t serial = 0;  // unique per loaded dictionary (caches keyed on it)
};

namespace {

nw_status set_err(nw_ctx* c, nw_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf; else g_create_error = buf;
  return st;
}

nw_status cuda_fail(nw_ctx* c, cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a non-sticky error
  return set_err(c, NW_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define NW_CK(call)                                                 \
  do {                                                              \
    cudaError_t e_ = (call);                                        \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call);          \
  } while (0)

#define NW_TRY(expr)                        \
  do {                                      \
    nw_status s_ = (expr);                  \
    if (s_ != NW_OK) return s_;             \
  } while (0)

nw_status ctx_alloc(nw_ctx* c, DevBuf& b, size_t bytes, const char* what) {
  if (bytes == 0) bytes = 16;
  if (c->fail_countdown) {
    if (--c->fail_countdown == 0)
      return set_err(c, NW_ENOMEM, "injected allocation failure for %s (%zu bytes)", what, bytes);
  }
  if (c->budget && c->used + bytes > c->budget)
    return set_err(c, NW_ENOMEM, "memory budget exceeded: %s needs %zu bytes, %zu of %zu in use", what,
                   bytes, c->used, c->budget);
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(c, NW_ENOMEM, "cudaMalloc(%zu) for %s failed: %s", bytes, what, cudaGetErrorString(e));
  }
  b.p = p;
  b.bytes = bytes;
  c->used += bytes;
  return NW_OK;
}

void ctx_free(nw_ctx* c, DevBuf& b) {
  if (b.p) {
    cudaFree(b.p);
    c->used -= b.bytes;
  }
  b = DevBuf{};
}

nw_status ctx_ensure(nw_ctx* c, DevBuf& b, size_t bytes, const char* what) {
  if (b.p && b.bytes >= bytes) return NW_OK;
  ctx_free(c, b);
  return ctx_alloc(c, b, bytes, what);
}

// RAII: one call at a time per context, on the context's device.
struct CallGuard {
  nw_ctx* c;
  bool ok = false;
  explicit CallGuard(nw_ctx* ctx) : c(ctx) {
    int expected = 0;
    ok = c->busy.compare_exchange_strong(expected, 1);
  }
  ~CallGuard() {
    if (ok) c->busy.store(0);
  }
};

// RAII: an NVTX range named after the entry point, so a timeline profiler
// (Nsight Systems) shows each library call around its copies and launches.
// Without a profiler attached the push and pop cost a few nanoseconds.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};

#define NW_ENTER(ctxp)                                                              \
  if (!(ctxp)) return NW_EINVAL;                                                    \
  NvtxRange nvtx_(__func__);                                                        \
  CallGuard guard_(ctxp);                                                           \
  if (!guard_.ok) return set_err(ctxp, NW_EBUSY, "context in use by another call"); \
  (ctxp)->err.clear();                                                              \
  {                                                                                 \
    cudaError_t e_ = cudaSetDevice((ctxp)->device);                                 \
    if (e_ != cudaSuccess) return cuda_fail(ctxp, e_, "cudaSetDevice");             \
  }

uint32_t pack16(int32_t v) {
  const uint32_t h = (uint32_t)v & 0xffffu;
  return h | (h << 16);
}

nw_status make_shifted(nw_ctx* c, const nw_scoring& s, uint32_t alphabet, ShiftedScoring& out) {
  if (std::abs(s.match) > 1024 || std::abs(s.mismatch) > 1024 || std::abs(s.gap) > 1024)
    return set_err(c, NW_EINVAL, "scoring values must lie in [-1024, 1024]");
  if (s.mismatch > s.match) return set_err(c, NW_EINVAL, "mismatch (%d) must not exceed match (%d)", s.mismatch, s.match);
  const int32_t sm = s.match - 2 * s.gap, sx = s.mismatch - 2 * s.gap;
  if (sm < 0) return set_err(c, NW_EINVAL, "2*gap (%d) must not exceed match (%d)", 2 * s.gap, s.match);
  if ((int64_t)sm * kMaxLen > 32767)
    return set_err(c, NW_ERANGE, "match - 2*gap = %d is too large for 16-bit cells at length %d", sm, kMaxLen);
  const int32_t delta = s.match - s.mismatch;
  uint32_t shift = 0;
  while ((1 << shift) < delta) ++shift;
  if (((alphabet - 1u) << shift) >= 32768u)
    return set_err(c, NW_EINVAL, "alphabet %u with match - mismatch = %d does not fit the 15-bit code encoding", alphabet, delta);
  out.sm = sm;
  out.sx = sx;
  out.shift = shift;
  out.C1 = pack16(sm + 1);
  out.C2 = pack16(std::max(sx, 0));  // a negative mismatch term never wins (see nw_dp.cuh)
  return NW_OK;
}

const uint16_t* dict_tab(const nw_dict* d) { return d->subst ? d->d_tab.as<uint16_t>() : nullptr; }

void pair_bounds(const nw_scoring& s, int la, int lb, int& lo, int& hi) {
  const int mn = std::min(la, lb), d = std::abs(la - lb);
  const int allgap = (la + lb) * s.gap;
  lo = std::max(allgap, mn * std::min(s.match, s.mismatch) + d * s.gap);
  hi = std::max(allgap, mn * std::max(s.match, s.mismatch) + d * s.gap);
}

// Buckets with every base filled from the counts.
void fill_buckets(Buckets& bk) {
  uint64_t pos = 0, aenc = 0, brec = 0;
  for (int L = 0; L < kBuckets; ++L) {
    bk.start[L] = (uint32_t)pos;
    bk.aenc_base[L] = (uint32_t)aenc;
    bk.brec_word_base[L] = (uint32_t)brec;
    pos += bk.count[L];
    aenc += (uint64_t)bk.count[L] * L;
    brec += (uint64_t)((bk.count[L] + 1) / 2) * (uint64_t)ceil4(L);
  }
  bk.start[kBuckets] = (uint32_t)pos;
}

uint64_t aenc_words(const Buckets& bk) {
  uint64_t s = 0;
  for (int L = 0; L < kBuckets; ++L) s += (uint64_t)bk.count[L] * L;
  return s;
}
uint64_t brec_words(const Buckets& bk) {
  uint64_t s = 0;
  for (int L = 0; L < kBuckets; ++L) s += (uint64_t)((bk.count[L] + 1) / 2) * (uint64_t)ceil4(L);
  return s;
}

uint64_t cdiv(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

Seg make_seg(const Buckets& A, int La, uint32_t a_beg, uint32_t a_end, const Buckets& B, int LB,
             uint32_t b_beg, uint32_t b_end, bool tri, uint32_t TA, uint64_t task0, uint64_t& ntasks) {
  Seg s{};
  s.a_beg = a_beg;
  s.a_end = a_end;
  s.b_beg = b_beg;
  s.b_end = b_end;
  s.aenc_base = A.aenc_base[La] + (a_beg - A.start[La]) * (uint32_t)La;
  const uint32_t rb = b_beg - B.start[LB];
  s.brec_base = (B.brec_word_base[LB] + (rb / 2) * (uint32_t)ceil4(LB)) / 4;
  s.la = (uint16_t)La;
  s.tri = tri ? 1 : 0;
  s.nca = (uint32_t)cdiv(a_end - a_beg, TA);
  s.task0 = task0;
  ntasks = (uint64_t)s.nca * cdiv(b_end - b_beg, kWarpB);
  return s;
}

// Launches run in increasing longer length: a word of length L first meets
// partners of its own length (the segment La == LB leads launch L), where its
// best neighbours usually are, so list thresholds rise before the many
// low-scoring pairs of very different lengths arrive.
void order_launches(Plan& p) {
  std::stable_sort(p.launches.begin(), p.launches.end(),
                   [](const LaunchPlan& x, const LaunchPlan& y) { return x.LB < y.LB; });
}

// Every unordered pair of one set, once: launch LB holds the pairs whose
// longer word has length LB; inside it the same-length rectangle comes first,
// then shorter A lengths in order of growing length difference.
void plan_all_pairs(const Buckets& bk, uint32_t TA, Plan& out) {
  out = Plan{};
  if (TA == 0) TA = kDefaultTA;
  TA = (TA + 1) & ~1u;  // A chunks start B chunks of the same bucket: keep them even
  for (int LB = 0; LB < kBuckets; ++LB) {
    const uint32_t nB = bk.count[LB];
    if (nB == 0) continue;
    LaunchPlan lp;
    lp.LB = LB;
    lp.role = 0;
    lp.seg_first = (uint32_t)out.segs.size();
    uint64_t task = 0;
    for (int La = LB; La >= 0; --La) {
      if (La == LB) {
        if (nB < 2) continue;
        const uint32_t s = bk.start[LB], e = s + nB;
        for (uint32_t a_beg = s; a_beg < e; a_beg += TA) {
          const uint32_t a_end = std::min(e, a_beg + TA);
          if (e - a_beg < 2) continue;
          uint64_t nt = 0;
          out.segs.push_back(make_seg(bk, LB, a_beg, a_end, bk, LB, a_beg, e, true, TA, task, nt));
          task += nt;
        }
        lp.pairs += (uint64_t)nB * (nB - 1) / 2;
        lp.cells += (uint64_t)nB * (nB - 1) / 2 * (uint64_t)(LB * LB);
      } else {
        const uint32_t nA = bk.count[La];
        if (nA == 0) continue;
        uint64_t nt = 0;
        out.segs.push_back(make_seg(bk, La, bk.start[La], bk.start[La] + nA, bk, LB, bk.start[LB],
                                    bk.start[LB] + nB, false, TA, task, nt));
        task += nt;
        lp.pairs += (uint64_t)nA * nB;
        lp.cells += (uint64_t)nA * nB * (uint64_t)(La * LB);
      }
    }
    lp.nsegs = (uint32_t)out.segs.size() - lp.seg_first;
    lp.ntasks = task;
    if (lp.nsegs) {
      out.pairs += lp.pairs;
      out.cells += lp.cells;
      out.launches.push_back(lp);
    }
  }
  order_launches(out);
}

// Tasks a query launch should have at least (a few per warp of a full GPU)
// before its A chunks are cut below the default size.
constexpr uint64_t kQueryMinTasks = 8192;

// Every (query, dictionary word) pair once; the longer word goes to the lanes.
// A launch whose B words are few (long dictionary words, or a small query
// set in the lanes) has few tasks at TA A words per task: with min_tasks > 0
// its chunk is halved, down to 32 words, until it has min_tasks tasks, and
// the launch records the chunk in its ta.
void plan_query(const Buckets& qb, const Buckets& db, uint32_t TA, Plan& out, uint64_t min_tasks = 0) {
  out = Plan{};
  for (int role = 1; role <= 2; ++role) {
    for (int LB = 0; LB < kBuckets; ++LB) {
      LaunchPlan lp;
      lp.LB = LB;
      lp.role = role;
      lp.seg_first = (uint32_t)out.segs.size();
      uint64_t task = 0;
      const Buckets& Bset = role == 1 ? db : qb;
      const Buckets& Aset = role == 1 ? qb : db;
      const uint32_t nB = Bset.count[LB];
      if (nB == 0) continue;
      // role 1: query length La <= LB (dictionary length); role 2: dictionary length La < LB (query length)
      const int La_hi = role == 1 ? LB : LB - 1;
      uint32_t ta = TA;
      if (min_tasks) {
        auto tasks_at = [&](uint32_t t) {
          uint64_t x = 0;
          for (int La = La_hi; La >= 0; --La) x += cdiv(Aset.count[La], t) * cdiv(nB, kWarpB);
          return x;
        };
        while (ta > 32 && tasks_at(ta) < min_tasks) ta /= 2;
        lp.ta = ta;
      }
      for (int La = La_hi; La >= 0; --La) {
        const uint32_t nA = Aset.count[La];
        if (nA == 0) continue;
        uint64_t nt = 0;
        out.segs.push_back(make_seg(Aset, La, Aset.start[La], Aset.start[La] + nA, Bset, LB, Bset.start[LB],
                                    Bset.start[LB] + nB, false, ta, task, nt));
        task += nt;
        lp.pairs += (uint64_t)nA * nB;
        lp.cells += (uint64_t)nA * nB * (uint64_t)(La * LB);
      }
      lp.nsegs = (uint32_t)out.segs.size() - lp.seg_first;
      lp.ntasks = task;
      if (lp.nsegs) {
        out.pairs += lp.pairs;
        out.cells += lp.cells;
        out.launches.push_back(lp);
      }
    }
  }
  order_launches(out);
}

uint32_t index_bits(uint32_t n) {
  uint32_t b = 1;
  while (b < 32 && ((uint64_t)1 << b) < (uint64_t)n) ++b;
  return b;
}

// Tables of the length-normalised ranking (Section 5 divides each score by
// the longer word's length).  Every value s/m that a pair whose longer word
// has m symbols can reach (s within that length's score bounds and within
// [lo, hi]) is ranked ascending by exact integer cross-multiplication; equal
// fractions share a rank.  Two empty words (m = 0) rank as s/1.
struct NormTables {
  int32_t lo = 0;              // score of row 0 of `rank`
  uint32_t nranks = 0;
  std::vector<uint16_t> rank;  // [(s - lo) * kBuckets + m]: rank of s/m (0 where s is out of reach for m)
  std::vector<int16_t> smin;   // [r * kBuckets + m]: smallest reachable s whose s/m has rank >= r, else above reach
  std::vector<int16_t> frac;   // [2r], [2r + 1]: numerator and denominator of rank r in lowest terms
};

void build_norm_tables(const nw_scoring& sc, int32_t lo, int32_t hi, NormTables& t) {
  int flo[kBuckets], fhi[kBuckets];
  std::vector<std::pair<int32_t, int32_t>> fr;  // reduced (numerator, denominator)
  for (int m = 0; m < kBuckets; ++m) {
    flo[m] = INT32_MAX;
    fhi[m] = INT32_MIN;
    for (int la = 0; la <= m; ++la) {
      int a, b;
      pair_bounds(sc, la, m, a, b);
      flo[m] = std::min(flo[m], a);
      fhi[m] = std::max(fhi[m], b);
    }
    flo[m] = std::max(flo[m], lo);
    fhi[m] = std::min(fhi[m], hi);
    const int32_t den = m > 0 ? m : 1;
    for (int s = flo[m]; s <= fhi[m]; ++s) {
      int32_t g = std::abs(s), h = den;
      while (h) { const int32_t r = g % h; g = h; h = r; }
      fr.push_back({s / g, den / g});
    }
  }
  auto less = [](const std::pair<int32_t, int32_t>& x, const std::pair<int32_t, int32_t>& y) {
    return (int64_t)x.first * y.second < (int64_t)y.first * x.second;
  };
  std::sort(fr.begin(), fr.end(), less);
  fr.erase(std::unique(fr.begin(), fr.end()), fr.end());  // reduced fractions are equal iff their parts are
  t.lo = lo;
  t.nranks = (uint32_t)fr.size();
  t.rank.assign((size_t)(hi - lo + 1) * kBuckets, 0);
  t.frac.resize(2 * fr.size());
  for (size_t r = 0; r < fr.size(); ++r) {
    t.frac[2 * r] = (int16_t)fr[r].first;
    t.frac[2 * r + 1] = (int16_t)fr[r].second;
  }
  for (int m = 0; m < kBuckets; ++m) {
    const int32_t den = m > 0 ? m : 1;
    for (int s = flo[m]; s <= fhi[m]; ++s) {
      const auto it = std::lower_bound(fr.begin(), fr.end(), std::make_pair((int32_t)s, den), less);
      t.rank[(size_t)(s - lo) * kBuckets + m] = (uint16_t)(it - fr.begin());
    }
  }
  // rank grows with s at fixed m, so the smallest s reaching rank r is found
  // by one sweep per length; above reach, the bound no G value attains
  t.smin.assign((size_t)fr.size() * kBuckets, INT16_MAX);
  for (int m = 0; m < kBuckets; ++m) {
    int s = flo[m];
    for (uint32_t r = 0; r < t.nranks; ++r) {
      while (s <= fhi[m] && t.rank[(size_t)(s - lo) * kBuckets + m] < r) ++s;
      if (s > fhi[m]) break;
      t.smin[(size_t)r * kBuckets + m] = (int16_t)s;
    }
  }
}

void free_wordset(nw_ctx* c, WordSet& w) {
  ctx_free(c, w.perm);
  ctx_free(c, w.rank);
  ctx_free(c, w.slen);
  ctx_free(c, w.aoff);
  ctx_free(c, w.brec_w);
  ctx_free(c, w.a_enc);
  ctx_free(c, w.b_rec);
  w = WordSet{};
}

uint64_t wordset_bytes(const WordSet& w) {
  return w.perm.bytes + w.rank.bytes + w.slen.bytes + w.aoff.bytes + w.brec_w.bytes + w.a_enc.bytes +
         w.b_rec.bytes;
}

// Copies (if needed), validates, buckets and encodes a word set.
nw_status ingest(nw_ctx* c, const uint8_t* codes, const uint32_t* offsets, uint32_t n, uint32_t alphabet,
                 uint32_t shift, uint32_t flags, WordSet& ws) {
  const bool dev = flags & NW_DEVICE_PTRS;
  cudaStream_t s = c->stream;
  std::vector<DevBuf> tmp;
  struct Cleanup {
    nw_ctx* c;
    std::vector<DevBuf>& t;
    ~Cleanup() {
      for (auto& b : t) ctx_free(c, b);
    }
  } cleanup{c, tmp};
  auto talloc = [&](size_t bytes, const char* what, void** out) -> nw_status {
    tmp.emplace_back();
    NW_TRY(ctx_alloc(c, tmp.back(), bytes, what));
    *out = tmp.back().p;
    return NW_OK;
  };

  uint32_t total = 0;
  const uint8_t* d_codes = codes;
  const uint32_t* d_offsets = offsets;
  if (dev) {
    NW_CK(cudaMemcpyAsync(&total, offsets + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    NW_CK(cudaStreamSynchronize(s));
  } else {
    if (offsets[0] != 0) return set_err(c, NW_EINVAL, "offsets[0] must be 0");
    for (uint32_t i = 0; i < n; ++i) {
      if (offsets[i + 1] < offsets[i]) return set_err(c, NW_EINVAL, "offsets decrease at word %u", i);
      if (offsets[i + 1] - offsets[i] > (uint32_t)kMaxLen)
        return set_err(c, NW_EINVAL, "word %u has %u codes; at most %d are supported", i, offsets[i + 1] - offsets[i], kMaxLen);
    }
    total = offsets[n];
    void* p;
    NW_TRY(talloc((size_t)total + 16, "input codes", &p));
    if (total) NW_CK(cudaMemcpyAsync(p, codes, total, cudaMemcpyHostToDevice, s));
    d_codes = static_cast<const uint8_t*>(p);
    NW_TRY(talloc(sizeof(uint32_t) * ((size_t)n + 1), "input offsets", &p));
    NW_CK(cudaMemcpyAsync(p, offsets, sizeof(uint32_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, s));
    d_offsets = static_cast<const uint32_t*>(p);
  }

  const uint32_t nblk = (uint32_t)cdiv(n, kIngestBlock);
  void *p_counts, *p_small;
  NW_TRY(talloc(sizeof(uint32_t) * (size_t)nblk * kBuckets, "ingest block counts", &p_counts));
  NW_TRY(talloc(sizeof(uint32_t) * (kBuckets + 4), "ingest counters", &p_small));
  uint32_t* d_counts = static_cast<uint32_t*>(p_counts);
  uint32_t* d_bucket = static_cast<uint32_t*>(p_small);
  uint32_t* d_err = d_bucket + kBuckets;
  NW_CK(cudaMemsetAsync(p_small, 0, sizeof(uint32_t) * (kBuckets + 4), s));
  NW_CK(launch_ingest_count(d_codes, d_offsets, n, alphabet, d_counts, d_err, s));
  NW_CK(launch_ingest_scan(d_counts, nblk, d_bucket, s));
  uint32_t host_small[kBuckets + 1];
  NW_CK(cudaMemcpyAsync(host_small, p_small, sizeof(uint32_t) * (kBuckets + 1), cudaMemcpyDeviceToHost, s));
  NW_CK(cudaStreamSynchronize(s));
  if (host_small[kBuckets])
    return set_err(c, NW_EINVAL,
                   "invalid words: offsets must start at 0 and not decrease, words have at most %d codes and "
                   "every code is < alphabet (%u)", kMaxLen, alphabet);

  ws.n = n;
  std::memcpy(ws.bk.count, host_small, sizeof(uint32_t) * kBuckets);
  fill_buckets(ws.bk);
  ws.min_len = kMaxLen;
  ws.max_len = 0;
  for (int L = 0; L < kBuckets; ++L)
    if (ws.bk.count[L]) { ws.min_len = std::min<uint32_t>(ws.min_len, L); ws.max_len = std::max<uint32_t>(ws.max_len, L); }
  if (n == 0) ws.min_len = 0;
  const uint64_t aw = aenc_words(ws.bk), bw = brec_words(ws.bk);
  if (aw >= (1ull << 32) || bw >= (1ull << 31))
    return set_err(c, NW_EINVAL, "word set too large for 32-bit symbol offsets");

  NW_TRY(ctx_alloc(c, ws.perm, sizeof(uint32_t) * (size_t)n, "word permutation"));
  NW_TRY(ctx_alloc(c, ws.rank, sizeof(uint32_t) * (size_t)n, "word ranks"));
  NW_TRY(ctx_alloc(c, ws.slen, (size_t)n + 16, "word lengths"));
  NW_TRY(ctx_alloc(c, ws.aoff, sizeof(uint32_t) * (size_t)n, "A-side offsets"));
  NW_TRY(ctx_alloc(c, ws.brec_w, sizeof(uint32_t) * (size_t)n, "B-side offsets"));
  NW_TRY(ctx_alloc(c, ws.a_enc, sizeof(uint32_t) * (size_t)(aw + 4), "A-side symbols"));
  NW_TRY(ctx_alloc(c, ws.b_rec, sizeof(uint32_t) * (size_t)(bw + 4), "B-side pair records"));
  NW_CK(cudaMemsetAsync(ws.b_rec.p, 0xff, ws.b_rec.bytes, s));
  if (n) {
    NW_CK(launch_ingest_scatter(d_offsets, n, d_counts, ws.bk, ws.perm.as<uint32_t>(), ws.rank.as<uint32_t>(),
                                ws.slen.as<uint8_t>(), s));
    NW_CK(launch_ingest_encode(d_codes, d_offsets, n, ws.perm.as<uint32_t>(), ws.slen.as<uint8_t>(), ws.bk,
                               shift, ws.a_enc.as<uint32_t>(), ws.aoff.as<uint32_t>(), ws.b_rec.as<uint32_t>(),
                               ws.brec_w.as<uint32_t>(), s));
  }
  NW_CK(cudaStreamSynchronize(s));  // temporaries are freed on return
  return NW_OK;
}

// ---------------------------------------------------------------------------
// profiling events

struct Timer {
  nw_ctx* c;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> dp, fin;
  cudaEvent_t first = nullptr, last = nullptr;
  size_t used = 0;
  cudaEvent_t get() {
    if (used == c->events.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
      c->events.push_back(e);
    }
    return c->events[used++];
  }
  void mark(cudaEvent_t e) {
    if (!e) return;
    cudaEventRecord(e, c->stream);
    if (!first) first = e;
    last = e;
  }
  void begin(bool dp_kind, cudaEvent_t& a) {
    a = c->profiling ? get() : nullptr;
    mark(a);
    (void)dp_kind;
  }
  void end(bool dp_kind, cudaEvent_t a) {
    if (!c->profiling) return;
    cudaEvent_t b = get();
    mark(b);
    if (a && b) (dp_kind ? dp : fin).emplace_back(a, b);
  }
  void collect() {
    if (!c->profiling) return;
    double dms = 0, fms = 0;
    for (auto& pr : dp) { float ms = 0; cudaEventElapsedTime(&ms, pr.first, pr.second); dms += ms; }
    for (auto& pr : fin) { float ms = 0; cudaEventElapsedTime(&ms, pr.first, pr.second); fms += ms; }
    c->prof.dp_ms = dms;
    c->prof.finalize_ms = fms;
    float tot = 0;
    if (first && last) cudaEventElapsedTime(&tot, first, last);
    c->prof.total_ms = tot;
  }
};

struct RunOut {
  uint32_t dp_launches = 0;
  uint64_t pairs = 0, cells = 0;
};

// Launches the alignment kernels of `plan` (shard `shard` of `nshards` of each
// launch's tasks) on `stream`.  The A and B sides of a launch come from the
// per-role tables: role 0 = one set against itself, 1 = queries (A) against the
// dictionary (B), 2 = dictionary (A) against queries (B).
nw_status run_plan(nw_ctx* c, cudaStream_t stream, const Plan& plan, const Seg* d_segs, const DpParams& base,
                   unsigned long long* counters, uint32_t shard, uint32_t nshards, Timer& tm, RunOut& ro,
                   const uint32_t* const a_enc_by_role[3], const SideView* const A_by_role[3],
                   const uint4* const b_rec_by_role[3], const SideView* const B_by_role[3]) {
  for (size_t li = 0; li < plan.launches.size(); ++li) {
    const LaunchPlan& lp = plan.launches[li];
    const uint64_t lo = lp.ntasks * shard / nshards, hi = lp.ntasks * (shard + 1) / nshards;
    if (lo >= hi) continue;
    DpParams P = base;
    P.dbg_insert_limit = c->dbg_insert_iters >= 0 ? (uint32_t)c->dbg_insert_iters + 1u : 0u;
    P.segs = d_segs + lp.seg_first;
    P.nsegs = lp.nsegs;
    if (lp.ta) P.TA = lp.ta;
    P.serial_a = lp.role == 1 ? 1u : 0u;  // query words are the A side
    P.task_lo = lo;
    P.task_hi = hi;
    P.counter = counters + li;
    P.a_enc = a_enc_by_role[lp.role];
    P.A = *A_by_role[lp.role];
    P.b_rec = b_rec_by_role[lp.role];
    P.B = *B_by_role[lp.role];
    const bool tab = P.sim_tab != nullptr;
    const size_t smem = hist_smem_bytes(P.hist_mode, P.nbins) + dp_stage_bytes(lp.LB) + (tab ? kTabBytes : 0);
    const int epi = P.terms ? kEpiBatchLists
                            : (P.mode == kModeMatrix ? kEpiMatrix
                                                     : (P.hist_mode == kHistLane ? kEpiListsLaneHist : kEpiLists));
    const void* fn = dp_kernel(lp.LB, epi, tab);
    if (!fn) return set_err(c, NW_EINVAL, "no kernel for length %d", lp.LB);
    NW_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    NW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kBlock, smem));
    if (occ < 1) occ = 1;
    if (lp.bps && occ > (int)lp.bps) occ = (int)lp.bps;
    uint64_t grid = (uint64_t)c->sm_count * occ;
    grid = std::min<uint64_t>(grid, cdiv(hi - lo, kWarpsPerBlock));
    void* args[] = {&P};
    cudaEvent_t e0 = nullptr;
    tm.begin(true, e0);
    NW_CK(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kBlock), args, smem, stream));
    tm.end(true, e0);
    ++ro.dp_launches;
    ro.pairs += lp.pairs;  // whole-launch figures; exact for nshards == 1
    ro.cells += lp.cells;
  }
  return NW_OK;
}

nw_status check_device_flags(nw_ctx* c, const uint32_t* d_small) {
  uint32_t err = 0;
  NW_CK(cudaMemcpyAsync(&err, d_small, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->stream));
  NW_CK(cudaStreamSynchronize(c->stream));
  if (err & kErrRetry) return set_err(c, NW_ETIMEOUT, "a neighbour-list update exceeded its retry bound");
  if (err & kErrWait) return set_err(c, NW_ETIMEOUT, "a pipeline wait on the device ran out");
  if (err & kErrInput) return set_err(c, NW_EINVAL, "invalid word index in the input (outputs may be partially written)");
  if (err & kErrCapacity) return set_err(c, NW_ERANGE, "a device buffer reached its capacity (outputs are not valid)");
  if (err & kErrHistRange) return set_err(c, NW_ERANGE, "a score fell outside the histogram range");
  return NW_OK;
}

nw_status topk_impl(nw_dict* d, uint32_t shard, uint32_t nshards, uint32_t k, uint32_t* nbr_idx,
                    int16_t* nbr_score, int64_t* hist, int32_t* hist_lo, uint32_t nbins, uint32_t flags) {
  nw_ctx* c = d->ctx;
  const uint32_t n = d->ws.n;
  if (n < 2) return set_err(c, NW_EINVAL, "the dictionary needs at least 2 words (has %u)", n);
  if (k == 0 || k > NW_MAX_K) return set_err(c, NW_EINVAL, "k must be in [1, %d]", NW_MAX_K);
  if (!nbr_idx || !nbr_score) return set_err(c, NW_EINVAL, "null output pointer");
  if (nshards == 0 || shard >= nshards) return set_err(c, NW_EINVAL, "shard %u of %u", shard, nshards);
  const uint32_t need_bins = (uint32_t)(d->score_hi - d->score_lo + 1);
  if (hist && nbins < need_bins)
    return set_err(c, NW_ERANGE, "histogram needs %u bins for scores [%d, %d], got %u", need_bins, d->score_lo,
                   d->score_hi, nbins);
  if (d->score_lo < INT16_MIN + 1 || d->score_hi > INT16_MAX)
    return set_err(c, NW_ERANGE, "scores [%d, %d] do not fit int16", d->score_lo, d->score_hi);
  const uint32_t ib = index_bits(n);
  const int32_t key_lo = d->score_lo - 1;
  const bool norm = flags & NW_RANK_NORMALISED;
  if (norm && nshards != 1)
    return set_err(c, NW_EINVAL, "the normalised ranking is not available for shards (lists merge by raw score)");
  NormTables nt;
  if (norm) {
    build_norm_tables(d->sc, d->score_lo, d->score_hi, nt);
    if (nt.nranks > 65535u || (uint64_t)nt.nranks >= (1ull << (32 - ib)))
      return set_err(c, NW_ERANGE, "%u normalised score values with %u words do not fit 32-bit list keys", nt.nranks,
                     n);
  } else if ((uint64_t)(d->score_hi - key_lo) >= (1ull << (32 - ib))) {
    return set_err(c, NW_ERANGE, "score range %d..%d with %u words does not fit 32-bit list keys", d->score_lo,
                   d->score_hi, n);
  }
  const bool dev = flags & NW_DEVICE_PTRS;
  cudaStream_t s = c->stream;
  const size_t nlaunch = d->plan.launches.size();

  NW_TRY(ctx_ensure(c, c->ws_slots, sizeof(uint32_t) * (size_t)n * k, "list slots"));
  NW_TRY(ctx_ensure(c, c->ws_thr, sizeof(uint32_t) * (size_t)n, "list thresholds"));
  NW_TRY(ctx_ensure(c, c->ws_small, 64 + sizeof(unsigned long long) * (nlaunch + 1), "task counters"));
  if (hist) NW_TRY(ctx_ensure(c, c->ws_hist, sizeof(unsigned long long) * need_bins, "histogram"));
  uint32_t* out_idx = nbr_idx;
  int16_t* out_score = nbr_score;
  if (!dev) {
    NW_TRY(ctx_ensure(c, c->ws_out_idx, sizeof(uint32_t) * (size_t)n * k, "output indices"));
    NW_TRY(ctx_ensure(c, c->ws_out_score, sizeof(int16_t) * (size_t)n * k, "output scores"));
    out_idx = c->ws_out_idx.as<uint32_t>();
    out_score = c->ws_out_score.as<int16_t>();
  }
  uint32_t* d_err = c->ws_small.as<uint32_t>();
  unsigned long long* d_stats = reinterpret_cast<unsigned long long*>(c->ws_small.as<char>() + 8);
  unsigned long long* d_counters = reinterpret_cast<unsigned long long*>(c->ws_small.as<char>() + 64);

  Timer tm{c};
  cudaEvent_t e_all = nullptr;
  tm.begin(false, e_all);
  NW_CK(cudaMemsetAsync(c->ws_small.p, 0, c->ws_small.bytes, s));
  NW_CK(cudaMemsetAsync(c->ws_slots.p, 0, sizeof(uint32_t) * (size_t)n * k, s));
  NW_CK(cudaMemsetAsync(c->ws_thr.p, 0, sizeof(uint32_t) * (size_t)n, s));
  if (hist) NW_CK(cudaMemsetAsync(c->ws_hist.p, 0, sizeof(unsigned long long) * need_bins, s));

  DpParams base{};
  base.TA = kDefaultTA;
  base.C1 = d->ss.C1;
  base.C2 = d->ss.C2;
  base.match = d->sc.match;
  base.mismatch = d->sc.mismatch;
  base.gap = d->sc.gap;
  base.sim_tab = dict_tab(d);
  base.mode = kModeLists;
  base.k = k;
  base.ib = ib;
  base.imask = (uint32_t)(((uint64_t)1 << ib) - 1);
  base.key_lo = key_lo;
  base.hist_mode = !hist ? kHistNone : hist_mode_for(need_bins);
  base.hist = hist ? c->ws_hist.as<unsigned long long>() : nullptr;
  base.hist_lo = d->score_lo;
  base.nbins = hist ? need_bins : 0;
  base.stats = d_stats;
  base.err = d_err;
  const int16_t* d_frac = nullptr;
  if (norm) {
    // one upload of the three tables, each at a 256-byte aligned offset
    const size_t rank_b = nt.rank.size() * sizeof(uint16_t), smin_b = nt.smin.size() * sizeof(int16_t);
    const size_t o_smin = (rank_b + 255) & ~(size_t)255, o_frac = (o_smin + smin_b + 255) & ~(size_t)255;
    const size_t total = o_frac + nt.frac.size() * sizeof(int16_t);
    NW_TRY(ctx_ensure(c, c->ws_norm, total, "normalised ranking tables"));
    std::vector<char> h(total, 0);
    std::memcpy(h.data(), nt.rank.data(), rank_b);
    std::memcpy(h.data() + o_smin, nt.smin.data(), smin_b);
    std::memcpy(h.data() + o_frac, nt.frac.data(), nt.frac.size() * sizeof(int16_t));
    NW_CK(cudaMemcpyAsync(c->ws_norm.p, h.data(), total, cudaMemcpyHostToDevice, s));
    NW_CK(cudaStreamSynchronize(s));  // the staging vector goes out of scope
    base.norm_rank = c->ws_norm.as<uint16_t>();
    base.norm_smin = reinterpret_cast<const int16_t*>(c->ws_norm.as<char>() + o_smin);
    base.norm_lo = nt.lo;
    d_frac = reinterpret_cast<const int16_t*>(c->ws_norm.as<char>() + o_frac);
  }
  SideView side{d->ws.perm.as<uint32_t>(), c->ws_slots.as<uint32_t>(), c->ws_thr.as<uint32_t>()};
  const uint32_t* a_enc[3] = {d->ws.a_enc.as<uint32_t>(), nullptr, nullptr};
  const uint4* b_rec[3] = {d->ws.b_rec.as<uint4>(), nullptr, nullptr};
  const SideView* views[3] = {&side, nullptr, nullptr};
  RunOut ro;
  NW_TRY(run_plan(c, c->stream, d->plan, d->d_segs.as<Seg>(), base, d_counters, shard, nshards, tm, ro, a_enc,
                  views, b_rec, views));
  cudaEvent_t e_fin = nullptr;
  tm.begin(false, e_fin);
  NW_CK(launch_finalize(c->ws_slots.as<uint32_t>(), n, k, d->ws.perm.as<uint32_t>(), ib, base.imask, key_lo,
                        out_idx, out_score, s, d_frac, d->ws.slen.as<uint8_t>(), d->ws.rank.as<uint32_t>()));
  tm.end(false, e_fin);
  if (hist && dev) NW_CK(cudaMemcpyAsync(hist, c->ws_hist.p, sizeof(int64_t) * need_bins, cudaMemcpyDeviceToDevice, s));
  if (!dev) {
    NW_CK(cudaMemcpyAsync(nbr_idx, out_idx, sizeof(uint32_t) * (size_t)n * k, cudaMemcpyDeviceToHost, s));
    NW_CK(cudaMemcpyAsync(nbr_score, out_score, sizeof(int16_t) * (size_t)n * k, cudaMemcpyDeviceToHost, s));
    if (hist) NW_CK(cudaMemcpyAsync(hist, c->ws_hist.p, sizeof(int64_t) * need_bins, cudaMemcpyDeviceToHost, s));
  }
  if (hist) {
    if (hist_lo) *hist_lo = d->score_lo;
    if (nbins > need_bins) {
      if (dev) NW_CK(cudaMemsetAsync(hist + need_bins, 0, sizeof(int64_t) * (nbins - need_bins), s));
      else std::memset(hist + need_bins, 0, sizeof(int64_t) * (nbins - need_bins));
    }
  }
  tm.mark(tm.c->profiling ? tm.get() : nullptr);
  if ((flags & NW_ASYNC) && dev) return NW_OK;
  NW_TRY(check_device_flags(c, d_err));
  if (c->profiling) {
    tm.collect();
    unsigned long long ins = 0;
    NW_CK(cudaMemcpy(&ins, d_stats, sizeof ins, cudaMemcpyDeviceToHost));
    c->prof.dp_launches = ro.dp_launches;
    c->prof.launches = ro.dp_launches + 1;
    c->prof.pairs = nshards == 1 ? d->plan.pairs : 0;
    c->prof.cells = nshards == 1 ? d->plan.cells : 0;
    c->prof.list_inserts = ins;
  }
  return NW_OK;
}

}  // namespace

