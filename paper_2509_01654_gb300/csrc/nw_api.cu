// nw_api.cu -- host runtime of libnw: the C ABI declared in include/nw.h.
//
// Contexts own a stream (or borrow the caller's), a device-memory budget and a
// grow-only workspace.  Dictionaries are word sets resident on the device,
// sorted by length into buckets and encoded for the alignment kernel, plus the
// plan of pair rectangles ("segments") the all-pairs launches walk.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <set>
#include <string>
#include <vector>

#include "nw.h"
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
  std::string err;
  bool profiling = false;
  nw_profile prof{};
  int sm_count = 0;
  std::set<nw_dict*> dicts;
  std::atomic<int> busy{0};
  // grow-only workspace
  DevBuf ws_slots, ws_thr, ws_hist, ws_small, ws_out_idx, ws_out_score, ws_mat, ws_pairs, ws_segs;
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

#define NW_ENTER(ctxp)                                                              \
  if (!(ctxp)) return NW_EINVAL;                                                    \
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

// Every (query, dictionary word) pair once; the longer word goes to the lanes.
void plan_query(const Buckets& qb, const Buckets& db, uint32_t TA, Plan& out) {
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
      for (int La = La_hi; La >= 0; --La) {
        const uint32_t nA = Aset.count[La];
        if (nA == 0) continue;
        uint64_t nt = 0;
        out.segs.push_back(make_seg(Aset, La, Aset.start[La], Aset.start[La] + nA, Bset, LB, Bset.start[LB],
                                    Bset.start[LB] + nB, false, TA, task, nt));
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

nw_status run_plan(nw_ctx* c, const Plan& plan, const Seg* d_segs, const DpParams& base, const WordSet* Aset_role,
                   const WordSet* Bset_role, unsigned long long* counters, uint32_t shard, uint32_t nshards,
                   Timer& tm, RunOut& ro,
                   // role-specific sides: [role] -> (a_enc, A view, b_rec, B view)
                   const uint32_t* const a_enc_by_role[3], const SideView* const A_by_role[3],
                   const uint4* const b_rec_by_role[3], const SideView* const B_by_role[3]) {
  (void)Aset_role;
  (void)Bset_role;
  for (size_t li = 0; li < plan.launches.size(); ++li) {
    const LaunchPlan& lp = plan.launches[li];
    const uint64_t lo = lp.ntasks * shard / nshards, hi = lp.ntasks * (shard + 1) / nshards;
    if (lo >= hi) continue;
    DpParams P = base;
    P.segs = d_segs + lp.seg_first;
    P.nsegs = lp.nsegs;
    P.task_lo = lo;
    P.task_hi = hi;
    P.counter = counters + li;
    P.a_enc = a_enc_by_role[lp.role];
    P.A = *A_by_role[lp.role];
    P.b_rec = b_rec_by_role[lp.role];
    P.B = *B_by_role[lp.role];
    const size_t smem = hist_smem_bytes(P.hist_mode, P.nbins) + dp_stage_bytes(lp.LB);
    const int epi = P.mode == kModeMatrix ? kEpiMatrix : (P.hist_mode == kHistLane ? kEpiListsLaneHist : kEpiLists);
    const void* fn = dp_kernel(lp.LB, epi);
    if (!fn) return set_err(c, NW_EINVAL, "no kernel for length %d", lp.LB);
    NW_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int occ = 0;
    NW_CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, fn, kBlock, smem));
    if (occ < 1) occ = 1;
    uint64_t grid = (uint64_t)c->sm_count * occ;
    grid = std::min<uint64_t>(grid, cdiv(hi - lo, kWarpsPerBlock));
    void* args[] = {&P};
    cudaEvent_t e0 = nullptr;
    tm.begin(true, e0);
    NW_CK(cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kBlock), args, smem, c->stream));
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
  if (err & kErrInput) return set_err(c, NW_EINVAL, "invalid word index in the input (outputs may be partially written)");
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
  if ((uint64_t)(d->score_hi - key_lo) >= (1ull << (32 - ib)))
    return set_err(c, NW_ERANGE, "score range %d..%d with %u words does not fit 32-bit list keys", d->score_lo,
                   d->score_hi, n);
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
  SideView side{d->ws.perm.as<uint32_t>(), c->ws_slots.as<uint32_t>(), c->ws_thr.as<uint32_t>()};
  const uint32_t* a_enc[3] = {d->ws.a_enc.as<uint32_t>(), nullptr, nullptr};
  const uint4* b_rec[3] = {d->ws.b_rec.as<uint4>(), nullptr, nullptr};
  const SideView* views[3] = {&side, nullptr, nullptr};
  RunOut ro;
  NW_TRY(run_plan(c, d->plan, d->d_segs.as<Seg>(), base, &d->ws, &d->ws, d_counters, shard, nshards, tm, ro, a_enc,
                  views, b_rec, views));
  cudaEvent_t e_fin = nullptr;
  tm.begin(false, e_fin);
  NW_CK(launch_finalize(c->ws_slots.as<uint32_t>(), n, k, d->ws.perm.as<uint32_t>(), ib, base.imask, key_lo,
                        out_idx, out_score, s));
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

// ===========================================================================
// C ABI

extern "C" {

nw_status nw_create(nw_ctx** out, int device, size_t mem_budget_bytes, void* cuda_stream) {
  if (!out) return set_err(nullptr, NW_EINVAL, "null output pointer");
  *out = nullptr;
  int ndev = 0;
  cudaError_t e = cudaGetDeviceCount(&ndev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return set_err(nullptr, NW_ECUDA, "cudaGetDeviceCount: %s", cudaGetErrorString(e));
  }
  if (device < 0 || device >= ndev) return set_err(nullptr, NW_EINVAL, "device %d of %d", device, ndev);
  e = cudaSetDevice(device);
  if (e != cudaSuccess) return set_err(nullptr, NW_ECUDA, "cudaSetDevice: %s", cudaGetErrorString(e));
  nw_ctx* c = new nw_ctx();
  c->device = device;
  c->budget = mem_budget_bytes;
  if (cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
    delete c;
    cudaGetLastError();
    return set_err(nullptr, NW_ECUDA, "cannot query the SM count");
  }
  if (cuda_stream) {
    c->stream = static_cast<cudaStream_t>(cuda_stream);
  } else {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete c;
      cudaGetLastError();
      return set_err(nullptr, NW_ECUDA, "cannot create a stream");
    }
    c->own_stream = true;
  }
  *out = c;
  return NW_OK;
}

void nw_destroy(nw_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  std::vector<nw_dict*> ds(c->dicts.begin(), c->dicts.end());
  for (nw_dict* d : ds) nw_dict_free(d);
  ctx_free(c, c->ws_slots);
  ctx_free(c, c->ws_thr);
  ctx_free(c, c->ws_hist);
  ctx_free(c, c->ws_small);
  ctx_free(c, c->ws_out_idx);
  ctx_free(c, c->ws_out_score);
  ctx_free(c, c->ws_mat);
  ctx_free(c, c->ws_pairs);
  ctx_free(c, c->ws_segs);
  for (cudaEvent_t e : c->events) cudaEventDestroy(e);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
}

const char* nw_last_error(const nw_ctx* c) { return c ? c->err.c_str() : g_create_error.c_str(); }

nw_status nw_set_profiling(nw_ctx* c, int enable) {
  if (!c) return NW_EINVAL;
  c->profiling = enable != 0;
  return NW_OK;
}

nw_status nw_last_profile(const nw_ctx* c, nw_profile* out) {
  if (!c || !out) return NW_EINVAL;
  *out = c->prof;
  return NW_OK;
}

nw_status nw_load_dictionary(nw_ctx* c, const uint8_t* codes, const uint32_t* offsets, uint32_t n,
                             uint32_t alphabet, const nw_scoring* scoring, uint32_t flags, nw_dict** out) {
  NW_ENTER(c);
  if (!out || !offsets || !scoring || (!codes && n)) return set_err(c, NW_EINVAL, "null pointer argument");
  *out = nullptr;
  if (alphabet == 0 || alphabet > 256) return set_err(c, NW_EINVAL, "alphabet must be in [1, 256]");
  nw_dict* d = new nw_dict();
  d->ctx = c;
  d->sc = *scoring;
  d->alphabet = alphabet;
  nw_status st = make_shifted(c, *scoring, alphabet, d->ss);
  if (st == NW_OK) st = ingest(c, codes, offsets, n, alphabet, d->ss.shift, flags, d->ws);
  if (st == NW_OK) {
    // score bounds over the length pairs present
    int lo = INT32_MAX, hi = INT32_MIN;
    for (int La = 0; La < kBuckets; ++La) {
      for (int Lb = La; Lb < kBuckets; ++Lb) {
        const uint32_t na = d->ws.bk.count[La], nb = d->ws.bk.count[Lb];
        if (!na || !nb || (La == Lb && na < 2)) continue;
        int l, h;
        pair_bounds(*scoring, La, Lb, l, h);
        lo = std::min(lo, l);
        hi = std::max(hi, h);
      }
    }
    if (lo > hi) lo = hi = 0;  // fewer than two words
    d->score_lo = lo;
    d->score_hi = hi;
    plan_all_pairs(d->ws.bk, kDefaultTA, d->plan);
    st = ctx_alloc(c, d->d_segs, sizeof(Seg) * std::max<size_t>(1, d->plan.segs.size()), "segment plan");
    if (st == NW_OK && !d->plan.segs.empty()) {
      cudaError_t e = cudaMemcpyAsync(d->d_segs.p, d->plan.segs.data(), sizeof(Seg) * d->plan.segs.size(),
                                      cudaMemcpyHostToDevice, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      if (e != cudaSuccess) st = cuda_fail(c, e, "uploading the segment plan");
    }
  }
  if (st != NW_OK) {
    free_wordset(c, d->ws);
    ctx_free(c, d->d_segs);
    delete d;
    return st;
  }
  c->dicts.insert(d);
  *out = d;
  return NW_OK;
}

nw_status nw_dict_info_get(const nw_dict* d, nw_dict_info* out) {
  if (!d || !out) return NW_EINVAL;
  nw_dict_info i{};
  i.n = d->ws.n;
  i.alphabet = d->alphabet;
  i.min_len = d->ws.min_len;
  i.max_len = d->ws.max_len;
  i.score_lo = d->score_lo;
  i.score_hi = d->score_hi;
  i.nbins = (uint32_t)(d->score_hi - d->score_lo + 1);
  i.pairs = d->plan.pairs;
  i.cells = d->plan.cells;
  i.device_bytes = wordset_bytes(d->ws) + d->d_segs.bytes;
  *out = i;
  return NW_OK;
}

void nw_dict_free(nw_dict* d) {
  if (!d) return;
  nw_ctx* c = d->ctx;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  free_wordset(c, d->ws);
  ctx_free(c, d->d_segs);
  c->dicts.erase(d);
  delete d;
}

nw_status nw_all_pairs_matrix(nw_dict* d, int8_t* out, uint32_t flags) {
  if (!d) return NW_EINVAL;
  nw_ctx* c = d->ctx;
  NW_ENTER(c);
  const uint32_t n = d->ws.n;
  if (!out) return set_err(c, NW_EINVAL, "null output pointer");
  if (n < 2) return set_err(c, NW_EINVAL, "the dictionary needs at least 2 words (has %u)", n);
  if (d->score_lo < -128 || d->score_hi > 127)
    return set_err(c, NW_ERANGE, "scores of this dictionary span [%d, %d], outside int8", d->score_lo, d->score_hi);
  const bool dev = flags & NW_DEVICE_PTRS;
  const uint64_t E = (uint64_t)n * (n - 1) / 2;
  cudaStream_t s = c->stream;
  int8_t* dst = out;
  if (!dev) {
    NW_TRY(ctx_ensure(c, c->ws_mat, E, "score matrix"));
    dst = c->ws_mat.as<int8_t>();
  }
  NW_TRY(ctx_ensure(c, c->ws_small, 64 + sizeof(unsigned long long) * (d->plan.launches.size() + 1), "task counters"));
  uint32_t* d_err = c->ws_small.as<uint32_t>();
  unsigned long long* d_counters = reinterpret_cast<unsigned long long*>(c->ws_small.as<char>() + 64);
  Timer tm{c};
  cudaEvent_t e0 = nullptr;
  tm.begin(false, e0);
  NW_CK(cudaMemsetAsync(c->ws_small.p, 0, c->ws_small.bytes, s));
  DpParams base{};
  base.TA = kDefaultTA;
  base.C1 = d->ss.C1;
  base.C2 = d->ss.C2;
  base.match = d->sc.match;
  base.mismatch = d->sc.mismatch;
  base.gap = d->sc.gap;
  base.mode = kModeMatrix;
  base.mat = dst;
  base.n = n;
  base.hist_mode = kHistNone;
  base.err = d_err;
  SideView side{d->ws.perm.as<uint32_t>(), nullptr, nullptr};
  const uint32_t* a_enc[3] = {d->ws.a_enc.as<uint32_t>(), nullptr, nullptr};
  const uint4* b_rec[3] = {d->ws.b_rec.as<uint4>(), nullptr, nullptr};
  const SideView* views[3] = {&side, nullptr, nullptr};
  RunOut ro;
  NW_TRY(run_plan(c, d->plan, d->d_segs.as<Seg>(), base, &d->ws, &d->ws, d_counters, 0, 1, tm, ro, a_enc, views,
                  b_rec, views));
  if (!dev) NW_CK(cudaMemcpyAsync(out, dst, E, cudaMemcpyDeviceToHost, s));
  tm.mark(c->profiling ? tm.get() : nullptr);
  if ((flags & NW_ASYNC) && dev) return NW_OK;
  NW_TRY(check_device_flags(c, d_err));
  if (c->profiling) {
    tm.collect();
    c->prof.dp_launches = ro.dp_launches;
    c->prof.launches = ro.dp_launches;
    c->prof.pairs = d->plan.pairs;
    c->prof.cells = d->plan.cells;
    c->prof.list_inserts = 0;
  }
  return NW_OK;
}

nw_status nw_all_pairs_topk(nw_dict* d, uint32_t k, uint32_t* nbr_idx, int16_t* nbr_score, int64_t* hist,
                            int32_t* hist_lo, uint32_t nbins, uint32_t flags) {
  if (!d) return NW_EINVAL;
  NW_ENTER(d->ctx);
  return topk_impl(d, 0, 1, k, nbr_idx, nbr_score, hist, hist_lo, nbins, flags);
}

nw_status nw_all_pairs_topk_shard(nw_dict* d, uint32_t shard, uint32_t nshards, uint32_t k, uint32_t* nbr_idx,
                                  int16_t* nbr_score, int64_t* hist, int32_t* hist_lo, uint32_t nbins,
                                  uint32_t flags) {
  if (!d) return NW_EINVAL;
  NW_ENTER(d->ctx);
  return topk_impl(d, shard, nshards, k, nbr_idx, nbr_score, hist, hist_lo, nbins, flags);
}

nw_status nw_topk_merge(uint32_t n, uint32_t k, uint32_t nparts, const uint32_t* const* idx_parts,
                        const int16_t* const* score_parts, uint32_t* idx_out, int16_t* score_out) {
  if (k == 0 || !idx_out || !score_out || (nparts && (!idx_parts || !score_parts))) return NW_EINVAL;
  for (uint32_t p = 0; p < nparts; ++p)
    if (!idx_parts[p] || !score_parts[p]) return NW_EINVAL;
  std::vector<std::pair<int32_t, uint32_t>> cand;
  cand.reserve((size_t)nparts * k);
  for (uint32_t w = 0; w < n; ++w) {
    cand.clear();
    for (uint32_t p = 0; p < nparts; ++p) {
      for (uint32_t r = 0; r < k; ++r) {
        const uint32_t j = idx_parts[p][(size_t)w * k + r];
        if (j == 0xffffffffu) continue;
        cand.emplace_back(score_parts[p][(size_t)w * k + r], j);
      }
    }
    std::sort(cand.begin(), cand.end(), [](const std::pair<int32_t, uint32_t>& x, const std::pair<int32_t, uint32_t>& y) {
      return x.first != y.first ? x.first > y.first : x.second < y.second;
    });
    uint32_t r = 0;
    for (size_t q = 0; q < cand.size() && r < k; ++q) {
      if (q > 0 && cand[q].second == cand[q - 1].second) continue;  // same neighbour from two parts
      idx_out[(size_t)w * k + r] = cand[q].second;
      score_out[(size_t)w * k + r] = (int16_t)cand[q].first;
      ++r;
    }
    for (; r < k; ++r) {
      idx_out[(size_t)w * k + r] = 0xffffffffu;
      score_out[(size_t)w * k + r] = INT16_MIN;
    }
  }
  return NW_OK;
}

nw_status nw_score_pairs(nw_dict* d, const uint32_t* i, const uint32_t* j, size_t m, int16_t* out, uint32_t flags) {
  if (!d) return NW_EINVAL;
  nw_ctx* c = d->ctx;
  NW_ENTER(c);
  if (m == 0) return NW_OK;
  if (!i || !j || !out) return set_err(c, NW_EINVAL, "null pointer argument");
  const bool dev = flags & NW_DEVICE_PTRS;
  const uint32_t n = d->ws.n;
  cudaStream_t s = c->stream;
  // every pair's score lies within the bounds of its lengths, all of which fit int16 by the scoring limits
  const uint32_t* di = i;
  const uint32_t* dj = j;
  int16_t* dout = out;
  if (!dev) {
    for (size_t p = 0; p < m; ++p)
      if (i[p] >= n || j[p] >= n) return set_err(c, NW_EINVAL, "pair %zu: index out of range (n = %u)", p, n);
    NW_TRY(ctx_ensure(c, c->ws_pairs, m * (2 * sizeof(uint32_t) + sizeof(int16_t)) + 64, "pair buffers"));
    char* base = c->ws_pairs.as<char>();
    NW_CK(cudaMemcpyAsync(base, i, m * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    NW_CK(cudaMemcpyAsync(base + m * sizeof(uint32_t), j, m * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
    di = reinterpret_cast<const uint32_t*>(base);
    dj = reinterpret_cast<const uint32_t*>(base + m * sizeof(uint32_t));
    dout = reinterpret_cast<int16_t*>(base + 2 * m * sizeof(uint32_t));
  }
  NW_TRY(ctx_ensure(c, c->ws_small, 64, "error flag"));
  NW_CK(cudaMemsetAsync(c->ws_small.p, 0, 64, s));
  PairsParams P{};
  P.pi = di;
  P.pj = dj;
  P.m = m;
  P.n = n;
  P.rank = d->ws.rank.as<uint32_t>();
  P.slen = d->ws.slen.as<uint8_t>();
  P.aoff = d->ws.aoff.as<uint32_t>();
  P.brec_w = d->ws.brec_w.as<uint32_t>();
  P.a_enc = d->ws.a_enc.as<uint32_t>();
  P.b_rec = d->ws.b_rec.as<uint32_t>();
  P.C1 = d->ss.C1;
  P.C2 = d->ss.C2;
  P.gap = d->sc.gap;
  P.out = dout;
  P.err = c->ws_small.as<uint32_t>();
  Timer tm{c};
  cudaEvent_t e0 = nullptr;
  tm.begin(true, e0);
  NW_CK(launch_pairs(P, s));
  tm.end(true, e0);
  if (!dev) NW_CK(cudaMemcpyAsync(out, dout, m * sizeof(int16_t), cudaMemcpyDeviceToHost, s));
  if ((flags & NW_ASYNC) && dev) return NW_OK;
  NW_TRY(check_device_flags(c, c->ws_small.as<uint32_t>()));
  if (c->profiling) {
    tm.collect();
    c->prof.dp_launches = 1;
    c->prof.launches = 1;
    c->prof.pairs = m;
    c->prof.cells = 0;
    c->prof.list_inserts = 0;
  }
  return NW_OK;
}

nw_status nw_query(nw_dict* d, const uint8_t* qcodes, const uint32_t* qoffsets, uint32_t nq, uint32_t k,
                   uint32_t* nbr_idx, int16_t* nbr_score, uint32_t flags) {
  if (!d) return NW_EINVAL;
  nw_ctx* c = d->ctx;
  NW_ENTER(c);
  if (nq == 0) return NW_OK;
  if (!qoffsets || !nbr_idx || !nbr_score) return set_err(c, NW_EINVAL, "null pointer argument");
  if (k == 0 || k > NW_MAX_K) return set_err(c, NW_EINVAL, "k must be in [1, %d]", NW_MAX_K);
  const uint32_t n = d->ws.n;
  const bool dev = flags & NW_DEVICE_PTRS;
  cudaStream_t s = c->stream;

  WordSet q;
  struct QFree {
    nw_ctx* c;
    WordSet& q;
    ~QFree() { free_wordset(c, q); }
  } qfree{c, q};
  NW_TRY(ingest(c, qcodes, qoffsets, nq, d->alphabet, d->ss.shift, flags & NW_DEVICE_PTRS, q));
  int lo = INT32_MAX, hi = INT32_MIN;
  for (int La = 0; La < kBuckets; ++La)
    for (int Lb = 0; Lb < kBuckets; ++Lb) {
      if (!q.bk.count[La] || !d->ws.bk.count[Lb]) continue;
      int l, h;
      pair_bounds(d->sc, La, Lb, l, h);
      lo = std::min(lo, l);
      hi = std::max(hi, h);
    }
  if (n == 0) lo = hi = 0;
  if (lo < INT16_MIN + 1 || hi > INT16_MAX) return set_err(c, NW_ERANGE, "query scores do not fit int16");
  const uint32_t ib = index_bits(std::max<uint32_t>(n, 2));
  const int32_t key_lo = lo - 1;
  if ((uint64_t)(hi - key_lo) >= (1ull << (32 - ib)))
    return set_err(c, NW_ERANGE, "score range with %u dictionary words does not fit 32-bit list keys", n);
  Plan plan;
  plan_query(q.bk, d->ws.bk, kDefaultTA, plan);
  NW_TRY(ctx_ensure(c, c->ws_segs, sizeof(Seg) * std::max<size_t>(1, plan.segs.size()), "query segments"));
  NW_TRY(ctx_ensure(c, c->ws_slots, sizeof(uint32_t) * (size_t)nq * k, "list slots"));
  NW_TRY(ctx_ensure(c, c->ws_thr, sizeof(uint32_t) * (size_t)nq, "list thresholds"));
  NW_TRY(ctx_ensure(c, c->ws_small, 64 + sizeof(unsigned long long) * (plan.launches.size() + 1), "task counters"));
  uint32_t* out_idx = nbr_idx;
  int16_t* out_score = nbr_score;
  if (!dev) {
    NW_TRY(ctx_ensure(c, c->ws_out_idx, sizeof(uint32_t) * (size_t)nq * k, "output indices"));
    NW_TRY(ctx_ensure(c, c->ws_out_score, sizeof(int16_t) * (size_t)nq * k, "output scores"));
    out_idx = c->ws_out_idx.as<uint32_t>();
    out_score = c->ws_out_score.as<int16_t>();
  }
  uint32_t* d_err = c->ws_small.as<uint32_t>();
  unsigned long long* d_stats = reinterpret_cast<unsigned long long*>(c->ws_small.as<char>() + 8);
  unsigned long long* d_counters = reinterpret_cast<unsigned long long*>(c->ws_small.as<char>() + 64);
  Timer tm{c};
  cudaEvent_t e_all = nullptr;
  tm.begin(false, e_all);
  if (!plan.segs.empty())
    NW_CK(cudaMemcpyAsync(c->ws_segs.p, plan.segs.data(), sizeof(Seg) * plan.segs.size(), cudaMemcpyHostToDevice, s));
  NW_CK(cudaMemsetAsync(c->ws_small.p, 0, c->ws_small.bytes, s));
  NW_CK(cudaMemsetAsync(c->ws_slots.p, 0, sizeof(uint32_t) * (size_t)nq * k, s));
  NW_CK(cudaMemsetAsync(c->ws_thr.p, 0, sizeof(uint32_t) * (size_t)nq, s));
  DpParams base{};
  base.TA = kDefaultTA;
  base.C1 = d->ss.C1;
  base.C2 = d->ss.C2;
  base.match = d->sc.match;
  base.mismatch = d->sc.mismatch;
  base.gap = d->sc.gap;
  base.mode = kModeLists;
  base.k = k;
  base.ib = ib;
  base.imask = (uint32_t)(((uint64_t)1 << ib) - 1);
  base.key_lo = key_lo;
  base.hist_mode = kHistNone;
  base.stats = d_stats;
  base.err = d_err;
  SideView qside{q.perm.as<uint32_t>(), c->ws_slots.as<uint32_t>(), c->ws_thr.as<uint32_t>()};
  SideView dside{d->ws.perm.as<uint32_t>(), nullptr, nullptr};
  const uint32_t* a_enc[3] = {nullptr, q.a_enc.as<uint32_t>(), d->ws.a_enc.as<uint32_t>()};
  const uint4* b_rec[3] = {nullptr, d->ws.b_rec.as<uint4>(), q.b_rec.as<uint4>()};
  const SideView* A_views[3] = {nullptr, &qside, &dside};
  const SideView* B_views[3] = {nullptr, &dside, &qside};
  RunOut ro;
  NW_TRY(run_plan(c, plan, c->ws_segs.as<Seg>(), base, nullptr, nullptr, d_counters, 0, 1, tm, ro, a_enc, A_views,
                  b_rec, B_views));
  cudaEvent_t e_fin = nullptr;
  tm.begin(false, e_fin);
  NW_CK(launch_finalize(c->ws_slots.as<uint32_t>(), nq, k, q.perm.as<uint32_t>(), ib, base.imask, key_lo, out_idx,
                        out_score, s));
  tm.end(false, e_fin);
  if (!dev) {
    NW_CK(cudaMemcpyAsync(nbr_idx, out_idx, sizeof(uint32_t) * (size_t)nq * k, cudaMemcpyDeviceToHost, s));
    NW_CK(cudaMemcpyAsync(nbr_score, out_score, sizeof(int16_t) * (size_t)nq * k, cudaMemcpyDeviceToHost, s));
  }
  tm.mark(c->profiling ? tm.get() : nullptr);
  // the query set is freed on return, so the stream is always synchronised here
  NW_TRY(check_device_flags(c, d_err));
  if (c->profiling) {
    tm.collect();
    unsigned long long ins = 0;
    NW_CK(cudaMemcpy(&ins, d_stats, sizeof ins, cudaMemcpyDeviceToHost));
    c->prof.dp_launches = ro.dp_launches;
    c->prof.launches = ro.dp_launches + 1;
    c->prof.pairs = plan.pairs;
    c->prof.cells = plan.cells;
    c->prof.list_inserts = ins;
  }
  return NW_OK;
}

nw_status nw_measure_int_rates(nw_ctx* c, double ms_target, nw_int_rates* out) {
  NW_ENTER(c);
  if (!out) return set_err(c, NW_EINVAL, "null output pointer");
  if (ms_target <= 0) ms_target = 200;
  cudaStream_t s = c->stream;
  const int max_blocks = c->sm_count * (2048 / kRateBlock);  // at most 2048 resident threads per SM
  DevBuf buf;
  NW_TRY(ctx_alloc(c, buf, 4096 + sizeof(uint32_t) * (size_t)max_blocks * kRateBlock, "rate buffers"));
  struct BFree {
    nw_ctx* c;
    DevBuf& b;
    ~BFree() { ctx_free(c, b); }
  } bfree{c, buf};
  uint32_t seeds[64];
  for (int q = 0; q < 64; ++q) seeds[q] = 0x01000100u * (q + 1) ^ (0x00030005u * q);
  uint32_t* d_in = buf.as<uint32_t>();
  unsigned long long* d_cyc = reinterpret_cast<unsigned long long*>(buf.as<char>() + 1024);
  uint32_t* d_out = reinterpret_cast<uint32_t*>(buf.as<char>() + 4096);
  NW_CK(cudaMemcpyAsync(d_in, seeds, sizeof seeds, cudaMemcpyHostToDevice, s));
  cudaEvent_t e0, e1;
  NW_CK(cudaEventCreate(&e0));
  NW_CK(cudaEventCreate(&e1));
  double rates[kRateOps] = {0};
  double clock_sum = 0;
  int clock_n = 0;
  for (int op = 0; op < kRateOps; ++op) {
    // exactly one wave, so every block runs for the whole kernel and
    // clock64 cycles per block over the event time give the SM clock
    const int blocks = std::min(max_blocks, c->sm_count * rate_blocks_per_sm(op));
    int iters = op == kRateCell ? 64 : 2048;
    double ms = 0;
    unsigned long long cyc = 0;
    for (int attempt = 0; attempt < 6; ++attempt) {
      NW_CK(cudaMemsetAsync(d_cyc, 0, sizeof(unsigned long long), s));
      NW_CK(cudaEventRecord(e0, s));
      NW_CK(launch_rate(op, blocks, iters, d_in, d_out, d_cyc, s));
      NW_CK(cudaEventRecord(e1, s));
      NW_CK(cudaEventSynchronize(e1));
      float f = 0;
      NW_CK(cudaEventElapsedTime(&f, e0, e1));
      ms = f;
      NW_CK(cudaMemcpy(&cyc, d_cyc, sizeof cyc, cudaMemcpyDeviceToHost));
      if (ms >= 0.5 * ms_target || attempt == 5) break;
      const double scale = std::min(64.0, std::max(2.0, ms_target / std::max(ms, 1e-3)));
      iters = (int)std::min(1e9, iters * scale);
    }
    rates[op] = (double)blocks * kRateBlock * (double)iters * rate_ops_per_iter(op) / (ms * 1e-3);
    clock_sum += (double)cyc / blocks / (ms * 1e3);
    ++clock_n;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  out->viaddmax_s16x2 = rates[kRateViaddmax];
  out->vimax3_s16x2 = rates[kRateVimax3];
  out->vimax_s16x2_relu = rates[kRateVimaxRelu];
  out->iadd3 = rates[kRateIadd3];
  out->lop3 = rates[kRateLop3];
  out->nw_cell_mix = rates[kRateCell];
  out->sm_clock_mhz = clock_sum / clock_n;
  out->sm_count = (uint32_t)c->sm_count;
  return NW_OK;
}

nw_status nw_debug_enumerate_pairs(const uint32_t* lengths, uint32_t n, uint32_t shard, uint32_t nshards, uint32_t* a,
                                   uint32_t* b, uint64_t cap, uint64_t* count) {
  if (!lengths || !count || nshards == 0 || shard >= nshards) return NW_EINVAL;
  if (cap && (!a || !b)) return NW_EINVAL;
  Buckets bk{};
  for (uint32_t i = 0; i < n; ++i) {
    if (lengths[i] > (uint32_t)kMaxLen) return NW_EINVAL;
    ++bk.count[lengths[i]];
  }
  fill_buckets(bk);
  std::vector<uint32_t> perm(n), fill(kBuckets, 0);
  for (uint32_t i = 0; i < n; ++i) perm[bk.start[lengths[i]] + fill[lengths[i]]++] = i;  // stable by length
  Plan plan;
  plan_all_pairs(bk, kDefaultTA, plan);
  uint64_t cnt = 0;
  for (const LaunchPlan& lp : plan.launches) {
    const uint64_t lo = lp.ntasks * shard / nshards, hi = lp.ntasks * (shard + 1) / nshards;
    const Seg* segs = plan.segs.data() + lp.seg_first;
    for (uint64_t t = lo; t < hi; ++t) {
      const Seg& S = segs[find_seg(segs, lp.nsegs, t)];
      const TaskGeom g = task_geom(S, t, kDefaultTA);
      for (uint32_t x = g.a0; x < g.a1; ++x) {
        for (uint32_t lane = 0; lane < 32; ++lane) {
          for (uint32_t h = 0; h < 2; ++h) {
            const uint32_t y = g.b0 + 2 * lane + h;
            if (!pair_valid(g, x, y)) continue;
            if (cnt < cap) {
              a[cnt] = perm[x];
              b[cnt] = perm[y];
            }
            ++cnt;
          }
        }
      }
    }
  }
  *count = cnt;
  return NW_OK;
}

nw_status nw_debug_fail_alloc(nw_ctx* c, uint32_t countdown) {
  if (!c) return NW_EINVAL;
  c->fail_countdown = countdown;
  return NW_OK;
}

}  // extern "C"

// ===========================================================================
// The all-pairs top-k reduction over a fixed scratch region (no allocation).

namespace nw {

nw_status topk_into_scratch(nw_dict* d, ScratchProvider provide, uint32_t k, uint32_t* nbr_idx,
                            int16_t* nbr_score, int64_t* hist, int32_t* hist_lo, uint32_t nbins,
                            uint32_t flags) {
  if (!d || !provide) return NW_EINVAL;
  nw_ctx* c = d->ctx;
  NW_ENTER(c);
  if (!(flags & NW_DEVICE_PTRS))
    return set_err(c, NW_EINVAL, "the no-allocation variant needs device output buffers (NW_DEVICE_PTRS)");
  const uint32_t n = d->ws.n;
  if (n < 2) return set_err(c, NW_EINVAL, "the dictionary needs at least 2 words (has %u)", n);
  if (k == 0 || k > NW_MAX_K) return set_err(c, NW_EINVAL, "k must be in [1, %d]", NW_MAX_K);
  if (!nbr_idx || !nbr_score) return set_err(c, NW_EINVAL, "null output pointer");
  const uint32_t need_bins = (uint32_t)(d->score_hi - d->score_lo + 1);
  if (hist && nbins < need_bins)
    return set_err(c, NW_ERANGE, "histogram needs %u bins for scores [%d, %d], got %u", need_bins, d->score_lo,
                   d->score_hi, nbins);
  if (d->score_lo < INT16_MIN + 1 || d->score_hi > INT16_MAX)
    return set_err(c, NW_ERANGE, "scores [%d, %d] do not fit int16", d->score_lo, d->score_hi);
  const uint32_t ib = index_bits(n);
  const int32_t key_lo = d->score_lo - 1;
  if ((uint64_t)(d->score_hi - key_lo) >= (1ull << (32 - ib)))
    return set_err(c, NW_ERANGE, "score range %d..%d with %u words does not fit 32-bit list keys", d->score_lo,
                   d->score_hi, n);

  // scratch layout: [error flag, insert count, task counters | 2 KiB][thresholds][list slots][histogram]
  const size_t nlaunch = d->plan.launches.size();
  auto up256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t off_thr = 2048;
  const size_t off_slots = off_thr + up256(sizeof(uint32_t) * (size_t)n);
  const size_t off_hist = off_slots + up256(sizeof(uint32_t) * (size_t)n * k);
  const size_t need = off_hist + (hist ? up256(sizeof(unsigned long long) * need_bins) : 0);
  if (64 + sizeof(unsigned long long) * (nlaunch + 1) > off_thr)
    return set_err(c, NW_ERANGE, "too many launches for the scratch header");
  void* base = nullptr;
  size_t cap = 0;
  const char* why = "";
  const nw_status pst = provide(c->device, &base, &cap, &why);
  if (pst != NW_OK) return set_err(c, pst, "static scratch region unavailable: %s", why);
  if (need > cap)
    return set_err(c, NW_ERANGE, "%u words with k = %u need %zu bytes of scratch; the static region holds %zu", n, k,
                   need, cap);
  char* sb = static_cast<char*>(base);
  uint32_t* d_err = reinterpret_cast<uint32_t*>(sb);
  unsigned long long* d_stats = reinterpret_cast<unsigned long long*>(sb + 8);
  unsigned long long* d_counters = reinterpret_cast<unsigned long long*>(sb + 64);
  uint32_t* d_thr = reinterpret_cast<uint32_t*>(sb + off_thr);
  uint32_t* d_slots = reinterpret_cast<uint32_t*>(sb + off_slots);
  unsigned long long* d_hist = hist ? reinterpret_cast<unsigned long long*>(sb + off_hist) : nullptr;
  cudaStream_t s = c->stream;

  // no events either: this path creates nothing
  const bool saved_profiling = c->profiling;
  c->profiling = false;
  struct Restore {
    nw_ctx* c;
    bool v;
    ~Restore() { c->profiling = v; }
  } restore{c, saved_profiling};

  NW_CK(cudaMemsetAsync(sb, 0, off_thr, s));
  NW_CK(cudaMemsetAsync(d_thr, 0, sizeof(uint32_t) * (size_t)n, s));
  NW_CK(cudaMemsetAsync(d_slots, 0, sizeof(uint32_t) * (size_t)n * k, s));
  if (hist) NW_CK(cudaMemsetAsync(d_hist, 0, sizeof(unsigned long long) * need_bins, s));

  DpParams P{};
  P.TA = kDefaultTA;
  P.C1 = d->ss.C1;
  P.C2 = d->ss.C2;
  P.match = d->sc.match;
  P.mismatch = d->sc.mismatch;
  P.gap = d->sc.gap;
  P.mode = kModeLists;
  P.k = k;
  P.ib = ib;
  P.imask = (uint32_t)(((uint64_t)1 << ib) - 1);
  P.key_lo = key_lo;
  P.hist_mode = !hist ? kHistNone : hist_mode_for(need_bins);
  P.hist = d_hist;
  P.hist_lo = d->score_lo;
  P.nbins = hist ? need_bins : 0;
  P.stats = d_stats;
  P.err = d_err;
  SideView side{d->ws.perm.as<uint32_t>(), d_slots, d_thr};
  const uint32_t* a_enc[3] = {d->ws.a_enc.as<uint32_t>(), nullptr, nullptr};
  const uint4* b_rec[3] = {d->ws.b_rec.as<uint4>(), nullptr, nullptr};
  const SideView* views[3] = {&side, nullptr, nullptr};
  Timer tm{c};
  RunOut ro;
  NW_TRY(run_plan(c, d->plan, d->d_segs.as<Seg>(), P, &d->ws, &d->ws, d_counters, 0, 1, tm, ro, a_enc, views, b_rec,
                  views));
  NW_CK(launch_finalize(d_slots, n, k, d->ws.perm.as<uint32_t>(), ib, P.imask, key_lo, nbr_idx, nbr_score, s));
  if (hist) {
    NW_CK(cudaMemcpyAsync(hist, d_hist, sizeof(int64_t) * need_bins, cudaMemcpyDeviceToDevice, s));
    if (nbins > need_bins) NW_CK(cudaMemsetAsync(hist + need_bins, 0, sizeof(int64_t) * (nbins - need_bins), s));
    if (hist_lo) *hist_lo = d->score_lo;
  }
  if (flags & NW_ASYNC) return NW_OK;
  return check_device_flags(c, d_err);
}

}  // namespace nw
