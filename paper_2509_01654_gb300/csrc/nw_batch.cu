// nw_batch.cu -- nw_batch_*: many independent dictionaries, each with an
// optional query set, reduced to top-k lists in one CUDA-graph launch.
//
// Every dictionary is loaded as usual (its own word set, scoring and score
// bounds), and its query set is ingested with the dictionary's alphabet and
// code shift.  The pair plans of all dictionaries and query sets are merged
// by longer length: the launch for length LB walks the LB segments of every
// dictionary and query set, each segment tagged with its terms (3d for
// dictionary d's own pairs, 3d + 1 for its queries as A words, 3d + 2 for its
// queries as B words), and the kernel (epilogue kEpiBatchLists) reads those
// terms' word sets, lists and scoring per task.  The A-chunk size of each
// launch is a tile-shape parameter that the autotuner picks by timing
// candidates on the batch.  The whole reduction is captured once into a CUDA
// graph and replayed by nw_batch_run / nw_batch_run_queries.
#include <chrono>
#include <map>
#include <mutex>

#include "nw_host.h"

struct nw_batch {
  nw_ctx* ctx = nullptr;
  cudaStream_t stream = nullptr;  // the batch's own stream (capture needs a non-legacy stream)
  std::vector<nw_dict*> dicts;
  std::vector<WordSet> qsets;     // each dictionary's query set (n = 0: none)
  std::vector<uint8_t> self;      // 1: the dictionary's own lists are computed
  uint32_t k = 0;
  uint32_t ta_by_lb[kBuckets] = {0};
  uint32_t bps_by_lb[kBuckets] = {0};  // resident blocks per SM at most (0: as many as fit)
  bool tune_cached = false;
  Plan plan;
  std::vector<size_t> list_off;   // first list of each dictionary's own lists in the combined arrays
  std::vector<size_t> qlist_off;  // first list of each query set in the combined arrays
  std::vector<int32_t> q_key_lo;  // list-key offset of each query set (its lowest score - 1)
  size_t nlists = 0;
  uint32_t query_words = 0;
  uint64_t query_pairs = 0, query_cells = 0;
  DevBuf d_segs, d_terms, d_slots, d_thr, d_small, d_out_idx, d_out_score;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double tune_ms = 0;
};

namespace {

constexpr uint32_t kTaCandidates[] = {64, 128, 256};

// Terms of dictionary d's own pairs (role 0) and of its query set as A words
// (role 1) or B words (role 2).
uint32_t term_index(size_t d, int role) { return (uint32_t)(3 * d + role); }

// Every dictionary's own plan and every query set's plan (launches of roles 1
// and 2), made with A chunks of `ta` words.
struct DictPlans {
  std::vector<Plan> self, query;
};

DictPlans dict_plans(const nw_batch* B, uint32_t ta) {
  DictPlans p;
  p.self.resize(B->dicts.size());
  p.query.resize(B->dicts.size());
  for (size_t d = 0; d < B->dicts.size(); ++d) {
    if (B->self[d]) plan_all_pairs(B->dicts[d]->ws.bk, ta, p.self[d]);
    if (B->qsets[d].n) plan_query(B->qsets[d].bk, B->dicts[d]->ws.bk, ta, p.query[d]);
  }
  return p;
}

// The segments of every dictionary and query set whose longer length is LB,
// taken from plans made with A chunks of `ta` words, appended as one launch
// (task0 rebased, terms tagged).
void append_launch(const nw_batch* B, const DictPlans& plans, int LB, uint32_t ta, Plan& out, uint32_t bps = 0) {
  LaunchPlan lp;
  lp.LB = LB;
  lp.role = 0;
  lp.ta = ta;
  lp.bps = bps;
  lp.seg_first = (uint32_t)out.segs.size();
  uint64_t task = 0;
  for (size_t d = 0; d < B->dicts.size(); ++d) {
    for (const Plan* p : {&plans.self[d], &plans.query[d]}) {
      for (const LaunchPlan& q : p->launches) {
        if (q.LB != LB) continue;
        for (uint32_t s = 0; s < q.nsegs; ++s) {
          Seg g = p->segs[q.seg_first + s];
          g.task0 += task;
          g.dict = term_index(d, q.role);
          out.segs.push_back(g);
        }
        task += q.ntasks;
        lp.pairs += q.pairs;
        lp.cells += q.cells;
      }
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

DpParams batch_params(nw_batch* B) {
  DpParams P{};
  P.TA = kDefaultTA;
  P.mode = kModeLists;
  P.k = B->k;
  P.hist_mode = kHistNone;
  P.stats = reinterpret_cast<unsigned long long*>(B->d_small.as<char>() + 8);
  P.err = B->d_small.as<uint32_t>();
  P.terms = B->d_terms.as<DictTerms>();
  return P;
}

nw_status upload_plan(nw_batch* B, const Plan& plan) {
  nw_ctx* c = B->ctx;
  NW_TRY(ctx_ensure(c, B->d_segs, sizeof(Seg) * std::max<size_t>(1, plan.segs.size()), "batch segments"));
  if (!plan.segs.empty())
    NW_CK(cudaMemcpyAsync(B->d_segs.p, plan.segs.data(), sizeof(Seg) * plan.segs.size(), cudaMemcpyHostToDevice,
                          B->stream));
  return NW_OK;
}

// List resets and the alignment launches of `plan` (shard `shard` of
// `nshards` of each launch's tasks) on the batch's stream.
nw_status issue_lists(nw_batch* B, const Plan& plan, uint32_t shard = 0, uint32_t nshards = 1) {
  nw_ctx* c = B->ctx;
  cudaStream_t s = B->stream;
  NW_CK(cudaMemsetAsync(B->d_small.p, 0, B->d_small.bytes, s));
  NW_CK(cudaMemsetAsync(B->d_slots.p, 0, sizeof(uint32_t) * B->nlists * B->k, s));
  NW_CK(cudaMemsetAsync(B->d_thr.p, 0, sizeof(uint32_t) * B->nlists, s));
  const DpParams P = batch_params(B);
  SideView none{nullptr, nullptr, nullptr};
  const uint32_t* a_enc[3] = {nullptr, nullptr, nullptr};
  const uint4* b_rec[3] = {nullptr, nullptr, nullptr};
  const SideView* views[3] = {&none, &none, &none};
  const bool saved = c->profiling;
  c->profiling = false;
  Timer tm{c};
  RunOut ro;
  const nw_status st = run_plan(c, s, plan, B->d_segs.as<Seg>(), P,
                                reinterpret_cast<unsigned long long*>(B->d_small.as<char>() + 64), shard, nshards,
                                tm, ro,
                                a_enc, views, b_rec, views);
  c->profiling = saved;
  return st;
}

nw_status issue_finalize(nw_batch* B) {
  nw_ctx* c = B->ctx;
  for (size_t d = 0; d < B->dicts.size(); ++d) {
    const nw_dict* D = B->dicts[d];
    const uint32_t n = D->ws.n;
    const uint32_t ib = index_bits(std::max<uint32_t>(n, 2));
    const uint32_t imask = (uint32_t)(((uint64_t)1 << ib) - 1);
    if (B->self[d] && n) {
      NW_CK(launch_finalize(B->d_slots.as<uint32_t>() + B->list_off[d] * B->k, n, B->k, D->ws.perm.as<uint32_t>(),
                            ib, imask, D->score_lo - 1, B->d_out_idx.as<uint32_t>() + B->list_off[d] * B->k,
                            B->d_out_score.as<int16_t>() + B->list_off[d] * B->k, B->stream));
    }
    const WordSet& Q = B->qsets[d];
    if (Q.n) {  // query lists name dictionary words, as nw_query's do
      NW_CK(launch_finalize(B->d_slots.as<uint32_t>() + B->qlist_off[d] * B->k, Q.n, B->k, Q.perm.as<uint32_t>(),
                            ib, imask, B->q_key_lo[d], B->d_out_idx.as<uint32_t>() + B->qlist_off[d] * B->k,
                            B->d_out_score.as<int16_t>() + B->qlist_off[d] * B->k, B->stream));
    }
  }
  return NW_OK;
}

// The autotuner's choices, kept for the life of the process and keyed by the
// batch's shape (tune_key): a batch of the same shape is not timed again.
struct TunedShape {
  uint32_t ta[kBuckets];
  uint32_t bps[kBuckets];
};
std::mutex& tune_mutex() {
  static std::mutex m;
  return m;
}
std::map<uint64_t, TunedShape>& tune_cache() {
  static std::map<uint64_t, TunedShape> m;
  return m;
}

// FNV-1a over the device's SM count, k, and every dictionary's and query
// set's length histogram, scoring and flags: what the launches' work and
// their timing follow.
uint64_t tune_key(const nw_batch* B) {
  uint64_t h = 1469598103934665603ull;
  auto mix = [&h](uint64_t v) {
    for (int i = 0; i < 8; ++i) {
      h ^= (v >> (8 * i)) & 0xffu;
      h *= 1099511628211ull;
    }
  };
  mix((uint64_t)B->ctx->sm_count);
  mix(B->k);
  mix(B->dicts.size());
  for (size_t d = 0; d < B->dicts.size(); ++d) {
    const nw_dict* D = B->dicts[d];
    mix(B->self[d]);
    mix(D->alphabet);
    mix((uint32_t)D->sc.match);
    mix((uint32_t)D->sc.mismatch);
    mix((uint32_t)D->sc.gap);
    mix(D->subst ? 1u : 0u);
    for (int L = 0; L < kBuckets; ++L) mix(D->ws.bk.count[L]);
    for (int L = 0; L < kBuckets; ++L) mix(B->qsets[d].bk.count[L]);
  }
  return h;
}

constexpr uint32_t kBpsCandidates[] = {3, 2};

// Per launch length: the fastest A-chunk candidate, then the fastest cap on
// resident blocks per SM at that chunk (whole launches timed on the batch).
nw_status autotune(nw_batch* B) {
  nw_ctx* c = B->ctx;
  const uint64_t key = tune_key(B);
  {
    std::lock_guard<std::mutex> lk(tune_mutex());
    auto it = tune_cache().find(key);
    if (it != tune_cache().end()) {
      std::copy(it->second.ta, it->second.ta + kBuckets, B->ta_by_lb);
      std::copy(it->second.bps, it->second.bps + kBuckets, B->bps_by_lb);
      B->tune_cached = true;
      B->tune_ms = 0;
      return NW_OK;
    }
  }
  const auto t0 = std::chrono::steady_clock::now();
  cudaEvent_t e0, e1;
  NW_CK(cudaEventCreate(&e0));
  NW_CK(cudaEventCreate(&e1));
  struct EvFree {
    cudaEvent_t a, b;
    ~EvFree() { cudaEventDestroy(a); cudaEventDestroy(b); }
  } evfree{e0, e1};
  constexpr size_t kNta = sizeof(kTaCandidates) / sizeof(kTaCandidates[0]);
  std::vector<DictPlans> plans;
  for (uint32_t ta : kTaCandidates) plans.push_back(dict_plans(B, ta));
  // one timed launch of length LB with chunk candidate ci and cap bps; false if the length has no pairs
  auto time_launch = [&](int LB, size_t ci, uint32_t bps, bool& warm, float& ms) -> nw_status {
    Plan p;
    append_launch(B, plans[ci], LB, kTaCandidates[ci], p, bps);
    ms = -1.f;
    if (p.launches.empty()) return NW_OK;
    NW_TRY(upload_plan(B, p));
    if (!warm) {  // the kernel's first launch pays its set-up; keep it out of the timings
      NW_TRY(issue_lists(B, p));
      warm = true;
    }
    NW_CK(cudaEventRecord(e0, B->stream));
    NW_TRY(issue_lists(B, p));
    NW_CK(cudaEventRecord(e1, B->stream));
    NW_CK(cudaEventSynchronize(e1));
    NW_CK(cudaEventElapsedTime(&ms, e0, e1));
    return NW_OK;
  };
  for (int LB = 0; LB < kBuckets; ++LB) {
    float best = 0;
    size_t best_ci = kNta;
    bool warm = false;
    for (size_t ci = 0; ci < kNta; ++ci) {
      float ms;
      NW_TRY(time_launch(LB, ci, 0, warm, ms));
      if (ms < 0) break;
      if (best_ci == kNta || ms < best) {
        best = ms;
        best_ci = ci;
      }
    }
    if (best_ci == kNta) continue;  // lengths without pairs keep the defaults
    B->ta_by_lb[LB] = kTaCandidates[best_ci];
    for (uint32_t bps : kBpsCandidates) {
      float ms;
      NW_TRY(time_launch(LB, best_ci, bps, warm, ms));
      if (ms >= 0 && ms < best) {
        best = ms;
        B->bps_by_lb[LB] = bps;
      }
    }
  }
  B->tune_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  TunedShape t;
  std::copy(B->ta_by_lb, B->ta_by_lb + kBuckets, t.ta);
  std::copy(B->bps_by_lb, B->bps_by_lb + kBuckets, t.bps);
  std::lock_guard<std::mutex> lk(tune_mutex());
  tune_cache()[key] = t;
  return NW_OK;
}

nw_status check_flags(nw_ctx* c, cudaStream_t stream, const uint32_t* d_err) {
  uint32_t err = 0;
  NW_CK(cudaMemcpyAsync(&err, d_err, sizeof err, cudaMemcpyDeviceToHost, stream));
  NW_CK(cudaStreamSynchronize(stream));
  if (err & kErrRetry) return set_err(c, NW_ETIMEOUT, "a neighbour-list update exceeded its retry bound");
  if (err) return set_err(c, NW_EINVAL, "device-side error flag %u", err);
  return NW_OK;
}

nw_status create_impl(nw_batch* B, const nw_batch_dict* dicts, uint32_t ndicts, uint32_t flags) {
  nw_ctx* c = B->ctx;
  for (uint32_t d = 0; d < ndicts; ++d) {
    nw_dict* D = nullptr;
    const nw_status st = nw_load_dictionary(c, dicts[d].codes, dicts[d].offsets, dicts[d].n, dicts[d].alphabet,
                                            &dicts[d].scoring, flags & NW_DEVICE_PTRS, &D);
    if (st != NW_OK) return st;
    B->dicts.push_back(D);
    B->qsets.emplace_back();
    B->self.push_back(dicts[d].queries_only ? 0 : 1);
    const uint32_t ib = index_bits(std::max<uint32_t>(D->ws.n, 2));
    if (B->self[d] && (D->score_lo < INT16_MIN + 1 || D->score_hi > INT16_MAX ||
                       (uint64_t)(D->score_hi - (D->score_lo - 1)) >= (1ull << (32 - ib))))
      return set_err(c, NW_ERANGE, "dictionary %u: scores [%d, %d] do not fit the list keys", d, D->score_lo,
                     D->score_hi);
    B->list_off.push_back(B->nlists);
    if (B->self[d]) B->nlists += D->ws.n;
    // the query set: ingested with the dictionary's alphabet and code shift;
    // its list keys span the scores of the (query length, dictionary length)
    // pairs present, as in nw_query
    int32_t key_lo = 0;
    if (dicts[d].nq) {
      if (!dicts[d].qoffsets) return set_err(c, NW_EINVAL, "dictionary %u: null query offsets", d);
      NW_TRY(ingest(c, dicts[d].qcodes, dicts[d].qoffsets, dicts[d].nq, D->alphabet, D->ss.shift,
                    flags & NW_DEVICE_PTRS, B->qsets[d]));
      const WordSet& Q = B->qsets[d];
      int lo = INT32_MAX, hi = INT32_MIN;
      for (int La = 0; La < kBuckets; ++La)
        for (int Lb = 0; Lb < kBuckets; ++Lb) {
          if (!Q.bk.count[La] || !D->ws.bk.count[Lb]) continue;
          int l, h;
          pair_bounds(D->sc, La, Lb, l, h);
          lo = std::min(lo, l);
          hi = std::max(hi, h);
        }
      if (D->ws.n == 0) lo = hi = 0;
      if (lo < INT16_MIN + 1 || hi > INT16_MAX || (uint64_t)(hi - (lo - 1)) >= (1ull << (32 - ib)))
        return set_err(c, NW_ERANGE, "query set %u: scores [%d, %d] do not fit the list keys", d, lo, hi);
      key_lo = lo - 1;
      B->query_words += Q.n;
    }
    B->q_key_lo.push_back(key_lo);
    B->qlist_off.push_back(B->nlists);
    B->nlists += B->qsets[d].n;
  }
  const size_t L = std::max<size_t>(1, B->nlists);
  NW_TRY(ctx_alloc(c, B->d_slots, sizeof(uint32_t) * L * B->k, "batch list slots"));
  NW_TRY(ctx_alloc(c, B->d_thr, sizeof(uint32_t) * L, "batch list bounds"));
  NW_TRY(ctx_alloc(c, B->d_out_idx, sizeof(uint32_t) * L * B->k, "batch output indices"));
  NW_TRY(ctx_alloc(c, B->d_out_score, sizeof(int16_t) * L * B->k, "batch output scores"));
  NW_TRY(ctx_alloc(c, B->d_small, 64 + sizeof(unsigned long long) * (kBuckets + 2), "batch counters"));
  std::vector<DictTerms> terms(std::max<size_t>(1, 3 * B->dicts.size()));
  for (size_t d = 0; d < B->dicts.size(); ++d) {
    const nw_dict* D = B->dicts[d];
    const WordSet& Q = B->qsets[d];
    const uint32_t ib = index_bits(std::max<uint32_t>(D->ws.n, 2));
    const SideView dict_side{D->ws.perm.as<uint32_t>(), B->d_slots.as<uint32_t>() + B->list_off[d] * B->k,
                             B->d_thr.as<uint32_t>() + B->list_off[d]};
    const SideView dict_nolists{D->ws.perm.as<uint32_t>(), nullptr, nullptr};
    const SideView query_side{Q.perm.as<uint32_t>(), B->d_slots.as<uint32_t>() + B->qlist_off[d] * B->k,
                              B->d_thr.as<uint32_t>() + B->qlist_off[d]};
    for (int role = 0; role < 3; ++role) {
      DictTerms& T = terms[term_index(d, role)];
      T.a_enc = role == 1 ? Q.a_enc.as<uint32_t>() : D->ws.a_enc.as<uint32_t>();
      T.b_rec = role == 2 ? Q.b_rec.as<uint4>() : D->ws.b_rec.as<uint4>();
      T.A = role == 0 ? dict_side : (role == 1 ? query_side : dict_nolists);
      T.B = role == 0 ? dict_side : (role == 1 ? dict_nolists : query_side);
      T.C1 = D->ss.C1;
      T.C2 = D->ss.C2;
      T.match = D->sc.match;
      T.mismatch = D->sc.mismatch;
      T.gap = D->sc.gap;
      T.key_lo = role == 0 ? D->score_lo - 1 : B->q_key_lo[d];
      T.ib = ib;
      T.imask = (uint32_t)(((uint64_t)1 << ib) - 1);
    }
    if (Q.n) {
      Plan qp;
      plan_query(Q.bk, D->ws.bk, kDefaultTA, qp);
      B->query_pairs += qp.pairs;
      B->query_cells += qp.cells;
    }
  }
  NW_TRY(ctx_alloc(c, B->d_terms, sizeof(DictTerms) * terms.size(), "batch terms"));
  NW_CK(cudaMemcpyAsync(B->d_terms.p, terms.data(), sizeof(DictTerms) * terms.size(), cudaMemcpyHostToDevice,
                        B->stream));

  for (int LB = 0; LB < kBuckets; ++LB) B->ta_by_lb[LB] = kDefaultTA;
  if (flags & NW_BATCH_AUTOTUNE) NW_TRY(autotune(B));
  B->plan = Plan{};
  {
    std::vector<uint32_t> tas;  // the distinct chunk sizes chosen, each planned once
    for (int LB = 0; LB < kBuckets; ++LB)
      if (std::find(tas.begin(), tas.end(), B->ta_by_lb[LB]) == tas.end()) tas.push_back(B->ta_by_lb[LB]);
    std::vector<DictPlans> plans;
    for (uint32_t ta : tas) plans.push_back(dict_plans(B, ta));
    for (int LB = 0; LB < kBuckets; ++LB) {
      const size_t ci = std::find(tas.begin(), tas.end(), B->ta_by_lb[LB]) - tas.begin();
      append_launch(B, plans[ci], LB, B->ta_by_lb[LB], B->plan, B->bps_by_lb[LB]);
    }
  }
  for (int LB = 0; LB < kBuckets; ++LB) {
    bool present = false;
    for (const LaunchPlan& lp : B->plan.launches) present |= lp.LB == LB;
    if (!present) B->ta_by_lb[LB] = B->bps_by_lb[LB] = 0;
  }
  NW_TRY(upload_plan(B, B->plan));
  // one uncaptured run sets the kernels' shared-memory attributes
  NW_TRY(issue_lists(B, B->plan));
  NW_TRY(issue_finalize(B));
  NW_TRY(check_flags(c, B->stream, B->d_small.as<uint32_t>()));

  NW_CK(cudaStreamBeginCapture(B->stream, cudaStreamCaptureModeThreadLocal));
  nw_status st = issue_lists(B, B->plan);
  if (st == NW_OK) st = issue_finalize(B);
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(B->stream, &g);
  if (st != NW_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaStreamEndCapture");
  B->graph = g;
  NW_CK(cudaGraphInstantiate(&B->exec, B->graph, 0));
  return NW_OK;
}

void destroy_impl(nw_batch* B) {
  nw_ctx* c = B->ctx;
  if (B->stream) cudaStreamSynchronize(B->stream);
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  for (DevBuf* b : {&B->d_segs, &B->d_terms, &B->d_slots, &B->d_thr, &B->d_small, &B->d_out_idx, &B->d_out_score})
    ctx_free(c, *b);
  for (WordSet& Q : B->qsets) free_wordset(c, Q);
  for (nw_dict* D : B->dicts) nw_dict_free(D);
  if (B->stream) cudaStreamDestroy(B->stream);
  delete B;
}

}  // namespace

extern "C" {

nw_status nw_batch_create(nw_ctx* ctx, const nw_batch_dict* dicts, uint32_t ndicts, uint32_t k, uint32_t flags,
                          nw_batch** out) {
  if (!ctx || !out) return NW_EINVAL;
  *out = nullptr;
  if (!dicts && ndicts) return set_err(ctx, NW_EINVAL, "null dictionary array");
  if (k == 0 || k > NW_MAX_K) return set_err(ctx, NW_EINVAL, "k must be in [1, %d]", NW_MAX_K);
  if (flags & NW_RANK_NORMALISED) return set_err(ctx, NW_EINVAL, "batches rank by raw score only");
  if (cudaSetDevice(ctx->device) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "cudaSetDevice");
  nw_batch* B = new nw_batch();
  B->ctx = ctx;
  B->k = k;
  nw_status st = NW_OK;
  if (cudaStreamCreateWithFlags(&B->stream, cudaStreamNonBlocking) != cudaSuccess)
    st = cuda_fail(ctx, cudaGetLastError(), "cudaStreamCreateWithFlags");
  if (st == NW_OK) st = create_impl(B, dicts, ndicts, flags);
  if (st != NW_OK) {
    const std::string msg = ctx->err;
    destroy_impl(B);
    ctx->err = msg;
    return st;
  }
  *out = B;
  return NW_OK;
}

nw_status nw_batch_run_queries(nw_batch* B, uint32_t* const* nbr_idx, int16_t* const* nbr_score,
                               uint32_t* const* qnbr_idx, int16_t* const* qnbr_score, uint32_t flags) {
  if (!B) return NW_EINVAL;
  nw_ctx* c = B->ctx;
  NW_ENTER(c);
  if (flags & NW_RANK_NORMALISED) return set_err(c, NW_EINVAL, "batches rank by raw score only");
  const bool want_q = qnbr_idx || qnbr_score;
  if (want_q && (!qnbr_idx || !qnbr_score)) return set_err(c, NW_EINVAL, "null query output arrays");
  // every buffer the copies need, checked before the graph runs
  for (size_t d = 0; d < B->dicts.size(); ++d) {
    if (B->self[d] && B->dicts[d]->ws.n &&
        (!nbr_idx || !nbr_score || !nbr_idx[d] || !nbr_score[d]))
      return set_err(c, NW_EINVAL, "null output for dictionary %zu", d);
    if (want_q && B->qsets[d].n && (!qnbr_idx[d] || !qnbr_score[d]))
      return set_err(c, NW_EINVAL, "null query output for dictionary %zu", d);
  }
  const bool dev = flags & NW_DEVICE_PTRS;
  const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  NW_CK(cudaGraphLaunch(B->exec, B->stream));
  auto copy_out = [&](uint32_t* idx, int16_t* score, size_t first, size_t lists) -> nw_status {
    const size_t cnt = lists * B->k;
    NW_CK(cudaMemcpyAsync(idx, B->d_out_idx.as<uint32_t>() + first * B->k, sizeof(uint32_t) * cnt, kind, B->stream));
    NW_CK(cudaMemcpyAsync(score, B->d_out_score.as<int16_t>() + first * B->k, sizeof(int16_t) * cnt, kind,
                          B->stream));
    return NW_OK;
  };
  for (size_t d = 0; d < B->dicts.size(); ++d) {
    if (B->self[d] && B->dicts[d]->ws.n) NW_TRY(copy_out(nbr_idx[d], nbr_score[d], B->list_off[d], B->dicts[d]->ws.n));
    if (want_q && B->qsets[d].n) NW_TRY(copy_out(qnbr_idx[d], qnbr_score[d], B->qlist_off[d], B->qsets[d].n));
  }
  if ((flags & NW_ASYNC) && dev) return NW_OK;
  return check_flags(c, B->stream, B->d_small.as<uint32_t>());
}

nw_status nw_batch_run(nw_batch* B, uint32_t* const* nbr_idx, int16_t* const* nbr_score, uint32_t flags) {
  return nw_batch_run_queries(B, nbr_idx, nbr_score, nullptr, nullptr, flags);
}

nw_status nw_batch_info_get(const nw_batch* B, nw_batch_info* out) {
  if (!B || !out) return NW_EINVAL;
  nw_batch_info i{};
  i.ndicts = (uint32_t)B->dicts.size();
  i.launches = (uint32_t)B->plan.launches.size();
  i.pairs = B->plan.pairs;
  i.cells = B->plan.cells;
  i.tune_ms = B->tune_ms;
  for (int L = 0; L < kBuckets; ++L) i.words_per_task[L] = B->ta_by_lb[L];
  for (int L = 0; L < kBuckets; ++L) i.blocks_per_sm[L] = B->bps_by_lb[L];
  i.tune_cached = B->tune_cached ? 1u : 0u;
  i.query_words = B->query_words;
  i.query_pairs = B->query_pairs;
  i.query_cells = B->query_cells;
  *out = i;
  return NW_OK;
}

void nw_batch_free(nw_batch* B) {
  if (!B) return;
  cudaSetDevice(B->ctx->device);
  destroy_impl(B);
}

}  // extern "C"
