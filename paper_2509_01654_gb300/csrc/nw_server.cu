// nw_server.cu -- nw_server_*: a continuous-batching query service over one
// device-resident dictionary.
//
// Requests queue on the host.  A worker thread packs queued requests (in
// arrival order) into batches of at most max_batch_queries words, prepares
// each batch on the host (length bucketing of the batch's words, the pair
// plan against the dictionary) and issues it on a free slot: H2D copies, the
// encode kernel, the alignment launches, list finalisation and the D2H copy of
// results, all on the slot's own stream, followed by a host callback that
// wakes the worker.  Slots are allocated once; their number is capped by the
// memory budget.  While batches run, new requests keep queueing and are
// admitted the moment a slot frees, so their GPU work overlaps the running
// batches'.
//
// A proposal server (nw_server_create_proposal) answers through the learned
// proposal instead.  Each of its slots owns a context (stream, workspace), a
// copy of the model's parameters and a view of the dictionary's device data,
// and a thread that runs nw_proposal_query for the batch it is given; a
// dispatcher packs queued requests into batches and hands each to a free
// slot, so batches run on the device side by side while new requests queue.
#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>

#include "nw_host.h"
#include "nw_proposal.h"
#include "nw_proposal_internal.h"

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t id = 0;
  uint32_t nq = 0;
  std::vector<uint8_t> codes;
  std::vector<uint32_t> offsets;
  std::vector<uint32_t> idx;
  std::vector<int16_t> score;
  nw_request_info info{};
  int state = 0;  // 0 queued, 1 on the GPU, 2 finished
  nw_status status = NW_OK;
};

struct Slot;

struct CallbackArg {
  nw_server* srv;
  Slot* slot;
};

// One batch in flight: its stream, pinned staging and device buffers.
struct Slot {
  cudaStream_t stream = nullptr;
  bool busy = false;
  std::atomic<int> gpu_done{0};
  CallbackArg cb{};
  uint8_t* h_codes = nullptr;
  uint32_t* h_offsets = nullptr;
  uint32_t* h_perm = nullptr;
  uint8_t* h_slen = nullptr;
  Seg* h_segs = nullptr;
  uint32_t* h_idx = nullptr;
  int16_t* h_score = nullptr;
  uint32_t* h_err = nullptr;
  DevBuf d_codes, d_offsets, d_perm, d_slen, d_aoff, d_brec_w, d_a_enc, d_b_rec, d_slots, d_thr, d_small, d_segs,
      d_idx, d_score;
  std::vector<Request*> reqs;
  std::vector<uint32_t> first;
  uint32_t nq = 0;
  Plan plan;
};

constexpr size_t kMaxSegs = 2u * kBuckets * kBuckets;  // plan_query makes at most one rectangle per (role, La, LB)

// One batch in flight through the proposal: a private context, the model's
// parameters copied into it, a non-owning view of the dictionary, and the
// thread that runs the slot's batches.
struct PropSlot {
  nw_ctx* ctx = nullptr;
  nw_model* model = nullptr;
  nw_dict* view = nullptr;
  std::thread th;
  std::vector<Request*> reqs;  // the batch handed to the slot
  bool busy = false;           // a batch is assigned and not yet finished
  bool taken = false;          // the slot's thread has taken the assigned batch
};

}  // namespace

struct nw_server {
  nw_dict* dict = nullptr;
  nw_model* model = nullptr;  // proposal mode: batches go through nw_proposal_query
  uint32_t C = 0;
  nw_ctx ictx;  // the server's own context: device, SM count, budget accounting, error text
  nw_server_config cfg{};
  std::vector<std::unique_ptr<Slot>> slots;
  std::mutex mu;
  std::condition_variable cv;       // wakes the worker: submissions and GPU completions
  std::condition_variable cv_done;  // wakes waiters: finished requests
  std::deque<Request*> queue;
  std::unordered_map<uint64_t, Request*> reqs;
  uint64_t next_id = 1;
  bool stop = false;
  std::thread worker;
  std::string err;  // guarded by mu
  std::vector<std::unique_ptr<PropSlot>> pslots;  // proposal mode
  std::condition_variable cv_slots;               // wakes proposal slot threads
};

namespace {

void CUDART_CB on_batch_done(void* p) {
  CallbackArg* a = static_cast<CallbackArg*>(p);
  a->slot->gpu_done.store(1);
  {
    std::lock_guard<std::mutex> lock(a->srv->mu);  // pairs with the worker's wait
  }
  a->srv->cv.notify_all();
}

size_t brec_capacity_words(uint32_t Q) { return ((size_t)Q / 2 + kBuckets) * (size_t)ceil4(kMaxLen) + 4; }

nw_status alloc_slot(nw_server* S, Slot& s) {
  nw_ctx* c = &S->ictx;
  const uint32_t Q = S->cfg.max_batch_queries, k = S->cfg.k;
  NW_CK(cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking));
  NW_CK(cudaMallocHost(&s.h_codes, (size_t)Q * kMaxLen + 16));
  NW_CK(cudaMallocHost(&s.h_offsets, sizeof(uint32_t) * ((size_t)Q + 1)));
  NW_CK(cudaMallocHost(&s.h_perm, sizeof(uint32_t) * Q));
  NW_CK(cudaMallocHost(&s.h_slen, (size_t)Q + 16));
  NW_CK(cudaMallocHost(&s.h_segs, sizeof(Seg) * kMaxSegs));
  NW_CK(cudaMallocHost(&s.h_idx, sizeof(uint32_t) * (size_t)Q * k));
  NW_CK(cudaMallocHost(&s.h_score, sizeof(int16_t) * (size_t)Q * k));
  NW_CK(cudaMallocHost(&s.h_err, 64));
  NW_TRY(ctx_alloc(c, s.d_codes, (size_t)Q * kMaxLen + 16, "batch codes"));
  NW_TRY(ctx_alloc(c, s.d_offsets, sizeof(uint32_t) * ((size_t)Q + 1), "batch offsets"));
  NW_TRY(ctx_alloc(c, s.d_perm, sizeof(uint32_t) * Q, "batch permutation"));
  NW_TRY(ctx_alloc(c, s.d_slen, (size_t)Q + 16, "batch lengths"));
  NW_TRY(ctx_alloc(c, s.d_aoff, sizeof(uint32_t) * Q, "batch A offsets"));
  NW_TRY(ctx_alloc(c, s.d_brec_w, sizeof(uint32_t) * Q, "batch B offsets"));
  NW_TRY(ctx_alloc(c, s.d_a_enc, sizeof(uint32_t) * ((size_t)Q * kMaxLen + 4), "batch A symbols"));
  NW_TRY(ctx_alloc(c, s.d_b_rec, sizeof(uint32_t) * brec_capacity_words(Q), "batch B records"));
  NW_TRY(ctx_alloc(c, s.d_slots, sizeof(uint32_t) * (size_t)Q * k, "batch list slots"));
  NW_TRY(ctx_alloc(c, s.d_thr, sizeof(uint32_t) * Q, "batch list bounds"));
  NW_TRY(ctx_alloc(c, s.d_small, 64 + sizeof(unsigned long long) * (2 * kBuckets + 2), "batch counters"));
  NW_TRY(ctx_alloc(c, s.d_segs, sizeof(Seg) * kMaxSegs, "batch segments"));
  NW_TRY(ctx_alloc(c, s.d_idx, sizeof(uint32_t) * (size_t)Q * k, "batch result indices"));
  NW_TRY(ctx_alloc(c, s.d_score, sizeof(int16_t) * (size_t)Q * k, "batch result scores"));
  return NW_OK;
}

void free_slot(nw_server* S, Slot& s) {
  nw_ctx* c = &S->ictx;
  if (s.stream) cudaStreamSynchronize(s.stream);
  for (DevBuf* b : {&s.d_codes, &s.d_offsets, &s.d_perm, &s.d_slen, &s.d_aoff, &s.d_brec_w, &s.d_a_enc, &s.d_b_rec,
                    &s.d_slots, &s.d_thr, &s.d_small, &s.d_segs, &s.d_idx, &s.d_score})
    ctx_free(c, *b);
  for (void* p : {(void*)s.h_codes, (void*)s.h_offsets, (void*)s.h_perm, (void*)s.h_slen, (void*)s.h_segs,
                  (void*)s.h_idx, (void*)s.h_score, (void*)s.h_err})
    if (p) cudaFreeHost(p);
  if (s.stream) cudaStreamDestroy(s.stream);
}

// A proposal slot's model, dictionary view (its device data stays with the
// caller's dictionary) and context.
void free_pslot(PropSlot& s) {
  if (s.model) nw_model_free(s.model);
  s.model = nullptr;
  delete s.view;
  s.view = nullptr;
  if (s.ctx) nw_destroy(s.ctx);
  s.ctx = nullptr;
}

// Prepares the slot's batch on the host and issues it on the slot's stream.
nw_status launch_batch(nw_server* S, Slot& s) {
  nw_ctx* c = &S->ictx;
  const nw_dict* d = S->dict;
  const uint32_t k = S->cfg.k;
  cudaStream_t st = s.stream;

  // concatenate the requests' words
  uint32_t nq = 0, ncodes = 0;
  s.first.clear();
  s.h_offsets[0] = 0;
  for (Request* r : s.reqs) {
    s.first.push_back(nq);
    std::memcpy(s.h_codes + ncodes, r->codes.data(), r->codes.size());
    for (uint32_t q = 0; q < r->nq; ++q) s.h_offsets[nq + q + 1] = ncodes + r->offsets[q + 1];
    nq += r->nq;
    ncodes += (uint32_t)r->codes.size();
  }
  s.nq = nq;
  // stable bucketing of the batch's words by length (host: the batch is small)
  Buckets bk{};
  for (uint32_t q = 0; q < nq; ++q) ++bk.count[s.h_offsets[q + 1] - s.h_offsets[q]];
  fill_buckets(bk);
  uint32_t fillc[kBuckets] = {0};
  for (uint32_t q = 0; q < nq; ++q) {
    const uint32_t L = s.h_offsets[q + 1] - s.h_offsets[q];
    const uint32_t pos = bk.start[L] + fillc[L]++;
    s.h_perm[pos] = q;
    s.h_slen[pos] = (uint8_t)L;
  }
  // score bounds of the (query, dictionary) length pairs present -> list keys
  int lo = INT32_MAX, hi = INT32_MIN;
  for (int La = 0; La < kBuckets; ++La)
    for (int Lb = 0; Lb < kBuckets; ++Lb) {
      if (!bk.count[La] || !d->ws.bk.count[Lb]) continue;
      int l, h;
      pair_bounds(d->sc, La, Lb, l, h);
      lo = std::min(lo, l);
      hi = std::max(hi, h);
    }
  if (lo > hi) lo = hi = 0;
  const uint32_t ib = index_bits(std::max<uint32_t>(d->ws.n, 2));
  const int32_t key_lo = lo - 1;
  if ((uint64_t)(hi - key_lo) >= (1ull << (32 - ib)))
    return set_err(c, NW_ERANGE, "score range with %u dictionary words does not fit 32-bit list keys", d->ws.n);
  plan_query(bk, d->ws.bk, kDefaultTA, s.plan, kQueryMinTasks);
  if (s.plan.segs.size() > kMaxSegs) return set_err(c, NW_ERANGE, "batch plan too large");
  std::memcpy(s.h_segs, s.plan.segs.data(), sizeof(Seg) * s.plan.segs.size());

  NW_CK(cudaMemcpyAsync(s.d_codes.p, s.h_codes, ncodes ? ncodes : 1, cudaMemcpyHostToDevice, st));
  NW_CK(cudaMemcpyAsync(s.d_offsets.p, s.h_offsets, sizeof(uint32_t) * ((size_t)nq + 1), cudaMemcpyHostToDevice, st));
  NW_CK(cudaMemcpyAsync(s.d_perm.p, s.h_perm, sizeof(uint32_t) * nq, cudaMemcpyHostToDevice, st));
  NW_CK(cudaMemcpyAsync(s.d_slen.p, s.h_slen, nq, cudaMemcpyHostToDevice, st));
  if (!s.plan.segs.empty())
    NW_CK(cudaMemcpyAsync(s.d_segs.p, s.h_segs, sizeof(Seg) * s.plan.segs.size(), cudaMemcpyHostToDevice, st));
  NW_CK(cudaMemsetAsync(s.d_b_rec.p, 0xff, sizeof(uint32_t) * brec_words(bk), st));
  NW_CK(launch_ingest_encode(s.d_codes.as<uint8_t>(), s.d_offsets.as<uint32_t>(), nq, s.d_perm.as<uint32_t>(),
                             s.d_slen.as<uint8_t>(), bk, d->ss.shift, s.d_a_enc.as<uint32_t>(),
                             s.d_aoff.as<uint32_t>(), s.d_b_rec.as<uint32_t>(), s.d_brec_w.as<uint32_t>(), st));
  NW_CK(cudaMemsetAsync(s.d_small.p, 0, s.d_small.bytes, st));
  NW_CK(cudaMemsetAsync(s.d_slots.p, 0, sizeof(uint32_t) * (size_t)nq * k, st));
  NW_CK(cudaMemsetAsync(s.d_thr.p, 0, sizeof(uint32_t) * nq, st));

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
  base.stats = reinterpret_cast<unsigned long long*>(s.d_small.as<char>() + 8);
  base.err = s.d_small.as<uint32_t>();
  SideView qside{s.d_perm.as<uint32_t>(), s.d_slots.as<uint32_t>(), s.d_thr.as<uint32_t>()};
  SideView dside{d->ws.perm.as<uint32_t>(), nullptr, nullptr};
  const uint32_t* a_enc[3] = {nullptr, s.d_a_enc.as<uint32_t>(), d->ws.a_enc.as<uint32_t>()};
  const uint4* b_rec[3] = {nullptr, d->ws.b_rec.as<uint4>(), s.d_b_rec.as<uint4>()};
  const SideView* A_views[3] = {nullptr, &qside, &dside};
  const SideView* B_views[3] = {nullptr, &dside, &qside};
  Timer tm{c};
  RunOut ro;
  NW_TRY(run_plan(c, st, s.plan, s.d_segs.as<Seg>(), base,
                  reinterpret_cast<unsigned long long*>(s.d_small.as<char>() + 64), 0, 1, tm, ro, a_enc, A_views,
                  b_rec, B_views));
  NW_CK(launch_finalize(s.d_slots.as<uint32_t>(), nq, k, s.d_perm.as<uint32_t>(), ib, base.imask, key_lo,
                        s.d_idx.as<uint32_t>(), s.d_score.as<int16_t>(), st));
  NW_CK(cudaMemcpyAsync(s.h_idx, s.d_idx.p, sizeof(uint32_t) * (size_t)nq * k, cudaMemcpyDeviceToHost, st));
  NW_CK(cudaMemcpyAsync(s.h_score, s.d_score.p, sizeof(int16_t) * (size_t)nq * k, cudaMemcpyDeviceToHost, st));
  NW_CK(cudaMemcpyAsync(s.h_err, s.d_small.p, sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
  s.cb.srv = S;
  s.cb.slot = &s;
  NW_CK(cudaLaunchHostFunc(st, on_batch_done, &s.cb));
  return NW_OK;
}

// Hands a finished batch's results to its requests (mu held).
void retire(nw_server* S, Slot& s) {
  const uint32_t k = S->cfg.k;
  const uint32_t err = s.h_err[0];
  const double t = now_s();
  for (size_t i = 0; i < s.reqs.size(); ++i) {
    Request* r = s.reqs[i];
    const size_t o = (size_t)s.first[i] * k;
    r->idx.assign(s.h_idx + o, s.h_idx + o + (size_t)r->nq * k);
    r->score.assign(s.h_score + o, s.h_score + o + (size_t)r->nq * k);
    r->info.done_s = t;
    r->status = err & kErrRetry ? NW_ETIMEOUT : (err ? NW_EINVAL : NW_OK);
    r->state = 2;
  }
  if (err) S->err = "a batch reported a device-side error";
  s.reqs.clear();
  s.busy = false;
  s.gpu_done.store(0);
  S->cv_done.notify_all();
}

// Proposal mode, one slot's thread: runs each batch the dispatcher assigns
// through nw_proposal_query on the slot's own context, then publishes the
// results and frees the slot.
void proposal_slot_main(nw_server* S, PropSlot* slot) {
  cudaSetDevice(S->ictx.device);
  const uint32_t k = S->cfg.k;
  std::vector<uint8_t> codes;
  std::vector<uint32_t> offsets, idx;
  std::vector<int16_t> score;
  std::unique_lock<std::mutex> lock(S->mu);
  for (;;) {
    S->cv_slots.wait(lock, [&] { return (slot->busy && !slot->taken) || (S->stop && !slot->busy); });
    if (!slot->busy) break;  // stopped with nothing assigned
    slot->taken = true;
    std::vector<Request*> batch = slot->reqs;
    lock.unlock();
    codes.clear();
    offsets.assign(1, 0u);
    uint32_t nq = 0;
    for (Request* r : batch) {
      const uint32_t base = (uint32_t)codes.size();
      codes.insert(codes.end(), r->codes.begin(), r->codes.end());
      for (uint32_t q = 0; q < r->nq; ++q) offsets.push_back(base + r->offsets[q + 1]);
      nq += r->nq;
    }
    if (codes.empty()) codes.push_back(0);
    idx.resize((size_t)nq * k);
    score.resize((size_t)nq * k);
    const nw_status st =
        nw_proposal_query(slot->model, slot->view, codes.data(), offsets.data(), nq, S->C, k, idx.data(), score.data(), 0);
    lock.lock();
    if (st != NW_OK) S->err = slot->ctx->err;
    const double t1 = now_s();
    uint32_t first = 0;
    for (Request* r : batch) {
      if (st == NW_OK) {
        r->idx.assign(idx.begin() + (size_t)first * k, idx.begin() + (size_t)(first + r->nq) * k);
        r->score.assign(score.begin() + (size_t)first * k, score.begin() + (size_t)(first + r->nq) * k);
      }
      first += r->nq;
      r->status = st;
      r->state = 2;
      r->info.done_s = t1;
    }
    slot->reqs.clear();
    slot->busy = false;
    slot->taken = false;
    S->cv_done.notify_all();
    S->cv.notify_all();
  }
}

// Proposal mode, the dispatcher: packs queued requests (in arrival order, at
// most max_batch_queries words) into a batch for the first free slot; requests
// arriving meanwhile are admitted as soon as a slot frees.
void worker_proposal(nw_server* S) {
  const uint32_t Q = S->cfg.max_batch_queries;
  std::unique_lock<std::mutex> lock(S->mu);
  while (!S->stop) {
    PropSlot* free_slot = nullptr;
    uint32_t inflight = 0;
    for (auto& sp : S->pslots) {
      if (sp->busy) ++inflight;
      else if (!free_slot) free_slot = sp.get();
    }
    if (!free_slot || S->queue.empty()) {
      S->cv.wait_for(lock, std::chrono::milliseconds(2));
      continue;
    }
    uint32_t nq = 0;
    while (!S->queue.empty() && nq + S->queue.front()->nq <= Q) {
      free_slot->reqs.push_back(S->queue.front());
      nq += S->queue.front()->nq;
      S->queue.pop_front();
    }
    const double t0 = now_s();
    for (Request* r : free_slot->reqs) {
      r->state = 1;
      r->info.start_s = t0;
      r->info.batch_queries = nq;
      r->info.batch_requests = (uint32_t)free_slot->reqs.size();
      r->info.inflight_at_start = inflight;
    }
    free_slot->busy = true;
    free_slot->taken = false;
    S->cv_slots.notify_all();
  }
  for (Request* r : S->queue) {
    r->status = NW_EINVAL;
    r->state = 2;
  }
  S->queue.clear();
  S->cv_done.notify_all();
  S->cv_slots.notify_all();
}

void worker_main(nw_server* S) {
  if (S->model) {
    worker_proposal(S);
    return;
  }
  cudaSetDevice(S->ictx.device);
  const uint32_t Q = S->cfg.max_batch_queries;
  std::unique_lock<std::mutex> lock(S->mu);
  for (;;) {
    uint32_t inflight = 0;
    for (auto& sp : S->slots) {
      if (sp->busy && sp->gpu_done.load()) retire(S, *sp);
      inflight += sp->busy ? 1u : 0u;
    }
    if (S->stop) {
      if (inflight == 0) break;
      S->cv.wait_for(lock, std::chrono::milliseconds(1));
      continue;
    }
    Slot* free_slot_p = nullptr;
    for (auto& sp : S->slots)
      if (!sp->busy) { free_slot_p = sp.get(); break; }
    if (free_slot_p && !S->queue.empty()) {
      Slot& s = *free_slot_p;
      uint32_t nq = 0;
      while (!S->queue.empty() && nq + S->queue.front()->nq <= Q) {
        Request* r = S->queue.front();
        S->queue.pop_front();
        nq += r->nq;
        s.reqs.push_back(r);
      }
      const double t = now_s();
      for (Request* r : s.reqs) {
        r->state = 1;
        r->info.start_s = t;
        r->info.batch_queries = nq;
        r->info.batch_requests = (uint32_t)s.reqs.size();
        r->info.inflight_at_start = inflight;
      }
      s.busy = true;
      lock.unlock();
      const nw_status st = launch_batch(S, s);
      // (never wait on a stream while holding mu: its host callback takes mu)
      if (st != NW_OK) cudaStreamSynchronize(s.stream);
      lock.lock();
      if (st != NW_OK) {
        S->err = S->ictx.err;
        for (Request* r : s.reqs) {
          r->status = st;
          r->state = 2;
          r->info.done_s = now_s();
        }
        s.reqs.clear();
        s.busy = false;
        S->cv_done.notify_all();
      }
      continue;
    }
    S->cv.wait_for(lock, std::chrono::milliseconds(2));
  }
  // stopped: requests that never reached the GPU fail
  for (Request* r : S->queue) {
    r->status = NW_EINVAL;
    r->state = 2;
  }
  S->queue.clear();
  S->cv_done.notify_all();
}

}  // namespace

extern "C" {

nw_status nw_server_create(nw_dict* dict, const nw_server_config* cfg, nw_server** out) {
  if (!out) return NW_EINVAL;
  *out = nullptr;
  if (!dict || !cfg) return set_err(nullptr, NW_EINVAL, "null argument");
  if (dict->subst) return set_err(nullptr, NW_EINVAL, "the server takes match / mismatch dictionaries only");
  if (cfg->k == 0 || cfg->k > NW_MAX_K) return set_err(nullptr, NW_EINVAL, "k must be in [1, %d]", NW_MAX_K);
  if (cfg->max_batch_queries == 0 || cfg->max_batch_queries > (1u << 20))
    return set_err(nullptr, NW_EINVAL, "max_batch_queries must be in [1, 2^20]");
  if (cfg->max_inflight == 0 || cfg->max_inflight > 64)
    return set_err(nullptr, NW_EINVAL, "max_inflight must be in [1, 64]");
  nw_server* S = new nw_server();
  S->dict = dict;
  S->cfg = *cfg;
  S->ictx.device = dict->ctx->device;
  S->ictx.sm_count = dict->ctx->sm_count;
  S->ictx.budget = cfg->mem_budget_bytes;
  if (cudaSetDevice(S->ictx.device) != cudaSuccess) {
    cudaGetLastError();
    delete S;
    return set_err(nullptr, NW_ECUDA, "cudaSetDevice failed");
  }
  // as many slots as the budget holds, at most max_inflight, at least one
  for (uint32_t i = 0; i < cfg->max_inflight; ++i) {
    auto sp = std::make_unique<Slot>();
    const size_t used_before = S->ictx.used;
    const nw_status st = alloc_slot(S, *sp);
    if (st != NW_OK) {
      free_slot(S, *sp);
      if (i == 0 || st != NW_ENOMEM) {
        const std::string msg = S->ictx.err;
        for (auto& q : S->slots) free_slot(S, *q);
        delete S;
        return set_err(nullptr, st, "server slot allocation: %s", msg.c_str());
      }
      (void)used_before;
      break;
    }
    S->slots.push_back(std::move(sp));
  }
  S->worker = std::thread(worker_main, S);
  *out = S;
  return NW_OK;
}

nw_status nw_server_create_proposal(nw_dict* dict, nw_model* model, uint32_t C, const nw_server_config* cfg,
                                    nw_server** out) {
  if (!out) return NW_EINVAL;
  *out = nullptr;
  if (!dict || !model || !cfg) return set_err(nullptr, NW_EINVAL, "null argument");
  if (nw::prop::model_ctx(model) != dict->ctx)
    return set_err(nullptr, NW_EINVAL, "the model and the dictionary belong to different contexts");
  if (C == 0 || C > NW_MAX_CANDIDATES) return set_err(nullptr, NW_EINVAL, "C must be in [1, %d]", NW_MAX_CANDIDATES);
  if (cfg->k == 0 || cfg->k > NW_MAX_K) return set_err(nullptr, NW_EINVAL, "k must be in [1, %d]", NW_MAX_K);
  if (cfg->max_batch_queries == 0 || cfg->max_batch_queries > (1u << 20))
    return set_err(nullptr, NW_EINVAL, "max_batch_queries must be in [1, 2^20]");
  if (cfg->max_inflight == 0 || cfg->max_inflight > 64)
    return set_err(nullptr, NW_EINVAL, "max_inflight must be in [1, 64]");
  const int device = dict->ctx->device;
  if (cudaSetDevice(device) != cudaSuccess) {
    cudaGetLastError();
    return set_err(nullptr, NW_ECUDA, "cudaSetDevice failed");
  }
  // slots: max_inflight, fewer when the memory budget does not hold that
  // many slots' device memory (at least one; each slot's context is capped at
  // its share of the budget)
  const uint32_t Q = cfg->max_batch_queries, n = dict->ws.n;
  const size_t per_slot = nw::prop::dot_topk_buffer_bytes(Q, std::max<uint32_t>(n, 1), C) +
                          nw::prop::dot_topk_qb_bytes(n) + nw::prop::dot_topk_qb_bytes(Q) + 8 * (size_t)n +
                          (size_t)Q * C * 16 + (size_t)Q * kMaxLen * 128 * 4 * 8;
  uint32_t nslots = cfg->max_inflight;
  if (cfg->mem_budget_bytes)
    nslots = (uint32_t)std::max<size_t>(1, std::min<size_t>(nslots, cfg->mem_budget_bytes / per_slot));
  const size_t slot_budget = cfg->mem_budget_bytes ? cfg->mem_budget_bytes / nslots : 0;
  nw_server* S = new nw_server();
  S->dict = dict;
  S->model = model;
  S->C = C;
  S->cfg = *cfg;
  S->ictx.device = device;
  S->ictx.sm_count = dict->ctx->sm_count;
  for (uint32_t i = 0; i < nslots; ++i) {
    auto sp = std::make_unique<PropSlot>();
    nw_status st = nw_create(&sp->ctx, device, slot_budget, nullptr);
    if (st == NW_OK) st = nw::prop::model_clone(model, sp->ctx, &sp->model);
    if (st != NW_OK) {
      const std::string msg = sp->ctx ? sp->ctx->err : g_create_error;
      free_pslot(*sp);
      for (auto& q : S->pslots) free_pslot(*q);
      delete S;
      return set_err(nullptr, st, "proposal server slot: %s", msg.c_str());
    }
    sp->view = new nw_dict(*dict);  // the dictionary's device data, owned by the caller's context
    sp->view->ctx = sp->ctx;
    S->pslots.push_back(std::move(sp));
  }
  for (auto& sp : S->pslots) sp->th = std::thread(proposal_slot_main, S, sp.get());
  S->worker = std::thread(worker_main, S);
  *out = S;
  return NW_OK;
}

nw_status nw_server_submit(nw_server* S, const uint8_t* qcodes, const uint32_t* qoffsets, uint32_t nq,
                           uint64_t* request_id) {
  if (!S || !qoffsets || !request_id) return NW_EINVAL;
  if (nq == 0 || nq > S->cfg.max_batch_queries) {
    std::lock_guard<std::mutex> lock(S->mu);
    S->err = "a request needs 1 to max_batch_queries query words";
    return NW_EINVAL;
  }
  if (qoffsets[0] != 0) return NW_EINVAL;
  const uint32_t alphabet = S->dict->alphabet;
  for (uint32_t q = 0; q < nq; ++q) {
    if (qoffsets[q + 1] < qoffsets[q] || qoffsets[q + 1] - qoffsets[q] > (uint32_t)kMaxLen) {
      std::lock_guard<std::mutex> lock(S->mu);
      S->err = "query words must have 0 to NW_MAX_WORD_LEN codes";
      return NW_EINVAL;
    }
  }
  const uint32_t total = qoffsets[nq];
  if (total && !qcodes) return NW_EINVAL;
  for (uint32_t i = 0; i < total; ++i)
    if (qcodes[i] >= alphabet) {
      std::lock_guard<std::mutex> lock(S->mu);
      S->err = "a query code is >= the dictionary's alphabet";
      return NW_EINVAL;
    }
  Request* r = new Request();
  r->nq = nq;
  r->codes.assign(qcodes, qcodes + total);
  r->offsets.assign(qoffsets, qoffsets + nq + 1);
  r->info.nq = nq;
  r->info.submit_s = now_s();
  {
    std::lock_guard<std::mutex> lock(S->mu);
    if (S->stop) {
      delete r;
      return NW_EINVAL;
    }
    r->id = S->next_id++;
    S->reqs[r->id] = r;
    S->queue.push_back(r);
    *request_id = r->id;
  }
  S->cv.notify_all();
  return NW_OK;
}

nw_status nw_server_wait(nw_server* S, uint64_t request_id, int timeout_ms, uint32_t* nbr_idx, int16_t* nbr_score,
                         nw_request_info* info) {
  if (!S) return NW_EINVAL;
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->reqs.find(request_id);
  if (it == S->reqs.end()) {
    S->err = "unknown request id";
    return NW_EINVAL;
  }
  Request* r = it->second;
  auto done = [&] { return r->state == 2; };
  if (timeout_ms < 0) S->cv_done.wait(lock, done);
  else if (!S->cv_done.wait_for(lock, std::chrono::milliseconds(timeout_ms), done)) return NW_EBUSY;
  const nw_status st = r->status;
  if (st == NW_OK) {
    if (nbr_idx) std::memcpy(nbr_idx, r->idx.data(), sizeof(uint32_t) * r->idx.size());
    if (nbr_score) std::memcpy(nbr_score, r->score.data(), sizeof(int16_t) * r->score.size());
  }
  if (info) *info = r->info;
  S->reqs.erase(it);
  delete r;
  return st;
}

const char* nw_server_last_error(const nw_server* S) { return S ? S->err.c_str() : g_create_error.c_str(); }

void nw_server_destroy(nw_server* S) {
  if (!S) return;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv.notify_all();
  if (S->worker.joinable()) S->worker.join();
  S->cv_slots.notify_all();
  for (auto& sp : S->pslots)
    if (sp->th.joinable()) sp->th.join();
  cudaSetDevice(S->ictx.device);
  for (auto& sp : S->slots) free_slot(S, *sp);
  for (auto& sp : S->pslots) free_pslot(*sp);
  for (auto& kv : S->reqs) delete kv.second;
  delete S;
}

}  // extern "C"
