// nw_api.cu -- host runtime of libnw: the C ABI declared in include/nw.h.
//
// Contexts own a stream (or borrow the caller's), a device-memory budget and a
// grow-only workspace.  Dictionaries are word sets resident on the device,
// sorted by length into buckets and encoded for the alignment kernel, plus the
// plan of pair rectangles ("segments") the all-pairs launches walk.
#include "nw_host.h"

using namespace nw;

// ===========================================================================
// C ABI

namespace {

// A dictionary from validated scoring: `scoring` gives the gap and the score
// bounds (match = the best and mismatch = the worst similarity), `tab` the
// substitution table of a similarity-matrix dictionary (else null).
nw_status load_impl(nw_ctx* c, const uint8_t* codes, const uint32_t* offsets, uint32_t n, uint32_t alphabet,
                    const nw_scoring& sc, const ShiftedScoring& ss, const std::vector<uint16_t>* tab, uint32_t flags,
                    nw_dict** out) {
  const nw_scoring* scoring = &sc;
  static std::atomic<uint64_t> next_serial{1};
  nw_dict* d = new nw_dict();
  d->serial = next_serial.fetch_add(1);
  d->ctx = c;
  d->sc = sc;
  d->ss = ss;
  d->alphabet = alphabet;
  d->subst = tab != nullptr;
  nw_status st = NW_OK;
  if (tab) {
    st = ctx_alloc(c, d->d_tab, kTabBytes, "substitution table");
    if (st == NW_OK) {
      cudaError_t e = cudaMemcpyAsync(d->d_tab.p, tab->data(), kTabBytes, cudaMemcpyHostToDevice, c->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
      if (e != cudaSuccess) st = cuda_fail(c, e, "uploading the substitution table");
    }
  }
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
    ctx_free(c, d->d_tab);
    delete d;
    return st;
  }
  c->dicts.insert(d);
  *out = d;
  return NW_OK;
}

}  // namespace

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
  const std::vector<nw_model*> ms(c->models.begin(), c->models.end());
  for (nw_model* m : ms) nw_model_free(m);
  ctx_free(c, c->ws_slots);
  ctx_free(c, c->ws_thr);
  ctx_free(c, c->ws_hist);
  ctx_free(c, c->ws_small);
  ctx_free(c, c->ws_out_idx);
  ctx_free(c, c->ws_out_score);
  ctx_free(c, c->ws_mat);
  ctx_free(c, c->ws_pairs);
  ctx_free(c, c->ws_segs);
  ctx_free(c, c->ws_norm);
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
  ShiftedScoring ss{};
  NW_TRY(make_shifted(c, *scoring, alphabet, ss));
  return load_impl(c, codes, offsets, n, alphabet, *scoring, ss, nullptr, flags, out);
}

nw_status nw_load_dictionary_sim(nw_ctx* c, const uint8_t* codes, const uint32_t* offsets, uint32_t n,
                                 uint32_t alphabet, const int32_t* sim, int32_t gap, uint32_t flags, nw_dict** out) {
  NW_ENTER(c);
  if (!out || !offsets || !sim || (!codes && n)) return set_err(c, NW_EINVAL, "null pointer argument");
  *out = nullptr;
  if (alphabet == 0 || alphabet > (uint32_t)kTabDim)
    return set_err(c, NW_EINVAL, "a similarity-matrix dictionary needs alphabet in [1, %d]", kTabDim);
  if (std::abs(gap) > 1024) return set_err(c, NW_EINVAL, "gap must lie in [-1024, 1024]");
  int smax = INT32_MIN, smin = INT32_MAX;
  std::vector<uint16_t> tab((size_t)kTabDim * kTabDim, 0);
  for (uint32_t a = 0; a < alphabet; ++a) {
    for (uint32_t b = 0; b < alphabet; ++b) {
      const int32_t v = sim[a * alphabet + b];
      if (std::abs(v) > 1024) return set_err(c, NW_EINVAL, "similarity values must lie in [-1024, 1024]");
      if (v != sim[b * alphabet + a]) return set_err(c, NW_EINVAL, "the similarity matrix must be symmetric");
      smax = std::max(smax, v);
      smin = std::min(smin, v);
      const int32_t sp = std::max(v - 2 * gap, 0);
      if ((int64_t)sp * kMaxLen > 32767)
        return set_err(c, NW_ERANGE, "sim - 2*gap = %d is too large for 16-bit cells at length %d", sp, kMaxLen);
      tab[(size_t)a * kTabDim + b] = (uint16_t)sp;
    }
  }
  // the bounds of a match / mismatch scoring with match = max sim and mismatch
  // = min sim hold for the matrix (the same two alignments bound the optimum)
  const nw_scoring bounds{smax, smin, gap};
  ShiftedScoring ss{};  // codes stay unshifted: the kernels look them up in the table
  return load_impl(c, codes, offsets, n, alphabet, bounds, ss, &tab, flags, out);
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
  ctx_free(c, d->d_tab);
  c->dicts.erase(d);
  delete d;
}

}  // extern "C"

namespace {

// The int8 matrix, written directly (chunk_bytes == 0 or >= the matrix) or in
// chunks of chunk_bytes of the row-major order: every pass scores all pairs
// and keeps the entries of one chunk, which is then copied to the host.
nw_status matrix_impl(nw_dict* d, int8_t* out, uint64_t chunk_bytes, uint32_t flags) {
  nw_ctx* c = d->ctx;
  const uint32_t n = d->ws.n;
  if (!out) return set_err(c, NW_EINVAL, "null output pointer");
  if (n < 2) return set_err(c, NW_EINVAL, "the dictionary needs at least 2 words (has %u)", n);
  if (d->score_lo < -128 || d->score_hi > 127)
    return set_err(c, NW_ERANGE, "scores of this dictionary span [%d, %d], outside int8", d->score_lo, d->score_hi);
  const bool dev = flags & NW_DEVICE_PTRS;
  const uint64_t E = (uint64_t)n * (n - 1) / 2;
  const bool chunked = chunk_bytes > 0 && chunk_bytes < E;
  if (chunked && dev) return set_err(c, NW_EINVAL, "chunked output goes to host memory (no NW_DEVICE_PTRS)");
  cudaStream_t s = c->stream;
  int8_t* dst = out;
  const uint64_t step = chunked ? chunk_bytes : E;
  if (!dev) {
    NW_TRY(ctx_ensure(c, c->ws_mat, step, "score matrix"));
    dst = c->ws_mat.as<int8_t>();
  }
  NW_TRY(ctx_ensure(c, c->ws_small, 64 + sizeof(unsigned long long) * (d->plan.launches.size() + 1), "task counters"));
  uint32_t* d_err = c->ws_small.as<uint32_t>();
  unsigned long long* d_counters = reinterpret_cast<unsigned long long*>(c->ws_small.as<char>() + 64);
  Timer tm{c};
  cudaEvent_t e0 = nullptr;
  tm.begin(false, e0);
  NW_CK(cudaMemsetAsync(c->ws_small.p, 0, c->ws_small.bytes, s));
  RunOut ro;
  for (uint64_t lo = 0; lo < E; lo += step) {
    const uint64_t hi = std::min(E, lo + step);
    if (lo > 0) NW_CK(cudaMemsetAsync(d_counters, 0, sizeof(unsigned long long) * d->plan.launches.size(), s));
    DpParams base{};
    base.TA = kDefaultTA;
    base.C1 = d->ss.C1;
    base.C2 = d->ss.C2;
    base.match = d->sc.match;
    base.mismatch = d->sc.mismatch;
    base.gap = d->sc.gap;
    base.sim_tab = dict_tab(d);
    base.mode = kModeMatrix;
    base.mat = dst - lo;  // entry `off` of the chunk [lo, hi) lands at dst[off - lo]
    base.n = n;
    base.mat_lo = lo;
    base.mat_hi = hi;
    base.hist_mode = kHistNone;
    base.err = d_err;
    SideView side{d->ws.perm.as<uint32_t>(), nullptr, nullptr};
    const uint32_t* a_enc[3] = {d->ws.a_enc.as<uint32_t>(), nullptr, nullptr};
    const uint4* b_rec[3] = {d->ws.b_rec.as<uint4>(), nullptr, nullptr};
    const SideView* views[3] = {&side, nullptr, nullptr};
    NW_TRY(run_plan(c, c->stream, d->plan, d->d_segs.as<Seg>(), base, d_counters, 0, 1, tm, ro, a_enc, views,
                    b_rec, views));
    if (!dev) {
      NW_CK(cudaMemcpyAsync(out + lo, dst, hi - lo, cudaMemcpyDeviceToHost, s));
      if (chunked) NW_CK(cudaStreamSynchronize(s));  // the chunk buffer is reused
    }
  }
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

}  // namespace

extern "C" {

nw_status nw_all_pairs_matrix(nw_dict* d, int8_t* out, uint32_t flags) {
  if (!d) return NW_EINVAL;
  NW_ENTER(d->ctx);
  return matrix_impl(d, out, 0, flags);
}

nw_status nw_all_pairs_matrix_chunked(nw_dict* d, int8_t* out, uint64_t chunk_bytes, uint32_t flags) {
  if (!d) return NW_EINVAL;
  NW_ENTER(d->ctx);
  if (chunk_bytes == 0) return set_err(d->ctx, NW_EINVAL, "chunk_bytes must be positive");
  return matrix_impl(d, out, chunk_bytes, flags);
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
  if (nparts > kMaxMergeParts) return NW_EINVAL;
  for (uint32_t p = 0; p < nparts; ++p)
    if (!idx_parts[p] || !score_parts[p]) return NW_EINVAL;
  for (uint32_t w = 0; w < n; ++w) {
    const size_t row = (size_t)w * k;
    merge_ranked_row(
        nparts, k,
        [&](uint32_t p, uint32_t r, uint32_t& j, int32_t& s) {
          j = idx_parts[p][row + r];
          s = score_parts[p][row + r];
        },
        idx_out + row, score_out + row);
  }
  return NW_OK;
}

nw_status nw_topk_merge_device(nw_ctx* c, uint32_t n, uint32_t k, uint32_t nparts, const uint32_t* idx_parts,
                               const int16_t* score_parts, uint32_t* idx_out, int16_t* score_out) {
  NW_ENTER(c);
  if (k == 0 || k > NW_MAX_K) return set_err(c, NW_EINVAL, "k must be in [1, %d]", NW_MAX_K);
  if (nparts == 0 || nparts > kMaxMergeParts)
    return set_err(c, NW_EINVAL, "nparts must be in [1, %u]", kMaxMergeParts);
  if (n == 0) return NW_OK;
  if (!idx_parts || !score_parts || !idx_out || !score_out) return set_err(c, NW_EINVAL, "null pointer argument");
  NW_CK(launch_topk_merge(n, k, nparts, idx_parts, score_parts, idx_out, score_out, c->stream));
  NW_CK(cudaStreamSynchronize(c->stream));
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
  P.tab = dict_tab(d);
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
  return nw::query_impl(d, qcodes, qoffsets, nq, k, nbr_idx, nbr_score, flags);
}

}  // extern "C"

namespace nw {

nw_status query_impl(nw_dict* d, const uint8_t* qcodes, const uint32_t* qoffsets, uint32_t nq, uint32_t k,
                     uint32_t* nbr_idx, int16_t* nbr_score, uint32_t flags) {
  nw_ctx* c = d->ctx;
  if (flags & NW_RANK_NORMALISED) return set_err(c, NW_EINVAL, "queries rank by raw score only");
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
  plan_query(q.bk, d->ws.bk, kDefaultTA, plan, kQueryMinTasks);
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
  base.sim_tab = dict_tab(d);
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
  NW_TRY(run_plan(c, c->stream, plan, c->ws_segs.as<Seg>(), base, d_counters, 0, 1, tm, ro, a_enc, A_views,
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

}  // namespace nw

extern "C" {

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

nw_status nw_debug_norm_tables(const nw_scoring* sc, int32_t lo, int32_t hi, uint16_t* rank, int16_t* smin,
                               int16_t* frac, uint32_t cap_ranks, uint32_t* nranks) {
  if (!sc || !rank || !smin || !frac || !nranks || lo > hi || lo < INT16_MIN || hi > INT16_MAX) return NW_EINVAL;
  NormTables t;
  build_norm_tables(*sc, lo, hi, t);
  *nranks = t.nranks;
  if (t.nranks > cap_ranks) return NW_ERANGE;
  std::copy(t.rank.begin(), t.rank.end(), rank);
  std::copy(t.smin.begin(), t.smin.end(), smin);
  std::copy(t.frac.begin(), t.frac.end(), frac);
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

nw_status nw_debug_enumerate_query_pairs(const uint32_t* q_lengths, uint32_t nq, const uint32_t* d_lengths,
                                         uint32_t nd, uint32_t ta, uint32_t* q, uint32_t* d, uint64_t cap,
                                         uint64_t* count) {
  if (!q_lengths || !d_lengths || !count) return NW_EINVAL;
  if (cap && (!q || !d)) return NW_EINVAL;
  // each set bucketed by length as ingest does (stable), then planned as nw_query plans it
  auto bucket = [](const uint32_t* len, uint32_t n, Buckets& bk, std::vector<uint32_t>& perm) -> bool {
    bk = Buckets{};
    for (uint32_t i = 0; i < n; ++i) {
      if (len[i] > (uint32_t)kMaxLen) return false;
      ++bk.count[len[i]];
    }
    fill_buckets(bk);
    perm.assign(n, 0);
    std::vector<uint32_t> fill(kBuckets, 0);
    for (uint32_t i = 0; i < n; ++i) perm[bk.start[len[i]] + fill[len[i]]++] = i;
    return true;
  };
  Buckets qb, db;
  std::vector<uint32_t> qperm, dperm;
  if (!bucket(q_lengths, nq, qb, qperm) || !bucket(d_lengths, nd, db, dperm)) return NW_EINVAL;
  const uint32_t TA = ta ? ta : kDefaultTA;
  Plan plan;
  plan_query(qb, db, TA, plan, kQueryMinTasks);
  uint64_t cnt = 0;
  for (const LaunchPlan& lp : plan.launches) {
    const Seg* segs = plan.segs.data() + lp.seg_first;
    for (uint64_t t = 0; t < lp.ntasks; ++t) {
      const Seg& S = segs[find_seg(segs, lp.nsegs, t)];
      const TaskGeom g = task_geom(S, t, lp.ta ? lp.ta : TA);
      for (uint32_t x = g.a0; x < g.a1; ++x) {
        for (uint32_t y = g.b0; y < g.bend; ++y) {
          if (!pair_valid(g, x, y)) continue;
          // role 1: queries are the A words; role 2: queries are the B words
          if (cnt < cap) {
            q[cnt] = lp.role == 1 ? qperm[x] : qperm[y];
            d[cnt] = lp.role == 1 ? dperm[y] : dperm[x];
          }
          ++cnt;
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

nw_status nw_debug_set_bounds(nw_ctx* c, int32_t insert_iters, int64_t wait_cycles, uint32_t withhold_tile) {
  if (!c) return NW_EINVAL;
  c->dbg_insert_iters = insert_iters < 0 ? -1 : insert_iters;
  c->dbg_wait_cycles = wait_cycles < 0 ? -1 : wait_cycles;
  c->dbg_withhold_tile = withhold_tile;
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
  if (flags & NW_RANK_NORMALISED)
    return set_err(c, NW_EINVAL, "the no-allocation variant ranks by raw score only");
  if (d->subst) return set_err(c, NW_EINVAL, "the no-allocation variant takes match / mismatch dictionaries only");
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
  // two error words: a synchronous call clears and reads word 0; an NW_ASYNC
  // call cannot read its flag, so its kernels raise word 1 instead, which is
  // never cleared by an NW_ASYNC call and is reported (then cleared) by the
  // next synchronous call
  const bool async = flags & NW_ASYNC;
  uint32_t* d_err = reinterpret_cast<uint32_t*>(sb);
  uint32_t* d_err_async = d_err + 1;
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

  if (!async) NW_CK(cudaMemsetAsync(d_err, 0, sizeof(uint32_t), s));
  NW_CK(cudaMemsetAsync(sb + 8, 0, off_thr - 8, s));
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
  P.err = async ? d_err_async : d_err;
  SideView side{d->ws.perm.as<uint32_t>(), d_slots, d_thr};
  const uint32_t* a_enc[3] = {d->ws.a_enc.as<uint32_t>(), nullptr, nullptr};
  const uint4* b_rec[3] = {d->ws.b_rec.as<uint4>(), nullptr, nullptr};
  const SideView* views[3] = {&side, nullptr, nullptr};
  Timer tm{c};
  RunOut ro;
  NW_TRY(run_plan(c, c->stream, d->plan, d->d_segs.as<Seg>(), P, d_counters, 0, 1, tm, ro, a_enc, views, b_rec,
                  views));
  NW_CK(launch_finalize(d_slots, n, k, d->ws.perm.as<uint32_t>(), ib, P.imask, key_lo, nbr_idx, nbr_score, s));
  if (hist) {
    NW_CK(cudaMemcpyAsync(hist, d_hist, sizeof(int64_t) * need_bins, cudaMemcpyDeviceToDevice, s));
    if (nbins > need_bins) NW_CK(cudaMemsetAsync(hist + need_bins, 0, sizeof(int64_t) * (nbins - need_bins), s));
    if (hist_lo) *hist_lo = d->score_lo;
  }
  if (async) return NW_OK;
  uint32_t words[2] = {0u, 0u};
  NW_CK(cudaMemcpyAsync(words, d_err, sizeof words, cudaMemcpyDeviceToHost, s));
  NW_CK(cudaStreamSynchronize(s));
  if (words[0]) return check_device_flags(c, d_err);
  if (words[1]) {
    NW_CK(cudaMemsetAsync(d_err_async, 0, sizeof(uint32_t), s));
    NW_CK(cudaStreamSynchronize(s));
    const char* what = (words[1] & (kErrRetry | kErrWait)) ? "a device-side bound ran out"
                       : (words[1] & kErrHistRange)        ? "a score fell outside the histogram range"
                                                           : "invalid input seen on the device";
    const nw_status st = (words[1] & (kErrRetry | kErrWait)) ? NW_ETIMEOUT
                         : (words[1] & kErrHistRange)        ? NW_ERANGE
                                                             : NW_EINVAL;
    return set_err(c, st,
                   "an earlier NW_ASYNC call of nw_all_pairs_topk_noalloc on this device failed (%s); its outputs "
                   "are not valid; this call's outputs are",
                   what);
  }
  return NW_OK;
}

}  // namespace nw
