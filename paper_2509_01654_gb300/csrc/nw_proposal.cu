// nw_proposal.cu -- the learned candidate proposal (include/nw_proposal.h):
// the model object, its forward and backward passes over a dictionary's
// device-resident words, the training loop (one captured CUDA graph per
// step, replayed), and the proposal path (embed, quantise, dot-product
// top-C, exact rescoring).
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <vector>

#include "nw_cnn.h"
#include "nw_host.h"
#include "nw_proposal.h"
#include "nw_proposal_internal.h"

using namespace nw;

struct nw_model {
  nw_ctx* ctx = nullptr;
  uint32_t alphabet = 0;
  cnn::Layout L{};
  cudaStream_t stream = nullptr;
  uint32_t steps_done = 0;  // mirror of the device step counter
  DevBuf params, grads, adam_m, adam_v, small;  // small: step counter, loss accumulator, error flags, amax
  // forward/backward scratch for cap_words words packed into cap_rows rows
  int cap_words = 0, cap_rows = 0;
  DevBuf widx, len, off, rinfo, rword, codes, X0, Y1, Y2, Y3, P, E, dE, dP, dYa, dYb, dX0;
  // training pairs
  uint32_t cap_pairs = 0;
  DevBuf pi, pj, target, score16;
  // proposal path
  DevBuf Eall, Qb, qbias, topbuf, cand, cand_dot, cand_score, nbr;
  // queries against a dictionary: its quantised rows, kept while the
  // dictionary (serial) and the parameters (gen) are unchanged
  uint64_t gen = 1, prep_serial = 0, prep_gen = 0;
  DevBuf dQb, dqbias, prep_small, qQb, qcand, qcand_dot, qscore, qbuf;
  // words of at least exact_len symbols take the exhaustive path (0: none);
  // their codes, offsets and (k + 1)-long exhaustive lists
  uint32_t exact_len = 0;
  DevBuf xcodes, xoffs, xidx, xscore;
  // the candidate sweep over the rows in a locality order (prop::sweep_order):
  // the rows and biases in that order, the order, its scratch
  bool sweep_order = true;
  DevBuf oQb, obias, operm, oscratch;
};

namespace {

// the context's debug bounds for the candidate kernel (nw_debug_set_bounds)
prop::DotDebug dot_debug(const nw_ctx* c) {
  prop::DotDebug d;
  d.wait_cycles = c->dbg_wait_cycles;
  d.withhold = c->dbg_withhold_tile;
  return d;
}

constexpr int kMaxRowsPerPass = 1 << 20;  // packed positions per forward pass of nw_model_embed

// codes of the dictionary's words from sorted position p0 on (contiguous in
// a_enc: every symbol e(c) = c << shift replicated in both 16-bit halves)
__global__ void extract_codes_kernel(const uint32_t* __restrict__ a_enc, uint32_t first, uint32_t total,
                                     uint32_t shift, uint8_t* __restrict__ codes) {
  const uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x < total) codes[x] = (uint8_t)((a_enc[first + x] & 0xffffu) >> shift);
}

// word w (sorted position p0 + w, original index perm[p0 + w]) gets the
// first k entries of its exhaustive (k + 1)-long list that are not itself
__global__ void splice_exact_kernel(const uint32_t* __restrict__ xi, const int16_t* __restrict__ xs, uint32_t m,
                                    uint32_t k, const uint32_t* __restrict__ perm, uint32_t p0,
                                    uint32_t* __restrict__ out_idx, int16_t* __restrict__ out_score) {
  const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= m) return;
  const uint32_t self = perm[p0 + w];
  uint32_t* oi = out_idx + (size_t)self * k;
  int16_t* os = out_score + (size_t)self * k;
  uint32_t j = 0;
  for (uint32_t x = 0; x <= k && j < k; ++x) {
    const uint32_t id = xi[(size_t)w * (k + 1) + x];
    if (id == self) continue;
    oi[j] = id;
    os[j] = xs[(size_t)w * (k + 1) + x];
    ++j;
  }
  for (; j < k; ++j) {
    oi[j] = 0xffffffffu;
    os[j] = INT16_MIN;
  }
}

float* fptr(const DevBuf& b, uint64_t off = 0) { return b.as<float>() + off; }

uint32_t* step_ptr(nw_model* M) { return M->small.as<uint32_t>(); }
float* loss_ptr(nw_model* M) { return reinterpret_cast<float*>(M->small.as<char>() + 4); }
uint32_t* err_ptr(nw_model* M) { return reinterpret_cast<uint32_t*>(M->small.as<char>() + 8); }
unsigned int* amax_ptr(nw_model* M) { return reinterpret_cast<unsigned int*>(M->small.as<char>() + 12); }
int* rows_ptr(nw_model* M) { return reinterpret_cast<int*>(M->small.as<char>() + 16); }
float* sumsq_ptr(nw_model* M) { return reinterpret_cast<float*>(M->small.as<char>() + 20); }

void model_free_buffers(nw_model* M) {
  nw_ctx* c = M->ctx;
  DevBuf* bufs[] = {&M->params, &M->grads, &M->adam_m, &M->adam_v, &M->small, &M->widx, &M->len, &M->off,
                    &M->rinfo, &M->rword, &M->codes, &M->X0, &M->Y1, &M->Y2, &M->Y3, &M->P, &M->E, &M->dE, &M->dP, &M->dYa,
                    &M->dYb, &M->dX0, &M->pi, &M->pj, &M->target, &M->score16, &M->Eall, &M->Qb,
                    &M->qbias, &M->topbuf, &M->cand, &M->cand_dot, &M->cand_score, &M->nbr,
                    &M->dQb, &M->dqbias, &M->prep_small, &M->qQb, &M->qcand, &M->qcand_dot, &M->qscore, &M->qbuf,
                    &M->xcodes, &M->xoffs, &M->xidx, &M->xscore, &M->oQb, &M->obias, &M->operm, &M->oscratch};
  for (DevBuf* b : bufs) ctx_free(c, *b);
}

// scratch for Bw words packed into at most Tmax rows
nw_status ensure_scratch(nw_model* M, int Bw, int Tmax) {
  nw_ctx* c = M->ctx;
  if (Bw <= M->cap_words && Tmax <= M->cap_rows) return NW_OK;
  const int W = std::max(Bw, M->cap_words);
  const size_t T = (size_t)std::max(Tmax, M->cap_rows);
  if (T > (size_t)INT32_MAX / cnn::kCh || W > (1 << 20))
    return set_err(c, NW_EINVAL, "batch of %d words in %zu rows too large", W, T);
  NW_TRY(ctx_ensure(c, M->widx, sizeof(uint32_t) * W, "model word indices"));
  NW_TRY(ctx_ensure(c, M->len, sizeof(int) * W, "model word lengths"));
  NW_TRY(ctx_ensure(c, M->off, sizeof(int) * W, "model word offsets"));
  NW_TRY(ctx_ensure(c, M->rinfo, sizeof(int) * T, "model row tables"));
  NW_TRY(ctx_ensure(c, M->rword, sizeof(int) * T, "model row tables"));
  NW_TRY(ctx_ensure(c, M->codes, sizeof(int32_t) * T, "model codes"));
  NW_TRY(ctx_ensure(c, M->X0, sizeof(float) * T * cnn::kEmb, "model activations"));
  NW_TRY(ctx_ensure(c, M->dX0, sizeof(float) * T * cnn::kEmb, "model activations"));
  DevBuf* big[] = {&M->Y1, &M->Y2, &M->Y3, &M->dYa, &M->dYb};
  for (DevBuf* b : big) NW_TRY(ctx_ensure(c, *b, sizeof(float) * T * cnn::kCh, "model activations"));
  NW_TRY(ctx_ensure(c, M->P, sizeof(float) * W * cnn::kCh, "model pooled"));
  NW_TRY(ctx_ensure(c, M->dP, sizeof(float) * W * cnn::kCh, "model pooled"));
  NW_TRY(ctx_ensure(c, M->E, sizeof(float) * W * cnn::kOut, "model embeddings"));
  NW_TRY(ctx_ensure(c, M->dE, sizeof(float) * W * cnn::kOut, "model embeddings"));
  M->cap_words = W;
  M->cap_rows = (int)T;
  return NW_OK;
}

nw_status ensure_pairs(nw_model* M, uint32_t m) {
  nw_ctx* c = M->ctx;
  if (m <= M->cap_pairs) return NW_OK;
  NW_TRY(ctx_ensure(c, M->pi, sizeof(uint32_t) * m, "training pairs"));
  NW_TRY(ctx_ensure(c, M->pj, sizeof(uint32_t) * m, "training pairs"));
  NW_TRY(ctx_ensure(c, M->target, sizeof(float) * m, "training targets"));
  NW_TRY(ctx_ensure(c, M->score16, sizeof(int16_t) * m, "training scores"));
  M->cap_pairs = m;
  return NW_OK;
}

// longest word of the dictionary (rows per word at most)
int max_len(const nw_dict* d) { return std::max<int>(1, (int)d->ws.max_len); }

cnn::Packed packed(nw_model* M, int Bw, int Tmax) {
  cnn::Packed pk;
  pk.len = M->len.as<int>();
  pk.off = M->off.as<int>();
  pk.T = rows_ptr(M);
  pk.rinfo = M->rinfo.as<int>();
  pk.rword = M->rword.as<int>();
  pk.Bw = Bw;
  pk.Tmax = Tmax;
  return pk;
}

cnn::WordSrc word_src(const WordSet& ws, uint32_t shift, const uint32_t* widx) {
  cnn::WordSrc s;
  s.widx = widx;
  s.rank = ws.rank.as<uint32_t>();
  s.slen = ws.slen.as<uint8_t>();
  s.aoff = ws.aoff.as<uint32_t>();
  s.a_enc = ws.a_enc.as<uint32_t>();
  s.shift = shift;
  s.n = ws.n;
  return s;
}

// embeddings of Bw words of `ws` (M->widx), packed into at most Tmax rows, into M->E
nw_status forward(nw_model* M, const WordSet& ws, uint32_t shift, int Bw, int Tmax, cudaStream_t s) {
  nw_ctx* c = M->ctx;
  const cnn::Layout& L = M->L;
  const float* W = fptr(M->params);
  const cnn::Packed pk = packed(M, Bw, Tmax);
  cnn::PackBufs pb{M->len.as<int>(), M->off.as<int>(), rows_ptr(M), M->rinfo.as<int>(), M->rword.as<int>(),
                   M->codes.as<int32_t>()};
  NW_CK(cnn::pack_words(word_src(ws, shift, M->widx.as<uint32_t>()), Bw, Tmax, W + L.emb, pb, fptr(M->X0),
                        err_ptr(M), M->alphabet, s));
  cnn::Epi e;
  e.relu = true;
  e.err = err_ptr(M);
  e.bias = W + L.b1;
  NW_CK(cnn::conv_fwd(fptr(M->X0), cnn::kEmb, W + L.W1, cnn::kCh, pk, fptr(M->Y1), e, s));
  e.bias = W + L.b2;
  NW_CK(cnn::conv_fwd(fptr(M->Y1), cnn::kCh, W + L.W2, cnn::kCh, pk, fptr(M->Y2), e, s));
  e.bias = W + L.b3;
  NW_CK(cnn::conv_fwd(fptr(M->Y2), cnn::kCh, W + L.W3, cnn::kCh, pk, fptr(M->Y3), e, s));
  NW_CK(cnn::mean_pool(fptr(M->Y3), pk, fptr(M->P), s));
  cnn::Epi el;
  el.bias = W + L.bl;
  el.err = err_ptr(M);
  NW_CK(cnn::lin_fwd(fptr(M->P), cnn::kCh, W + L.Wl, cnn::kOut, Bw, fptr(M->E), el, s));
  return NW_OK;
}

nw_status forward(nw_model* M, const nw_dict* d, int Bw, int Tmax, cudaStream_t s) {
  return forward(M, d->ws, d->ss.shift, Bw, Tmax, s);
}

// gradient of the pair loss (pairs = word slots 2p, 2p + 1; targets in M->target) into M->grads
nw_status backward(nw_model* M, int m, int Tmax, cudaStream_t s) {
  nw_ctx* c = M->ctx;
  const cnn::Layout& L = M->L;
  const int Bw = 2 * m;
  const float* W = fptr(M->params);
  float* G = fptr(M->grads);
  const cnn::Packed pk = packed(M, Bw, Tmax);
  const int nsm = c->sm_count;
  NW_CK(cudaMemsetAsync(G, 0, sizeof(float) * L.total, s));
  NW_CK(cnn::pair_loss(fptr(M->E), fptr(M->target), m, fptr(M->dE), loss_ptr(M), s));
  NW_CK(cnn::lin_dw(fptr(M->dE), cnn::kOut, fptr(M->P), cnn::kCh, Bw, G + L.Wl, nsm, s));
  NW_CK(cnn::col_sum(fptr(M->dE), Bw, nullptr, cnn::kOut, G + L.bl, s));
  NW_CK(cnn::lin_dx(fptr(M->dE), cnn::kOut, W + L.Wl, cnn::kCh, Bw, fptr(M->dP), s));
  NW_CK(cnn::mean_pool_bwd(fptr(M->dP), fptr(M->Y3), pk, fptr(M->dYa), s));
  // layer 3: dYa = dY3
  NW_CK(cnn::conv_dw(fptr(M->dYa), cnn::kCh, fptr(M->Y2), cnn::kCh, pk, G + L.W3, nsm, s));
  NW_CK(cnn::col_sum(fptr(M->dYa), Tmax, pk.T, cnn::kCh, G + L.b3, s));
  cnn::Epi e;
  e.gate = fptr(M->Y2);
  NW_CK(cnn::conv_dx(fptr(M->dYa), cnn::kCh, W + L.W3, cnn::kCh, pk, fptr(M->dYb), e, s));
  // layer 2: dYb = dY2
  NW_CK(cnn::conv_dw(fptr(M->dYb), cnn::kCh, fptr(M->Y1), cnn::kCh, pk, G + L.W2, nsm, s));
  NW_CK(cnn::col_sum(fptr(M->dYb), Tmax, pk.T, cnn::kCh, G + L.b2, s));
  e.gate = fptr(M->Y1);
  NW_CK(cnn::conv_dx(fptr(M->dYb), cnn::kCh, W + L.W2, cnn::kCh, pk, fptr(M->dYa), e, s));
  // layer 1: dYa = dY1
  NW_CK(cnn::conv_dw(fptr(M->dYa), cnn::kCh, fptr(M->X0), cnn::kEmb, pk, G + L.W1, nsm, s));
  NW_CK(cnn::col_sum(fptr(M->dYa), Tmax, pk.T, cnn::kCh, G + L.b1, s));
  e.gate = nullptr;
  NW_CK(cnn::conv_dx(fptr(M->dYa), cnn::kCh, W + L.W1, cnn::kEmb, pk, fptr(M->dX0), e, s));
  NW_CK(cnn::emb_scatter(fptr(M->dX0), M->codes.as<int32_t>(), pk, G + L.emb, s));
  return NW_OK;
}

nw_status check_err(nw_model* M, cudaStream_t s) {
  nw_ctx* c = M->ctx;
  uint32_t err = 0;
  NW_CK(cudaMemcpyAsync(&err, err_ptr(M), sizeof err, cudaMemcpyDeviceToHost, s));
  NW_CK(cudaStreamSynchronize(s));
  if (err) {
    NW_CK(cudaMemsetAsync(err_ptr(M), 0, sizeof(uint32_t), s));
    if (err & kErrWait) return set_err(c, NW_ETIMEOUT, "a pipeline wait on the device ran out");
    return set_err(c, NW_EINVAL, "invalid word index or code in the input");
  }
  return NW_OK;
}

nw_status check_model_dict(nw_model* M, nw_dict* d) {
  nw_ctx* c = M->ctx;
  if (d->ctx != c) return set_err(c, NW_EINVAL, "the dictionary belongs to another context");
  if (d->alphabet > M->alphabet)
    return set_err(c, NW_EINVAL, "dictionary alphabet %u exceeds the model's %u", d->alphabet, M->alphabet);
  // the dictionary's uploads ran on the context stream
  NW_CK(cudaStreamSynchronize(c->stream));
  return NW_OK;
}

// copy n elements of T between host/device according to `dev`
template <class T>
nw_status copy_in(nw_ctx* c, T* dst, const T* src, size_t n, bool dev, cudaStream_t s) {
  if (n) NW_CK(cudaMemcpyAsync(dst, src, sizeof(T) * n, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  return NW_OK;
}
template <class T>
nw_status copy_out(nw_ctx* c, T* dst, const T* src, size_t n, bool dev, cudaStream_t s) {
  if (n) NW_CK(cudaMemcpyAsync(dst, src, sizeof(T) * n, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  return NW_OK;
}

uint64_t splitmix64_next(uint64_t& st) {
  uint64_t z = (st += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// embeddings of all n words into M->Eall (n x 64): chunks of consecutive
// sorted positions (words of similar length), each at most kMaxRowsPerPass
// packed rows, scattered back to original order
nw_status embed_all(nw_model* M, const WordSet& ws, uint32_t shift, cudaStream_t s) {
  nw_ctx* c = M->ctx;
  const uint32_t n = ws.n;
  const Buckets& bk = ws.bk;
  // chunk boundaries on the host from the bucket table
  std::vector<std::pair<uint32_t, uint32_t>> chunks;  // (first sorted position, words)
  int max_words = 1;
  {
    uint32_t p0 = 0;
    uint64_t rows = 0;
    for (int Lb = 0; Lb < kBuckets; ++Lb) {
      for (uint32_t k = 0; k < bk.count[Lb]; ++k) {
        const uint32_t p = bk.start[Lb] + k;
        if (rows + (uint64_t)Lb > (uint64_t)kMaxRowsPerPass || p - p0 >= (uint32_t)kMaxRowsPerPass) {
          chunks.push_back({p0, p - p0});
          max_words = std::max<int>(max_words, (int)(p - p0));
          p0 = p;
          rows = 0;
        }
        rows += (uint64_t)Lb;
      }
    }
    if (n > p0) {
      chunks.push_back({p0, n - p0});
      max_words = std::max<int>(max_words, (int)(n - p0));
    }
  }
  NW_TRY(ensure_scratch(M, max_words, kMaxRowsPerPass));
  NW_TRY(ctx_ensure(c, M->Eall, sizeof(float) * std::max<size_t>(1, (size_t)n * cnn::kOut), "embeddings"));
  for (const auto& ch : chunks) {
    const int Bw = (int)ch.second;
    NW_CK(cnn::take(ws.perm.as<uint32_t>(), ch.first, Bw, M->widx.as<uint32_t>(), s));
    NW_TRY(forward(M, ws, shift, Bw, kMaxRowsPerPass, s));
    NW_CK(cnn::scatter_rows(fptr(M->E), M->widx.as<uint32_t>(), Bw, fptr(M->Eall), s));
  }
  return NW_OK;
}

nw_status embed_all(nw_model* M, nw_dict* d, cudaStream_t s) { return embed_all(M, d->ws, d->ss.shift, s); }

// the dictionary's encoded words as the pairs kernel reads them
PairsParams pairs_params(const nw_dict* d, uint32_t* err) {
  PairsParams P{};
  P.n = d->ws.n;
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
  P.err = err;
  return P;
}

// candidate rescoring + selection on the model's or context's buffers
nw_status rescore_select(nw_ctx* c, nw_dict* d, const uint32_t* cand, uint32_t C, uint32_t k, DevBuf& score_buf,
                         uint32_t* out_idx, int16_t* out_score, uint32_t* err, cudaStream_t s) {
  const uint32_t n = d->ws.n;
  // scores, then the length-sorted candidates they belong to and the work lists
  NW_TRY(ctx_ensure(c, score_buf, prop::rescore_scratch_bytes(n, C), "candidate scores"));
  int32_t* score = score_buf.as<int32_t>();
  uint32_t* sorted = nullptr;
  NW_CK(prop::rescore_sorted(pairs_params(d, err), cand, C, (int)d->ws.max_len, score, &sorted, s));
  NW_CK(prop::select_topk(sorted, score, n, C, k, out_idx, out_score, s));
  return NW_OK;
}

// The exhaustive (k + 1)-long lists of the dictionary's words with at least
// M->exact_len symbols (their sorted positions p0 .. n - 1) into M->xidx /
// M->xscore, on the context's stream, synchronised; *m receives their number
// and *ms the pass's time.  splice_long_rows then puts them over the proposal
// lists.
nw_status exact_long_rows(nw_model* M, nw_dict* d, uint32_t k, uint32_t* m_out, float* ms) {
  *ms = 0.f;
  *m_out = 0;
  nw_ctx* c = M->ctx;
  const uint32_t L0 = M->exact_len;
  if (L0 == 0) return NW_OK;
  const Buckets& bk = d->ws.bk;
  const uint32_t n = d->ws.n, p0 = bk.start[L0], m = n - p0;
  if (m == 0) return NW_OK;
  if (k + 1 > NW_MAX_K) return set_err(c, NW_EINVAL, "k must be below %d on the exact path", NW_MAX_K);
  std::vector<uint32_t> offs(m + 1, 0u);
  uint32_t w = 0;
  for (int Lb = (int)L0; Lb < kBuckets; ++Lb)
    for (uint32_t r = 0; r < bk.count[Lb]; ++r, ++w) offs[w + 1] = offs[w] + (uint32_t)Lb;
  const uint32_t total = offs[m];
  NW_TRY(ctx_ensure(c, M->xcodes, std::max<size_t>(16, total), "long-word codes"));
  NW_TRY(ctx_ensure(c, M->xoffs, sizeof(uint32_t) * (m + 1), "long-word offsets"));
  NW_TRY(ctx_ensure(c, M->xidx, sizeof(uint32_t) * (size_t)m * (k + 1), "long-word lists"));
  NW_TRY(ctx_ensure(c, M->xscore, sizeof(int16_t) * (size_t)m * (k + 1), "long-word lists"));
  cudaStream_t cs = c->stream;
  cudaEvent_t ev[2];
  for (auto& e : ev) NW_CK(cudaEventCreate(&e));
  struct FreeEv {
    cudaEvent_t* e;
    ~FreeEv() {
      cudaEventDestroy(e[0]);
      cudaEventDestroy(e[1]);
    }
  } fe{ev};
  NW_CK(cudaEventRecord(ev[0], cs));
  NW_CK(cudaMemcpyAsync(M->xoffs.p, offs.data(), sizeof(uint32_t) * (m + 1), cudaMemcpyHostToDevice, cs));
  if (total)
    extract_codes_kernel<<<(total + 255) / 256, 256, 0, cs>>>(d->ws.a_enc.as<uint32_t>(), bk.aenc_base[L0], total,
                                                            d->ss.shift, M->xcodes.as<uint8_t>());
  NW_CK(cudaGetLastError());
  // as nw_query with k + 1 neighbours (the word itself is among them); returns synchronised
  NW_TRY(query_impl(d, M->xcodes.as<uint8_t>(), M->xoffs.as<uint32_t>(), m, k + 1, M->xidx.as<uint32_t>(),
                    M->xscore.as<int16_t>(), NW_DEVICE_PTRS));
  NW_CK(cudaEventRecord(ev[1], cs));
  NW_CK(cudaEventSynchronize(ev[1]));
  NW_CK(cudaEventElapsedTime(ms, ev[0], ev[1]));
  *m_out = m;
  return NW_OK;
}

// the m exhaustive lists of exact_long_rows over the proposal lists in
// out_idx / out_score (device, n x k), on stream s after the work queued there
nw_status splice_long_rows(nw_model* M, nw_dict* d, uint32_t m, uint32_t k, uint32_t* out_idx, int16_t* out_score,
                           cudaStream_t s) {
  nw_ctx* c = M->ctx;
  if (m == 0) return NW_OK;
  const uint32_t p0 = d->ws.n - m;
  splice_exact_kernel<<<(m + 127) / 128, 128, 0, s>>>(M->xidx.as<uint32_t>(), M->xscore.as<int16_t>(), m, k,
                                                       d->ws.perm.as<uint32_t>(), p0, out_idx, out_score);
  NW_CK(cudaGetLastError());
  return NW_OK;
}

}  // namespace

namespace nw {
namespace prop {
nw_ctx* model_ctx(const nw_model* M) { return M->ctx; }
}  // namespace prop
}  // namespace nw

extern "C" {

nw_status nw_model_create(nw_ctx* c, uint32_t alphabet, uint64_t seed, nw_model** out) {
  if (!out) return NW_EINVAL;
  *out = nullptr;
  NW_ENTER(c);
  if (alphabet == 0 || alphabet > 256) return set_err(c, NW_EINVAL, "alphabet must be in [1, 256]");
  nw_model* M = new nw_model();
  M->ctx = c;
  M->alphabet = alphabet;
  M->L = cnn::layout(alphabet);
  auto fail = [&](nw_status st) {
    const std::string msg = c->err;
    model_free_buffers(M);
    if (M->stream) cudaStreamDestroy(M->stream);
    delete M;
    c->err = msg;
    return st;
  };
  if (cudaStreamCreateWithFlags(&M->stream, cudaStreamNonBlocking) != cudaSuccess)
    return fail(cuda_fail(c, cudaGetLastError(), "cudaStreamCreateWithFlags"));
  const size_t pb = sizeof(float) * M->L.total;
  nw_status st = ctx_alloc(c, M->params, pb, "model parameters");
  if (st == NW_OK) st = ctx_alloc(c, M->grads, pb, "model gradients");
  if (st == NW_OK) st = ctx_alloc(c, M->adam_m, pb, "Adam moments");
  if (st == NW_OK) st = ctx_alloc(c, M->adam_v, pb, "Adam moments");
  if (st == NW_OK) st = ctx_alloc(c, M->small, 64, "model counters");
  if (st != NW_OK) return fail(st);
  // initial parameters from one SplitMix64 stream, block by block
  std::vector<float> h(M->L.total, 0.f);
  uint64_t state = seed;
  auto uniform = [&](float a) {
    const double u = (double)(splitmix64_next(state) >> 11) * (1.0 / 9007199254740992.0);  // [0, 1)
    return (float)((2.0 * u - 1.0) * a);
  };
  const cnn::Layout& L = M->L;
  for (uint64_t x = L.emb; x < L.W1; ++x) h[x] = uniform((float)std::sqrt(3.0));
  for (uint64_t x = L.W1; x < L.b1; ++x) h[x] = uniform((float)std::sqrt(6.0 / (3 * cnn::kEmb)));
  for (uint64_t x = L.W2; x < L.b2; ++x) h[x] = uniform((float)std::sqrt(6.0 / (3 * cnn::kCh)));
  for (uint64_t x = L.W3; x < L.b3; ++x) h[x] = uniform((float)std::sqrt(6.0 / (3 * cnn::kCh)));
  for (uint64_t x = L.Wl; x < L.bl; ++x) h[x] = uniform((float)(0.1 * std::sqrt(6.0 / cnn::kCh)));
  cudaError_t e = cudaMemcpy(M->params.p, h.data(), pb, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(M->adam_m.p, 0, pb);
  if (e == cudaSuccess) e = cudaMemset(M->adam_v.p, 0, pb);
  if (e == cudaSuccess) e = cudaMemset(M->small.p, 0, 64);
  if (e != cudaSuccess) return fail(cuda_fail(c, e, "model initialisation"));
  c->models.insert(M);
  *out = M;
  return NW_OK;
}

void nw_model_free(nw_model* M) {
  if (!M) return;
  nw_ctx* c = M->ctx;
  cudaSetDevice(c->device);
  if (M->stream) {
    cudaStreamSynchronize(M->stream);
    cudaStreamDestroy(M->stream);
  }
  model_free_buffers(M);
  c->models.erase(M);
  delete M;
}

uint64_t nw_model_param_count(const nw_model* M) { return M ? M->L.total : 0; }

nw_status nw_model_get_params(nw_model* M, float* params, uint32_t flags) {
  if (!M) return NW_EINVAL;
  nw_ctx* c = M->ctx;
  NW_ENTER(c);
  if (!params) return set_err(c, NW_EINVAL, "null parameter buffer");
  NW_TRY(copy_out(c, params, fptr(M->params), M->L.total, flags & NW_DEVICE_PTRS, M->stream));
  NW_CK(cudaStreamSynchronize(M->stream));
  return NW_OK;
}

nw_status nw_model_set_params(nw_model* M, const float* params, uint32_t flags) {
  if (!M) return NW_EINVAL;
  nw_ctx* c = M->ctx;
  NW_ENTER(c);
  if (!params) return set_err(c, NW_EINVAL, "null parameter buffer");
  NW_TRY(copy_in(c, fptr(M->params), params, M->L.total, flags & NW_DEVICE_PTRS, M->stream));
  NW_CK(cudaMemsetAsync(M->adam_m.p, 0, M->adam_m.bytes, M->stream));
  NW_CK(cudaMemsetAsync(M->adam_v.p, 0, M->adam_v.bytes, M->stream));
  NW_CK(cudaMemsetAsync(step_ptr(M), 0, sizeof(uint32_t), M->stream));
  M->steps_done = 0;
  ++M->gen;
  NW_CK(cudaStreamSynchronize(M->stream));
  return NW_OK;
}

nw_status nw_model_embed(nw_model* M, nw_dict* d, float* out, uint32_t flags) {
  if (!M || !d) return NW_EINVAL;
  nw_ctx* c = M->ctx;
  NW_ENTER(c);
  if (!out) return set_err(c, NW_EINVAL, "null output buffer");
  NW_TRY(check_model_dict(M, d));
  NW_TRY(embed_all(M, d, M->stream));
  NW_TRY(copy_out(c, out, fptr(M->Eall), (size_t)d->ws.n * cnn::kOut, flags & NW_DEVICE_PTRS, M->stream));
  return check_err(M, M->stream);
}

nw_status nw_model_loss_grad(nw_model* M, nw_dict* d, const uint32_t* pi, const uint32_t* pj, const float* target,
                             uint32_t m, float* loss, float* grad, uint32_t flags) {
  if (!M || !d) return NW_EINVAL;
  nw_ctx* c = M->ctx;
  NW_ENTER(c);
  if (!pi || !pj || !target || m == 0) return set_err(c, NW_EINVAL, "need m >= 1 pairs and their targets");
  if (m > (1u << 20)) return set_err(c, NW_EINVAL, "at most 2^20 pairs per call");
  NW_TRY(check_model_dict(M, d));
  const bool dev = flags & NW_DEVICE_PTRS;
  cudaStream_t s = M->stream;
  const int Tmax = (int)(2 * m) * max_len(d);
  NW_TRY(ensure_pairs(M, m));
  NW_TRY(ensure_scratch(M, (int)(2 * m), Tmax));
  NW_TRY(copy_in(c, M->pi.as<uint32_t>(), pi, m, dev, s));
  NW_TRY(copy_in(c, M->pj.as<uint32_t>(), pj, m, dev, s));
  NW_TRY(copy_in(c, fptr(M->target), target, m, dev, s));
  NW_CK(cnn::interleave_pairs(M->pi.as<uint32_t>(), M->pj.as<uint32_t>(), (int)m, M->widx.as<uint32_t>(), s));
  NW_CK(cudaMemsetAsync(loss_ptr(M), 0, sizeof(float), s));
  NW_TRY(forward(M, d, (int)(2 * m), Tmax, s));
  NW_TRY(backward(M, (int)m, Tmax, s));
  if (grad) NW_TRY(copy_out(c, grad, fptr(M->grads), M->L.total, dev, s));
  float h_loss = 0.f;
  NW_CK(cudaMemcpyAsync(&h_loss, loss_ptr(M), sizeof(float), cudaMemcpyDeviceToHost, s));
  NW_TRY(check_err(M, s));
  if (loss) *loss = h_loss;
  return NW_OK;
}

nw_status nw_model_train(nw_model* M, nw_dict* d, const nw_train_config* cfg, const uint32_t* nbr, uint32_t knb,
                         float* losses, uint32_t flags) {
  if (!M || !d || !cfg) return NW_EINVAL;
  nw_ctx* c = M->ctx;
  NW_ENTER(c);
  const uint32_t n = d->ws.n;
  if (n < 2) return set_err(c, NW_EINVAL, "training needs at least 2 words");
  if (cfg->batch_pairs == 0 || cfg->batch_pairs > 65536) return set_err(c, NW_EINVAL, "batch_pairs must be in [1, 65536]");
  if (!(cfg->nbr_fraction >= 0.f && cfg->nbr_fraction <= 1.f)) return set_err(c, NW_EINVAL, "nbr_fraction in [0, 1]");
  if (!(cfg->long_fraction >= 0.f && cfg->long_fraction <= 1.f)) return set_err(c, NW_EINVAL, "long_fraction in [0, 1]");
  if (cfg->long_fraction > 0.f && cfg->long_len > (uint32_t)kMaxLen)
    return set_err(c, NW_EINVAL, "long_len must be at most %d", kMaxLen);
  if (!(cfg->raw_scale >= 0.f)) return set_err(c, NW_EINVAL, "raw_scale must be >= 0");
  if (!(cfg->clip_norm >= 0.f) || !(cfg->lr_final >= 0.f)) return set_err(c, NW_EINVAL, "clip_norm, lr_final >= 0");
  if (nbr && knb == 0) return set_err(c, NW_EINVAL, "neighbour lists need knb >= 1");
  if (cfg->steps == 0) return NW_OK;
  ++M->gen;  // the parameters change from here on
  NW_TRY(check_model_dict(M, d));
  const bool dev = flags & NW_DEVICE_PTRS;
  cudaStream_t s = M->stream;
  const uint32_t m = cfg->batch_pairs;
  const int Tmax = (int)(2 * m) * max_len(d);
  NW_TRY(ensure_pairs(M, m));
  NW_TRY(ensure_scratch(M, (int)(2 * m), Tmax));
  DevBuf loss_buf;
  NW_TRY(ctx_alloc(c, loss_buf, sizeof(float) * cfg->steps, "training losses"));
  struct Free {
    nw_ctx* c;
    DevBuf& b;
    ~Free() { ctx_free(c, b); }
  } free_losses{c, loss_buf};
  const uint32_t* d_nbr = nullptr;
  if (nbr) {
    NW_TRY(ctx_ensure(c, M->nbr, sizeof(uint32_t) * (size_t)n * knb, "neighbour lists"));
    NW_TRY(copy_in(c, M->nbr.as<uint32_t>(), nbr, (size_t)n * knb, dev, s));
    d_nbr = M->nbr.as<uint32_t>();
  }
  NW_CK(cudaMemsetAsync(loss_ptr(M), 0, sizeof(float), s));
  NW_CK(cudaStreamSynchronize(s));

  cnn::PairDraw pd;
  pd.seed = cfg->seed;
  pd.step = step_ptr(M);
  pd.n = n;
  pd.m = m;
  pd.nbr = d_nbr;
  pd.knb = knb;
  pd.n_nbr = d_nbr ? (uint32_t)std::lround((double)cfg->nbr_fraction * m) : 0u;
  pd.perm = d->ws.perm.as<uint32_t>();
  pd.long0 = 0;
  pd.nlong = 0;
  pd.long_thresh = 0;
  if (cfg->long_fraction > 0.f && cfg->long_len <= (uint32_t)kMaxLen) {
    pd.long0 = d->ws.bk.start[cfg->long_len];
    pd.nlong = n - pd.long0;
    pd.long_thresh = (uint32_t)std::lround((double)cfg->long_fraction * (double)(1u << 20));
  }
  PairsParams pp = pairs_params(d, err_ptr(M));
  pp.pi = M->pi.as<uint32_t>();
  pp.pj = M->pj.as<uint32_t>();
  pp.m = m;
  pp.out = M->score16.as<int16_t>();

  cnn::AdamCfg ac;
  ac.lr = cfg->lr;
  ac.lr_final = cfg->lr_final > 0.f ? cfg->lr_final : cfg->lr;
  ac.b1 = cfg->beta1;
  ac.b2 = cfg->beta2;
  ac.eps = cfg->eps;
  ac.clip = cfg->clip_norm;
  ac.sumsq = sumsq_ptr(M);
  ac.step0 = M->steps_done;
  ac.nsteps = cfg->steps;

  // one step, captured once and replayed
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  NW_CK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  nw_status st = NW_OK;
  auto step_body = [&]() -> nw_status {
    NW_CK(cnn::draw_pairs(pd, M->pi.as<uint32_t>(), M->pj.as<uint32_t>(), M->widx.as<uint32_t>(), s));
    NW_CK(launch_pairs(pp, s));
    NW_CK(cnn::pair_targets(M->score16.as<int16_t>(), M->pi.as<uint32_t>(), M->pj.as<uint32_t>(),
                            d->ws.rank.as<uint32_t>(), d->ws.slen.as<uint8_t>(), (int)m, cfg->raw_scale,
                            fptr(M->target), s));
    NW_TRY(forward(M, d, (int)(2 * m), Tmax, s));
    NW_TRY(backward(M, (int)m, Tmax, s));
    NW_CK(cnn::bump_step(step_ptr(M), s));
    NW_CK(cnn::adam(fptr(M->params), fptr(M->grads), fptr(M->adam_m), fptr(M->adam_v), M->L.total, step_ptr(M),
                    ac, s));
    NW_CK(cnn::record_loss(loss_ptr(M), loss_buf.as<float>(), step_ptr(M), M->steps_done, cfg->steps, s));
    return NW_OK;
  };
  st = step_body();
  const cudaError_t ec = cudaStreamEndCapture(s, &graph);
  if (st != NW_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (ec != cudaSuccess) return cuda_fail(c, ec, "cudaStreamEndCapture");
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) return cuda_fail(c, e, "cudaGraphInstantiate");
  for (uint32_t x = 0; x < cfg->steps && e == cudaSuccess; ++x) e = cudaGraphLaunch(exec, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  cudaGraphExecDestroy(exec);
  if (e != cudaSuccess) return cuda_fail(c, e, "training graph");
  M->steps_done += cfg->steps;
  if (losses) NW_TRY(copy_out(c, losses, loss_buf.as<float>(), cfg->steps, dev, s));
  return check_err(M, s);
}

nw_status nw_quantize_embeddings(nw_ctx* c, const float* E, uint32_t n, int8_t* q, int32_t* bias, float* scale,
                                 uint32_t flags) {
  NW_ENTER(c);
  if (!E || !q || !bias || !scale) return set_err(c, NW_EINVAL, "null pointer argument");
  const bool dev = flags & NW_DEVICE_PTRS;
  cudaStream_t s = c->stream;
  const size_t cnt = (size_t)n * NW_EMBED_DIM;
  DevBuf dE, dq, db, dsmall;
  struct Free {
    nw_ctx* c;
    DevBuf* b[4];
    ~Free() {
      for (DevBuf* x : b) ctx_free(c, *x);
    }
  } fr{c, {&dE, &dq, &db, &dsmall}};
  const float* srcE = E;
  int8_t* dstq = q;
  int32_t* dstb = bias;
  if (!dev) {
    NW_TRY(ctx_alloc(c, dE, sizeof(float) * std::max<size_t>(1, cnt), "embeddings"));
    NW_TRY(ctx_alloc(c, dq, std::max<size_t>(1, cnt), "quantised embeddings"));
    NW_TRY(ctx_alloc(c, db, sizeof(int32_t) * std::max<size_t>(1, n), "quantised biases"));
    NW_TRY(copy_in(c, dE.as<float>(), E, cnt, false, s));
    srcE = dE.as<float>();
    dstq = dq.as<int8_t>();
    dstb = db.as<int32_t>();
  }
  NW_TRY(ctx_alloc(c, dsmall, 16, "quantisation scratch"));
  float* dscale = reinterpret_cast<float*>(dsmall.as<char>() + 4);
  NW_CK(prop::quantize(srcE, n, dsmall.as<unsigned int>(), dstq, nullptr, dstb, dscale, s));
  if (!dev) {
    NW_TRY(copy_out(c, q, dstq, cnt, false, s));
    NW_TRY(copy_out(c, bias, dstb, n, false, s));
  }
  NW_TRY(copy_out(c, scale, dscale, 1, dev, s));
  NW_CK(cudaStreamSynchronize(s));
  return NW_OK;
}

nw_status nw_dot_topk(nw_ctx* c, const int8_t* q, const int32_t* bias, uint32_t n, uint32_t C, uint32_t* idx,
                      int32_t* val, uint32_t flags) {
  NW_ENTER(c);
  if (!q || !idx || !val) return set_err(c, NW_EINVAL, "null pointer argument");
  if (C == 0 || C > NW_MAX_CANDIDATES) return set_err(c, NW_EINVAL, "C must be in [1, %d]", NW_MAX_CANDIDATES);
  if (n == 0) return NW_OK;
  const bool dev = flags & NW_DEVICE_PTRS;
  cudaStream_t s = c->stream;
  const size_t cnt = (size_t)n * NW_EMBED_DIM, outc = (size_t)n * C;
  DevBuf dq, db, qb, buf, oi, od;
  struct Free {
    nw_ctx* c;
    DevBuf* b[6];
    ~Free() {
      for (DevBuf* x : b) ctx_free(c, *x);
    }
  } fr{c, {&dq, &db, &qb, &buf, &oi, &od}};
  const int8_t* srcq = q;
  const int32_t* srcb = bias;
  if (!dev) {
    NW_TRY(ctx_alloc(c, dq, cnt, "quantised embeddings"));
    NW_TRY(copy_in(c, dq.as<int8_t>(), q, cnt, false, s));
    srcq = dq.as<int8_t>();
  }
  // the kernel reads biases in 16-byte chunks: host or unaligned device biases are copied
  if (bias && (!dev || (reinterpret_cast<uintptr_t>(bias) & 15u))) {
    NW_TRY(ctx_alloc(c, db, sizeof(int32_t) * n, "biases"));
    NW_CK(cudaMemcpyAsync(db.p, bias, sizeof(int32_t) * n, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          s));
    srcb = db.as<int32_t>();
  }
  NW_TRY(ctx_alloc(c, qb, prop::dot_topk_qb_bytes(n), "bf16 embeddings"));
  NW_TRY(ctx_alloc(c, buf, prop::dot_topk_buffer_bytes(n, C), "candidate buffers"));
  const bool locality = flags & NW_LOCALITY_ORDER;
  DevBuf oq, ob, op, osc;
  struct FreeOrder {
    nw_ctx* c;
    DevBuf* b[4];
    ~FreeOrder() {
      for (DevBuf* x : b) ctx_free(c, *x);
    }
  } fro{c, {&oq, &ob, &op, &osc}};
  if (locality) {
    NW_TRY(ctx_alloc(c, oq, prop::dot_topk_qb_bytes(n), "bf16 embeddings in sweep order"));
    NW_TRY(ctx_alloc(c, ob, sizeof(int32_t) * n, "biases in sweep order"));
    NW_TRY(ctx_alloc(c, op, sizeof(uint32_t) * prop::sweep_perm_entries(n), "sweep order"));
    NW_TRY(ctx_alloc(c, osc, prop::sweep_order_bytes(n), "sweep order scratch"));
  }
  uint32_t* out_i = idx;
  int32_t* out_v = val;
  if (!dev) {
    NW_TRY(ctx_alloc(c, oi, sizeof(uint32_t) * outc, "candidate lists"));
    NW_TRY(ctx_alloc(c, od, sizeof(int32_t) * outc, "candidate lists"));
    out_i = oi.as<uint32_t>();
    out_v = od.as<int32_t>();
  }
  uint32_t* derr = prop::dot_topk_err_word(buf.as<uint64_t>(), n);
  NW_CK(cudaMemsetAsync(derr, 0, sizeof(uint32_t), s));
  NW_CK(prop::widen(srcq, n, qb.as<__nv_bfloat16>(), s));
  if (locality) {
    NW_CK(prop::sweep_order(qb.as<__nv_bfloat16>(), srcb, nullptr, nullptr, n, osc.p, op.as<uint32_t>(),
                            oq.as<__nv_bfloat16>(), srcb ? ob.as<int32_t>() : nullptr, s));
    NW_CK(prop::dot_topk(oq.as<__nv_bfloat16>(), srcb ? ob.as<int32_t>() : nullptr, n, C, buf.as<uint64_t>(), out_i,
                         out_v, derr, s, dot_debug(c), op.as<uint32_t>()));
  } else {
    NW_CK(prop::dot_topk(qb.as<__nv_bfloat16>(), srcb, n, C, buf.as<uint64_t>(), out_i, out_v, derr, s,
                         dot_debug(c)));
  }
  NW_TRY(check_device_flags(c, derr));
  if (!dev) {
    NW_TRY(copy_out(c, idx, out_i, outc, false, s));
    NW_TRY(copy_out(c, val, out_v, outc, false, s));
  }
  NW_CK(cudaStreamSynchronize(s));
  return NW_OK;
}

nw_status nw_rescore_topk(nw_dict* d, const uint32_t* cand, uint32_t C, uint32_t k, uint32_t* nbr_idx,
                          int16_t* nbr_score, uint32_t flags) {
  if (!d) return NW_EINVAL;
  nw_ctx* c = d->ctx;
  NW_ENTER(c);
  if (!cand || !nbr_idx || !nbr_score) return set_err(c, NW_EINVAL, "null pointer argument");
  if (C == 0 || C > NW_MAX_CANDIDATES) return set_err(c, NW_EINVAL, "C must be in [1, %d]", NW_MAX_CANDIDATES);
  if (k == 0 || k > NW_MAX_K) return set_err(c, NW_EINVAL, "k must be in [1, %d]", NW_MAX_K);
  if (d->score_lo < INT16_MIN + 1 || d->score_hi > INT16_MAX)
    return set_err(c, NW_ERANGE, "scores [%d, %d] do not fit int16", d->score_lo, d->score_hi);
  const uint32_t n = d->ws.n;
  if (n == 0) return NW_OK;
  const bool dev = flags & NW_DEVICE_PTRS;
  cudaStream_t s = c->stream;
  DevBuf dc, sc, oi, os, small;
  struct Free {
    nw_ctx* c;
    DevBuf* b[5];
    ~Free() {
      for (DevBuf* x : b) ctx_free(c, *x);
    }
  } fr{c, {&dc, &sc, &oi, &os, &small}};
  const uint32_t* srcc = cand;
  if (!dev) {
    NW_TRY(ctx_alloc(c, dc, sizeof(uint32_t) * (size_t)n * C, "candidates"));
    NW_TRY(copy_in(c, dc.as<uint32_t>(), cand, (size_t)n * C, false, s));
    srcc = dc.as<uint32_t>();
  }
  uint32_t* out_i = nbr_idx;
  int16_t* out_s = nbr_score;
  if (!dev) {
    NW_TRY(ctx_alloc(c, oi, sizeof(uint32_t) * (size_t)n * k, "neighbour lists"));
    NW_TRY(ctx_alloc(c, os, sizeof(int16_t) * (size_t)n * k, "neighbour lists"));
    out_i = oi.as<uint32_t>();
    out_s = os.as<int16_t>();
  }
  NW_TRY(ctx_alloc(c, small, 16, "error flags"));
  NW_CK(cudaMemsetAsync(small.p, 0, 16, s));
  NW_TRY(rescore_select(c, d, srcc, C, k, sc, out_i, out_s, small.as<uint32_t>(), s));
  if (!dev) {
    NW_TRY(copy_out(c, nbr_idx, out_i, (size_t)n * k, false, s));
    NW_TRY(copy_out(c, nbr_score, out_s, (size_t)n * k, false, s));
  }
  NW_TRY(check_device_flags(c, small.as<uint32_t>()));
  return NW_OK;
}

nw_status nw_dot_topk_cross(nw_ctx* c, const int8_t* qa, uint32_t na, const int8_t* qb, const int32_t* bias,
                           uint32_t nb, uint32_t C, uint32_t* idx, int32_t* val, uint32_t flags) {
  NW_ENTER(c);
  if (!qa || !idx || !val || (nb && !qb)) return set_err(c, NW_EINVAL, "null pointer argument");
  if (C == 0 || C > NW_MAX_CANDIDATES) return set_err(c, NW_EINVAL, "C must be in [1, %d]", NW_MAX_CANDIDATES);
  if (na == 0) return NW_OK;
  const bool dev = flags & NW_DEVICE_PTRS;
  cudaStream_t s = c->stream;
  const size_t outc = (size_t)na * C;
  DevBuf dqa, dqb, db, qab, qbb, buf, oi, od;
  struct Free {
    nw_ctx* c;
    DevBuf* b[8];
    ~Free() {
      for (DevBuf* x : b) ctx_free(c, *x);
    }
  } fr{c, {&dqa, &dqb, &db, &qab, &qbb, &buf, &oi, &od}};
  const int8_t* sa = qa;
  const int8_t* sb = qb;
  const int32_t* sbias = bias;
  if (!dev) {
    NW_TRY(ctx_alloc(c, dqa, (size_t)na * NW_EMBED_DIM, "quantised rows"));
    NW_TRY(copy_in(c, dqa.as<int8_t>(), qa, (size_t)na * NW_EMBED_DIM, false, s));
    sa = dqa.as<int8_t>();
    if (nb) {
      NW_TRY(ctx_alloc(c, dqb, (size_t)nb * NW_EMBED_DIM, "quantised columns"));
      NW_TRY(copy_in(c, dqb.as<int8_t>(), qb, (size_t)nb * NW_EMBED_DIM, false, s));
      sb = dqb.as<int8_t>();
    }
  }
  // the kernel reads biases in 16-byte chunks: host or unaligned device biases are copied
  if (bias && nb && (!dev || (reinterpret_cast<uintptr_t>(bias) & 15u))) {
    NW_TRY(ctx_alloc(c, db, sizeof(int32_t) * nb, "biases"));
    NW_CK(cudaMemcpyAsync(db.p, bias, sizeof(int32_t) * nb, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                          s));
    sbias = db.as<int32_t>();
  }
  NW_TRY(ctx_alloc(c, qab, prop::dot_topk_qb_bytes(na), "bf16 rows"));
  NW_TRY(ctx_alloc(c, qbb, std::max<size_t>(128, prop::dot_topk_qb_bytes(nb)), "bf16 columns"));
  NW_TRY(ctx_alloc(c, buf, prop::dot_topk_buffer_bytes(na, nb, C), "candidate buffers"));
  uint32_t* out_i = idx;
  int32_t* out_v = val;
  if (!dev) {
    NW_TRY(ctx_alloc(c, oi, sizeof(uint32_t) * outc, "candidate lists"));
    NW_TRY(ctx_alloc(c, od, sizeof(int32_t) * outc, "candidate lists"));
    out_i = oi.as<uint32_t>();
    out_v = od.as<int32_t>();
  }
  uint32_t* derr = prop::dot_topk_err_word(buf.as<uint64_t>(), na, nb);
  NW_CK(cudaMemsetAsync(derr, 0, sizeof(uint32_t), s));
  NW_CK(prop::widen(sa, na, qab.as<__nv_bfloat16>(), s));
  NW_CK(prop::widen(sb, nb, qbb.as<__nv_bfloat16>(), s));
  NW_CK(prop::dot_topk_rect(qab.as<__nv_bfloat16>(), na, qbb.as<__nv_bfloat16>(), sbias, nb, C, false,
                            buf.as<uint64_t>(), out_i, out_v, derr, s, dot_debug(c)));
  NW_TRY(check_device_flags(c, derr));
  if (!dev) {
    NW_TRY(copy_out(c, idx, out_i, outc, false, s));
    NW_TRY(copy_out(c, val, out_v, outc, false, s));
  }
  NW_CK(cudaStreamSynchronize(s));
  return NW_OK;
}

}  // extern "C"

namespace {

// nw_proposal_query for every query word through the proposal (the context
// is held by the caller)
nw_status proposal_query_impl(nw_model* M, nw_dict* d, const uint8_t* qcodes, const uint32_t* qoffsets, uint32_t nq,
                              uint32_t C, uint32_t k, uint32_t* nbr_idx, int16_t* nbr_score, uint32_t flags) {
  nw_ctx* c = M->ctx;
  if (flags & NW_RANK_NORMALISED) return set_err(c, NW_EINVAL, "queries rank by raw score only");
  if (nq == 0) return NW_OK;
  if (!qoffsets || !nbr_idx || !nbr_score) return set_err(c, NW_EINVAL, "null pointer argument");
  if (C == 0 || C > NW_MAX_CANDIDATES) return set_err(c, NW_EINVAL, "C must be in [1, %d]", NW_MAX_CANDIDATES);
  if (k == 0 || k > NW_MAX_K) return set_err(c, NW_EINVAL, "k must be in [1, %d]", NW_MAX_K);
  NW_TRY(check_model_dict(M, d));
  const uint32_t n = d->ws.n;
  const bool dev = flags & NW_DEVICE_PTRS;
  cudaStream_t s = M->stream;

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
  NW_CK(cudaStreamSynchronize(c->stream));  // the query words were uploaded on the context stream

  // the dictionary's quantised rows, kept until the dictionary or the parameters change
  unsigned int* amax = M->prep_small.p ? M->prep_small.as<unsigned int>() : nullptr;
  if (M->prep_serial != d->serial || M->prep_gen != M->gen) {
    M->prep_serial = 0;
    NW_TRY(ctx_ensure(c, M->dQb, std::max<size_t>(128, prop::dot_topk_qb_bytes(n)), "dictionary bf16 rows"));
    NW_TRY(ctx_ensure(c, M->dqbias, sizeof(int32_t) * std::max<size_t>(1, n), "dictionary biases"));
    NW_TRY(ctx_ensure(c, M->prep_small, 16, "dictionary scale"));
    amax = M->prep_small.as<unsigned int>();
    NW_TRY(embed_all(M, d, s));
    NW_CK(prop::quantize(fptr(M->Eall), n, amax, nullptr, M->dQb.as<__nv_bfloat16>(), M->dqbias.as<int32_t>(),
                         nullptr, s));
    M->prep_serial = d->serial;
    M->prep_gen = M->gen;
  }
  // the queries, quantised on the dictionary's scale
  NW_TRY(embed_all(M, q, d->ss.shift, s));
  NW_TRY(ctx_ensure(c, M->qQb, prop::dot_topk_qb_bytes(nq), "query bf16 rows"));
  NW_CK(prop::quantize(fptr(M->Eall), nq, amax, nullptr, M->qQb.as<__nv_bfloat16>(), nullptr, nullptr, s, true));

  const size_t outc = (size_t)nq * C;
  NW_TRY(ctx_ensure(c, M->qbuf, prop::dot_topk_buffer_bytes(nq, n, C), "candidate buffers"));
  NW_TRY(ctx_ensure(c, M->qcand, sizeof(uint32_t) * outc, "candidate lists"));
  NW_TRY(ctx_ensure(c, M->qcand_dot, sizeof(int32_t) * outc, "candidate lists"));
  NW_TRY(ctx_ensure(c, M->qscore, sizeof(int32_t) * outc, "candidate scores"));
  uint32_t* derr = prop::dot_topk_err_word(M->qbuf.as<uint64_t>(), nq, n);
  NW_CK(cudaMemsetAsync(derr, 0, sizeof(uint32_t), s));
  NW_CK(prop::dot_topk_rect(M->qQb.as<__nv_bfloat16>(), nq, M->dQb.as<__nv_bfloat16>(), M->dqbias.as<int32_t>(), n,
                            C, false, M->qbuf.as<uint64_t>(), M->qcand.as<uint32_t>(), M->qcand_dot.as<int32_t>(),
                            derr, s, dot_debug(c), nullptr, nullptr, /*sorted=*/false));
  NW_CK(cudaStreamSynchronize(s));
  NW_TRY(check_device_flags(c, derr));

  // exact rescoring of (query, candidate) and the k best
  prop::CrossParams X{};
  X.QD = pairs_params(d, err_ptr(M));
  X.QD.aoff = q.aoff.as<uint32_t>();
  X.QD.a_enc = q.a_enc.as<uint32_t>();
  X.DQ = pairs_params(d, err_ptr(M));
  X.DQ.brec_w = q.brec_w.as<uint32_t>();
  X.DQ.b_rec = q.b_rec.as<uint32_t>();
  X.q_rank = q.rank.as<uint32_t>();
  X.q_slen = q.slen.as<uint8_t>();
  X.d_rank = d->ws.rank.as<uint32_t>();
  X.d_slen = d->ws.slen.as<uint8_t>();
  X.nq = nq;
  X.nd = n;
  DevBuf oi, os;
  struct Free {
    nw_ctx* c;
    DevBuf* b[2];
    ~Free() {
      for (DevBuf* x : b) ctx_free(c, *x);
    }
  } fr{c, {&oi, &os}};
  uint32_t* out_i = nbr_idx;
  int16_t* out_s = nbr_score;
  if (!dev) {
    NW_TRY(ctx_alloc(c, oi, sizeof(uint32_t) * (size_t)nq * k, "neighbour lists"));
    NW_TRY(ctx_alloc(c, os, sizeof(int16_t) * (size_t)nq * k, "neighbour lists"));
    out_i = oi.as<uint32_t>();
    out_s = os.as<int16_t>();
  }
  NW_CK(prop::cross_rescore(X, M->qcand.as<uint32_t>(), C, M->qscore.as<int32_t>(), s));
  NW_CK(prop::select_topk(M->qcand.as<uint32_t>(), M->qscore.as<int32_t>(), nq, C, k, out_i, out_s, s));
  if (!dev) {
    NW_TRY(copy_out(c, nbr_idx, out_i, (size_t)nq * k, false, s));
    NW_TRY(copy_out(c, nbr_score, out_s, (size_t)nq * k, false, s));
  }
  NW_TRY(check_err(M, s));
  return NW_OK;
}

}  // namespace

extern "C" {

nw_status nw_proposal_query(nw_model* M, nw_dict* d, const uint8_t* qcodes, const uint32_t* qoffsets, uint32_t nq,
                            uint32_t C, uint32_t k, uint32_t* nbr_idx, int16_t* nbr_score, uint32_t flags) {
  if (!M || !d) return NW_EINVAL;
  nw_ctx* c = M->ctx;
  NW_ENTER(c);
  const uint32_t L0 = M->exact_len;
  if (L0 == 0 || nq == 0 || !qoffsets || !nbr_idx || !nbr_score)
    return proposal_query_impl(M, d, qcodes, qoffsets, nq, C, k, nbr_idx, nbr_score, flags);
  if (k == 0 || k > NW_MAX_K) return set_err(c, NW_EINVAL, "k must be in [1, %d]", NW_MAX_K);
  // long query words take the exhaustive path: split the set on the host
  const bool dev = flags & NW_DEVICE_PTRS;
  std::vector<uint32_t> off(nq + 1);
  if (dev) NW_CK(cudaMemcpy(off.data(), qoffsets, sizeof(uint32_t) * (nq + 1), cudaMemcpyDeviceToHost));
  else std::memcpy(off.data(), qoffsets, sizeof(uint32_t) * (nq + 1));
  for (uint32_t q = 0; q < nq; ++q)
    if (off[q + 1] < off[q]) return set_err(c, NW_EINVAL, "query offsets must not decrease");
  const uint32_t total = off[nq] - off[0];
  std::vector<uint8_t> codes(std::max<uint32_t>(1u, total));
  if (total) {
    if (!qcodes) return set_err(c, NW_EINVAL, "null query codes");
    if (dev) NW_CK(cudaMemcpy(codes.data(), qcodes + off[0], total, cudaMemcpyDeviceToHost));
    else std::memcpy(codes.data(), qcodes + off[0], total);
  }
  std::vector<uint8_t> sc, lc;
  std::vector<uint32_t> so(1, 0u), lo(1, 0u), which;  // which: query -> (long << 31) | position in its set
  for (uint32_t q = 0; q < nq; ++q) {
    const uint32_t a = off[q] - off[0], len = off[q + 1] - off[q];
    const bool is_long = len >= L0;
    std::vector<uint8_t>& dst = is_long ? lc : sc;
    std::vector<uint32_t>& o = is_long ? lo : so;
    which.push_back((is_long ? 0x80000000u : 0u) | (uint32_t)(o.size() - 1));
    dst.insert(dst.end(), codes.begin() + a, codes.begin() + a + len);
    o.push_back((uint32_t)dst.size());
  }
  const uint32_t ns = (uint32_t)so.size() - 1, nl = (uint32_t)lo.size() - 1;
  if (sc.empty()) sc.push_back(0);
  if (lc.empty()) lc.push_back(0);
  std::vector<uint32_t> si((size_t)ns * k), li((size_t)nl * k), ri((size_t)nq * k);
  std::vector<int16_t> ss((size_t)ns * k), ls((size_t)nl * k), rs((size_t)nq * k);
  if (ns) NW_TRY(proposal_query_impl(M, d, sc.data(), so.data(), ns, C, k, si.data(), ss.data(), 0));
  if (nl) NW_TRY(query_impl(d, lc.data(), lo.data(), nl, k, li.data(), ls.data(), 0));
  for (uint32_t q = 0; q < nq; ++q) {
    const bool is_long = which[q] >> 31;
    const size_t src = (size_t)(which[q] & 0x7fffffffu) * k;
    std::memcpy(ri.data() + (size_t)q * k, (is_long ? li.data() : si.data()) + src, sizeof(uint32_t) * k);
    std::memcpy(rs.data() + (size_t)q * k, (is_long ? ls.data() : ss.data()) + src, sizeof(int16_t) * k);
  }
  if (dev) {
    NW_CK(cudaMemcpy(nbr_idx, ri.data(), sizeof(uint32_t) * ri.size(), cudaMemcpyHostToDevice));
    NW_CK(cudaMemcpy(nbr_score, rs.data(), sizeof(int16_t) * rs.size(), cudaMemcpyHostToDevice));
  } else {
    std::memcpy(nbr_idx, ri.data(), sizeof(uint32_t) * ri.size());
    std::memcpy(nbr_score, rs.data(), sizeof(int16_t) * rs.size());
  }
  return NW_OK;
}

}  // extern "C"

namespace nw {
namespace prop {

nw_status model_clone(nw_model* src, nw_ctx* c, nw_model** out) {
  *out = nullptr;
  NW_TRY(nw_model_create(c, src->alphabet, 0, out));
  nw_model* M = *out;
  cudaSetDevice(c->device);
  cudaError_t e = cudaMemcpyAsync(M->params.p, src->params.p, src->params.bytes, cudaMemcpyDeviceToDevice, M->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(M->stream);
  if (e != cudaSuccess) {
    nw_model_free(M);
    *out = nullptr;
    return cuda_fail(c, e, "copying model parameters");
  }
  M->exact_len = src->exact_len;
  M->sweep_order = src->sweep_order;
  return NW_OK;
}

}  // namespace prop
}  // namespace nw

extern "C" {

nw_status nw_proposal_set_exact_length(nw_model* M, uint32_t min_len) {
  if (!M) return NW_EINVAL;
  if (min_len > (uint32_t)kMaxLen) return set_err(M->ctx, NW_EINVAL, "min_len must be at most %d", kMaxLen);
  M->exact_len = min_len;
  return NW_OK;
}

nw_status nw_proposal_set_sweep_order(nw_model* M, int locality) {
  if (!M) return NW_EINVAL;
  M->sweep_order = locality != 0;
  return NW_OK;
}

nw_status nw_proposal_topk(nw_model* M, nw_dict* d, uint32_t C, uint32_t k, uint32_t* nbr_idx, int16_t* nbr_score,
                           nw_proposal_profile* prof, uint32_t flags) {
  if (!M || !d) return NW_EINVAL;
  nw_ctx* c = M->ctx;
  NW_ENTER(c);
  if (!nbr_idx || !nbr_score) return set_err(c, NW_EINVAL, "null output buffer");
  if (C == 0 || C > NW_MAX_CANDIDATES) return set_err(c, NW_EINVAL, "C must be in [1, %d]", NW_MAX_CANDIDATES);
  if (k == 0 || k > NW_MAX_K) return set_err(c, NW_EINVAL, "k must be in [1, %d]", NW_MAX_K);
  if (d->score_lo < INT16_MIN + 1 || d->score_hi > INT16_MAX)
    return set_err(c, NW_ERANGE, "scores [%d, %d] do not fit int16", d->score_lo, d->score_hi);
  NW_TRY(check_model_dict(M, d));
  const uint32_t n = d->ws.n;
  if (n == 0) return NW_OK;
  const bool dev = flags & NW_DEVICE_PTRS;
  cudaStream_t s = M->stream;
  const size_t outc = (size_t)n * C;
  NW_TRY(ctx_ensure(c, M->Qb, prop::dot_topk_qb_bytes(n), "bf16 embeddings"));
  NW_TRY(ctx_ensure(c, M->qbias, sizeof(int32_t) * (size_t)n, "quantised biases"));
  NW_TRY(ctx_ensure(c, M->topbuf, prop::dot_topk_buffer_bytes(n, C), "candidate buffers"));
  NW_TRY(ctx_ensure(c, M->cand, sizeof(uint32_t) * outc, "candidate lists"));
  NW_TRY(ctx_ensure(c, M->cand_dot, sizeof(int32_t) * outc, "candidate lists"));
  if (M->sweep_order) {
    NW_TRY(ctx_ensure(c, M->oQb, prop::dot_topk_qb_bytes(n), "bf16 embeddings in sweep order"));
    NW_TRY(ctx_ensure(c, M->obias, sizeof(int32_t) * (size_t)n, "quantised biases in sweep order"));
    NW_TRY(ctx_ensure(c, M->operm, sizeof(uint32_t) * prop::sweep_perm_entries(n), "sweep order"));
    NW_TRY(ctx_ensure(c, M->oscratch, prop::sweep_order_bytes(n), "sweep order scratch"));
  }
  DevBuf oi, os;
  struct Free {
    nw_ctx* c;
    DevBuf* b[2];
    ~Free() {
      for (DevBuf* x : b) ctx_free(c, *x);
    }
  } fr{c, {&oi, &os}};
  uint32_t* out_i = nbr_idx;
  int16_t* out_s = nbr_score;
  if (!dev) {
    NW_TRY(ctx_alloc(c, oi, sizeof(uint32_t) * (size_t)n * k, "neighbour lists"));
    NW_TRY(ctx_alloc(c, os, sizeof(int16_t) * (size_t)n * k, "neighbour lists"));
    out_i = oi.as<uint32_t>();
    out_s = os.as<int16_t>();
  }
  // scratch sized before the timed stages
  NW_TRY(ctx_ensure(c, M->Eall, sizeof(float) * (size_t)n * cnn::kOut, "embeddings"));
  NW_TRY(ctx_ensure(c, M->cand_score, sizeof(int32_t) * outc, "candidate scores"));
  cudaEvent_t ev[5];
  for (auto& e : ev) NW_CK(cudaEventCreate(&e));
  struct FreeEv {
    cudaEvent_t* e;
    ~FreeEv() {
      for (int x = 0; x < 5; ++x) cudaEventDestroy(e[x]);
    }
  } fe{ev};
  // the long words' exhaustive lists first (their own stream, timed on their own)
  float exact_ms = 0.f;
  uint32_t nlong = 0;
  NW_TRY(exact_long_rows(M, d, k, &nlong, &exact_ms));
  NW_CK(cudaEventRecord(ev[0], s));
  NW_TRY(embed_all(M, d, s));
  NW_CK(cudaEventRecord(ev[1], s));
  NW_CK(prop::quantize(fptr(M->Eall), n, amax_ptr(M), nullptr, M->Qb.as<__nv_bfloat16>(), M->qbias.as<int32_t>(),
                       nullptr, s));
  NW_CK(cudaEventRecord(ev[2], s));
  if (M->sweep_order) {  // the rows in a locality order; the lists come back in the original rows and ids
    NW_CK(prop::sweep_order(M->Qb.as<__nv_bfloat16>(), M->qbias.as<int32_t>(), d->ws.rank.as<uint32_t>(),
                            d->ws.slen.as<uint8_t>(), n, M->oscratch.p, M->operm.as<uint32_t>(),
                            M->oQb.as<__nv_bfloat16>(), M->obias.as<int32_t>(), s));
    NW_CK(prop::dot_topk(M->oQb.as<__nv_bfloat16>(), M->obias.as<int32_t>(), n, C, M->topbuf.as<uint64_t>(),
                         M->cand.as<uint32_t>(), M->cand_dot.as<int32_t>(), err_ptr(M), s, dot_debug(c),
                         M->operm.as<uint32_t>(), /*sorted=*/false));
  } else {
    NW_CK(prop::dot_topk(M->Qb.as<__nv_bfloat16>(), M->qbias.as<int32_t>(), n, C, M->topbuf.as<uint64_t>(),
                         M->cand.as<uint32_t>(), M->cand_dot.as<int32_t>(), err_ptr(M), s, dot_debug(c), nullptr,
                         /*sorted=*/false));
  }
  NW_CK(cudaEventRecord(ev[3], s));
  // (the candidates of a row come in no particular order: the rescoring
  // regroups them by length and the k best are taken by score, then index)
  NW_TRY(rescore_select(c, d, M->cand.as<uint32_t>(), C, k, M->cand_score, out_i, out_s, err_ptr(M), s));
  NW_CK(cudaEventRecord(ev[4], s));
  NW_TRY(splice_long_rows(M, d, nlong, k, out_i, out_s, s));
  if (!dev) {
    NW_TRY(copy_out(c, nbr_idx, out_i, (size_t)n * k, false, s));
    NW_TRY(copy_out(c, nbr_score, out_s, (size_t)n * k, false, s));
  }
  NW_TRY(check_err(M, s));
  if (prof) {
    float ms[4];
    for (int x = 0; x < 4; ++x) NW_CK(cudaEventElapsedTime(&ms[x], ev[x], ev[x + 1]));
    prof->embed_ms = ms[0];
    prof->quantize_ms = ms[1];
    prof->candidates_ms = ms[2];
    prof->rescore_ms = ms[3];
    prof->exact_ms = exact_ms;
    prof->total_ms = (double)ms[0] + ms[1] + ms[2] + ms[3] + exact_ms;
  }
  return NW_OK;
}

}  // extern "C"
