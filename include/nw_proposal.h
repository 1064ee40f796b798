/*
 * nw_proposal.h -- learned neighbour-candidate proposal for libnw.
 *
 * The paper scores every pair (Section 4) and notes that this cost grows
 * with the square of the dictionary.  This part of the library adds a
 * learned shortcut that it does not have: a character CNN maps each word to
 * 64 values, read as 63 features phi and a bias beta, and models the
 * similarity of two words as pred(a, b) = phi_a . phi_b + beta_a + beta_b
 * (trained on Algorithm 1's raw score or on Section 5's normalised weight;
 * the biases carry the -len(A) - len(B) part of a raw score, which no dot
 * product of one embedding per word can express).  Each word's C best
 * phi_a . phi_b + beta_b propose candidates, and Algorithm 1 rescores only
 * those exactly.  The result is an approximate top-k whose scores are exact.
 *
 * Network (fixed shape; float32 parameters, float32 arithmetic):
 *   x_t = emb[code_t]                      (32 values per position)
 *   three times: x_t <- ReLU(b + sum_{tap=0..2} W[., tap, .] x_{t+tap-1})
 *                (128 channels, zero outside the word)
 *   p = mean over the word's positions of x_t (zero for an empty word)
 *   e = Wl p + bl                          (64 values)
 * Flat parameter layout, in order: emb[alphabet][32], W1[128][3][32],
 * b1[128], W2[128][3][128], b2[128], W3[128][3][128], b3[128], Wl[64][128],
 * bl[64].
 *
 * Conventions as in nw.h: status codes, NW_DEVICE_PTRS / NW_ASYNC flags,
 * original word indices, missing list entries (UINT32_MAX, INT16_MIN).
 */
#ifndef NW_PROPOSAL_H
#define NW_PROPOSAL_H

#include <stddef.h>
#include <stdint.h>

#include "nw.h"

#ifdef __cplusplus
extern "C" {
#endif

#define NW_EMBED_DIM 64
#define NW_MAX_CANDIDATES 512

typedef struct nw_model nw_model;

/* A model for codes < alphabet (<= 256) with parameters drawn from a
 * SplitMix64 stream of `seed` (embedding uniform on [-sqrt(3), sqrt(3)],
 * convolution weights uniform on +-sqrt(6 / fan_in), output weights on
 * +-0.1 sqrt(6 / fan_in), biases zero) and Adam moments at zero.  Owned by
 * the caller; freed by nw_model_free. */
nw_status nw_model_create(nw_ctx *ctx, uint32_t alphabet, uint64_t seed, nw_model **out);
void nw_model_free(nw_model *model);

/* Number of float32 parameters (the flat layout above). */
uint64_t nw_model_param_count(const nw_model *model);

/* Copies the flat parameters out of / into the model (nparams floats; host
 * buffers, or device buffers with NW_DEVICE_PTRS).  Setting parameters also
 * resets the Adam moments and step. */
nw_status nw_model_get_params(nw_model *model, float *params, uint32_t flags);
nw_status nw_model_set_params(nw_model *model, const float *params, uint32_t flags);

/* Embeddings of every word of `dict` (whose alphabet must not exceed the
 * model's): out[i * 64 + d], original order. */
nw_status nw_model_embed(nw_model *model, nw_dict *dict, float *out, uint32_t flags);

/* Loss and gradient of m pairs without changing the model:
 *   loss = (1/m) sum_p (pred(pi[p], pj[p]) - target[p])^2
 * grad receives nparams floats (NULL to skip).  pi, pj: original indices;
 * m >= 1. */
nw_status nw_model_loss_grad(nw_model *model, nw_dict *dict, const uint32_t *pi, const uint32_t *pj,
                             const float *target, uint32_t m, float *loss, float *grad, uint32_t flags);

/* Training by Adam on pairs drawn on the device, each labelled by Algorithm
 * 1 with the dictionary's scoring: target = s / max(len_i, len_j, 1).
 * With raw_scale > 0 the target is s * raw_scale instead.
 * Each step draws batch_pairs pairs from a SplitMix64 stream of `seed`: a
 * fraction nbr_fraction take j from the given neighbour lists of a uniform i
 * (nbr: n x knb original indices, UINT32_MAX entries skipped; NULL for
 * none), the rest are uniform pairs i != j.  With long_fraction > 0, each
 * pair's i is drawn, with that probability, uniformly among the dictionary's
 * words of at least long_len symbols instead (long words are rare in a
 * dictionary, and the proposal ranks them worst).  `losses` (steps floats, may be
 * NULL) receives each step's mean loss.  Steps run as one captured CUDA
 * graph replayed `steps` times. */
typedef struct {
    uint32_t steps;
    uint32_t batch_pairs;   /* <= 65536 */
    float lr, beta1, beta2, eps;
    float nbr_fraction;     /* in [0, 1] */
    float raw_scale;        /* > 0: target s * raw_scale; 0: s / max(len) */
    float lr_final;         /* > 0: the rate falls linearly from lr to lr_final over the steps; 0: constant */
    float clip_norm;        /* > 0: each step's gradient is scaled to norm <= clip_norm; 0: off */
    uint64_t seed;
    uint32_t long_len;      /* with long_fraction: the words of at least long_len symbols ... */
    float long_fraction;    /* ... give a pair's first word with this probability (0: uniform words) */
} nw_train_config;

nw_status nw_model_train(nw_model *model, nw_dict *dict, const nw_train_config *cfg, const uint32_t *nbr,
                         uint32_t knb, float *losses, uint32_t flags);

/* Quantisation of n x 64 float embeddings, all arithmetic in float32:
 * scale = max|phi| / 127 over the 63 features of every row,
 * q[i][d] = round-half-even(phi[i][d] / scale) clamped to [-127, 127] for
 * d < 63, q[i][63] = 0, and bias[i] = round-half-even(beta_i / (scale *
 * scale)) clamped to +-2^23 (so q_a . q_b + bias_b is phi_a . phi_b + beta_b
 * in units of scale^2).  All zero when scale is 0.  q: n * 64 int8; bias: n
 * int32; scale: one float. */
nw_status nw_quantize_embeddings(nw_ctx *ctx, const float *E, uint32_t n, int8_t *q, int32_t *bias,
                                 float *scale, uint32_t flags);

/* nw_dot_topk flag: sweep the rows in a locality order (sorted by their
 * first two principal components, so that a row's best columns tend to come
 * early and its threshold rises sooner).  Changes the time, never the
 * result.  Without it the rows are swept in their given order. */
#define NW_LOCALITY_ORDER 0x8u

/* For every row i of the n x 64 int8 matrix q, the C other rows j with the
 * largest value q_i . q_j + bias[j] (exact integers; bias may be NULL for
 * 0, |bias| <= 2^23), higher first and lower j first on equal values:
 * idx[i * C + r], val[i * C + r].  Rows with fewer than C others end in
 * (UINT32_MAX, INT32_MIN).  1 <= C <= NW_MAX_CANDIDATES.  The products run
 * on the tensor cores in bf16 with float32 accumulation, which is exact for
 * these integers.  flags: NW_DEVICE_PTRS, NW_LOCALITY_ORDER. */
nw_status nw_dot_topk(nw_ctx *ctx, const int8_t *q, const int32_t *bias, uint32_t n, uint32_t C, uint32_t *idx,
                      int32_t *val, uint32_t flags);

/* Rectangular form: for every row i of qa (na x 64 int8), the C rows j of
 * qb (nb x 64 int8) with the largest q_a[i] . q_b[j] + bias[j] (bias: nb
 * int32 or NULL for 0), higher first and lower j first on equal values; no
 * row is skipped (qa and qb are different sets).  Rows with fewer than C
 * columns end in (UINT32_MAX, INT32_MIN).  Same arithmetic as nw_dot_topk. */
nw_status nw_dot_topk_cross(nw_ctx *ctx, const int8_t *qa, uint32_t na, const int8_t *qb, const int32_t *bias,
                            uint32_t nb, uint32_t C, uint32_t *idx, int32_t *val, uint32_t flags);

/* Exact rescoring: for every word i of `dict`, Algorithm 1's score against
 * each candidate cand[i * C + r] (original indices; UINT32_MAX entries are
 * skipped; candidates of a row must be distinct and differ from i), and the
 * k best (higher score first, lower index on ties) into nbr_idx / nbr_score
 * (n * k each).  1 <= k <= NW_MAX_K, 1 <= C <= NW_MAX_CANDIDATES. */
nw_status nw_rescore_topk(nw_dict *dict, const uint32_t *cand, uint32_t C, uint32_t k, uint32_t *nbr_idx,
                          int16_t *nbr_score, uint32_t flags);

/* Stage times of the last nw_proposal_topk call, milliseconds.  exact_ms is
 * the exhaustive pass over the long words (nw_proposal_set_exact_length);
 * total_ms includes it. */
typedef struct {
    double embed_ms, quantize_ms, candidates_ms, rescore_ms, total_ms, exact_ms;
} nw_proposal_profile;

/* Words and query words with at least `min_len` symbols (0: none, the
 * default) take their k neighbours from the exhaustive kernel instead of the
 * learned proposal: exact lists, as nw_all_pairs_topk gives for a dictionary
 * word (itself excluded) and nw_query for a query word.  The proposal ranks
 * long words poorly (a mean over positions cannot see their longest shared
 * stretches), and long words are rare in a dictionary, so the exhaustive pass
 * over them is cheap there; for query words its cost follows the share of
 * long queries.  Applies to nw_proposal_topk, nw_proposal_query and the
 * proposal server.  NW_EINVAL for min_len > NW_MAX_WORD_LEN. */
nw_status nw_proposal_set_exact_length(nw_model *model, uint32_t min_len);

/* The row order of the candidate sweep in nw_proposal_topk: nonzero (the
 * default) sorts the words by (length, first principal component of their
 * embeddings in 16 equal-count buckets, second principal component) and
 * sweeps each row block's column tiles outward from its own, so that a
 * word's best candidates tend to come first and its threshold rises early;
 * 0 sweeps the words in dictionary order.  The candidates, and so every
 * result, are the same either way (ties still go to the lower original
 * index); only the time of the candidate stage, which includes building the
 * order, changes. */
nw_status nw_proposal_set_sweep_order(nw_model *model, int locality);

/* The whole proposal path for `dict`: embed every word, quantise, take C
 * candidates per word by dot product, rescore them exactly and keep the k
 * best (as nw_rescore_topk).  `prof` may be NULL. */
nw_status nw_proposal_topk(nw_model *model, nw_dict *dict, uint32_t C, uint32_t k, uint32_t *nbr_idx,
                           int16_t *nbr_score, nw_proposal_profile *prof, uint32_t flags);

/* Queries through the proposal: the nq query words (codes and offsets as
 * nw_query) get their k best words of `dict` (raw score, higher first, lower
 * index on ties; UINT32_MAX / INT16_MIN past the candidates).  The
 * dictionary's embeddings are quantised once and kept on the device while
 * neither the dictionary nor the model's parameters change; each call
 * embeds the queries, quantises them on the dictionary's scale (features
 * beyond it clamp to +-127), takes each query's C dictionary words with the
 * largest q_query . q_j + bias_j, and rescores those exactly (Algorithm 1).
 * The scores are exact; the lists equal nw_query's when C >= the
 * dictionary's size.  1 <= C <= NW_MAX_CANDIDATES, 1 <= k <= NW_MAX_K;
 * NW_ERANGE when query scores may not fit int16; NW_RANK_NORMALISED is
 * refused. */
nw_status nw_proposal_query(nw_model *model, nw_dict *dict, const uint8_t *qcodes, const uint32_t *qoffsets,
                            uint32_t nq, uint32_t C, uint32_t k, uint32_t *nbr_idx, int16_t *nbr_score,
                            uint32_t flags);

/* A query server (nw_server_submit / nw_server_wait / nw_server_destroy of
 * nw.h) that answers through the proposal, with continuous batching: each
 * batch holds the queued requests that fit cfg->max_batch_queries (in arrival
 * order) and runs as nw_proposal_query(model, dict, ..., C, cfg->k) on one of
 * the server's slots; up to cfg->max_inflight batches run on the device side
 * by side, and requests arriving meanwhile are admitted the moment a slot
 * frees (nw_request_info.inflight_at_start counts the batches already
 * running).  Each slot owns a context of its own (stream, workspace; capped
 * at mem_budget_bytes / slots when a budget is given, and the slot count is
 * lowered until the budget holds an estimate of a slot's memory), a copy of
 * the model's parameters and exact-path length taken at creation, and a
 * view of the dictionary's device data.  A request's lists equal
 * nw_proposal_query's for its words alone (a word's embedding, candidates and
 * scores do not depend on the rest of its batch).  The model and the
 * dictionary must share a context; the dictionary must outlive the server;
 * later changes to the model do not reach the server. */
nw_status nw_server_create_proposal(nw_dict *dict, nw_model *model, uint32_t C, const nw_server_config *cfg,
                                    nw_server **out);

#ifdef __cplusplus
}
#endif

#endif /* NW_PROPOSAL_H */
