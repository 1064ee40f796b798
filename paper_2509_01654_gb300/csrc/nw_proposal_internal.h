// nw_proposal_internal.h -- kernels of the candidate proposal path
// (quantisation, dot-product top-C, exact rescoring; see nw_proposal.h).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "nw_launch.h"

struct nw_ctx;
struct nw_model;

namespace nw {
namespace prop {

// the context a model was created on (its allocations, stream and error text)
nw_ctx* model_ctx(const nw_model* M);
// a model on context c with src's alphabet, parameters (copied on the
// device) and exact-path length; src's context must not be in use
nw_status model_clone(nw_model* src, nw_ctx* c, nw_model** out);

constexpr int kCap = 2048;       // keys per append buffer of the dot-product top-C (two buffers per row)
constexpr int kFeat = 63;        // embedding outputs 0..62 are features, 63 is the bias
constexpr int kBiasLimit = 1 << 23;

// Quantisation of n x 64 embeddings (see nw_quantize_embeddings): q (int8,
// row-major, may be null), qb (the candidate kernel's bf16 rows,
// dot_topk_qb_bytes(n), may be null), bias (int32, may be null), scale
// (device float, may be null); amax_bits is device scratch.  given_scale:
// *amax_bits already holds the largest |feature| to scale by (another set's,
// e.g. the dictionary's for its queries; larger features clamp to +-127).
cudaError_t quantize(const float* E, uint32_t n, unsigned int* amax_bits, int8_t* q, __nv_bfloat16* qb,
                     int32_t* bias, float* scale, cudaStream_t s, bool given_scale = false);
// int8 rows (row-major) -> the candidate kernel's bf16 rows
cudaError_t widen(const int8_t* q, uint32_t n, __nv_bfloat16* qb, cudaStream_t s);
// bf16 rows: row-major rows of 64 values, zero-padded to whole 256-row tiles
size_t dot_topk_qb_bytes(uint32_t n);
// scratch of a launch over nA rows, nB columns and C candidates (the err
// word must follow the returned layout: use dot_topk_err_word)
uint32_t dot_topk_splits(uint32_t nA, uint32_t nB);
size_t dot_topk_buffer_bytes(uint32_t nA, uint32_t nB, uint32_t C);
inline size_t dot_topk_buffer_bytes(uint32_t n, uint32_t C) { return dot_topk_buffer_bytes(n, n, C); }
// the device error word inside a dot_topk buffer (zero it before a launch)
uint32_t* dot_topk_err_word(uint64_t* buf, uint32_t nA, uint32_t nB);
inline uint32_t* dot_topk_err_word(uint64_t* buf, uint32_t n) { return dot_topk_err_word(buf, n, n); }
// debug settings of the candidate kernel: wait_cycles < 0 keeps the kernel's
// own bound on a pipeline wait; withhold names a column tile the producer
// never issues (UINT32_MAX: none), so that the waits for it run out with no
// copy in flight
struct DotDebug {
  long long wait_cycles = -1;
  uint32_t withhold = 0xffffffffu;
};
// each row's C best q_i . q_j + bias_j over the other rows (bias may be
// null: 0); a pipeline wait that runs out sets kErrWait in *err.  ids
// (nullable): the rows are stored in another order and ids[p] is the
// original id of the row at position p (sweep_order's perm); the lists are
// then written to the original rows and name original ids, ties broken by
// the lower original id, exactly as for the rows in their own order.
// sorted: each list in descending order (value, then lower id); otherwise
// the same C entries in an order that may differ from call to call.
cudaError_t dot_topk(const __nv_bfloat16* Qb, const int32_t* bias, uint32_t n, uint32_t C, uint64_t* buf,
                     uint32_t* idx, int32_t* dot, uint32_t* err, cudaStream_t s, DotDebug dbg = DotDebug{},
                     const uint32_t* ids = nullptr, bool sorted = true);
// each row i of QA's C best QA_i . QB_j + biasB_j over all nB columns (self:
// the two are one set and column i is skipped).  col_ids / row_ids
// (nullable): original ids of the columns (at least ceil(nB / 128) * 128
// entries) and of the rows, when either set is stored in another order.
cudaError_t dot_topk_rect(const __nv_bfloat16* QA, uint32_t nA, const __nv_bfloat16* QB, const int32_t* biasB,
                          uint32_t nB, uint32_t C, bool self, uint64_t* buf, uint32_t* idx, int32_t* dot,
                          uint32_t* err, cudaStream_t s, DotDebug dbg = DotDebug{}, const uint32_t* col_ids = nullptr,
                          const uint32_t* row_ids = nullptr, bool sorted = true);

// The sweep order of the self product: the rows' positions sorted by
// (word length, first principal component of the rows in 16 equal-count
// buckets, second principal component rising in even buckets and falling in
// odd ones), so that most of a row's best columns lie in the tiles near its
// own.  The order changes only the time of dot_topk, never its result.
// rank / slen (nullable: every length 0) give word i's length as
// slen[rank[i]].  Writes perm[p] = the row at position p (sweep_perm_entries
// entries, UINT32_MAX past n) and Qp / bp = the rows (dot_topk_qb_bytes) and
// biases (n entries, bias nullable: none) in that order.  scratch holds
// sweep_order_bytes(n) bytes.  Positions within one sort key follow the
// order of atomic arrival.
size_t sweep_order_bytes(uint32_t n);
size_t sweep_perm_entries(uint32_t n);
cudaError_t sweep_order(const __nv_bfloat16* Qb, const int32_t* bias, const uint32_t* rank, const uint8_t* slen,
                        uint32_t n, void* scratch, uint32_t* perm, __nv_bfloat16* Qp, int32_t* bp, cudaStream_t s);

// Algorithm 1's scores of every row i against its candidates cand[i * C +
// r] (UINT32_MAX entries score INT32_MIN; out-of-range or self candidates
// raise kErrInput; P supplies the encoded dictionary, its pi/pj/m/out
// unused), two candidates per thread: each row's candidates are first
// reordered by length (*sorted_out, n * C), and score[i * C + r] is the
// score of (*sorted_out)[i * C + r].  score points at the start of a region
// of rescore_scratch_bytes(n, C) (the scores, then the reordered candidates
// and the work lists grouped by DP width).  max_len: the dictionary's
// longest word (the widest DP; one launch per width up to it).
size_t rescore_scratch_bytes(uint32_t n, uint32_t C);
cudaError_t rescore_sorted(const PairsParams& P, const uint32_t* cand, uint32_t C, int max_len, int32_t* score,
                           uint32_t** sorted_out, cudaStream_t s);
// Words of a query set Q against a dictionary D for cross_rescore: QD reads
// its streamed (A) words from Q and its register (B) words from D, DQ the
// reverse; both carry D's scoring.  Ranks and lengths of either set map
// original indices to sorted positions.
struct CrossParams {
  PairsParams QD, DQ;
  const uint32_t* q_rank;
  const uint8_t* q_slen;
  const uint32_t* d_rank;
  const uint8_t* d_slen;
  uint32_t nq, nd;
};
// Algorithm 1's score of (query i, dictionary word cand[i * C + r]) into
// score[i * C + r] (INT32_MIN for UINT32_MAX entries; out-of-range
// candidates raise kErrInput)
cudaError_t cross_rescore(const CrossParams& X, const uint32_t* cand, uint32_t C, int32_t* score, cudaStream_t s);
// each row's k best (score desc, index asc) of its C scored candidates
cudaError_t select_topk(const uint32_t* cand, const int32_t* score, uint32_t n, uint32_t C, uint32_t k,
                        uint32_t* out_idx, int16_t* out_score, cudaStream_t s);

}  // namespace prop
}  // namespace nw
