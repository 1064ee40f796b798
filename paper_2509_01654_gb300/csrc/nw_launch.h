// nw_launch.h -- host-side entry points of the kernel translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nw_internal.cuh"

namespace nw {

// alignment kernel for the longer length LB (0 .. kMaxLen), epilogue kind and
// scoring (tab: substitution table); nullptr if there is none
const void* dp_kernel(int LB, int epi, bool tab = false);

// ingest: stable bucketing by length and encoding of a word set
cudaError_t launch_ingest_count(const uint8_t* codes, const uint32_t* offsets, uint32_t n,
                                uint32_t alphabet, uint32_t* block_counts, uint32_t* err,
                                cudaStream_t s);
cudaError_t launch_ingest_scan(uint32_t* block_counts, uint32_t nblk, uint32_t* bucket_count,
                               cudaStream_t s);
cudaError_t launch_ingest_scatter(const uint32_t* offsets, uint32_t n, const uint32_t* block_base,
                                  const Buckets& bk, uint32_t* perm, uint32_t* rank, uint8_t* slen,
                                  cudaStream_t s);
cudaError_t launch_ingest_encode(const uint8_t* codes, const uint32_t* offsets, uint32_t n,
                                 const uint32_t* perm, const uint8_t* slen, const Buckets& bk,
                                 uint32_t shift, uint32_t* a_enc, uint32_t* aoff,
                                 uint32_t* b_rec, uint32_t* brec_w, cudaStream_t s);
constexpr uint32_t kIngestBlock = 256;

// lists -> ranked (index, score) rows.  With norm_frac (normalised ranking),
// a key carries the rank r of s/m, whose reduced fraction is norm_frac[2r] /
// norm_frac[2r+1]; the raw score is rebuilt from m = the longer length of the
// pair (slen by sorted position, rank maps the partner to its position).
cudaError_t launch_finalize(const uint32_t* slots, uint32_t nlists, uint32_t k, const uint32_t* perm,
                            uint32_t ib, uint32_t imask, int32_t key_lo, uint32_t* out_idx,
                            int16_t* out_score, cudaStream_t s, const int16_t* norm_frac = nullptr,
                            const uint8_t* slen = nullptr, const uint32_t* rank = nullptr);

// per word, the k best distinct neighbours of nparts ranked lists stored one
// after another (part p of word w at p * n * k + w * k), one thread per word
cudaError_t launch_topk_merge(uint32_t n, uint32_t k, uint32_t nparts, const uint32_t* idx_parts,
                              const int16_t* score_parts, uint32_t* idx_out, int16_t* score_out, cudaStream_t s);

// explicit pairs of one encoded set
struct PairsParams {
  const uint32_t* pi;
  const uint32_t* pj;
  uint64_t m;
  uint32_t n;
  const uint32_t* rank;
  const uint8_t* slen;
  const uint32_t* aoff;
  const uint32_t* brec_w;
  const uint32_t* a_enc;
  const uint32_t* b_rec;
  uint32_t C1, C2;
  int32_t gap;
  int16_t* out;
  uint32_t* err;
  const uint16_t* tab;  // substitution table (device, kTabDim x kTabDim) or null
};
cudaError_t launch_pairs(const PairsParams& p, cudaStream_t s);

// the all-pairs top-k reduction with every scratch buffer taken from a
// caller-supplied device region; `provide` is called with the dictionary's
// device current and returns the region (see nw_all_pairs_topk_noalloc)
typedef nw_status (*ScratchProvider)(int device, void** base, size_t* bytes, const char** why);
nw_status topk_into_scratch(nw_dict* d, ScratchProvider provide, uint32_t k, uint32_t* nbr_idx,
                            int16_t* nbr_score, int64_t* hist, int32_t* hist_lo, uint32_t nbins,
                            uint32_t flags);

// nw_query without entering the context (for library calls that hold it):
// the k best dictionary words of each query word
nw_status query_impl(nw_dict* d, const uint8_t* qcodes, const uint32_t* qoffsets, uint32_t nq, uint32_t k,
                     uint32_t* nbr_idx, int16_t* nbr_score, uint32_t flags);

// microbenchmarks of the integer instruction rates
enum RateOp { kRateViaddmax = 0, kRateVimax3, kRateVimaxRelu, kRateIadd3, kRateLop3, kRateCell, kRateOps };
cudaError_t launch_rate(int op, int blocks, int iters, const uint32_t* in, uint32_t* out,
                        unsigned long long* cycles, cudaStream_t s);
// operations per thread per iteration of launch_rate for `op`
double rate_ops_per_iter(int op);
// resident blocks of launch_rate's kernel per SM (one full wave = SMs x this)
int rate_blocks_per_sm(int op);
constexpr int kRateBlock = 256;

}  // namespace nw
