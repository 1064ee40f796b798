// nw_pairs.cu -- scores an explicit list of word pairs of one encoded set.
// One thread per pair: the longer word's symbols come from its pair record
// (its own 16-bit half, copied into both halves), the shorter word is
// streamed row by row, and the same shifted recurrence as the all-pairs
// kernel is evaluated; the result is read from the low half.
#include <cuda_runtime.h>

#include "nw_dp.cuh"
#include "nw_launch.h"
#include "nw_proposal.h"
#include "nw_proposal_internal.h"

namespace nw {

template <int LB, bool TAB>
__device__ __forceinline__ int pair_score(const PairsParams& P, uint32_t pa, int la, uint32_t pb) {
  BRow<LB> b;
  if constexpr (LB > 0) {
    const uint32_t w = __ldg(P.brec_w + pb);     // record offset | half (bit 0)
    const uint32_t sh = (w & 1u) * 16u;
    const uint32_t* rec = P.b_rec + (w & ~3u);
#pragma unroll
    for (int j = 0; j < LB; ++j) {
      uint32_t v = (__ldg(rec + j) >> sh) & 0xffffu;
      if constexpr (TAB) v = ~v & 0xffffu;  // the code itself (unshifted)
      b.v[j] = v | (v << 16);
    }
  }
  const uint32_t* arow = P.a_enc + __ldg(P.aoff + pa);
  const uint32_t res = dp_word<LB, TAB>(arow, la, b, P.C1, P.C2, P.tab);
  return (int)(int16_t)(res & 0xffffu) + P.gap * (la + LB);
}

template <bool TAB>
__device__ int pair_dispatch_t(int LB, const PairsParams& P, uint32_t pa, int la, uint32_t pb) {
  switch (LB) {
#define NW_CASE(L) case L: return pair_score<L, TAB>(P, pa, la, pb);
    NW_CASE(0) NW_CASE(1) NW_CASE(2) NW_CASE(3) NW_CASE(4) NW_CASE(5) NW_CASE(6) NW_CASE(7)
    NW_CASE(8) NW_CASE(9) NW_CASE(10) NW_CASE(11) NW_CASE(12) NW_CASE(13) NW_CASE(14)
    NW_CASE(15) NW_CASE(16) NW_CASE(17) NW_CASE(18) NW_CASE(19) NW_CASE(20) NW_CASE(21)
    NW_CASE(22) NW_CASE(23) NW_CASE(24) NW_CASE(25) NW_CASE(26) NW_CASE(27) NW_CASE(28)
    NW_CASE(29) NW_CASE(30) NW_CASE(31) NW_CASE(32) NW_CASE(33) NW_CASE(34) NW_CASE(35)
    NW_CASE(36) NW_CASE(37) NW_CASE(38) NW_CASE(39) NW_CASE(40)
#undef NW_CASE
    default: return INT_MIN;
  }
}
static_assert(kMaxLen == 40, "pair_dispatch lists every length up to kMaxLen");

__device__ int pair_dispatch(int LB, const PairsParams& P, uint32_t pa, int la, uint32_t pb) {
  return P.tab ? pair_dispatch_t<true>(LB, P, pa, la, pb) : pair_dispatch_t<false>(LB, P, pa, la, pb);
}

__global__ void __launch_bounds__(128) pairs_kernel(const PairsParams P) {
  const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= P.m) return;
  const uint32_t i = P.pi[p], j = P.pj[p];
  if (i >= P.n || j >= P.n) {
    atomicOr(P.err, kErrInput);
    P.out[p] = INT16_MIN;
    return;
  }
  const uint32_t ri = __ldg(P.rank + i), rj = __ldg(P.rank + j);
  const int li = __ldg(P.slen + ri), lj = __ldg(P.slen + rj);
  uint32_t pa = ri, pb = rj;
  int la = li, lb = lj;
  if (li > lj) { pa = rj; pb = ri; la = lj; lb = li; }
  P.out[p] = (int16_t)pair_dispatch(lb, P, pa, la, pb);
}

// one thread per candidate of a query: Algorithm 1 between query i of set
// Q and dictionary word cand[i * C + r] of set D, the shorter word streamed
// (QD: query streamed, dictionary word in registers; DQ: the reverse)
__global__ void __launch_bounds__(128) cross_rescore_kernel(const prop::CrossParams X, const uint32_t* __restrict__ cand,
                                                            uint32_t C, int32_t* __restrict__ score) {
  const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= (uint64_t)X.nq * C) return;
  const uint32_t i = (uint32_t)(p / C);
  const uint32_t j = cand[p];
  if (j == 0xffffffffu) {
    score[p] = INT32_MIN;
    return;
  }
  if (j >= X.nd) {
    atomicOr(X.QD.err, kErrInput);
    score[p] = INT32_MIN;
    return;
  }
  const uint32_t ri = __ldg(X.q_rank + i), rj = __ldg(X.d_rank + j);
  const int li = __ldg(X.q_slen + ri), lj = __ldg(X.d_slen + rj);
  score[p] = li <= lj ? pair_dispatch(lj, X.QD, ri, li, rj) : pair_dispatch(li, X.DQ, rj, lj, ri);
}

constexpr int kSelPerLane = NW_MAX_CANDIDATES / 32;

// one warp per row: repeated warp-wide maximum over (score, reversed index) keys
__global__ void select_topk_kernel(const uint32_t* __restrict__ cand, const int32_t* __restrict__ score, uint32_t n,
                                   uint32_t C, uint32_t k, uint32_t* __restrict__ out_idx,
                                   int16_t* __restrict__ out_score) {
  const uint32_t row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  uint64_t keys[kSelPerLane];
#pragma unroll
  for (int q = 0; q < kSelPerLane; ++q) {
    const uint32_t c = (uint32_t)lane + 32u * q;
    keys[q] = 0ull;
    if (c < C) {
      const int32_t s = score[(size_t)row * C + c];
      if (s != INT32_MIN)
        keys[q] = ((uint64_t)(uint32_t)(s + 0x80000000) << 32) | (0xffffffffu - cand[(size_t)row * C + c]);
    }
  }
  for (uint32_t r = 0; r < k; ++r) {
    uint64_t best = 0ull;
    int bq = -1;
#pragma unroll
    for (int q = 0; q < kSelPerLane; ++q)
      if (keys[q] > best) { best = keys[q]; bq = q; }
    uint64_t wb = best;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const uint64_t other = __shfl_xor_sync(0xffffffffu, wb, o);
      wb = other > wb ? other : wb;
    }
    if (wb != 0ull && best == wb) {
#pragma unroll
      for (int q = 0; q < kSelPerLane; ++q)
        if (q == bq) keys[q] = 0ull;
    }
    if (lane == 0) {
      const size_t o = (size_t)row * k + r;
      out_idx[o] = wb ? 0xffffffffu - (uint32_t)wb : 0xffffffffu;
      out_score[o] = wb ? (int16_t)(int32_t)((uint32_t)(wb >> 32) - 0x80000000u) : (int16_t)INT16_MIN;
    }
  }
}

namespace prop {

cudaError_t cross_rescore(const CrossParams& X, const uint32_t* cand, uint32_t C, int32_t* score, cudaStream_t s) {
  const uint64_t m = (uint64_t)X.nq * C;
  if (m == 0) return cudaSuccess;
  cross_rescore_kernel<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(X, cand, C, score);
  return cudaGetLastError();
}

cudaError_t select_topk(const uint32_t* cand, const int32_t* score, uint32_t n, uint32_t C, uint32_t k,
                        uint32_t* out_idx, int16_t* out_score, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  select_topk_kernel<<<(n + 7) / 8, 256, 0, s>>>(cand, score, n, C, k, out_idx, out_score);
  return cudaGetLastError();
}

}  // namespace prop

cudaError_t launch_pairs(const PairsParams& p, cudaStream_t s) {
  if (p.m == 0) return cudaSuccess;
  const uint32_t blk = 128;
  const uint64_t grid = (p.m + blk - 1) / blk;
  pairs_kernel<<<(unsigned)grid, blk, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace nw
