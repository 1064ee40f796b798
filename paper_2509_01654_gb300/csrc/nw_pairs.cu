// nw_pairs.cu -- scores an explicit list of word pairs of one encoded set.
// One thread per pair: the longer word's symbols come from its pair record
// (its own 16-bit half, copied into both halves), the shorter word is
// streamed row by row, and the same shifted recurrence as the all-pairs
// kernel is evaluated; the result is read from the low half.
#include <cuda_runtime.h>

#include "nw_dp.cuh"
#include "nw_launch.h"

namespace nw {

template <int LB>
__device__ __forceinline__ int pair_score(const PairsParams& P, uint32_t pa, int la, uint32_t pb) {
  BRow<LB> b;
  if constexpr (LB > 0) {
    const uint32_t w = __ldg(P.brec_w + pb);     // record offset | half (bit 0)
    const uint32_t sh = (w & 1u) * 16u;
    const uint32_t* rec = P.b_rec + (w & ~3u);
#pragma unroll
    for (int j = 0; j < LB; ++j) {
      const uint32_t v = (__ldg(rec + j) >> sh) & 0xffffu;
      b.v[j] = v | (v << 16);
    }
  }
  const uint32_t* arow = P.a_enc + __ldg(P.aoff + pa);
  const uint32_t res = dp_word<LB>(arow, la, b, P.C1, P.C2);
  return (int)(int16_t)(res & 0xffffu) + P.gap * (la + LB);
}

__device__ int pair_dispatch(int LB, const PairsParams& P, uint32_t pa, int la, uint32_t pb) {
  switch (LB) {
#define NW_CASE(L) case L: return pair_score<L>(P, pa, la, pb);
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

cudaError_t launch_pairs(const PairsParams& p, cudaStream_t s) {
  if (p.m == 0) return cudaSuccess;
  const uint32_t blk = 128;
  const uint64_t grid = (p.m + blk - 1) / blk;
  pairs_kernel<<<(unsigned)grid, blk, 0, s>>>(p);
  return cudaGetLastError();
}

}  // namespace nw
