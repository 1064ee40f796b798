// nw_rescore.cu -- exact rescoring of proposal candidates, two per thread:
// each row's candidates are reordered by length, and consecutive entries
// share one thread's int16 halves (the row's word streamed, both candidates
// in registers), so neither half of the packed DP idles.
#include <algorithm>
#include <climits>
#include <cuda_runtime.h>
#include <stdint.h>

#include "nw_dp.cuh"
#include "nw_launch.h"
#include "nw_proposal.h"
#include "nw_proposal_internal.h"

namespace nw {
namespace {

// Two alignments in the int16 halves: the low half's B word has l0 symbols
// and the high half's l1 (both <= LB; columns past a word's end only extend
// its DP to the right and do not change its earlier columns).  Returns the
// low half's cell at column l0 and the high half's at column l1 (0 for an
// empty word).
template <int LB, bool TAB = false>
__device__ __forceinline__ uint32_t dp_word2(const uint32_t* __restrict__ arow, int la, const BRow<LB>& b,
                                             uint32_t C1, uint32_t C2, const uint16_t* tab, int l0, int l1) {
  if constexpr (LB == 0) {
    return 0u;
  } else {
    uint32_t G[LB];
#pragma unroll
    for (int j = 0; j < LB; ++j) G[j] = 0u;
    int i = 0;
#pragma unroll 1
    for (; i + 1 < la; i += 2) {
      const uint32_t a0 = __ldg(arow + i);
      const uint32_t a1 = __ldg(arow + i + 1);
      dp_row<LB, TAB>(G, a0, b, C1, C2, tab);
      dp_row<LB, TAB>(G, a1, b, C1, C2, tab);
    }
    if (i < la) dp_row<LB, TAB>(G, __ldg(arow + i), b, C1, C2, tab);
    uint32_t lo = 0u, hi = 0u;
#pragma unroll
    for (int j = 0; j < LB; ++j) {
      if (j == l0 - 1) lo = G[j] & 0xffffu;
      if (j == l1 - 1) hi = G[j] >> 16;
    }
    return lo | (hi << 16);
  }
}

// Two candidates of one row in one thread (int16 halves): the row's word
// streams, the candidates sit in registers; s0 / s1 their scores.
template <int LB, bool TAB>
__device__ __forceinline__ int2 pair2_score(const PairsParams& P, uint32_t ra, int la, bool ok0, uint32_t rb0, int l0,
                                            bool ok1, uint32_t rb1, int l1) {
  BRow<LB> b;
  if constexpr (LB > 0) {
    const uint32_t w0 = ok0 ? __ldg(P.brec_w + rb0) : 0u, w1 = ok1 ? __ldg(P.brec_w + rb1) : 0u;
    const uint32_t sh0 = (w0 & 1u) * 16u, sh1 = (w1 & 1u) * 16u;
    const uint32_t* rec0 = P.b_rec + (w0 & ~3u);
    const uint32_t* rec1 = P.b_rec + (w1 & ~3u);
#pragma unroll
    for (int j = 0; j < LB; ++j) {
      // padding past a word's end: code 0 (any valid code: those columns
      // do not reach the word's own score)
      uint32_t v0 = 0u, v1 = 0u;
      if (ok0 && j < l0) {
        v0 = (__ldg(rec0 + j) >> sh0) & 0xffffu;
        if constexpr (TAB) v0 = ~v0 & 0xffffu;
      }
      if (ok1 && j < l1) {
        v1 = (__ldg(rec1 + j) >> sh1) & 0xffffu;
        if constexpr (TAB) v1 = ~v1 & 0xffffu;
      }
      b.v[j] = v0 | (v1 << 16);
    }
  }
  const uint32_t* arow = P.a_enc + __ldg(P.aoff + ra);
  const uint32_t res = dp_word2<LB, TAB>(arow, la, b, P.C1, P.C2, P.tab, l0, l1);
  return make_int2((int)(int16_t)(res & 0xffffu) + P.gap * (la + l0), (int)(int16_t)(res >> 16) + P.gap * (la + l1));
}

template <bool TAB>
__device__ int2 pair2_dispatch_t(int LB, const PairsParams& P, uint32_t ra, int la, bool ok0, uint32_t rb0, int l0,
                                 bool ok1, uint32_t rb1, int l1) {
  switch (LB) {
#define NW_CASE(L) case L: return pair2_score<L, TAB>(P, ra, la, ok0, rb0, l0, ok1, rb1, l1);
    NW_CASE(0) NW_CASE(1) NW_CASE(2) NW_CASE(3) NW_CASE(4) NW_CASE(5) NW_CASE(6) NW_CASE(7)
    NW_CASE(8) NW_CASE(9) NW_CASE(10) NW_CASE(11) NW_CASE(12) NW_CASE(13) NW_CASE(14)
    NW_CASE(15) NW_CASE(16) NW_CASE(17) NW_CASE(18) NW_CASE(19) NW_CASE(20) NW_CASE(21)
    NW_CASE(22) NW_CASE(23) NW_CASE(24) NW_CASE(25) NW_CASE(26) NW_CASE(27) NW_CASE(28)
    NW_CASE(29) NW_CASE(30) NW_CASE(31) NW_CASE(32) NW_CASE(33) NW_CASE(34) NW_CASE(35)
    NW_CASE(36) NW_CASE(37) NW_CASE(38) NW_CASE(39) NW_CASE(40)
#undef NW_CASE
    default: return make_int2(INT_MIN, INT_MIN);
  }
}

constexpr int kSortWarps = 8;
constexpr int kLenBins = kMaxLen + 2;  // lengths 0..kMaxLen, then missing or invalid entries

// one warp per row: the row's candidates reordered by length (counting
// sort; order within a length is arbitrary), so that neighbours in the list
// share a DP width when paired
__global__ void __launch_bounds__(kSortWarps * 32) sort_cands_kernel(const PairsParams P,
                                                                   const uint32_t* __restrict__ cand, uint32_t C,
                                                                   uint32_t* __restrict__ out) {
  __shared__ unsigned bins[kSortWarps][kLenBins];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t i = blockIdx.x * kSortWarps + warp;
  if (i >= P.n) return;  // warp-uniform
  unsigned* h = bins[warp];
  for (int b = lane; b < kLenBins; b += 32) h[b] = 0u;
  __syncwarp();
  const uint32_t* row = cand + (size_t)i * C;
  auto len_of = [&](uint32_t j) { return j < P.n ? (int)__ldg(P.slen + __ldg(P.rank + j)) : kMaxLen + 1; };
  for (uint32_t x = lane; x < C; x += 32) atomicAdd(&h[len_of(row[x])], 1u);
  __syncwarp();
  if (lane == 0) {
    unsigned acc = 0;
    for (int b = 0; b < kLenBins; ++b) {
      const unsigned c = h[b];
      h[b] = acc;
      acc += c;
    }
  }
  __syncwarp();
  for (uint32_t x = lane; x < C; x += 32) {
    const uint32_t j = row[x];
    out[(size_t)i * C + atomicAdd(&h[len_of(j)], 1u)] = j;
  }
}

// DP width of pair item p = (row i, pair r): the longer of sorted[i * C +
// 2r] and sorted[i * C + 2r + 1] (missing or invalid entries count as empty)
__device__ __forceinline__ int item_width(const PairsParams& P, const uint32_t* __restrict__ cs, uint32_t C, uint32_t Ch,
                                          uint32_t p) {
  const uint32_t i = p / Ch, r = p - i * Ch;
  const size_t o = (size_t)i * C + 2 * r;
  const uint32_t j0 = cs[o], j1 = 2 * r + 1 < C ? cs[o + 1] : 0xffffffffu;
  const int l0 = j0 < P.n ? (int)__ldg(P.slen + __ldg(P.rank + j0)) : 0;
  const int l1 = j1 < P.n ? (int)__ldg(P.slen + __ldg(P.rank + j1)) : 0;
  return max(l0, l1);
}

constexpr int kBinThreads = 256;

// items per DP width, summed into bins[width]
__global__ void __launch_bounds__(kBinThreads) count_widths_kernel(const PairsParams P, const uint32_t* __restrict__ cs,
                                                                   uint32_t C, uint32_t m, unsigned* __restrict__ bins) {
  __shared__ unsigned h[kLenBins];
  for (int b = threadIdx.x; b < kLenBins; b += kBinThreads) h[b] = 0u;
  __syncthreads();
  const uint32_t p = blockIdx.x * kBinThreads + threadIdx.x;
  if (p < m) atomicAdd(&h[item_width(P, cs, C, (C + 1) / 2, p)], 1u);
  __syncthreads();
  for (int b = threadIdx.x; b < kLenBins; b += kBinThreads)
    if (h[b]) atomicAdd(&bins[b], h[b]);
}

// bins: counts -> exclusive starts (one thread)
__global__ void scan_widths_kernel(unsigned* bins) {
  unsigned acc = 0;
  for (int b = 0; b < kLenBins; ++b) {
    const unsigned c = bins[b];
    bins[b] = acc;
    acc += c;
  }
}

// items grouped by DP width; a block reserves one range per width, so the
// items of a block (consecutive pairs, mostly of one row) stay together
__global__ void __launch_bounds__(kBinThreads) scatter_widths_kernel(const PairsParams P, const uint32_t* __restrict__ cs,
                                                                     uint32_t C, uint32_t m, unsigned* __restrict__ cursor,
                                                                     uint32_t* __restrict__ items) {
  __shared__ unsigned h[kLenBins], base[kLenBins];
  for (int b = threadIdx.x; b < kLenBins; b += kBinThreads) h[b] = 0u;
  __syncthreads();
  const uint32_t p = blockIdx.x * kBinThreads + threadIdx.x;
  int w = 0;
  unsigned local = 0;
  if (p < m) {
    w = item_width(P, cs, C, (C + 1) / 2, p);
    local = atomicAdd(&h[w], 1u);
  }
  __syncthreads();
  for (int b = threadIdx.x; b < kLenBins; b += kBinThreads) base[b] = h[b] ? atomicAdd(&cursor[b], h[b]) : 0u;
  __syncthreads();
  if (p < m) items[base[w] + local] = p;
}

// Scores of pair item p (two consecutive entries of a row's length-sorted
// candidates) with DP width LB >= both candidates' lengths.
template <int LB, bool TAB>
__device__ __forceinline__ void rescore_item(const PairsParams& P, const uint32_t* __restrict__ cs, uint32_t C,
                                             uint64_t p, int32_t* __restrict__ score) {
  const uint32_t Ch = (C + 1) / 2;
  const uint32_t i = (uint32_t)(p / Ch), r = (uint32_t)(p - (uint64_t)i * Ch);
  const size_t o = (size_t)i * C + 2 * r;
  const bool two = 2 * r + 1 < C;
  const uint32_t j0 = cs[o], j1 = two ? cs[o + 1] : 0xffffffffu;
  bool ok0 = j0 != 0xffffffffu, ok1 = j1 != 0xffffffffu;
  if (ok0 && (j0 >= P.n || j0 == i)) {
    atomicOr(P.err, kErrInput);
    ok0 = false;
  }
  if (ok1 && (j1 >= P.n || j1 == i)) {
    atomicOr(P.err, kErrInput);
    ok1 = false;
  }
  int s0 = INT32_MIN, s1 = INT32_MIN;
  if (ok0 || ok1) {
    const uint32_t ri = __ldg(P.rank + i);
    const int la = __ldg(P.slen + ri);
    const uint32_t rb0 = ok0 ? __ldg(P.rank + j0) : 0u, rb1 = ok1 ? __ldg(P.rank + j1) : 0u;
    const int l0 = ok0 ? __ldg(P.slen + rb0) : 0, l1 = ok1 ? __ldg(P.slen + rb1) : 0;
    const int2 t = pair2_score<LB, TAB>(P, ri, la, ok0, rb0, l0, ok1, rb1, l1);
    if (ok0) s0 = t.x;
    if (ok1) s1 = t.y;
  }
  score[o] = s0;
  if (two) score[o + 1] = s1;
}

// The pair items of DP width LB: items[ends[LB - 1] .. ends[LB]) after the
// grouping by width (ends[w] = first item past width w).  One launch per
// width, so that each kernel's registers follow its own width (a single
// kernel switching over every width is held to the widest case's registers
// and occupancy).  The table variant keeps a table row pointer and code
// halves live and gets twice the registers per thread.
template <bool TAB>
constexpr int rescore_min_blocks(int LB) { return TAB ? dp_min_blocks(LB) : 2 * dp_min_blocks(LB); }

template <int LB, bool TAB>
__global__ void __launch_bounds__(128, rescore_min_blocks<TAB>(LB)) rescore_width_kernel(
    const PairsParams P, const uint32_t* __restrict__ cs, uint32_t C, const uint32_t* __restrict__ items,
    const unsigned* __restrict__ ends, int32_t* __restrict__ score) {
  const uint32_t beg = LB == 0 ? 0u : ends[LB - 1], end = ends[LB];
  for (uint32_t t = beg + blockIdx.x * blockDim.x + threadIdx.x; t < end; t += gridDim.x * blockDim.x)
    rescore_item<LB, TAB>(P, cs, C, items[t], score);
}

template <bool TAB>
cudaError_t launch_rescore_width(int LB, unsigned grid, const PairsParams& P, const uint32_t* cs, uint32_t C,
                                 const uint32_t* items, const unsigned* ends, int32_t* score, cudaStream_t s) {
  switch (LB) {
#define NW_CASE(L) \
  case L: rescore_width_kernel<L, TAB><<<grid, 128, 0, s>>>(P, cs, C, items, ends, score); break;
    NW_CASE(0) NW_CASE(1) NW_CASE(2) NW_CASE(3) NW_CASE(4) NW_CASE(5) NW_CASE(6) NW_CASE(7)
    NW_CASE(8) NW_CASE(9) NW_CASE(10) NW_CASE(11) NW_CASE(12) NW_CASE(13) NW_CASE(14)
    NW_CASE(15) NW_CASE(16) NW_CASE(17) NW_CASE(18) NW_CASE(19) NW_CASE(20) NW_CASE(21)
    NW_CASE(22) NW_CASE(23) NW_CASE(24) NW_CASE(25) NW_CASE(26) NW_CASE(27) NW_CASE(28)
    NW_CASE(29) NW_CASE(30) NW_CASE(31) NW_CASE(32) NW_CASE(33) NW_CASE(34) NW_CASE(35)
    NW_CASE(36) NW_CASE(37) NW_CASE(38) NW_CASE(39) NW_CASE(40)
#undef NW_CASE
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

// one thread per two consecutive entries of a row's length-sorted candidates
// (work item t; used when the items are too many to group by width)
__global__ void __launch_bounds__(128) rescore2_kernel(const PairsParams P, const uint32_t* __restrict__ cs, uint32_t C,
                                                       const uint32_t* __restrict__ items, uint64_t m,
                                                       int32_t* __restrict__ score) {
  const uint32_t Ch = (C + 1) / 2;
  const uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const uint64_t p = items ? (uint64_t)items[t] : t;
  const uint32_t i = (uint32_t)(p / Ch), r = (uint32_t)(p - (uint64_t)i * Ch);
  const size_t o = (size_t)i * C + 2 * r;
  const bool two = 2 * r + 1 < C;
  const uint32_t j0 = cs[o], j1 = two ? cs[o + 1] : 0xffffffffu;
  bool ok0 = j0 != 0xffffffffu, ok1 = j1 != 0xffffffffu;
  if (ok0 && (j0 >= P.n || j0 == i)) {
    atomicOr(P.err, kErrInput);
    ok0 = false;
  }
  if (ok1 && (j1 >= P.n || j1 == i)) {
    atomicOr(P.err, kErrInput);
    ok1 = false;
  }
  int s0 = INT32_MIN, s1 = INT32_MIN;
  if (ok0 || ok1) {
    const uint32_t ri = __ldg(P.rank + i);
    const int la = __ldg(P.slen + ri);
    const uint32_t rb0 = ok0 ? __ldg(P.rank + j0) : 0u, rb1 = ok1 ? __ldg(P.rank + j1) : 0u;
    const int l0 = ok0 ? __ldg(P.slen + rb0) : 0, l1 = ok1 ? __ldg(P.slen + rb1) : 0;
    const int2 t = P.tab ? pair2_dispatch_t<true>(max(l0, l1), P, ri, la, ok0, rb0, l0, ok1, rb1, l1)
                         : pair2_dispatch_t<false>(max(l0, l1), P, ri, la, ok0, rb0, l0, ok1, rb1, l1);
    if (ok0) s0 = t.x;
    if (ok1) s1 = t.y;
  }
  score[o] = s0;
  if (two) score[o + 1] = s1;
}

}  // namespace

namespace prop {

size_t rescore_scratch_bytes(uint32_t n, uint32_t C) {
  const size_t m = (size_t)n * ((C + 1) / 2);
  return ((size_t)n * C * 2 + m) * sizeof(uint32_t) + 256;
}

cudaError_t rescore_sorted(const PairsParams& P, const uint32_t* cand, uint32_t C, int max_len, int32_t* score,
                           uint32_t** sorted_out, cudaStream_t s) {
  uint32_t* sorted = reinterpret_cast<uint32_t*>(score + (size_t)P.n * C);
  *sorted_out = sorted;
  if (P.n == 0) return cudaSuccess;
  sort_cands_kernel<<<(P.n + kSortWarps - 1) / kSortWarps, kSortWarps * 32, 0, s>>>(P, cand, C, sorted);
  const uint64_t m = (uint64_t)P.n * ((C + 1) / 2);
  uint32_t* items = nullptr;
  if (m < (1ull << 32)) {  // group the pair items by DP width, so that a warp runs one width
    items = sorted + (size_t)P.n * C;
    unsigned* bins = reinterpret_cast<unsigned*>(items + m);
    cudaError_t e = cudaMemsetAsync(bins, 0, sizeof(unsigned) * kLenBins, s);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((m + kBinThreads - 1) / kBinThreads);
    count_widths_kernel<<<blocks, kBinThreads, 0, s>>>(P, sorted, C, (uint32_t)m, bins);
    scan_widths_kernel<<<1, 1, 0, s>>>(bins);
    scatter_widths_kernel<<<blocks, kBinThreads, 0, s>>>(P, sorted, C, (uint32_t)m, bins, items);
    // the scatter left bins[w] at the end of width w's items: one launch per
    // width up to the dictionary's longest word, each a grid of resident blocks
    static int sms = 0;
    if (sms == 0) {
      int dev = 0;
      if (cudaGetDevice(&dev) != cudaSuccess ||
          cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return cudaGetLastError();
    }
    const int top = max_len < 0 ? 0 : (max_len > kMaxLen ? kMaxLen : max_len);
    for (int LB = 0; LB <= top; ++LB) {
      const uint64_t cap = (uint64_t)sms * (uint64_t)(P.tab ? rescore_min_blocks<true>(LB)
                                                            : rescore_min_blocks<false>(LB));
      const unsigned grid = (unsigned)std::min<uint64_t>(cap, (m + 127) / 128);
      e = P.tab ? launch_rescore_width<true>(LB, grid, P, sorted, C, items, bins, score, s)
                : launch_rescore_width<false>(LB, grid, P, sorted, C, items, bins, score, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  rescore2_kernel<<<(unsigned)((m + 127) / 128), 128, 0, s>>>(P, sorted, C, items, m, score);
  return cudaGetLastError();
}

}  // namespace prop
}  // namespace nw
