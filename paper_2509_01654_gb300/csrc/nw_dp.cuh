// nw_dp.cuh -- the all-pairs alignment kernel (sm_103a), templated on the
// length LB of the longer word of every pair it scores.
//
// Recurrence.  Algorithm 1 of the paper fills H[i][j] = max(H[i-1][j-1] +
// sim(A[i-1], B[j-1]), H[i-1][j] + p, H[i][j-1] + p) from H[i][0] = p*i and
// H[0][j] = p*j and returns H[la][lb].  With G[i][j] = H[i][j] - p*(i + j)
// the same recurrence reads
//     G[i][j] = max(G[i-1][j-1] + s'(a, b), G[i-1][j], G[i][j-1]),
//     G[i][0] = G[0][j] = 0,   s'(a, b) = sim(a, b) - 2p,
// so the gap terms vanish, every G is >= 0 and the score is
// G[la][lb] + p*(la + lb).  This is an exact rewrite (same maximising paths).
//
// Packing.  A lane holds two B words of length LB (lo and hi 16-bit halves
// of each register) and their DP row G[i][1..LB] in LB registers; the warp
// streams one A word at a time (the same symbol in both halves), so each
// packed instruction advances two alignments by one cell.  Per packed cell:
//     xt = a2 ^ b2[j]                    per half: -1 - (e(a) ^ e(b))
//     f  = viaddmax(xt, s'_m + 1, s'_x+) per half: s'_m if a == b else s'_x+
//     d  = diag + f                      plain 32-bit add (both halves >= 0)
//     h  = vimax3(d, up, left)           max(G[i-1][j-1] + s', G[i-1][j], G[i][j-1])
// The codes are stored shifted (e(c) = c << shift, 2^shift >= match -
// mismatch), so for different codes e(a) ^ e(b) >= match - mismatch and
// s'_m - (e(a) ^ e(b)) <= s'_x: the max with s'_x then selects the mismatch
// value.  s'_x+ = max(s'_x, 0): G is non-decreasing along rows and columns,
// so G[i-1][j-1] + s'_x < 0 + G[i-1][j-1] <= G[i-1][j] whenever s'_x < 0 and
// raising the mismatch term to 0 changes no maximum; it keeps f >= 0, so the
// packed add never carries between halves (G + f <= s'_m * LB < 2^15).
// Per two cells: one LOP3, one add and two DPX instructions; rows go two at
// a time so the two rows' dependency chains interleave.
//
// Substitution-matrix scoring (TAB): the lane holds its B words' codes
// (lo / hi halves) and the per-cell term is read from the table row of the A
// symbol, f = s'+(a, b_lo) | s'+(a, b_hi) << 16 with s'+ = max(s', 0) (the
// same argument as above makes the clamp exact and keeps the add carry-free).
#pragma once

#include <cuda_runtime.h>
#include <limits.h>

#include "nw_internal.cuh"

namespace nw {

template <int LB>
struct BRow {
  uint32_t v[LB > 0 ? LB : 1];
};

// the packed per-cell term of symbol pair column j
template <int LB, bool TAB>
__device__ __forceinline__ uint32_t cell_term(uint32_t a2, const BRow<LB>& b, int j, uint32_t C1, uint32_t C2,
                                              const uint16_t* trow) {
  if constexpr (TAB) {
    const uint32_t bv = b.v[j];
    return (uint32_t)trow[bv & 0xffffu] | ((uint32_t)trow[bv >> 16] << 16);
  } else {
    return __viaddmax_s16x2(a2 ^ b.v[j], C1, C2);
  }
}

// the table row of A symbol a2 (codes stored unshifted in TAB dictionaries)
template <bool TAB>
__device__ __forceinline__ const uint16_t* tab_row(const uint16_t* tab, uint32_t a2) {
  if constexpr (TAB) return tab + ((a2 & 0xffffu) * (uint32_t)kTabDim);
  return nullptr;
}

// One row of the shifted recurrence: G[1..LB] of row i-1 becomes row i.
template <int LB, bool TAB = false>
__device__ __forceinline__ void dp_row(uint32_t (&G)[LB], uint32_t a2, const BRow<LB>& b, uint32_t C1,
                                       uint32_t C2, const uint16_t* tab = nullptr) {
  const uint16_t* trow = tab_row<TAB>(tab, a2);
  uint32_t diag = 0u, left = 0u;
#pragma unroll
  for (int j = 0; j < LB; ++j) {
    const uint32_t f = cell_term<LB, TAB>(a2, b, j, C1, C2, trow);
    const uint32_t up = G[j];
    const uint32_t h = __vimax3_s16x2(diag + f, up, left);
    diag = up;
    G[j] = h;
    left = h;
  }
}

// The first row (i = 1): diag and up are G[0][*] = 0 and f, left >= 0, so
// the cell is max(f, left) and no row of zeros needs setting up.
template <int LB, bool TAB = false>
__device__ __forceinline__ void dp_row_first(uint32_t (&G)[LB], uint32_t a2, const BRow<LB>& b, uint32_t C1,
                                             uint32_t C2, const uint16_t* tab = nullptr) {
  const uint16_t* trow = tab_row<TAB>(tab, a2);
  uint32_t left = 0u;
#pragma unroll
  for (int j = 0; j < LB; ++j) {
    const uint32_t f = cell_term<LB, TAB>(a2, b, j, C1, C2, trow);
    left = __vimax_s16x2_relu(f, left);
    G[j] = left;
  }
}

// DP over the la rows of one A word against the lane's two B words; returns
// the packed G[la][LB] (0 when la == 0 or LB == 0).
template <int LB, bool TAB = false>
__device__ __forceinline__ uint32_t dp_word(const uint32_t* __restrict__ arow, int la,
                                            const BRow<LB>& b, uint32_t C1, uint32_t C2,
                                            const uint16_t* tab = nullptr) {
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
    return G[LB - 1];
  }
}

// The same DP with the A word's symbols in shared memory, symbol i at
// acol[32 * i] (the staging layout of the all-pairs kernel; every lane reads
// the same address, so each load is a broadcast).
template <int LB, bool TAB = false>
__device__ __forceinline__ uint32_t dp_word_staged(const uint32_t* acol, int la, const BRow<LB>& b, uint32_t C1,
                                                   uint32_t C2, const uint16_t* tab = nullptr) {
  if constexpr (LB == 0) {
    return 0u;
  } else {
    if (la == 0) return 0u;
    uint32_t G[LB];
    dp_row_first<LB, TAB>(G, acol[0], b, C1, C2, tab);
    int i = 1;
    // four rows per iteration: their dependency chains interleave as a
    // wavefront, and the loop control is paid once per four rows
#pragma unroll 1
    for (; i + 3 < la; i += 4) {
      const uint32_t a0 = acol[32 * i];
      const uint32_t a1 = acol[32 * (i + 1)];
      const uint32_t a2 = acol[32 * (i + 2)];
      const uint32_t a3 = acol[32 * (i + 3)];
      dp_row<LB, TAB>(G, a0, b, C1, C2, tab);
      dp_row<LB, TAB>(G, a1, b, C1, C2, tab);
      dp_row<LB, TAB>(G, a2, b, C1, C2, tab);
      dp_row<LB, TAB>(G, a3, b, C1, C2, tab);
    }
    if (i + 1 < la) {
      const uint32_t a0 = acol[32 * i];
      const uint32_t a1 = acol[32 * (i + 1)];
      dp_row<LB, TAB>(G, a0, b, C1, C2, tab);
      dp_row<LB, TAB>(G, a1, b, C1, C2, tab);
      i += 2;
    }
    if (i < la) dp_row<LB, TAB>(G, acol[32 * i], b, C1, C2, tab);
    return G[LB - 1];
  }
}

template <int LB>
__device__ __forceinline__ void load_brow(const uint4* __restrict__ rec, BRow<LB>& b) {
  if constexpr (LB > 0) {
    constexpr int Q = ceil4(LB) / 4;
#pragma unroll
    for (int q = 0; q < Q; ++q) {
      const uint4 v = __ldg(rec + q);
      if (4 * q + 0 < LB) b.v[4 * q + 0] = v.x;
      if (4 * q + 1 < LB) b.v[4 * q + 1] = v.y;
      if (4 * q + 2 < LB) b.v[4 * q + 2] = v.z;
      if (4 * q + 3 < LB) b.v[4 * q + 3] = v.w;
    }
  }
}

// Offers `key` to a word's list of k slots.  The slots always hold the k
// largest keys offered so far (0 = empty); keys of one list are distinct.
// The smallest slot is replaced by compare-and-swap; a failed swap means
// another thread changed that slot, so the scan repeats (bounded).  Slots only
// grow, so a stale read can only make the swap fail, never corrupt the set.
// Returns a lower bound of the list's current smallest key and raises it in
// *thr.
__device__ __forceinline__ uint32_t list_offer(uint32_t* row, uint32_t* thr, uint32_t k,
                                               uint32_t key, uint32_t* err, uint32_t& inserts, int max_iters) {
  for (int it = 0; it < max_iters; ++it) {
    uint32_t m1 = 0xffffffffu, m2 = 0xffffffffu, mi = 0;
    for (uint32_t s = 0; s < k; ++s) {
      const uint32_t v = __ldcg(row + s);
      if (v < m1) { m2 = m1; m1 = v; mi = s; }
      else if (v < m2) { m2 = v; }
    }
    if (key <= m1) {
      atomicMax(thr, m1);
      return m1;
    }
    if (atomicCAS(row + mi, m1, key) == m1) {
      const uint32_t nm = m2 < key ? m2 : key;
      atomicMax(thr, nm);
      ++inserts;
      return nm;
    }
  }
  atomicOr(err, kErrRetry);
  return 0xffffffffu;
}

// global -> shared 4-byte asynchronous copy (cp.async.ca; 4-byte aligned)
__device__ __forceinline__ void cp_async4(uint32_t* dst, const uint32_t* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

__device__ __forceinline__ uint64_t upper_offset(uint64_t i, uint64_t j, uint64_t n) {
  // pair (i, j), i < j, in the row-major upper triangle: S(i-1) + (j - i - 1)
  return i * (2 * n - i - 1) / 2 + (j - i - 1);
}

// Histogram accumulation.  kHistLane: every lane owns a column of the warp's
// shared array (bin b of lane l at b*32 + l), so the shared atomics of a warp
// never collide; kHistSmem: one shared array per warp; kHistGlobal: global
// atomics.  `bin` is the score minus the histogram's lowest score.
__device__ __forceinline__ void hist_add(const DpParams& P, uint32_t* wh, int lane, int bin) {
  const uint32_t bi = (uint32_t)bin;
  if (bi >= P.nbins) { atomicOr(P.err, kErrHistRange); return; }
  if (P.hist_mode == kHistLane) atomicAdd(wh + bi * 32u + (uint32_t)lane, 1u);
  else if (P.hist_mode == kHistSmem) atomicAdd(wh + bi, 1u);
  else atomicAdd(P.hist + bi, 1ull);
}

__device__ __forceinline__ void hist_flush(const DpParams& P, uint32_t* wh, int lane) {
  __syncwarp();
  if (P.hist_mode == kHistLane) {
    for (uint32_t b = lane; b < P.nbins; b += 32) {
      uint32_t c = 0;
      for (int l = 0; l < 32; ++l) {
        const uint32_t q = b * 32u + (uint32_t)((l + lane) & 31);  // rotated: no bank conflicts
        c += wh[q];
      }
      if (c) atomicAdd(P.hist + b, (unsigned long long)c);
    }
    __syncwarp();
    for (uint32_t q = lane; q < P.nbins * 32u; q += 32) wh[q] = 0u;
  } else {
    for (uint32_t b = lane; b < P.nbins; b += 32) {
      const uint32_t c = wh[b];
      if (c) { atomicAdd(P.hist + b, (unsigned long long)c); wh[b] = 0u; }
    }
  }
  __syncwarp();
}

// Lowest and highest score any pair of lengths la <= lb can reach: the
// all-gap alignment and the alignment with min(la, lb) diagonal columns bound
// the optimum from below, and no alignment beats the diagonal one with every
// diagonal column a match from above (for gap <= 0; with gap > 0 the all-gap
// alignment is the larger).
__device__ __forceinline__ void pair_score_bounds(int match, int mismatch, int gap, int la, int lb, int& lo,
                                                  int& hi) {
  const int allgap = (la + lb) * gap;
  const int diag_lo = la * mismatch + (lb - la) * gap;
  const int diag_hi = la * match + (lb - la) * gap;
  lo = allgap > diag_lo ? allgap : diag_lo;
  hi = allgap > diag_hi ? allgap : diag_hi;
}

// Word sets, lists and scoring of one task: the kernel parameters, or in a
// batched launch the terms of the segment (its dictionary or query set).
struct TaskTerms {
  const uint32_t* a_enc;
  const uint4* b_rec;
  SideView A, B;
  uint32_t C1, C2;
  int32_t match, mismatch, gap, key_lo;
  uint32_t ib, imask;
};

// List key of a pair with score s whose longer word has m symbols: the raw
// score, or the rank of s/m in the normalised ranking, above the partner's
// reversed index (higher key = better neighbour).
__device__ __forceinline__ uint32_t list_key(const DpParams& P, const TaskTerms& T, int s, int m,
                                             uint32_t partner) {
  const uint32_t v = P.norm_rank ? (uint32_t)P.norm_rank[(s - P.norm_lo) * kBuckets + m] + 1u
                                 : (uint32_t)(s - T.key_lo);
  return (v << T.ib) | (T.imask - partner);
}

// G-space candidate bound of a list whose smallest key is >= thr_key, for
// pairs whose longer word has m symbols: a pair can enter the list only if its
// G value (score - pconst) reaches this bound.  With raw keys that is the
// threshold's own score; with normalised keys, the smallest score whose s/m
// has the threshold's rank (a lower rank makes a key below any key of that
// rank, whatever the partner).
__device__ __forceinline__ int g_bound(const DpParams& P, const TaskTerms& T, uint32_t thr_key, int m, int pconst) {
  if (thr_key == 0u) return INT_MIN;
  if (P.norm_rank) return (int)P.norm_smin[((thr_key >> T.ib) - 1u) * kBuckets + m] - pconst;
  return (int)(thr_key >> T.ib) + T.key_lo - pconst;
}

// Packed candidate prefilter.  A G-space bound t (a pair is a candidate for
// a list when G >= t) is held as 1 - t, clamped so that t = 0 admits every G
// (G >= 0) and t = 0x7fff none (G <= 819 * 40 < 0x7fff: the host bounds
// s'_m * NW_MAX_WORD_LEN by 32767).  For the lane's two results packed in res,
// viaddmax_relu(res, 1 - t, 0) is non-zero in a half exactly when G >= t there.
__device__ __forceinline__ uint32_t neg_bound16(int t) {
  const int c = t < 0 ? 0 : (t > 0x7fff ? 0x7fff : t);
  return (uint32_t)(1 - c) & 0xffffu;
}
__device__ __forceinline__ uint32_t neg_bound2(int t_lo, int t_hi) {
  return neg_bound16(t_lo) | (neg_bound16(t_hi) << 16);
}

// The all-pairs kernel.  TAB selects substitution-matrix scoring (the table
// is copied to shared memory after the staging area).  EPI selects the
// per-pair epilogue at compile time:
// kEpiMatrix writes the int8 upper triangle, kEpiLists updates neighbour lists
// (and a shared or global histogram), kEpiListsLaneHist updates lists and the
// per-lane shared histogram columns, kEpiBatchLists updates the lists named
// by the segment's terms (a dictionary's own lists, or a query set's lists
// against a dictionary) in a launch spanning many dictionaries.
template <int LB, int EPI, bool TAB = false>
__global__ void __launch_bounds__(kBlock, dp_min_blocks(LB)) nw_dp_kernel(const DpParams P) {
  extern __shared__ uint32_t s_dyn[];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  constexpr bool kLists = EPI != kEpiMatrix;
  const bool smem_hist = EPI == kEpiListsLaneHist || (EPI == kEpiLists && P.hist_mode == kHistSmem);
  const uint32_t wstride = EPI == kEpiListsLaneHist ? P.nbins * 32u : (smem_hist ? P.nbins : 0u);
  uint32_t* wh = s_dyn + (size_t)wib * wstride;
  // this warp's staging area: symbol i of the chunk's word w at sA[32 * i + w],
  // followed by the 32 words' list bounds (raw keys) at sT[w]
  uint32_t* sA = s_dyn + (size_t)kWarpsPerBlock * wstride + (size_t)wib * 32u * (uint32_t)(LB + 1);
  uint32_t* sT = sA + 32u * (uint32_t)LB;
  uint16_t* sTab = nullptr;
  if constexpr (TAB) {
    sTab = reinterpret_cast<uint16_t*>(s_dyn + (size_t)kWarpsPerBlock * wstride +
                                       (size_t)kWarpsPerBlock * 32u * (uint32_t)(LB + 1));
    const uint4* src = reinterpret_cast<const uint4*>(P.sim_tab);
    uint4* dst = reinterpret_cast<uint4*>(sTab);
    for (int q = threadIdx.x; q < (int)(kTabBytes / sizeof(uint4)); q += blockDim.x) dst[q] = __ldg(src + q);
    __syncthreads();
  }
  if (smem_hist) {
    for (uint32_t q = lane; q < wstride; q += 32) wh[q] = 0u;
    __syncwarp();
  }
  uint64_t wpairs = 0;
  uint32_t inserts = 0;
  const int max_iters = P.dbg_insert_limit ? (int)(P.dbg_insert_limit - 1u) : kInsertMaxIters;

  for (;;) {
    unsigned long long t = 0;
    if (lane == 0) t = atomicAdd(P.counter, 1ull);
    t = __shfl_sync(0xffffffffu, t, 0) + P.task_lo;
    if (t >= P.task_hi) break;

    const Seg S = P.segs[find_seg(P.segs, P.nsegs, t)];
    const TaskGeom g = task_geom(S, t, P.TA);
    TaskTerms T;
    if constexpr (EPI == kEpiBatchLists) {
      const DictTerms& D = P.terms[S.dict];
      T = TaskTerms{D.a_enc, D.b_rec, D.A, D.B, D.C1, D.C2, D.match, D.mismatch, D.gap, D.key_lo, D.ib, D.imask};
    } else {
      T = TaskTerms{P.a_enc, P.b_rec, P.A, P.B, P.C1, P.C2, P.match, P.mismatch, P.gap, P.key_lo, P.ib, P.imask};
    }
    const bool listsA = kLists && T.A.slots != nullptr;
    // (queries run without a histogram: the histogram kernels keep the lanes' own offers)
    const bool serialA = EPI == kEpiLists && listsA && P.serial_a != 0u;
    const bool listsB = kLists && T.B.slots != nullptr;
    const uint32_t blo = g.b0 + 2u * lane;
    const uint32_t bhi = blo + 1u;
    const bool vlo = blo < g.bend;
    const bool vhi = bhi < g.bend;
    const bool check = g.tri && g.a1 > g.b0;  // the task straddles the diagonal: test a < b
    const int la = S.la;
    const int pconst = T.gap * (la + LB);  // score = G + pconst
    const int hoff = pconst - P.hist_lo;   // histogram bin = G + hoff

    // every bin this task can produce lies inside the histogram (proven
    // bounds); checked once here instead of per pair
    bool hist_on = (EPI == kEpiLists || EPI == kEpiListsLaneHist) && P.hist_mode != kHistNone;
    if (hist_on) {
      int lo, hi;
      pair_score_bounds(T.match, T.mismatch, T.gap, la, LB, lo, hi);
      if (lo < P.hist_lo || hi - P.hist_lo >= (int)P.nbins) {
        if (lane == 0) atomicOr(P.err, kErrHistRange);
        hist_on = false;
      }
    }
    uint32_t* hcol = wh + (ptrdiff_t)lane + (ptrdiff_t)hoff * 32;  // lane column shifted so bin = G

    BRow<LB> brow;
    if constexpr (LB > 0) {
#pragma unroll
      for (int j = 0; j < LB; ++j) brow.v[j] = 0xffffffffu;
      if (vlo) load_brow<LB>(T.b_rec + S.brec_base + (size_t)(g.cb * (kWarpB / 2) + lane) * (ceil4(LB) / 4), brow);
      if constexpr (TAB) {
        // records hold ~code per half (unshifted codes): back to codes, and
        // code 0 for halves without a word (their results are discarded)
        const uint32_t keep = (vlo ? 0x0000ffffu : 0u) | (vhi ? 0xffff0000u : 0u);
#pragma unroll
        for (int j = 0; j < LB; ++j) brow.v[j] = ~brow.v[j] & keep;
      }
    }
    const uint32_t ob_lo = vlo ? __ldg(T.B.perm + blo) : 0u;
    const uint32_t ob_hi = vhi ? __ldg(T.B.perm + bhi) : 0u;
    // B-side lists: cached smallest keys and their G-space candidate bounds
    uint32_t thrB_lo = 0u, thrB_hi = 0u;
    int tB_lo = INT_MAX, tB_hi = INT_MAX;
    if (listsB) {
      if (vlo) { thrB_lo = __ldcg(T.B.thr + blo); tB_lo = g_bound(P, T, thrB_lo, LB, pconst); }
      if (vhi) { thrB_hi = __ldcg(T.B.thr + bhi); tB_hi = g_bound(P, T, thrB_hi, LB, pconst); }
    }
    // packed form of the B bounds for the prefilter, and the halves holding a word
    uint32_t nB2 = neg_bound2(tB_lo, tB_hi);
    const uint32_t okmask = (vlo ? 0x0000ffffu : 0u) | (vhi ? 0xffff0000u : 0u);

    for (uint32_t c0 = g.a0; c0 < g.a1; c0 += 32u) {
      // Stage 32 A words: lane l copies word c0 + l (la symbols) and its list
      // bound; the warp then reads symbols as shared-memory broadcasts and the
      // G-space bound by shuffle.
      const uint32_t nA = g.a1 - c0 < 32u ? g.a1 - c0 : 32u;
      const uint32_t my_a = c0 + (uint32_t)lane;
      const bool have = (uint32_t)lane < nA;
      const uint32_t my_orig = (EPI == kEpiMatrix && have) ? __ldg(T.A.perm + my_a) : 0u;
      const uint32_t my_thr = (listsA && have) ? __ldcg(T.A.thr + my_a) : 0u;
      const int my_tA = listsA ? g_bound(P, T, my_thr, LB, pconst) : INT_MAX;
      const uint32_t my_nA2 = neg_bound2(my_tA, my_tA);
      __syncwarp();
      if (have) {
        // asynchronous 4-byte copies: the word's symbol loads are in flight together
        const uint32_t* src = T.a_enc + S.aenc_base + (size_t)(my_a - S.a_beg) * (uint32_t)la;
        for (int i = 0; i < la; ++i) cp_async4(sA + 32 * i + lane, src + i);
        sT[lane] = my_thr;
      }
      cp_async_wait_all();
      __syncwarp();

      for (uint32_t w = 0; w < nA; ++w) {
        const uint32_t a = c0 + w;
        const uint32_t res = dp_word_staged<LB, TAB>(sA + w, la, brow, T.C1, T.C2, sTab);
        const int g_lo = (int)(res & 0xffffu);  // G >= 0
        const int g_hi = (int)(res >> 16);
        bool ok_lo = vlo, ok_hi = vhi;
        if (check) {
          ok_lo = ok_lo && a < blo;
          ok_hi = ok_hi && a < bhi;
        }

        if constexpr (EPI == kEpiMatrix) {
          const uint32_t oa = __shfl_sync(0xffffffffu, my_orig, (int)w);
          if (ok_lo) {
            const uint64_t i = oa < ob_lo ? oa : ob_lo, j = oa < ob_lo ? ob_lo : oa;
            const uint64_t off = upper_offset(i, j, P.n);
            if (off >= P.mat_lo && off < P.mat_hi) P.mat[off] = (int8_t)(g_lo + pconst);
          }
          if (ok_hi) {
            const uint64_t i = oa < ob_hi ? oa : ob_hi, j = oa < ob_hi ? ob_hi : oa;
            const uint64_t off = upper_offset(i, j, P.n);
            if (off >= P.mat_lo && off < P.mat_hi) P.mat[off] = (int8_t)(g_hi + pconst);
          }
        } else {
          if (hist_on) {
            if constexpr (EPI == kEpiListsLaneHist) {
              // lane columns are private to their lane: plain increments
              if (ok_lo) hcol[32 * g_lo] += 1u;
              if (ok_hi) hcol[32 * g_hi] += 1u;
            } else {
              if (ok_lo) hist_add(P, wh, lane, g_lo + hoff);
              if (ok_hi) hist_add(P, wh, lane, g_hi + hoff);
            }
          }
          // Both halves tested at once against the lower of the two lists'
          // bounds (packed prefilter, exact: see neg_bound16); tasks on the
          // diagonal, which must also test a < b, skip it.  Exact keys are
          // formed only for the rare candidates.
          const uint32_t nA2 = __shfl_sync(0xffffffffu, my_nA2, (int)w);
          const bool pre = check || (__viaddmax_s16x2_relu(res, __vmaxs2(nB2, nA2), 0u) & okmask) != 0u;
          uint32_t ka_lo = 0u, ka_hi = 0u;  // this lane's keys for the A word's list
          if (pre) {
            const uint32_t thrA = sT[w];
            const int tA = listsA ? g_bound(P, T, thrA, LB, pconst) : INT_MAX;
            const bool c_lo = ok_lo && g_lo >= min(tB_lo, tA);
            const bool c_hi = ok_hi && g_hi >= min(tB_hi, tA);
            if (c_lo || c_hi) {
              const uint32_t oa = __ldg(T.A.perm + a);
              if (c_lo) {
                const int s = g_lo + pconst;
                if (g_lo >= tB_lo) {  // the lane's word takes the A word as a neighbour
                  const uint32_t key = list_key(P, T, s, LB, oa);
                  if (key > thrB_lo) {
                    const uint32_t nm = list_offer(T.B.slots + (size_t)blo * P.k, T.B.thr + blo, P.k, key, P.err, inserts, max_iters);
                    if (nm > thrB_lo) {
                      thrB_lo = nm;
                      tB_lo = g_bound(P, T, nm, LB, pconst);
                      nB2 = neg_bound2(tB_lo, tB_hi);
                    }
                  }
                }
                if (g_lo >= tA) {  // the A word takes the lane's word as a neighbour
                  const uint32_t key = list_key(P, T, s, LB, ob_lo);
                  if (key > thrA) {
                    if (serialA) ka_lo = key;
                    else list_offer(T.A.slots + (size_t)a * P.k, T.A.thr + a, P.k, key, P.err, inserts, max_iters);
                  }
                }
              }
              if (c_hi) {
                const int s = g_hi + pconst;
                if (g_hi >= tB_hi) {
                  const uint32_t key = list_key(P, T, s, LB, oa);
                  if (key > thrB_hi) {
                    const uint32_t nm = list_offer(T.B.slots + (size_t)bhi * P.k, T.B.thr + bhi, P.k, key, P.err, inserts, max_iters);
                    if (nm > thrB_hi) {
                      thrB_hi = nm;
                      tB_hi = g_bound(P, T, nm, LB, pconst);
                      nB2 = neg_bound2(tB_lo, tB_hi);
                    }
                  }
                }
                if (g_hi >= tA) {
                  const uint32_t key = list_key(P, T, s, LB, ob_hi);
                  if (key > thrA) {
                    if (serialA) ka_hi = key;
                    else list_offer(T.A.slots + (size_t)a * P.k, T.A.thr + a, P.k, key, P.err, inserts, max_iters);
                  }
                }
              }
            }
          }
          if (serialA) {
            // Every lane may hold keys for the same A word's list.  The warp
            // offers them one at a time from the best down, each against the
            // bound the previous offer returned, and stops at the first key
            // below it: the lanes never race on that list, and a list that
            // is already full costs one offer.
            uint32_t best = ka_lo > ka_hi ? ka_lo : ka_hi;
            uint32_t thrW = sT[w];
            while (__any_sync(0xffffffffu, best > thrW)) {
              const uint32_t m = __reduce_max_sync(0xffffffffu, best);
              const int src = __ffs(__ballot_sync(0xffffffffu, best == m)) - 1;
              uint32_t nm = 0u;
              if (lane == src) {
                nm = list_offer(T.A.slots + (size_t)a * P.k, T.A.thr + a, P.k, m, P.err, inserts, max_iters);
                if (ka_lo == m) ka_lo = 0u; else ka_hi = 0u;
                best = ka_lo > ka_hi ? ka_lo : ka_hi;
              }
              nm = __shfl_sync(0xffffffffu, nm, src);
              thrW = nm > thrW ? nm : thrW;
            }
          }
        }
      }
    }
    if (smem_hist) {  // 32-bit shared counters: flush long before they could wrap
      wpairs += (uint64_t)(g.a1 - g.a0) * 64u;
      if (wpairs >= (1ull << 30)) { hist_flush(P, wh, lane); wpairs = 0; }
    }
  }

  if (smem_hist) hist_flush(P, wh, lane);
  if (P.stats) {
    for (int o = 16; o > 0; o >>= 1) inserts += __shfl_xor_sync(0xffffffffu, inserts, o);
    if (lane == 0 && inserts) atomicAdd(P.stats, (unsigned long long)inserts);
  }
}

}  // namespace nw
