// nw_internal.cuh -- data layout, task geometry and kernel parameters of libnw.
//
// Words of a set (a dictionary or a batch of queries) are sorted stably by
// length into buckets (bucket L holds the words of length L in original-index
// order).  A word is addressed by its sorted position.  Every unordered pair
// of words is scored once: by the alignment kernel instantiated for LB = the
// longer length, with the longer word held by a lane ("B side") and the
// shorter word streamed to the whole warp ("A side").
//
// Encoded symbols (both built at load time for the scoring of the set):
//   e(c)  = c << shift, with 2^shift >= match - mismatch, so two different
//           codes differ by at least match - mismatch after XOR.
//   a_enc = e(c) replicated into both 16-bit halves, one uint32 per symbol,
//           each word's symbols contiguous.
//   b_rec = pair records: the words at even/odd positions 2m, 2m+1 of a bucket
//           share a record of ceil4(L) uint32, entry j = (~e(c_2m[j]) & 0xffff)
//           | (~e(c_2m+1[j]) << 16); a lane loads one record with 16-byte loads.
#pragma once

#include <stdint.h>

#include "nw.h"

#ifndef __CUDACC__
#define __host__
#define __device__
#define __forceinline__ inline
#endif

namespace nw {

constexpr int kMaxLen = NW_MAX_WORD_LEN;
constexpr int kBuckets = kMaxLen + 1;  // lengths 0 .. kMaxLen
constexpr int kBlock = 256;            // threads per block of the alignment kernel
constexpr int kWarpB = 64;             // B words per warp task (two per lane)
constexpr int kWarpsPerBlock = kBlock / 32;
constexpr uint32_t kDefaultTA = 256;   // A words per task
constexpr uint32_t kHistSmemMaxBins = 1024;
constexpr int kInsertMaxIters = 1 << 20;

// error bits raised by kernels (read back by the host)
constexpr uint32_t kErrRetry = 1u;      // a list insertion exceeded its retry bound
constexpr uint32_t kErrHistRange = 2u;  // a score fell outside the histogram bins
constexpr uint32_t kErrInput = 4u;      // invalid input seen on the device (code/length/index)
constexpr uint32_t kErrWait = 8u;       // a pipeline wait ran out (the kernel stopped early)
constexpr uint32_t kErrCapacity = 16u;  // a buffer would have overflowed (the access was skipped)

__host__ __device__ constexpr int ceil4(int x) { return (x + 3) & ~3; }

// Bucket tables of a word set, by length.
struct Buckets {
  uint32_t count[kBuckets];      // words of length L
  uint32_t start[kBuckets + 1];  // first sorted position of bucket L
  uint32_t aenc_base[kBuckets];  // a_enc index of the bucket's first symbol
  uint32_t brec_word_base[kBuckets];  // b_rec uint32 offset of the bucket's first record (multiple of 4)
};

// A rectangle of pairs: A positions [a_beg, a_end) x B positions [b_beg, b_end),
// all A words of length la and all B words of the launch's length LB.  With tri,
// A and B are the same bucket of the same set and only pairs a < b are scored.
struct Seg {
  uint32_t a_beg, a_end;
  uint32_t b_beg, b_end;
  uint32_t aenc_base;   // a_enc index of word a_beg's first symbol
  uint32_t brec_base;   // uint4 index into b_rec of the record holding b_beg
                        // (b_beg - bucket start is even; records of bucket LB are ceil4(LB)/4 uint4 apart)
  uint16_t la;
  uint16_t tri;
  uint32_t nca;         // A chunks (tasks = nca * ceil((b_end - b_beg) / kWarpB))
  uint32_t dict;        // terms of the segment in a batched launch (else 0)
  uint64_t task0;       // first task of the segment within its launch
};

// One side of a launch: the word set providing A (or B) words.
struct SideView {
  const uint32_t* perm;   // sorted position -> original index of the set
  uint32_t* slots;        // k list slots per word (sorted position), or null
  uint32_t* thr;          // per-word lower bound of the k-th best key, or null
};

// Terms of one kind of segment in a batched launch (indexed by Seg::dict):
// the A and B word sets with their lists and the scoring constants.  A
// dictionary's own pairs take A = B = the dictionary with its lists; a query
// set against a dictionary takes the query words on one side (with the
// queries' lists) and the dictionary on the other (no lists).
struct DictTerms {
  const uint32_t* a_enc;
  const uint4* b_rec;
  SideView A, B;
  uint32_t C1, C2;
  int32_t match, mismatch, gap;
  int32_t key_lo;
  uint32_t ib, imask;
};

struct TaskGeom {
  uint32_t a0, a1;      // A positions of the task
  uint32_t b0, bend;    // B chunk [b0, bend)
  uint32_t ca, cb;      // chunk coordinates
  bool tri;
};

__host__ __device__ __forceinline__ uint32_t find_seg(const Seg* segs, uint32_t nsegs, uint64_t t) {
  uint32_t lo = 0, hi = nsegs;
  while (hi - lo > 1) {
    uint32_t mid = (lo + hi) >> 1;
    if (segs[mid].task0 <= t) lo = mid; else hi = mid;
  }
  return lo;
}

__host__ __device__ __forceinline__ TaskGeom task_geom(const Seg& S, uint64_t t, uint32_t TA) {
  TaskGeom g;
  uint64_t local = t - S.task0;
  g.ca = (uint32_t)(local % S.nca);
  g.cb = (uint32_t)(local / S.nca);
  g.a0 = S.a_beg + g.ca * TA;
  g.a1 = S.a_end < g.a0 + TA ? S.a_end : g.a0 + TA;
  g.b0 = S.b_beg + g.cb * (uint32_t)kWarpB;
  g.bend = S.b_end < g.b0 + (uint32_t)kWarpB ? S.b_end : g.b0 + (uint32_t)kWarpB;
  g.tri = S.tri != 0;
  if (g.tri && g.a1 > g.bend - 1) g.a1 = g.bend - 1;  // some b > a must exist
  if (g.a1 < g.a0) g.a1 = g.a0;
  return g;
}

__host__ __device__ __forceinline__ bool pair_valid(const TaskGeom& g, uint32_t a, uint32_t b) {
  return b < g.bend && (!g.tri || a < b);
}

// The k best distinct neighbours of one word from nparts ranked lists (each
// sorted by score descending, then index ascending, UINT32_MAX entries
// ending it): a k-way merge.  at(p, r) gives entry r of list p as
// (index, score); an index met in two lists carries the same score there and
// is kept once (the two copies are adjacent in the merged order).
constexpr uint32_t kMaxMergeParts = 64;
template <class At>
__host__ __device__ inline void merge_ranked_row(uint32_t nparts, uint32_t k, At at, uint32_t* out_idx,
                                                 int16_t* out_score) {
  uint32_t pos[kMaxMergeParts];
  for (uint32_t p = 0; p < nparts; ++p) pos[p] = 0;
  uint32_t r = 0, last = 0xffffffffu;
  while (r < k) {
    int best = -1;
    int32_t bs = 0;
    uint32_t bi = 0;
    for (uint32_t p = 0; p < nparts; ++p) {
      if (pos[p] >= k) continue;
      uint32_t j;
      int32_t s;
      at(p, pos[p], j, s);
      if (j == 0xffffffffu) continue;
      if (best < 0 || s > bs || (s == bs && j < bi)) {
        best = (int)p;
        bs = s;
        bi = j;
      }
    }
    if (best < 0) break;
    ++pos[best];
    if (bi == last) continue;  // the same neighbour from two lists
    out_idx[r] = bi;
    out_score[r] = (int16_t)bs;
    last = bi;
    ++r;
  }
  for (; r < k; ++r) {
    out_idx[r] = 0xffffffffu;
    out_score[r] = (int16_t)-32768;
  }
}

enum { kModeMatrix = 0, kModeLists = 1 };
enum { kHistNone = 0, kHistSmem = 1, kHistGlobal = 2, kHistLane = 3 };

// Blocks per SM the alignment kernel is compiled for: the register budget
// shrinks with LB (the lane keeps LB registers of B symbols and LB of DP row).
__host__ __device__ constexpr int dp_min_blocks(int LB) { return LB <= 10 ? 4 : (LB <= 20 ? 3 : 2); }

// Shared memory each block of the LB kernel stages A words in: every warp
// holds 32 words of at most LB symbols and their 32 list bounds (after the
// histogram area).
__host__ __device__ constexpr size_t dp_stage_bytes(int LB) {
  return (size_t)kWarpsPerBlock * 32u * (size_t)(LB + 1) * sizeof(uint32_t);
}

// per-pair epilogue of the all-pairs kernel (a template parameter);
// kEpiBatchLists takes word sets, lists and scoring per task from DpParams::terms
enum { kEpiMatrix = 0, kEpiLists = 1, kEpiListsLaneHist = 2, kEpiBatchLists = 3, kEpiKinds = 4 };

// Histogram accumulation mode for `nbins` bins and the dynamic shared memory
// it needs per block: per-lane columns while they fit in 48 KiB, else one
// shared array per warp, else global atomics.
inline int hist_mode_for(uint32_t nbins) {
  if ((size_t)nbins * 32u * sizeof(uint32_t) * kWarpsPerBlock <= 48u * 1024u) return kHistLane;
  if (nbins <= kHistSmemMaxBins) return kHistSmem;
  return kHistGlobal;
}
inline size_t hist_smem_bytes(int mode, uint32_t nbins) {
  if (mode == kHistLane) return (size_t)kWarpsPerBlock * nbins * 32u * sizeof(uint32_t);
  if (mode == kHistSmem) return (size_t)kWarpsPerBlock * nbins * sizeof(uint32_t);
  return 0;
}

struct DpParams {
  const Seg* segs;
  uint32_t nsegs;
  uint32_t TA;
  uint64_t task_lo, task_hi;      // task slice handled by this launch
  unsigned long long* counter;    // zeroed before the launch
  const uint32_t* a_enc;          // A set
  const uint4* b_rec;             // B set
  SideView A, B;
  uint32_t C1, C2;                // packed (s'_m + 1) and max(s'_x, 0), see the kernel
  int32_t match, mismatch, gap;
  int32_t mode;
  int8_t* mat;                    // matrix mode: row-major upper triangle, entries [mat_lo, mat_hi) stored
  uint64_t n;
  uint64_t mat_lo, mat_hi;        // (mat points at the buffer holding entry mat_lo, minus mat_lo)
  uint32_t k, ib, imask;          // list key = ((s - key_lo) << ib) | (imask - partner)
  int32_t key_lo;
  int32_t hist_mode;
  unsigned long long* hist;
  int32_t hist_lo;
  uint32_t nbins;
  unsigned long long* stats;      // [0] list inserts
  uint32_t* err;
  const DictTerms* terms;         // batched launches: per-dictionary terms (device), else null
  // length-normalised ranking (null = raw scores): rank of s / max(la, lb) at
  // norm_rank[(s - norm_lo) * kBuckets + m], and the smallest s reaching rank r
  // for longer length m at norm_smin[r * kBuckets + m]
  const uint16_t* norm_rank;
  const int16_t* norm_smin;
  int32_t norm_lo;
  // substitution-matrix scoring (null = match / mismatch): kTabDim x kTabDim
  // table of s'+(a, b) = max(sim(a, b) - 2p, 0), copied to shared memory
  const uint16_t* sim_tab;
  // debug setting: 0 = list insertions retry up to kInsertMaxIters times;
  // otherwise they give up after dbg_insert_limit - 1 tries (NW_ETIMEOUT)
  uint32_t dbg_insert_limit;
  // nonzero: the A words' list offers of one A word go through the warp one at
  // a time (A words that many tasks share, such as query words, whose lists
  // the 64 lanes of a task would otherwise race on)
  uint32_t serial_a;
};

// The substitution table of a dictionary scored with a full similarity
// matrix: row a holds s'+(a, b) for b < kTabDim (zero past the alphabet).  A
// row of 64 16-bit entries covers the 32 shared-memory banks once, so the 32
// lanes' lookups into one row never conflict.
constexpr int kTabDim = 64;
constexpr size_t kTabBytes = (size_t)kTabDim * kTabDim * sizeof(uint16_t);

// Scoring constants of the shifted recurrence (see the kernel).
struct ShiftedScoring {
  int32_t sm, sx;   // s'_m = match - 2*gap, s'_x = mismatch - 2*gap
  uint32_t shift;   // code shift of the XOR encoding
  uint32_t C1, C2;  // packed 16x2 constants
};

}  // namespace nw
