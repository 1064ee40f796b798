// nw_dot_topk.cu -- candidate proposal by quantised embedding products, on the
// fifth-generation tensor cores (tcgen05, accumulators in tensor memory).
//
// Exactness.  Features are quantised to integers in [-127, 127] (exact in
// bf16) and a column's bias b (|b| <= 2^23) is split into three bf16-exact
// digits, b = b2 * 2^16 + b1 * 2^8 + b0 with b0, b1 in [0, 256) and b2 in
// [-128, 128]; a row carries the matching weights (2^16, 2^8, 1).  The products
// of one output are then integers, and so is every partial sum (|.| < 2^24), so
// the tensor cores' float32 accumulation gives q_i . q_j + b_j exactly, in any
// order, and the top-C selection is an exact, deterministic function of the
// integers (ties: lower column index first).
//
// dot_topk_kernel: a CTA owns two blocks of 128 rows (each block fills the
// 128 lanes of tensor memory) and sweeps column tiles of 128.  Fourteen warps
// with fixed roles:
//   * a producer thread streams each tile (128 rows of 128 B by a 2-D
//     tensor-map copy, cp.async.bulk.tensor, whose 128-byte swizzle lays them
//     out as the K-major operand, plus 4 KiB of bias digits by cp.async.bulk)
//     into a four-stage shared-memory ring, counted on mbarriers; the CTA's
//     own 256 rows arrive once the same way; every tile feeds both row blocks;
//   * an MMA thread issues, per tile and row block, four tcgen05.mma
//     (M = 128, N = 128, K = 16, bf16 -> f32) over the 64 features and a fifth
//     over the bias digits into one of the block's two accumulators, then
//     commits the stage back to the producer and the accumulators to the
//     epilogue;
//   * eight epilogue warps (two per SM sub-partition, so each hides the
//     other's latency), one thread per row, read the accumulator with
//     tcgen05.ld (32 columns at a time, the next load in flight while the
//     current values are tested), release it, and append every value that
//     reaches the row's threshold to one of the row's two global buffers;
//   * compactor warps: when a row's active buffer passes its trigger, the
//     epilogue thread hands the buffer over and keeps appending to the other
//     one; a compactor stages the handed keys and the other buffer's kept keys
//     in shared memory, raises the row's threshold to a value at or below the
//     C-th best of them and drops the handed keys below it, off the path of
//     the tensor pipe.
// A key is appended when its value is >= the threshold, so the column order
// does not change the result, only the time: every key of the final top C is
// always kept (each threshold is at most the C-th best value among keys
// already seen).  A CTA visits its column tiles outward from its own diagonal
// tile; with the rows in a locality order (sweep_order: sorted by length and
// principal components, keys carrying the original ids) a row's best columns
// come early and its threshold rises sooner.  A final pass selects each row's
// C best keys from its two buffers exactly (a value histogram, then the exact
// select among the keys of the boundary bin) and sorts them when the caller
// wants sorted lists.  Every wait is bounded and sets kErrWait when it runs
// out; the CTA then stops, waits (bounded) for the copies and products it
// issued, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <algorithm>
#include <cstring>
#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

#include "nw_internal.cuh"
#include "nw_proposal.h"
#include "nw_proposal_internal.h"
#include "nw_tc.cuh"

namespace nw {
namespace prop {
namespace {

constexpr int kDim = 64;                  // values per row (bf16)
constexpr int kRowBytes = kDim * 2;       // 128
constexpr int kRows = 128;                // rows of one MMA = tensor-memory lanes
constexpr int kBlocksPerCta = 2;          // row blocks per CTA (each B tile feeds both)
constexpr int kCtaRows = kRows * kBlocksPerCta;
constexpr int kTileN = 128;               // columns per tile (MMA N)
constexpr int kPadRows = 256;             // row and column sets are zero-padded to this
constexpr int kExtK = 16;                 // bias-digit K (one MMA K-step)
constexpr int kStages = 4;
constexpr int kMainBytes = kTileN * kRowBytes;          // 16 KiB
constexpr int kExtBytes = kTileN * kExtK * 2;           // 4 KiB
constexpr int kStageBytes = kMainBytes + kExtBytes;     // 20 KiB
constexpr int kAMainBytes = kRows * kRowBytes;          // 16 KiB per row block
constexpr int kAExtBytes = kRows * kExtK * 2;           // 4 KiB (the same for both blocks)
constexpr int kEpiWarps = 8;                            // warps 0..7: block = warp / 4, lanes 32 * (warp % 4)
constexpr int kProducerWarp = 8;
constexpr int kMmaWarp = 9;
constexpr int kCompWarps = 4;                           // warps 10..13
constexpr int kWarps = kEpiWarps + 2 + kCompWarps;
constexpr int kThreads = kWarps * 32;
constexpr int kChunks = kTileN / 32;                    // 32-column chunks of a tile
constexpr int kSel = NW_MAX_CANDIDATES;                 // per-warp gather/sort area (keys)
constexpr uint32_t kTmemCols = 2 * kBlocksPerCta * kTileN;  // two accumulators per block: 512

// dynamic shared memory (bytes from a 1024-aligned base)
constexpr int kOffAMain = 0;
constexpr int kOffAExt = kOffAMain + kBlocksPerCta * kAMainBytes;
constexpr int kOffStages = kOffAExt + kAExtBytes;
// compactor warps: a 256-bin histogram each and one staging area for the
// handed-over keys and the kept keys of the row's other buffer, split into
// kCompWarps areas of 1,536 keys (hand-overs of up to 1,024 keys, C <= 256) or
// two of 3,072 (hand-overs of up to 2,048 keys, larger C: two compactors)
constexpr int kStageKeysTotal = 6144;
constexpr int kOffCompHist = kOffStages + kStages * kStageBytes;
constexpr int kOffCompKeys = kOffCompHist + kCompWarps * 1024;
// epilogue: each thread's 32 values of a chunk with hits, staged so that the
// hits can be read by index (row stride 36 floats: conflict-free 16-byte stores)
constexpr int kValStride = 36;
constexpr int kOffVals = kOffCompKeys + kStageKeysTotal * 8;
constexpr int kOffRow = kOffVals + kCtaRows * kValStride * 4;
constexpr int kFinalSort = 2 * NW_MAX_CANDIDATES;      // final pass: keys sorted per row at most
constexpr int kFinalBytes = 256 * 4 + kFinalSort * 8;  // final pass: histogram + sort area per warp
// row state: threshold, kept counts of the two buffers, hand-over request, final state
constexpr int kOffThr = kOffRow;
constexpr int kOffKept = kOffThr + kCtaRows * 4;
constexpr int kOffReq = kOffKept + kCtaRows * 8;
constexpr int kOffFin = kOffReq + kCtaRows * 4;
constexpr int kOffHi = kOffFin + kCtaRows * 4;          // per row: a bound on every value appended
constexpr int kOffMisc = kOffHi + kCtaRows * 4;        // request masks, done flags, tmem address, progress
constexpr int kOffBars = kOffMisc + 128;
constexpr int kNumBars = 2 * kStages + 4 + 1;          // full, empty, acc full x2, acc empty x2, A loaded
// per epilogue warp: the original ids of the current tile's columns (sweeps
// over rows in a locality order)
constexpr int kOffIds = (kOffBars + kNumBars * 8 + 15) / 16 * 16;
constexpr int kSmemUsed = kOffIds + kEpiWarps * kTileN * 4;
constexpr int kSmemTotal = kSmemUsed + 1024;           // slack for aligning the base
static_assert(kSmemTotal <= 227 * 1024, "one CTA per SM");
// the final pass reuses the ring, compactor and value areas: per warp a
// histogram and a sort area
static_assert(kOffStages + kWarps * kFinalBytes <= kOffRow, "final-pass scratch stays below the row state");
static_assert(kCap >= 2 * NW_MAX_CANDIDATES + 256, "a buffer holds a compaction's keys and a tile");
static_assert(kPadRows % kCtaRows == 0 && kPadRows % kTileN == 0, "padding covers whole row blocks and tiles");
// a pipeline wait gives up after this many SM clock cycles (about a second)
constexpr long long kWaitCycles = 2000000000ll;

using tc::bulk_g2s;
using tc::mbar_arrive;
using tc::mbar_expect_tx;
using tc::mbar_init;
using tc::mbar_wait;
using tc::smem_desc;
using tc::smem_u32;
using tc::tmem_ld32;
using tc::tmem_wait;
__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(smem_u32(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// instruction descriptor of the products: f32 accumulator, bf16 A and B,
// both K-major, M = 128 rows, N = one 128-column tile
constexpr uint32_t kIdesc = tc::idesc_bf16(kRows, kTileN);
__device__ __forceinline__ void tc_fence_before() { tc::fence_before(); }
__device__ __forceinline__ void tc_fence_after() { tc::fence_after(); }
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t accumulate) {
  tc::mma(d, a, b, kIdesc, accumulate);
}
__device__ __forceinline__ void tc_commit(uint32_t bar) { tc::commit(bar); }

__device__ __forceinline__ float fmax3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;\n" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Byte offset of element (row r, k) of a K = 16 bf16 tile in the canonical
// K-major layout without swizzle: 8-row x 16-byte core matrices, the two K
// halves 128 bytes apart, 8-row groups 256 bytes apart.
__host__ __device__ __forceinline__ uint32_t ext_offset(uint32_t r, uint32_t k) {
  return (r >> 3) * 256u + (k >> 3) * 128u + (r & 7u) * 16u + (k & 7u) * 2u;
}

// key: higher value first, then lower index; 0 sorts below every real key
__device__ __forceinline__ uint64_t make_key(int v, uint32_t j) {
  return ((uint64_t)(uint32_t)(v + 0x80000000) << 32) | (uint64_t)(0xffffffffu - j);
}
__device__ __forceinline__ int key_val(uint64_t k) { return (int)((uint32_t)(k >> 32) - 0x80000000u); }
__device__ __forceinline__ uint32_t key_idx(uint64_t k) { return 0xffffffffu - (uint32_t)k; }

// Sorts s[0, size) descending (size a power of two) with the warp.
__device__ void warp_bitonic_desc(uint64_t* s, int size, int lane) {
  __syncwarp();
  for (int k = 2; k <= size; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = lane; i < size; i += 32) {
        const int p = i ^ j;
        if (p > i) {
          const uint64_t a = s[i], b = s[p];
          const bool desc = (i & k) == 0;
          if (desc ? (a < b) : (a > b)) {
            s[i] = b;
            s[p] = a;
          }
        }
      }
      __syncwarp();
    }
  }
}

// A warp's 256-bin histogram scanned from the top bin down: the bin in which
// the running count reaches need (1 <= need <= total), and the count of the
// bins above it.
__device__ __forceinline__ void hist_find_desc(const unsigned* hist, unsigned need, int lane, int& bin,
                                               unsigned& before) {
  // lane l holds bins 255 - 8l .. 248 - 8l (descending order)
  unsigned c[8], tot = 0;
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    c[q] = hist[255 - 8 * lane - q];
    tot += c[q];
  }
  unsigned incl = tot;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  const unsigned excl = incl - tot;
  const bool mine = excl < need && need <= incl;
  const unsigned ball = __ballot_sync(0xffffffffu, mine);
  const int src = __ffs(ball) - 1;
  int b = 0;
  unsigned bef = 0;
  if (mine) {
    unsigned acc = excl;
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if (acc + c[q] >= need) {
        b = 255 - 8 * lane - q;
        bef = acc;
        break;
      }
      acc += c[q];
    }
  }
  bin = __shfl_sync(0xffffffffu, b, src);
  before = __shfl_sync(0xffffffffu, bef, src);
}

// Row-buffer passes read kBatch keys per lane before using any of them, so
// their loads are in flight together.
constexpr int kBatch = 8;

// The r-th largest (1-based) of the cnt distinct keys buf[0, cnt), r <= cnt:
// one 8-bit digit per pass from the top, counting only keys that share the
// digits found so far.
__device__ uint64_t warp_select_kth(const uint64_t* buf, int cnt, int r, unsigned* hist, int lane) {
  uint64_t prefix = 0;
  unsigned need = (unsigned)r;
  for (int byte = 7; byte >= 0; --byte) {
    const int sh = byte * 8;
    const uint64_t hmask = byte == 7 ? 0ull : (~0ull << (sh + 8));
    for (int b = lane; b < 256; b += 32) hist[b] = 0u;
    __syncwarp();
    for (int i0 = 0; i0 < cnt; i0 += 32 * kBatch) {
      uint64_t k[kBatch];
#pragma unroll
      for (int u = 0; u < kBatch; ++u) {
        const int i = i0 + 32 * u + lane;
        k[u] = i < cnt ? buf[i] : 0ull;
      }
#pragma unroll
      for (int u = 0; u < kBatch; ++u)
        if (i0 + 32 * u + lane < cnt && (k[u] & hmask) == prefix) atomicAdd(&hist[(uint32_t)(k[u] >> sh) & 255u], 1u);
    }
    __syncwarp();
    int bin;
    unsigned before;
    hist_find_desc(hist, need, lane, bin, before);
    prefix |= (uint64_t)bin << sh;
    need -= before;
    __syncwarp();
  }
  return prefix;
}

// Copies the keys >= kmin of buf[0, cnt) into s (in their order); returns
// how many.  s may be buf itself (each key moves down or stays).
__device__ int warp_gather_ge(const uint64_t* buf, int cnt, uint64_t kmin, uint64_t* s, int lane) {
  int base = 0;
  for (int i0 = 0; i0 < cnt; i0 += 32 * kBatch) {
    uint64_t k[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int i = i0 + 32 * u + lane;
      k[u] = i < cnt ? buf[i] : 0ull;
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const bool keep = i0 + 32 * u + lane < cnt && k[u] >= kmin;
      const unsigned ball = __ballot_sync(0xffffffffu, keep);
      if (keep) s[base + __popc(ball & ((1u << lane) - 1u))] = k[u];
      base += __popc(ball);
    }
  }
  __syncwarp();
  return base;
}

// Smallest and largest value among the keys buf[0, cnt), cnt >= 1.
__device__ void warp_value_range(const uint64_t* buf, int cnt, int lane, int& lo, int& hi) {
  int mn = INT32_MAX, mx = INT32_MIN;
  for (int i0 = 0; i0 < cnt; i0 += 32 * kBatch) {
    uint64_t k[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int i = i0 + 32 * u + lane;
      k[u] = i < cnt ? buf[i] : 0ull;
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u)
      if (i0 + 32 * u + lane < cnt) {
        mn = min(mn, key_val(k[u]));
        mx = max(mx, key_val(k[u]));
      }
  }
  lo = __reduce_min_sync(0xffffffffu, mn);
  hi = __reduce_max_sync(0xffffffffu, mx);
}

// hist[b] = number of keys of buf[0, cnt) whose value v is >= lo and has
// (v - lo) >> sh == b (keys below lo are skipped; a value past the last bin
// counts in it); returns how many were counted.
__device__ unsigned warp_value_hist_ge(const uint64_t* buf, int cnt, int lo, int sh, unsigned* hist, int lane) {
  for (int b = lane; b < 256; b += 32) hist[b] = 0u;
  __syncwarp();
  unsigned mine = 0u;
  for (int i0 = 0; i0 < cnt; i0 += 32 * kBatch) {
    uint64_t k[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int i = i0 + 32 * u + lane;
      k[u] = i < cnt ? buf[i] : 0ull;
    }
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int v = key_val(k[u]);
      if (i0 + 32 * u + lane < cnt && v >= lo) {
        atomicAdd(&hist[min((uint32_t)(v - lo) >> sh, 255u)], 1u);
        ++mine;
      }
    }
  }
  __syncwarp();
  return __reduce_add_sync(0xffffffffu, mine);
}

__device__ __forceinline__ int pow2_at_least(int x) {
  int p = 32;
  while (p < x) p <<= 1;
  return p;
}


// One launch: rows QA[0, nA) against columns QB[0, nB) (both bf16 rows of
// 128 bytes, zero-padded to whole 256-row tiles), loaded through the tensor
// maps tmA (boxes of the CTA's 256 rows) and tmB (boxes of a 128-column
// tile), whose 128-byte swizzle lays them out as the products' K-major
// operands; ext holds the columns' bias digits in the K = 16 layout of
// ext_offset.  self: rows and columns are one set, and row i
// skips column i.  With splits > 1, CTA (x, y) sweeps only the column tiles
// [y * tps, (y + 1) * tps) and writes its rows' C best keys, sorted, to part
// (a merge kernel then takes each row's C best of its splits' lists).
struct DotArgs {
  CUtensorMap tmA;  // QA as [rows][64] bf16, boxes of kCtaRows rows, 128-byte swizzle
  CUtensorMap tmB;  // QB likewise, boxes of kTileN rows
  const unsigned char* ext;
  uint32_t nA, nB, C;
  uint32_t splits, tps;
  uint64_t* buf;   // (nA x splits) x 2 buffers x kCap keys
  uint64_t* part;  // (nA x splits) x C keys when splits > 1
  // original ids when the rows or columns are stored in another order
  // (nullptr: position = id): col_ids covers every column tile (tiles x 128
  // entries) and names the columns in the keys; row_ids places the output rows
  const uint32_t* col_ids;
  const uint32_t* row_ids;
  bool sorted;  // lists in descending key order (else in any order)
  uint32_t* out_idx;
  int32_t* out_val;
  uint32_t* err;
  long long wait_cycles;  // bound of every wait (SM clock cycles)
  uint32_t withhold;      // debug: a column tile never issued (UINT32_MAX: none)
};

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t* p) { return *reinterpret_cast<const volatile uint32_t*>(p); }

// Copies the keys of src[0, cnt) whose value is >= t to dst (in their order);
// returns how many.  dst may be src itself (each key moves down or stays).
__device__ int warp_keep_value_ge_to(const uint64_t* src, int cnt, int t, uint64_t* dst, int lane) {
  int base = 0;
  for (int i0 = 0; i0 < cnt; i0 += 32 * kBatch) {
    uint64_t k[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int i = i0 + 32 * u + lane;
      k[u] = i < cnt ? src[i] : 0ull;
    }
    __syncwarp();
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const bool keep = i0 + 32 * u + lane < cnt && key_val(k[u]) >= t;
      const unsigned ball = __ballot_sync(0xffffffffu, keep);
      if (keep) dst[base + __popc(ball & ((1u << lane) - 1u))] = k[u];
      base += __popc(ball);
    }
  }
  __syncwarp();
  return base;
}

// A warp compacts one handed-over buffer keys[0, c) (C < c <= the hand-over
// cap).  The keys, and the kept keys other[0, co) of the row's other buffer
// (a prefix the epilogue no longer writes), are staged into shared memory
// with one round of asynchronous copies; every pass runs there.  The
// threshold t is at or below the C-th best value of the two together (the
// lower edge of the 256-bin value-histogram bin holding it, or the exact C-th
// key when that bin is crowded), so it is at or below the row's C-th best
// value so far; the handed-over keys that reach it are written back to the
// front of their buffer.  Returns the number kept there.
//
// thr_now is the row's current threshold and hi_now a bound on every value
// the row has appended.  Once the row has a threshold, keys below it cannot
// reach its C best, so the histogram covers [thr_now, hi_now] and skips them
// (no pass for the range); if fewer than C keys reach thr_now, it stays.
__device__ int compact_buffer(uint64_t* keys, int c, const uint64_t* other, int co, uint32_t C, unsigned keep_limit,
                              float thr_now, float hi_now, unsigned* hist, uint64_t* stage, int lane, int& t) {
  for (int x = lane; x < c; x += 32) cp_async8(stage + x, keys + x);
  for (int x = lane; x < co; x += 32) cp_async8(stage + c + x, other + x);
  cp_async_wait_all();
  __syncwarp();
  const int n = c + co;
  int lo, hi;
  if (thr_now > -FLT_MAX && hi_now >= thr_now) {  // integers held exactly in float
    lo = (int)thr_now;
    hi = (int)hi_now;
  } else {
    warp_value_range(stage, n, lane, lo, hi);
  }
  const unsigned span = (unsigned)(hi - lo);
  const int sh = span < 256u ? 0 : 24 - __clz((int)span);
  const unsigned counted = warp_value_hist_ge(stage, n, lo, sh, hist, lane);
  int kept;
  if (counted < C) {
    t = lo;
    kept = warp_keep_value_ge_to(stage, c, lo, keys, lane);
  } else {
    int bin;
    unsigned above;
    hist_find_desc(hist, C, lane, bin, above);
    const unsigned keep = above + hist[bin];
    __syncwarp();
    if (keep <= keep_limit) {
      t = lo + (bin << sh);
      kept = warp_keep_value_ge_to(stage, c, t, keys, lane);
    } else {
      const uint64_t kth = warp_select_kth(stage, n, (int)C, hist, lane);
      kept = warp_gather_ge(stage, c, kth, keys, lane);
      t = key_val(kth);
    }
  }
  __syncwarp();
  return kept;
}

template <bool kSplit, bool kSelf>
__global__ void __launch_bounds__(kThreads, 1) dot_topk_kernel(const __grid_constant__ DotArgs P) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t C = P.C;
  uint32_t* __restrict__ err = P.err;
  const long long wait_lim = P.wait_cycles;

  float* sThr = reinterpret_cast<float*>(smem + kOffThr);
  float* sHi = reinterpret_cast<float*>(smem + kOffHi);
  int* sKept = reinterpret_cast<int*>(smem + kOffKept);          // [row][buffer]
  uint32_t* sReq = reinterpret_cast<uint32_t*>(smem + kOffReq);  // buffer | count << 1 of a hand-over
  uint32_t* sFin = reinterpret_cast<uint32_t*>(smem + kOffFin);  // active buffer | count << 1 at the end
  uint32_t* sMisc = reinterpret_cast<uint32_t*>(smem + kOffMisc);
  uint32_t* sMask = sMisc;                  // [kEpiWarps]: rows of each epilogue warp awaiting compaction
  uint32_t* sDone = sMisc + kEpiWarps;      // epilogue warps that finished their sweep
  uint32_t* sTmem = sMisc + kEpiWarps + 1;  // tensor-memory base (written by tcgen05.alloc)
  uint32_t* sProg = sMisc + kEpiWarps + 2;  // [kEpiWarps]: tiles each epilogue warp has finished
  const uint32_t bar0 = smem_u32(smem + kOffBars);
  auto full_bar = [&](uint32_t s) { return bar0 + 8u * s; };
  auto empty_bar = [&](uint32_t s) { return bar0 + 8u * (kStages + s); };
  auto accf_bar = [&](uint32_t b) { return bar0 + 8u * (2 * kStages + b); };
  auto acce_bar = [&](uint32_t b) { return bar0 + 8u * (2 * kStages + 2 + b); };
  const uint32_t a_bar = bar0 + 8u * (2 * kStages + 4);

  const uint32_t row0 = blockIdx.x * (uint32_t)kCtaRows;
  const uint32_t ys = kSplit ? blockIdx.y : 0u;
  const uint32_t tall = (P.nB + kTileN - 1) / kTileN;
  const uint32_t tlo = kSplit ? min(tall, ys * P.tps) : 0u;
  const uint32_t ntiles = kSplit ? min(tall - tlo, P.tps) : tall;
  // A square sweep starts at the CTA's own diagonal tile and moves outward
  // in both directions (start, +1, -1, +2, -2, ..., then the longer side
  // alone): with rows in a locality order the tiles nearest the diagonal hold
  // most of a row's best columns, so its threshold rises early.
  uint32_t start = 0;
  if (kSelf) {
    const uint32_t d = row0 / kTileN;
    if (d >= tlo && d < tlo + ntiles) start = d - tlo;
  }
  const uint32_t side_lo = start, side_hi = ntiles - 1u - start, side = min(side_lo, side_hi);
  auto tile_of = [&](uint32_t u) {
    uint32_t x;
    if (u <= 2u * side) {
      const uint32_t k = (u + 1u) >> 1;
      x = (u & 1u) ? start + k : start - k;
    } else {
      x = side_hi > side_lo ? start + (u - side) : start - (u - side);
    }
    return tlo + x;
  };
  auto row_buf = [&](uint32_t i, uint32_t b) { return P.buf + (((size_t)i * P.splits + ys) * 2 + b) * kCap; };
  // compactors and their staging capacity (keys a hand-over may carry)
  const int ncomp = C <= 256u ? kCompWarps : 2;
  // a hand-over carries at most stage_keys keys, and the other buffer's kept
  // keys number at most keep_limit <= C + trigger / 2 <= area / 3: the two fit
  // one compactor's area of kStageKeysTotal / ncomp keys
  const int stage_keys = kStageKeysTotal / ncomp * 2 / 3;  // keys a hand-over may carry
  const int trigger = min(stage_keys - kTileN, (int)C + (int)C / 2);
  const unsigned keep_limit = (C + (unsigned)trigger) / 2;  // a compaction frees at least this much

  // ---- set-up: row state, the rows' bias-digit weights (2^16, 2^8, 1),
  // barriers, tensor memory
  for (int r = tid; r < kCtaRows; r += kThreads) {
    sThr[r] = -FLT_MAX;
    sKept[2 * r] = 0;
    sKept[2 * r + 1] = 0;
    sReq[r] = 0u;
    sFin[r] = 0u;
  }
  if (tid <= kEpiWarps) sMisc[tid] = 0u;  // request masks, done flags (not the tensor-memory word)
  if (tid < kEpiWarps) sProg[tid] = 0u;
  for (int x = tid; x < kRows * kExtK; x += kThreads) {
    const uint32_t r = (uint32_t)x / kExtK, k = (uint32_t)x % kExtK;
    const float w = k == 0 ? 65536.f : (k == 1 ? 256.f : (k == 2 ? 1.f : 0.f));
    *reinterpret_cast<__nv_bfloat16*>(smem + kOffAExt + ext_offset(r, k)) = __float2bfloat16_rn(w);
  }
  if (tid == 0) {
    for (uint32_t s = 0; s < (uint32_t)kStages; ++s) {
      mbar_init(full_bar(s), 1);
      mbar_init(empty_bar(s), 1);
    }
    for (uint32_t b = 0; b < 2; ++b) {
      mbar_init(accf_bar(b), 1);
      mbar_init(acce_bar(b), kEpiWarps);
    }
    mbar_init(a_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(sTmem)),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // the weights above, for the tensor cores
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *sTmem;

  if (warp == kProducerWarp) {
    // ---- producer: the CTA's rows once, then the column tiles into the ring
    if (lane == 0) {
      mbar_expect_tx(a_bar, kBlocksPerCta * kAMainBytes);
      tc::tma_load_2d(smem_u32(smem + kOffAMain), &P.tmA, 0, (int)row0, a_bar);
      uint32_t u = 0;
      for (; u < ntiles; ++u) {
        const uint32_t s = u % kStages;
        // stage s last held tile u - kStages: free once its products are done
        if (u >= (uint32_t)kStages && !mbar_wait(empty_bar(s), ((u / kStages) - 1u) & 1u, wait_lim)) {
          atomicOr(err, kErrWait);
          break;
        }
        if (u == P.withhold) continue;  // debug: never issued; the waits for it run out
        const uint32_t t = tile_of(u);
        unsigned char* st = smem + kOffStages + s * kStageBytes;
        mbar_expect_tx(full_bar(s), kStageBytes);
        tc::tma_load_2d(smem_u32(st), &P.tmB, 0, (int)(t * (uint32_t)kTileN), full_bar(s));
        bulk_g2s(smem_u32(st + kMainBytes), P.ext + (size_t)t * kExtBytes, kExtBytes, full_bar(s));
      }
      // every copy issued has landed before the CTA's shared memory is reused (bounded)
      if (!mbar_wait(a_bar, 0u, wait_lim)) atomicOr(err, kErrWait);
      for (uint32_t v = u > (uint32_t)kStages ? u - kStages : 0u; v < u; ++v) {
        if (v == P.withhold) continue;
        if (!mbar_wait(full_bar(v % kStages), (v / kStages) & 1u, wait_lim)) {
          atomicOr(err, kErrWait);
          break;
        }
      }
    }
  } else if (warp == kMmaWarp) {
    // ---- one thread issues the products of each tile for both row blocks
    // into their accumulators u & 1
    if (lane == 0) {
      bool ok = mbar_wait(a_bar, 0u, wait_lim);
      if (!ok) atomicOr(err, kErrWait);
      const uint32_t a_main = smem_u32(smem + kOffAMain), a_ext = smem_u32(smem + kOffAExt);
      uint32_t u = 0;
      for (; ok && u < ntiles; ++u) {
        const uint32_t s = u % kStages, b = u & 1u;
        if (!mbar_wait(full_bar(s), (u / kStages) & 1u, wait_lim)) {
          atomicOr(err, kErrWait);
          break;
        }
        if (u >= 2 && !mbar_wait(acce_bar(b), ((u >> 1) - 1u) & 1u, wait_lim)) {
          atomicOr(err, kErrWait);
          break;
        }
        tc_fence_after();
        const uint32_t st = smem_u32(smem + kOffStages + s * kStageBytes);
#pragma unroll
        for (uint32_t rb = 0; rb < (uint32_t)kBlocksPerCta; ++rb) {
          const uint32_t d = tbase + (2u * rb + b) * (uint32_t)kTileN;
          const uint32_t am = a_main + rb * (uint32_t)kAMainBytes;
#pragma unroll
          for (uint32_t ks = 0; ks < 4; ++ks)
            tc_mma(d, smem_desc(am + 32u * ks, 16u, 1024u, 2u), smem_desc(st + 32u * ks, 16u, 1024u, 2u),
                   ks > 0 ? 1u : 0u);
          tc_mma(d, smem_desc(a_ext, 128u, 256u, 0u), smem_desc(st + kMainBytes, 128u, 256u, 0u), 1u);
        }
        tc_commit(empty_bar(s));
        tc_commit(accf_bar(b));
      }
      // the products issued have completed before tensor memory is freed
      if (u > 0 && !mbar_wait(accf_bar((u - 1u) & 1u), ((u - 1u) >> 1) & 1u, wait_lim)) atomicOr(err, kErrWait);
    }
  } else if (warp < kEpiWarps) {
    // ---- epilogue: thread = row; warp w reads row block w / 4, tensor-memory
    // lanes 32 * (w % 4) + lane (two warps per SM sub-partition)
    const int r = warp * 32 + lane;
    const uint32_t blk = (uint32_t)warp >> 2;
    const uint32_t i = row0 + (uint32_t)r;
    bool live = i < P.nA;
    uint32_t act = 0;  // the buffer being appended to
    int cnt = 0;
    uint64_t* rb = live ? row_buf(i, 0) : nullptr;
    float thr = -FLT_MAX;
    float amax = -FLT_MAX;  // at least every value this row has appended
    const uint32_t lane_base = tbase + ((uint32_t)((warp & 3) * 32) << 16);
    const uint32_t bit = 1u << lane;

    float* sv = reinterpret_cast<float*>(smem + kOffVals) + r * kValStride;
    // the original ids of the tile's columns, loaded one tile ahead
    uint32_t* sid = reinterpret_cast<uint32_t*>(smem + kOffIds) + warp * kTileN;
    const uint32_t* __restrict__ col_ids = P.col_ids;
    uint4 idn = make_uint4(0u, 0u, 0u, 0u);
    if (col_ids && ntiles > 0) {
      *reinterpret_cast<uint4*>(sid + 4 * lane) = __ldg(reinterpret_cast<const uint4*>(col_ids + (size_t)tile_of(0) * kTileN) + lane);
      if (ntiles > 1) idn = __ldg(reinterpret_cast<const uint4*>(col_ids + (size_t)tile_of(1) * kTileN) + lane);
      __syncwarp();
    }
    // values of one 32-column chunk (column colbase + k in v[k]) that reach
    // the threshold are appended.  The chunk's maximum is tested first; a
    // thread whose maximum passes builds its hit mask with two instructions
    // per value (the sign bit of x - thr: values and threshold are integers,
    // so the difference has the exact sign, and it is +0 when they are equal)
    // and reads the hits back from shared memory, so the work beyond the test
    // follows the number of hits.
    auto process = [&](const uint32_t (&v)[32], uint32_t colbase, uint32_t cofs) {
      float m[11];
#pragma unroll
      for (int x = 0; x < 10; ++x)
        m[x] = fmax3(__uint_as_float(v[3 * x]), __uint_as_float(v[3 * x + 1]), __uint_as_float(v[3 * x + 2]));
      m[10] = fmaxf(__uint_as_float(v[30]), __uint_as_float(v[31]));
      const float m2 = fmax3(fmax3(m[0], m[1], m[2]), fmax3(m[3], m[4], m[5]), fmax3(m[6], m[7], m[8]));
      const float mx = fmax3(m2, m[9], m[10]);
      if (live && mx >= thr) {
        uint32_t ms[4] = {0u, 0u, 0u, 0u};  // bit k: x_k < thr, in four independent chains
#pragma unroll
        for (int k = 7; k >= 0; --k)
#pragma unroll
          for (int g = 0; g < 4; ++g)
            ms[g] = __funnelshift_l(__float_as_uint(__uint_as_float(v[8 * g + k]) - thr), ms[g], 1);
        uint32_t hit = ~(ms[0] | (ms[1] << 8) | (ms[2] << 16) | (ms[3] << 24));
        if (colbase + 32u > P.nB || (kSelf && i - colbase < 32u)) {
          uint32_t valid = 0u;
#pragma unroll
          for (int k = 0; k < 32; ++k) {
            const uint32_t j = colbase + (uint32_t)k;
            if (j < P.nB && !(kSelf && j == i)) valid |= 1u << k;
          }
          hit &= valid;
        }
        if (hit) {
          amax = fmaxf(amax, mx);
#pragma unroll
          for (int q4 = 0; q4 < 8; ++q4)
            *reinterpret_cast<uint4*>(sv + 4 * q4) = make_uint4(v[4 * q4], v[4 * q4 + 1], v[4 * q4 + 2], v[4 * q4 + 3]);
          do {
            const int k = __ffs(hit) - 1;
            hit &= hit - 1u;
            rb[cnt++] = make_key(__float2int_rn(sv[k]), col_ids ? sid[cofs + (uint32_t)k] : colbase + (uint32_t)k);
          } while (hit);
        }
      }
    };

    for (uint32_t u = 0; u < ntiles; ++u) {
      const uint32_t b = u & 1u;
      const bool got = mbar_wait(accf_bar(b), (u >> 1) & 1u, wait_lim);
      if (!__all_sync(0xffffffffu, got)) {
        if (lane == 0) atomicOr(err, kErrWait);
        break;
      }
      tc_fence_after();
      if (live && cnt > kCap - kTileN) {  // cannot happen (hand-overs cap the count); never write past the buffer
        atomicOr(err, kErrCapacity);
        live = false;
      }
      thr = fmaxf(thr, *reinterpret_cast<volatile float*>(sThr + r));
      const uint32_t col0 = tile_of(u) * (uint32_t)kTileN;
      const uint32_t tcol = lane_base + (2u * blk + b) * (uint32_t)kTileN;
      uint32_t va[32], vb[32];
      tmem_ld32(tcol, va);
      tmem_wait(va);
#pragma unroll
      for (int c = 0; c < kChunks; c += 2) {
        tmem_ld32(tcol + 32u * (uint32_t)(c + 1), vb);
        process(va, col0 + 32u * (uint32_t)c, 32u * (uint32_t)c);
        tmem_wait(vb);
        if (c + 2 < kChunks) {
          tmem_ld32(tcol + 32u * (uint32_t)(c + 2), va);
        } else {  // every column of the accumulator is in registers: release it
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(acce_bar(b));
        }
        process(vb, col0 + 32u * (uint32_t)(c + 1), 32u * (uint32_t)(c + 1));
        if (c + 2 < kChunks) tmem_wait(va);
      }
      if (lane == 0) *reinterpret_cast<volatile uint32_t*>(sProg + warp) = u + 1u;  // seen by the compactors
      if (col_ids && u + 1u < ntiles) {  // the next tile's ids, once every hit of this one is appended
        __syncwarp();
        *reinterpret_cast<uint4*>(sid + 4 * lane) = idn;
        __syncwarp();
        if (u + 2u < ntiles) idn = __ldg(reinterpret_cast<const uint4*>(col_ids + (size_t)tile_of(u + 2u) * kTileN) + lane);
      }
      // a full buffer goes to the compactor, unless it still holds the other one
      if (live && cnt > trigger) {
        bool pending = (ld_volatile(sMask + warp) & bit) != 0u;
        if (pending && cnt > stage_keys - kTileN) {  // a hand-over must fit the staging area: wait (bounded)
          const long long t0 = clock64();
          while (pending && clock64() - t0 <= wait_lim) pending = (ld_volatile(sMask + warp) & bit) != 0u;
          if (pending) {
            atomicOr(err, kErrWait);
            live = false;
          }
        }
        if (live && !pending) {
          sHi[r] = amax;
          sReq[r] = act | ((uint32_t)cnt << 1);
          __threadfence_block();
          atomicOr(sMask + warp, bit);
          act ^= 1u;
          cnt = (int)ld_volatile(reinterpret_cast<const uint32_t*>(sKept + 2 * r + act));
          rb = row_buf(i, act);
        }
      }
      __syncwarp();
    }
    // the last hand-over completes before the final state is published
    if (live) {
      const long long t0 = clock64();
      bool pending = true;
      while ((pending = (ld_volatile(sMask + warp) & bit) != 0u) && clock64() - t0 <= wait_lim) {
      }
      if (pending) atomicOr(err, kErrWait);
    }
    sHi[r] = amax;  // for the final pass
    sFin[r] = act | ((uint32_t)cnt << 1);
    __threadfence_block();
    __syncwarp();
    if (lane == 0) atomicOr(sDone, 1u << warp);
  } else if (warp >= kEpiWarps + 2) {
    // ---- compactor q serves the rows of epilogue warps [q * per, (q + 1) * per)
    const int q = warp - (kEpiWarps + 2);
    if (q < ncomp) {
      const int per = kEpiWarps / ncomp;
      const uint32_t served = ((1u << per) - 1u) << (q * per);
      unsigned* hist = reinterpret_cast<unsigned*>(smem + kOffCompHist + q * 1024);
      const int area = kStageKeysTotal / ncomp;  // staging keys of this compactor
      uint64_t* stage = reinterpret_cast<uint64_t*>(smem + kOffCompKeys) + (size_t)q * area;
      long long t0 = clock64();
      uint32_t last_prog = 0u;
      for (;;) {
        uint32_t done = 0u, any = 0u;
        if (lane == 0) {
          done = ld_volatile(sDone) & served;
          for (int e = 0; e < per; ++e) any |= ld_volatile(sMask + q * per + e);
          if (any == 0u && done == served)  // a last request raced with the done flags
            for (int e = 0; e < per; ++e) any |= ld_volatile(sMask + q * per + e);
        }
        any = __shfl_sync(0xffffffffu, any, 0);
        done = __shfl_sync(0xffffffffu, done, 0);
        if (any == 0u) {
          if (done == served) break;
          // no request: the bound runs only while the epilogue warps served
          // make no progress either (a sweep may go long without a hand-over)
          uint32_t prog = 0u;
          if (lane == 0)
            for (int e = 0; e < per; ++e) prog += ld_volatile(sProg + q * per + e);
          prog = __shfl_sync(0xffffffffu, prog, 0);
          if (prog != last_prog) {
            last_prog = prog;
            t0 = clock64();
          } else if (clock64() - t0 > wait_lim) {
            if (lane == 0) atomicOr(err, kErrWait);
            break;
          }
          __nanosleep(64);
          continue;
        }
        for (int e = 0; e < per; ++e) {
          const int ew = q * per + e;  // an epilogue warp served
          uint32_t m = lane == 0 ? ld_volatile(sMask + ew) : 0u;
          m = __shfl_sync(0xffffffffu, m, 0);
          while (m) {
            const int l = __ffs(m) - 1;
            m &= m - 1u;
            const int r = ew * 32 + l;
            const uint32_t rq = ld_volatile(sReq + r);
            const uint32_t b = rq & 1u;
            uint64_t* keys = row_buf(row0 + (uint32_t)r, b);
            int co = (int)ld_volatile(reinterpret_cast<const uint32_t*>(sKept + 2 * r + (b ^ 1u)));
            int c = (int)(rq >> 1);
            if (c > stage_keys || co > area - stage_keys) {  // cannot happen; never stage past the area
              if (lane == 0) atomicOr(err, kErrCapacity);
              c = min(c, stage_keys);
              co = min(co, area - stage_keys);
            }
            int t = 0;
            const float thr_now = *reinterpret_cast<volatile float*>(sThr + r);
            const float hi_now = *reinterpret_cast<volatile float*>(sHi + r);
            const int kept = compact_buffer(keys, c, row_buf(row0 + (uint32_t)r, b ^ 1u), co, C, keep_limit,
                                            thr_now, hi_now, hist, stage, lane, t);
            __threadfence_block();
            if (lane == 0) {
              sKept[2 * r + b] = kept;
              sThr[r] = fmaxf(sThr[r], (float)t);
              __threadfence_block();
              atomicAnd(sMask + ew, ~(1u << l));
            }
            __syncwarp();
          }
        }
        t0 = clock64();
      }
    }
  }

  // ---- tear-down: tensor memory freed once every product and load is done
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tbase), "r"(kTmemCols));

  // ---- final lists: each row's C best keys of its two buffers, sorted (the
  // ring, compactor and value areas are free: every copy landed)
  unsigned* hist = reinterpret_cast<unsigned*>(smem + kOffStages + warp * kFinalBytes);
  uint64_t* sort = reinterpret_cast<uint64_t*>(smem + kOffStages + warp * kFinalBytes + 1024);
  for (int r = warp; r < kCtaRows; r += kWarps) {
    const uint32_t i = row0 + (uint32_t)r;
    if (i >= P.nA) break;
    const uint32_t fin = sFin[r];
    const uint32_t act = fin & 1u;
    const int ca = (int)(fin >> 1), co = sKept[2 * r + (act ^ 1u)];
    const int c0 = act == 0 ? ca : co, c1 = act == 0 ? co : ca;
    uint64_t* b0 = row_buf(i, 0);
    // buffer 1's keys move down to follow buffer 0's (reads of a batch before its writes)
    for (int x0 = 0; x0 < c1; x0 += 32 * kBatch) {
      uint64_t k[kBatch];
#pragma unroll
      for (int v = 0; v < kBatch; ++v) {
        const int x = x0 + 32 * v + lane;
        k[v] = x < c1 ? b0[kCap + x] : 0ull;
      }
      __syncwarp();
#pragma unroll
      for (int v = 0; v < kBatch; ++v) {
        const int x = x0 + 32 * v + lane;
        if (x < c1) b0[c0 + x] = k[v];
      }
      __syncwarp();
    }
    // The C best keys: a 256-bin histogram of the values finds the bin that
    // holds the C-th; the keys at or above that bin's lower edge (C or more,
    // at most kFinalSort) are gathered into shared memory, and when there
    // are more than C the exact select of the C-th key runs there, among
    // them.  A bin too crowded for the area falls back to the exact select
    // over the buffers.  Sorted only when the caller wants it.
    const int total = c0 + c1;
    int kept;
    if (total <= (int)C) {
      kept = warp_gather_ge(b0, total, 1ull, sort, lane);
    } else {
      // with a threshold, every key of the C best is at or above it and at
      // most the row's value bound: the histogram covers that range only
      int lo, hi;
      const float thr_f = sThr[r], hi_f = sHi[r];
      if (thr_f > -FLT_MAX && hi_f >= thr_f) {
        lo = (int)thr_f;
        hi = (int)hi_f;
      } else {
        warp_value_range(b0, total, lane, lo, hi);
      }
      const unsigned span = (unsigned)(hi - lo);
      const int sh = span < 256u ? 0 : 24 - __clz((int)span);
      const unsigned counted = warp_value_hist_ge(b0, total, lo, sh, hist, lane);
      int bin = 0;
      unsigned above = 0u, cand = 0xffffffffu;
      if (counted >= C) {
        hist_find_desc(hist, C, lane, bin, above);
        cand = above + hist[bin];
      }
      __syncwarp();
      if (cand <= (unsigned)kFinalSort) {
        kept = warp_keep_value_ge_to(b0, total, lo + (bin << sh), sort, lane);
        if (kept > (int)C) {
          const uint64_t kth = warp_select_kth(sort, kept, (int)C, hist, lane);
          kept = warp_gather_ge(sort, kept, kth, sort, lane);
        }
      } else {
        const uint64_t kth = warp_select_kth(b0, total, (int)C, hist, lane);
        kept = warp_gather_ge(b0, total, kth, sort, lane);
      }
    }
    if (P.sorted) {
      const int size = pow2_at_least(kept);
      for (int x = kept + lane; x < size; x += 32) sort[x] = 0ull;
      warp_bitonic_desc(sort, size, lane);
    }
    if (kSplit) {
      uint64_t* dst = P.part + ((size_t)i * P.splits + ys) * C;
      for (uint32_t x = lane; x < C; x += 32) dst[x] = (int)x < kept ? sort[x] : 0ull;
    } else {
      const size_t orow = P.row_ids ? P.row_ids[i] : i;
      for (uint32_t x = lane; x < C; x += 32) {
        const bool have = (int)x < kept;
        P.out_idx[orow * C + x] = have ? key_idx(sort[x]) : 0xffffffffu;
        P.out_val[orow * C + x] = have ? key_val(sort[x]) : INT32_MIN;
      }
    }
    __syncwarp();
  }
}

// one warp per row: the C best of the row's splits' lists (S x C keys, 0
// for missing) by the exact select, sorted when asked
constexpr int kMergeWarps = 8;
__global__ void __launch_bounds__(kMergeWarps * 32)
    merge_splits_kernel(const uint64_t* __restrict__ part, uint32_t nA, uint32_t S, uint32_t C, bool sorted,
                        const uint32_t* __restrict__ row_ids, uint32_t* __restrict__ out_idx,
                        int32_t* __restrict__ out_val) {
  __shared__ unsigned hist[kMergeWarps][256];
  __shared__ uint64_t keep[kMergeWarps][kSel];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t i = blockIdx.x * kMergeWarps + warp;
  if (i >= nA) return;  // warp-uniform
  const uint64_t* keys = part + (size_t)i * S * C;
  const int cnt = (int)(S * C);
  // missing entries are key 0, below every real key: select among all of them
  const uint64_t kth = warp_select_kth(keys, cnt, (int)C, hist[warp], lane);
  const uint64_t kmin = kth ? kth : 1ull;
  const int kept = warp_gather_ge(keys, cnt, kmin, keep[warp], lane);  // <= C
  if (sorted) {
    const int size = pow2_at_least(kept);
    for (int x = kept + lane; x < size; x += 32) keep[warp][x] = 0ull;
    warp_bitonic_desc(keep[warp], size, lane);
  }
  const size_t orow = row_ids ? row_ids[i] : i;
  for (uint32_t x = lane; x < C; x += 32) {
    const bool have = (int)x < kept;
    out_idx[orow * C + x] = have ? key_idx(keep[warp][x]) : 0xffffffffu;
    out_val[orow * C + x] = have ? key_val(keep[warp][x]) : INT32_MIN;
  }
}

__global__ void absmax_kernel(const float* __restrict__ E, uint32_t n, unsigned int* amax_bits) {
  float m = 0.f;
  const size_t count = (size_t)n * kFeat;
  for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < count; x += (size_t)gridDim.x * blockDim.x) {
    const size_t r = x / kFeat, c = x - r * kFeat;
    m = fmaxf(m, fabsf(E[r * kDim + c]));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax_bits, __float_as_uint(m));  // non-negative floats order as integers
}

// Element (r, c) of the bf16 rows the candidate kernel reads: row-major
// rows of 64 values (128 bytes), padded with zeros to whole 256-row tiles.
// The kernel's tensor-map loads apply the 128-byte shared-memory swizzle.
__device__ __forceinline__ size_t qb_index(size_t r, int c) { return r * kDim + (size_t)c; }

// one thread per (row, value) of the padded rows: the quantised values
// (row-major int8, optional), their bf16 copy (optional) and the biases
__global__ void quantize_kernel(const float* __restrict__ E, uint32_t n, uint32_t npad, const unsigned int* amax_bits,
                                int8_t* q, __nv_bfloat16* qb, int32_t* bias, float* scale_out) {
  const float scale = __uint_as_float(*amax_bits) / 127.0f;
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x == 0 && scale_out) *scale_out = scale;
  if (x >= (size_t)npad * kDim) return;
  const size_t r = x / kDim;
  const int c = (int)(x - r * kDim);
  float v = 0.f;
  if (r < n) {
    if (c < kFeat) {
      if (scale > 0.f) v = fminf(fmaxf(rintf(E[x] / scale), -127.f), 127.f);
    } else if (bias) {
      int32_t bv = 0;
      if (scale > 0.f) {
        const float s2 = scale * scale;
        bv = (int32_t)fminf(fmaxf(rintf(E[x] / s2), -(float)kBiasLimit), (float)kBiasLimit);
      }
      bias[r] = bv;
    }
    if (q) q[x] = (int8_t)v;
  }
  if (qb) qb[qb_index(r, c)] = __float2bfloat16_rn(v);
}

__global__ void widen_kernel(const int8_t* __restrict__ q, uint32_t n, uint32_t npad, __nv_bfloat16* qb) {
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (size_t)npad * kDim) return;
  const size_t r = x / kDim;
  qb[qb_index(r, (int)(x - r * kDim))] = __float2bfloat16_rn(r < n ? (float)q[x] : 0.f);
}

// one thread per (column, K half) of the padded columns: the bias digits
// (b >> 16, (b >> 8) & 255, b & 255 at K = 0, 1, 2; zero elsewhere and past n)
__global__ void bias_digits_kernel(const int32_t* __restrict__ bias, uint32_t n, uint32_t npad, unsigned char* ext) {
  const uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= 2u * npad) return;
  const uint32_t j = x >> 1, h = x & 1u;
  const int32_t b = (bias && j < n) ? bias[j] : 0;
  __nv_bfloat16 v[8];
#pragma unroll
  for (int e = 0; e < 8; ++e) v[e] = __float2bfloat16_rn(0.f);
  if (h == 0) {
    v[0] = __float2bfloat16_rn((float)(b >> 16));
    v[1] = __float2bfloat16_rn((float)((b >> 8) & 255));
    v[2] = __float2bfloat16_rn((float)(b & 255));
  }
  *reinterpret_cast<uint4*>(ext + ext_offset(j, 8u * h)) = *reinterpret_cast<const uint4*>(v);
}

size_t bias_pad(uint32_t n) { return ((size_t)n + kPadRows - 1) / kPadRows * kPadRows; }

// ---- sweep order of the self product (see sweep_order)
constexpr int kOrdBins = 4096;     // histogram of the first projection
constexpr int kOrdBuckets = 16;    // equal-count buckets of the first projection
constexpr int kOrdLevels = 256;    // levels of the second projection
constexpr int kOrdLens = NW_MAX_WORD_LEN + 1;
constexpr int kOrdKeys = kOrdLens * kOrdBuckets * kOrdLevels;
constexpr int kMomRows = 32;       // rows staged per step of moments_kernel (one 16-byte load per thread)
constexpr uint32_t kMomMaxRows = 1u << 17;  // rows per block at most: 2^17 x 127^2 < 2^31
static_assert(kOrdKeys % 4096 == 0 && kOrdBins % 4096 == 0, "block_exclusive_scan tiles of 4,096");
static_assert(kMomRows * 8 == 256, "one 16-byte chunk per thread of moments_kernel");

// sums over the rows of x and of x x^T, x = a row's 64 values (integers in
// [-127, 127], so integer sums are exact and order-free): mom[0, 64) and
// mom[64 + 64 k + l].  A step stages kMomRows rows with one 16-byte load per
// thread; thread t owns entries (t / 4, 16 (t % 4) + 0..15) and sums them in
// 32 bits (a block covers at most kMomMaxRows rows: |sum| < 2^31), then adds
// them to the 64-bit totals.
__global__ void __launch_bounds__(256) moments_kernel(const __nv_bfloat16* __restrict__ Qb, uint32_t n,
                                                      unsigned long long* mom) {
  __shared__ int row[kMomRows][kDim];
  const int t = threadIdx.x, k = t >> 2, l0 = (t & 3) * 16;
  int acc[16], s1 = 0;
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j] = 0;
  const uint32_t per = (n + gridDim.x - 1) / gridDim.x;
  const uint32_t rbeg = min(n, blockIdx.x * per), rend = min(n, rbeg + per);
  for (uint32_t r0 = rbeg; r0 < rend; r0 += kMomRows) {
    __syncthreads();
    {  // kMomRows x 8 chunks of 16 bytes: chunk ch of row r holds values 8 ch .. 8 ch + 7
      const uint32_t rr = (uint32_t)t >> 3, ch = (uint32_t)t & 7u, r = r0 + rr;
      uint4 u = make_uint4(0u, 0u, 0u, 0u);
      if (r < rend) u = __ldg(reinterpret_cast<const uint4*>(Qb + (size_t)r * kDim) + ch);
      const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&u);
      const int lc = (int)(ch * 8u);
#pragma unroll
      for (int e = 0; e < 8; ++e) row[rr][lc + e] = (int)__bfloat162float(h[e]);
    }
    __syncthreads();
#pragma unroll 4
    for (int rr = 0; rr < kMomRows; ++rr) {
      const int a = row[rr][k];
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] += a * row[rr][l0 + j];
      s1 += a;
    }
  }
#pragma unroll
  for (int j = 0; j < 16; ++j)
    if (acc[j]) atomicAdd(&mom[kDim + k * kDim + l0 + j], (unsigned long long)(long long)acc[j]);
  if ((t & 3) == 0 && s1) atomicAdd(&mom[k], (unsigned long long)(long long)s1);
}

// One block of 64 threads: the covariance of the rows from their moments and
// its two leading eigenvectors by power iteration (the second after
// deflating the first), written to dirs[0, 64) and dirs[64, 128); also resets
// the projection ranges that project_kernel raises.
__global__ void __launch_bounds__(kDim) pca_kernel(const unsigned long long* __restrict__ mom, uint32_t n,
                                                   float* dirs, unsigned* range) {
  __shared__ float cov[kDim][kDim + 1];
  __shared__ float v[kDim], w[kDim];
  const int t = threadIdx.x;
  const double inv = 1.0 / (double)max(n, 1u);
  const double mt = (double)(long long)mom[t] * inv;
  for (int l = 0; l < kDim; ++l)
    cov[t][l] = (float)((double)(long long)mom[kDim + t * kDim + l] * inv - mt * ((double)(long long)mom[l] * inv));
  if (t < 4) range[t] = (t & 1) ? 0u : 0xffffffffu;  // min, max, min, max of the ordered float bits
  for (int e = 0; e < 2; ++e) {
    v[t] = 1.f + (e ? -0.013f : 0.011f) * (float)t;  // fixed starting vectors
    __syncthreads();
    for (int it = 0; it < 256; ++it) {
      float x = 0.f;
      for (int l = 0; l < kDim; ++l) x = fmaf(cov[t][l], v[l], x);
      w[t] = x;
      __syncthreads();
      float nn = 0.f;
      for (int l = 0; l < kDim; ++l) nn = fmaf(w[l], w[l], nn);
      v[t] = nn > 0.f ? w[t] * rsqrtf(nn) : 0.f;
      __syncthreads();
    }
    dirs[e * kDim + t] = v[t];
    float x = 0.f;
    for (int l = 0; l < kDim; ++l) x = fmaf(cov[t][l], v[l], x);
    w[t] = x;
    __syncthreads();
    float lam = 0.f;
    for (int l = 0; l < kDim; ++l) lam = fmaf(v[l], w[l], lam);
    for (int l = 0; l < kDim; ++l) cov[t][l] -= lam * v[t] * v[l];
    __syncthreads();
  }
}

// floats as unsigned integers of the same order
__device__ __forceinline__ unsigned ord_bits(float f) {
  const unsigned b = __float_as_uint(f);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord_float(unsigned u) {
  return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// one thread per row: its projections on the two directions, and their
// ranges (range[0..3] = min, max of the first, min, max of the second)
__global__ void __launch_bounds__(256) project_kernel(const __nv_bfloat16* __restrict__ Qb, uint32_t n,
                                                      const float* __restrict__ dirs, float2* proj,
                                                      unsigned* range) {
  __shared__ float d[2 * kDim];
  if (threadIdx.x < 2 * kDim) d[threadIdx.x] = dirs[threadIdx.x];
  __syncthreads();
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  float a = 0.f, b = 0.f;
  if (r < n) {
    const uint4* row = reinterpret_cast<const uint4*>(Qb + (size_t)r * kDim);
#pragma unroll
    for (int ch = 0; ch < 8; ++ch) {
      const uint4 u = __ldg(row + ch);
      const int lc = ch * 8;  // chunk ch holds values lc .. lc + 7
      const __nv_bfloat16* h = reinterpret_cast<const __nv_bfloat16*>(&u);
#pragma unroll
      for (int e = 0; e < 8; ++e) {
        const float x = __bfloat162float(h[e]);
        a = fmaf(x, d[lc + e], a);
        b = fmaf(x, d[kDim + lc + e], b);
      }
    }
    proj[r] = make_float2(a, b);
  }
  unsigned mn1 = r < n ? ord_bits(a) : 0xffffffffu, mx1 = r < n ? ord_bits(a) : 0u;
  unsigned mn2 = r < n ? ord_bits(b) : 0xffffffffu, mx2 = r < n ? ord_bits(b) : 0u;
  mn1 = __reduce_min_sync(0xffffffffu, mn1);
  mx1 = __reduce_max_sync(0xffffffffu, mx1);
  mn2 = __reduce_min_sync(0xffffffffu, mn2);
  mx2 = __reduce_max_sync(0xffffffffu, mx2);
  if ((threadIdx.x & 31) == 0) {
    atomicMin(range + 0, mn1);
    atomicMax(range + 1, mx1);
    atomicMin(range + 2, mn2);
    atomicMax(range + 3, mx2);
  }
}

__device__ __forceinline__ int ord_level(float x, float lo, float hi, int levels) {
  if (!(hi > lo)) return 0;
  const int v = (int)((x - lo) / (hi - lo) * (float)levels);
  return min(max(v, 0), levels - 1);
}

// histogram of the first projection over kOrdBins equal-width bins
__global__ void __launch_bounds__(256) proj_hist_kernel(const float2* __restrict__ proj, uint32_t n,
                                                        const unsigned* __restrict__ range, unsigned* hist) {
  __shared__ unsigned h[kOrdBins];
  for (int x = threadIdx.x; x < kOrdBins; x += blockDim.x) h[x] = 0u;
  __syncthreads();
  const float lo = ord_float(range[0]), hi = ord_float(range[1]);
  for (uint32_t r = blockIdx.x * blockDim.x + threadIdx.x; r < n; r += gridDim.x * blockDim.x)
    atomicAdd(&h[ord_level(proj[r].x, lo, hi, kOrdBins)], 1u);
  __syncthreads();
  for (int x = threadIdx.x; x < kOrdBins; x += blockDim.x)
    if (h[x]) atomicAdd(&hist[x], h[x]);
}

// one block of 1024 threads: an exclusive scan of a[0, m) in place, m a
// multiple of 4096 (a 16-byte-aligned array), in coalesced tiles of 4,096
__device__ void block_exclusive_scan(unsigned* a, int m) {
  __shared__ unsigned part[1024];
  __shared__ unsigned carry;
  const int t = threadIdx.x;
  if (t == 0) carry = 0u;
  __syncthreads();
  for (int base = 0; base < m; base += 4096) {
    uint4 v = reinterpret_cast<const uint4*>(a + base)[t];
    const unsigned sum = v.x + v.y + v.z + v.w;
    part[t] = sum;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {
      const unsigned x = t >= o ? part[t - o] : 0u;
      __syncthreads();
      part[t] += x;
      __syncthreads();
    }
    const unsigned e = carry + part[t] - sum;
    uint4 w;
    w.x = e;
    w.y = e + v.x;
    w.z = w.y + v.y;
    w.w = w.z + v.z;
    reinterpret_cast<uint4*>(a + base)[t] = w;
    __syncthreads();
    if (t == 1023) carry += part[1023];
    __syncthreads();
  }
}

// one block of 1024: hist[b] becomes the equal-count bucket of bin b (by the
// rank of the bin's middle row)
__global__ void __launch_bounds__(1024) proj_buckets_kernel(unsigned* hist, uint32_t n) {
  __shared__ unsigned cnt[kOrdBins];
  for (int x = threadIdx.x; x < kOrdBins; x += blockDim.x) cnt[x] = hist[x];
  __syncthreads();
  block_exclusive_scan(hist, kOrdBins);
  __syncthreads();
  for (int x = threadIdx.x; x < kOrdBins; x += blockDim.x) {
    const unsigned long long mid = (unsigned long long)hist[x] + cnt[x] / 2u;
    const unsigned long long bk = mid * kOrdBuckets / max(n, 1u);
    hist[x] = bk < (unsigned long long)(kOrdBuckets - 1) ? (unsigned)bk : (unsigned)(kOrdBuckets - 1);
  }
}

// one thread per row: its sort key and the key's count
__global__ void __launch_bounds__(256) order_key_kernel(const float2* __restrict__ proj, uint32_t n,
                                                        const unsigned* __restrict__ range,
                                                        const unsigned* __restrict__ bucket_of,
                                                        const uint32_t* __restrict__ rank,
                                                        const uint8_t* __restrict__ slen, uint32_t* key,
                                                        unsigned* cnt) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
  const float2 p = proj[r];
  const unsigned b = bucket_of[ord_level(p.x, ord_float(range[0]), ord_float(range[1]), kOrdBins)];
  int lv = ord_level(p.y, ord_float(range[2]), ord_float(range[3]), kOrdLevels);
  if (b & 1u) lv = kOrdLevels - 1 - lv;
  const unsigned len = (rank && slen) ? min((unsigned)(kOrdLens - 1), (unsigned)slen[rank[r]]) : 0u;
  const uint32_t k = (len * kOrdBuckets + b) * kOrdLevels + (uint32_t)lv;
  key[r] = k;
  atomicAdd(&cnt[k], 1u);
}

__global__ void __launch_bounds__(1024) key_scan_kernel(unsigned* cnt) { block_exclusive_scan(cnt, kOrdKeys); }

__global__ void __launch_bounds__(256) order_scatter_kernel(const uint32_t* __restrict__ key, uint32_t n,
                                                            unsigned* cursor, uint32_t* perm) {
  const uint32_t r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) perm[atomicAdd(&cursor[key[r]], 1u)] = r;
}

// one thread per (position, 16-byte chunk) of the padded rows: row perm[p]
// moved to position p, and its bias
__global__ void __launch_bounds__(256) order_gather_kernel(const __nv_bfloat16* __restrict__ Qb,
                                                           const int32_t* __restrict__ bias, uint32_t n,
                                                           uint32_t npad, const uint32_t* __restrict__ perm,
                                                           __nv_bfloat16* Qp, int32_t* bp) {
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (size_t)npad * 8) return;
  const uint32_t p = (uint32_t)(x >> 3), ch = (uint32_t)(x & 7u);
  uint4 v = make_uint4(0u, 0u, 0u, 0u);
  if (p < n) {
    const uint32_t r = perm[p];
    v = __ldg(reinterpret_cast<const uint4*>(Qb + (size_t)r * kDim) + ch);
    if (ch == 0 && bp) bp[p] = bias ? bias[r] : 0;
  }
  *(reinterpret_cast<uint4*>(Qp + (size_t)p * kDim) + ch) = v;
}


}  // namespace

size_t dot_topk_qb_bytes(uint32_t n) { return bias_pad(n) * kRowBytes; }

// column splits of a launch over nA rows and nB columns on the current
// device: enough CTAs for one per SM when the row blocks alone are fewer,
// each split at least four tiles of 128 columns
uint32_t dot_topk_splits(uint32_t nA, uint32_t nB) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess || sms <= 0) {
    cudaGetLastError();
    sms = 152;
  }
  const uint32_t blocks = (nA + kCtaRows - 1) / kCtaRows;
  const uint32_t tiles = (nB + kTileN - 1) / kTileN;
  const uint32_t want = ((uint32_t)sms + blocks - 1) / std::max(blocks, 1u);
  return std::max(1u, std::min(want, tiles / 4));
}

// scratch layout: [row buffers: nA x S x 2 x kCap keys][column bias digits:
// bias_pad(nB) x 32 B][error word: 16 B][split lists: nA x S x C keys]
static size_t ext_offset_bytes(uint32_t nA, uint32_t nB) {
  return (size_t)nA * dot_topk_splits(nA, nB) * 2 * kCap * sizeof(uint64_t);
}

size_t dot_topk_buffer_bytes(uint32_t nA, uint32_t nB, uint32_t C) {
  const size_t S = dot_topk_splits(nA, nB);
  return ext_offset_bytes(nA, nB) + bias_pad(nB) * (size_t)kExtK * 2 + 16 +
         (S > 1 ? (size_t)nA * S * C * sizeof(uint64_t) : 0);
}

uint32_t* dot_topk_err_word(uint64_t* buf, uint32_t nA, uint32_t nB) {
  return reinterpret_cast<uint32_t*>(reinterpret_cast<char*>(buf) + ext_offset_bytes(nA, nB) +
                                     bias_pad(nB) * (size_t)kExtK * 2);
}

// the driver's tensor-map encoder, looked up once through the runtime
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled_fn() {
  static const EncodeTiledFn fn = []() -> EncodeTiledFn {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// `rows` bf16 rows of 64 values (128 bytes) at base, loaded in boxes of
// box_rows rows with the 128-byte swizzle of the products' K-major operands
static cudaError_t encode_rows(CUtensorMap* m, const void* base, uint64_t rows, uint32_t box_rows) {
  const EncodeTiledFn fn = encode_tiled_fn();
  if (!fn) return cudaErrorNotSupported;
  const cuuint64_t dims[2] = {(cuuint64_t)kDim, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)kRowBytes};
  const cuuint32_t box[2] = {(cuuint32_t)kDim, box_rows};
  const cuuint32_t elem[2] = {1, 1};
  const CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, elem,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

cudaError_t dot_topk_rect(const __nv_bfloat16* QA, uint32_t nA, const __nv_bfloat16* QB, const int32_t* biasB,
                          uint32_t nB, uint32_t C, bool self, uint64_t* buf, uint32_t* idx, int32_t* val,
                          uint32_t* err, cudaStream_t s, DotDebug dbg, const uint32_t* col_ids,
                          const uint32_t* row_ids, bool sorted) {
  if (nA == 0) return cudaSuccess;
  const uint32_t S = dot_topk_splits(nA, nB);
  const auto kernel = S > 1 ? (self ? dot_topk_kernel<true, true> : dot_topk_kernel<true, false>)
                            : (self ? dot_topk_kernel<false, true> : dot_topk_kernel<false, false>);
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotal);
  if (e != cudaSuccess) return e;
  const uint32_t tiles = (nB + kTileN - 1) / kTileN;
  unsigned char* ext = reinterpret_cast<unsigned char*>(buf) + ext_offset_bytes(nA, nB);
  DotArgs P;
  std::memset(&P, 0, sizeof P);
  // the row sets as allocated: zero-padded to whole 256-row tiles
  e = encode_rows(&P.tmA, QA, bias_pad(nA), (uint32_t)kCtaRows);
  if (e == cudaSuccess && nB) e = encode_rows(&P.tmB, QB, bias_pad(nB), (uint32_t)kTileN);
  if (e != cudaSuccess) return e;
  P.ext = ext;
  P.nA = nA;
  P.nB = nB;
  P.C = C;
  P.splits = S;
  P.tps = (tiles + S - 1) / S;
  P.buf = buf;
  P.part = S > 1 ? reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(dot_topk_err_word(buf, nA, nB)) + 16) : nullptr;
  P.out_idx = idx;
  P.out_val = val;
  P.err = err;
  P.wait_cycles = dbg.wait_cycles >= 0 ? dbg.wait_cycles : kWaitCycles;
  P.withhold = dbg.withhold;
  P.col_ids = col_ids;
  P.row_ids = row_ids;
  P.sorted = sorted;
  const uint32_t npad = (uint32_t)bias_pad(nB);
  if (npad) bias_digits_kernel<<<(2 * npad + 255) / 256, 256, 0, s>>>(biasB, nB, npad, ext);
  const dim3 grid((nA + kCtaRows - 1) / kCtaRows, S);
  kernel<<<grid, kThreads, kSmemTotal, s>>>(P);
  if (S > 1)
    merge_splits_kernel<<<(nA + kMergeWarps - 1) / kMergeWarps, kMergeWarps * 32, 0, s>>>(P.part, nA, S, C, sorted, row_ids, idx,
                                                                                         val);
  return cudaGetLastError();
}

cudaError_t dot_topk(const __nv_bfloat16* Qb, const int32_t* bias, uint32_t n, uint32_t C, uint64_t* buf,
                     uint32_t* idx, int32_t* val, uint32_t* err, cudaStream_t s, DotDebug dbg,
                     const uint32_t* ids, bool sorted) {
  return dot_topk_rect(Qb, n, Qb, bias, n, C, true, buf, idx, val, err, s, dbg, ids, ids, sorted);
}

cudaError_t quantize(const float* E, uint32_t n, unsigned int* amax_bits, int8_t* q, __nv_bfloat16* qb,
                     int32_t* bias, float* scale, cudaStream_t s, bool given_scale) {
  const size_t count = (size_t)bias_pad(n) * kDim;
  if (!given_scale) {
    cudaError_t e = cudaMemsetAsync(amax_bits, 0, sizeof(unsigned int), s);
    if (e != cudaSuccess) return e;
    if (n) absmax_kernel<<<1024, 256, 0, s>>>(E, n, amax_bits);
  }
  quantize_kernel<<<(unsigned)((count + 255) / 256 + (count == 0)), 256, 0, s>>>(E, n, (uint32_t)bias_pad(n),
                                                                                   amax_bits, q, qb, bias, scale);
  return cudaGetLastError();
}

// sweep-order scratch: [moments 64 + 64 x 64 x 8 B][directions 128 floats][ranges 4]
// [p1 histogram / buckets][key counts / cursors][projections n x 8 B][keys n x 4 B]
namespace {
constexpr size_t kOrdMomBytes = (kDim + kDim * kDim) * 8;
constexpr size_t kOrdDirOff = kOrdMomBytes;
constexpr size_t kOrdRangeOff = kOrdDirOff + 2 * kDim * 4;
constexpr size_t kOrdHistOff = kOrdRangeOff + 16;
constexpr size_t kOrdCntOff = kOrdHistOff + kOrdBins * 4;
constexpr size_t kOrdProjOff = kOrdCntOff + (size_t)kOrdKeys * 4;
}  // namespace

size_t sweep_perm_entries(uint32_t n) { return bias_pad(n); }
size_t sweep_order_bytes(uint32_t n) { return kOrdProjOff + (size_t)n * 8 + (size_t)n * 4 + 16; }

cudaError_t sweep_order(const __nv_bfloat16* Qb, const int32_t* bias, const uint32_t* rank, const uint8_t* slen,
                        uint32_t n, void* scratch, uint32_t* perm, __nv_bfloat16* Qp, int32_t* bp, cudaStream_t s) {
  const uint32_t npad = (uint32_t)bias_pad(n);
  char* sc = static_cast<char*>(scratch);
  auto* mom = reinterpret_cast<unsigned long long*>(sc);
  auto* dirs = reinterpret_cast<float*>(sc + kOrdDirOff);
  auto* range = reinterpret_cast<unsigned*>(sc + kOrdRangeOff);
  auto* hist = reinterpret_cast<unsigned*>(sc + kOrdHistOff);
  auto* cnt = reinterpret_cast<unsigned*>(sc + kOrdCntOff);
  auto* proj = reinterpret_cast<float2*>(sc + kOrdProjOff);
  auto* key = reinterpret_cast<uint32_t*>(sc + kOrdProjOff + (size_t)n * 8);
  cudaError_t e = cudaMemsetAsync(sc, 0, kOrdProjOff, s);  // moments, histogram, counts
  if (e == cudaSuccess) e = cudaMemsetAsync(perm, 0xff, sizeof(uint32_t) * npad, s);
  if (e != cudaSuccess) return e;
  if (n) {
    // enough blocks to hide the loads, and never more than kMomMaxRows rows per block
    const unsigned rows_grid = std::max<unsigned>(std::min<unsigned>(1216u, (n + kMomRows - 1) / kMomRows),
                                                  (unsigned)((n + kMomMaxRows - 1) / kMomMaxRows));
    const unsigned grid = (n + 255) / 256;
    moments_kernel<<<rows_grid, 256, 0, s>>>(Qb, n, mom);
    pca_kernel<<<1, kDim, 0, s>>>(mom, n, dirs, range);
    project_kernel<<<grid, 256, 0, s>>>(Qb, n, dirs, proj, range);
    proj_hist_kernel<<<std::min(grid, 608u), 256, 0, s>>>(proj, n, range, hist);
    proj_buckets_kernel<<<1, 1024, 0, s>>>(hist, n);
    order_key_kernel<<<grid, 256, 0, s>>>(proj, n, range, hist, rank, slen, key, cnt);
    key_scan_kernel<<<1, 1024, 0, s>>>(cnt);
    order_scatter_kernel<<<grid, 256, 0, s>>>(key, n, cnt, perm);
  }
  if (npad)
    order_gather_kernel<<<(unsigned)(((size_t)npad * 8 + 255) / 256), 256, 0, s>>>(Qb, bias, n, npad, perm, Qp, bp);
  return cudaGetLastError();
}

cudaError_t widen(const int8_t* q, uint32_t n, __nv_bfloat16* qb, cudaStream_t s) {
  const size_t count = (size_t)bias_pad(n) * kDim;
  if (!count) return cudaSuccess;
  widen_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(q, n, (uint32_t)bias_pad(n), qb);
  return cudaGetLastError();
}

}  // namespace prop
}  // namespace nw
