// nw_dot_topk.cu -- candidate proposal by quantised embedding products.
//
// Features are quantised to integers in [-127, 127] and stored as bf16, which
// holds them exactly; a product of two is at most 16,129, a sum of 64 at most
// 1,032,256, and a per-column bias is an integer of magnitude <= 2^23, so
// every partial sum stays below 2^24 and the tensor cores' float32
// accumulation gives the exact integer q_i . q_j + bias_j in any order.  The
// top-C selection is then an exact, deterministic function of the integers
// (ties: lower index).
//
// dot_topk_kernel: a CTA owns 256 rows (8 warps x 32 rows, A fragments held
// in registers for the whole sweep) and sweeps every column in tiles of 64:
// a three-stage cp.async ring into swizzled shared memory (one barrier per
// tile), ldmatrix, bf16 m16n8k16 mma.sync whose first k-step starts from the
// columns' biases.  Each row keeps an append buffer of kCap keys in global
// memory and a threshold; a value enters when it beats the threshold (a row
// group's maximum is tested first, so most tiles cost one compare per value
// and no branch).  A row's values in a tile belong to the four lanes of one
// quad, so its key count lives in their registers and appends take slots by
// a prefix sum over the quad, with no atomics.  When a row holds more than
// 2C keys (or its buffer could overflow during the next tile), its warp
// raises the row's threshold to the lower edge t of the value-histogram bin
// that holds the C-th best key and drops the keys below t (an exact 8-pass
// radix select when that bin is crowded).  Later columns have higher
// indices, so a later value equal to the C-th best never displaces a kept
// key: the comparison is strict, and the final pass, an exact select and
// sort of each row's buffer, gives exact lists.
#include <cuda_bf16.h>
#include <algorithm>
#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

#include "nw_internal.cuh"
#include "nw_proposal.h"
#include "nw_proposal_internal.h"

namespace nw {
namespace prop {
namespace {

constexpr int kDim = 64;                 // values per row (bf16)
constexpr int kRowBytes = kDim * 2;      // 128
// 32 rows (two 16-row slabs) per warp: 16 rows with three CTAs per SM measured 5% slower
constexpr int kRowsPerWarp = 32;
constexpr int kSlabs = kRowsPerWarp / 16;
constexpr int kCtasPerSm = kSlabs == 2 ? 2 : 3;
constexpr int kWarps = 8;
constexpr int kRowsPerCta = kRowsPerWarp * kWarps;  // 256
constexpr int kTileCols = 64;
constexpr int kThreads = kWarps * 32;
constexpr int kSel = NW_MAX_CANDIDATES;  // per-warp gather/sort area (keys)

// dynamic shared memory layout (bytes)
constexpr int kStages = kSlabs == 2 ? 6 : 4;             // column tiles in flight
constexpr int kTileBytes = kTileCols * kRowBytes;        // 8 KiB per tile
constexpr int kTileBiasBytes = kTileCols * 4;            // its biases (float)
constexpr int kSmemB = kStages * kTileBytes;
constexpr int kSmemBias = kStages * kTileBiasBytes;
constexpr int kSmemSort = kWarps * kSel * 8;             // 32 KiB (A staging at start)
constexpr int kSmemHist = kWarps * 256 * 4;              // radix histograms
constexpr int kSmemCnt = kRowsPerCta * 4;
constexpr int kSmemThr = kRowsPerCta * 4;
constexpr int kSmemBars = 2 * kStages * 8 + 16;          // full / empty mbarriers, next tile to issue
constexpr int kOffBias = kSmemB;
constexpr int kOffSort = kOffBias + kSmemBias;
constexpr int kOffHist = kOffSort + kSmemSort;
constexpr int kOffCnt = kOffHist + kSmemHist;
constexpr int kOffThr = kOffCnt + kSmemCnt;
constexpr int kOffBars = kOffThr + kSmemThr;
constexpr int kSmemTotal = kOffBars + kSmemBars;
static_assert(kSmemTotal * kCtasPerSm <= 224 * 1024, "kCtasPerSm CTAs per SM");
// a pipeline wait gives up after this many SM clock cycles (about a second)
constexpr long long kWaitCycles = 2000000000ll;
static_assert(kRowsPerCta * kRowBytes <= kSmemSort, "A staging fits the sort area");
static_assert(kCap - kTileCols > NW_MAX_CANDIDATES, "a compaction leaves room for a tile");
static_assert(kTileCols == 64, "a row's own column is found by i >> 6");
static_assert(kSel * 8 >= 32 * 32 * 4, "a warp's sort area stages 32 values per lane");

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// 16-byte chunk c of row r in a swizzled [rows][8 chunks] tile
__device__ __forceinline__ uint32_t swz(int r, int c) { return (uint32_t)(r * kRowBytes + ((c ^ (r & 7)) << 4)); }

__device__ __forceinline__ void cp_async16(uint32_t dst, const void* src, bool valid) {
  const int n = valid ? 16 : 0;
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(dst), "l"(src), "r"(n));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

// ---- mbarriers and bulk copies
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}
// whether the barrier's phase of this parity has completed (never blocks)
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0u;
}
// waits for the phase of this parity to complete; false once `limit` SM clock cycles have passed
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, long long limit) {
  const long long t0 = clock64();
  for (;;) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    if (ok) return true;
    if (clock64() - t0 > limit) return false;
  }
}
// global -> shared, 16-byte aligned addresses, bytes a multiple of 16; counted on bar
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void ldmatrix_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(addr));
}

// d = a . b + (c0, c1, c0, c1): the first k-step, accumulating onto the columns' biases
__device__ __forceinline__ void mma_bf16_init(float* d, const uint32_t* a, uint32_t b0, uint32_t b1, float c0,
                                              float c1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%10, %11, %10, %11};\n"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(c0), "f"(c1));
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// key: higher value first, then lower index; 0 sorts below every real key
__device__ __forceinline__ uint64_t make_key(int v, uint32_t j) {
  return ((uint64_t)(uint32_t)(v + 0x80000000) << 32) | (uint64_t)(0xffffffffu - j);
}
__device__ __forceinline__ int key_val(uint64_t k) { return (int)((uint32_t)(k >> 32) - 0x80000000u); }
__device__ __forceinline__ uint32_t key_idx(uint64_t k) { return 0xffffffffu - (uint32_t)k; }

// Sorts s[0, size) descending (size a power of two) with the warp.
__device__ void warp_bitonic_desc(uint64_t* s, int size, int lane) {
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

// Copies the keys >= kmin of buf[0, cnt) into s (in any order); returns how many.
__device__ int warp_gather_ge(const uint64_t* buf, int cnt, uint64_t kmin, uint64_t* s, int lane) {
  int base = 0;
  for (int i0 = 0; i0 < cnt; i0 += 32 * kBatch) {
    uint64_t k[kBatch];
#pragma unroll
    for (int u = 0; u < kBatch; ++u) {
      const int i = i0 + 32 * u + lane;
      k[u] = i < cnt ? buf[i] : 0ull;
    }
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

// hist[b] = number of keys of buf[0, cnt) with (value - lo) >> sh == b; every
// value lies in [lo, lo + (256 << sh)).
__device__ void warp_value_hist(const uint64_t* buf, int cnt, int lo, int sh, unsigned* hist, int lane) {
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
      if (i0 + 32 * u + lane < cnt) atomicAdd(&hist[(uint32_t)(key_val(k[u]) - lo) >> sh], 1u);
  }
  __syncwarp();
}

// Keeps the keys of buf[0, cnt) whose value is >= t at the front of buf, in
// their order; returns how many.  A batch's writes land below the end of the
// batch, which its lanes have already read.
__device__ int warp_keep_value_ge(uint64_t* buf, int cnt, int t, int lane) {
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
      const bool keep = i0 + 32 * u + lane < cnt && key_val(k[u]) >= t;
      const unsigned ball = __ballot_sync(0xffffffffu, keep);
      if (keep) buf[base + __popc(ball & ((1u << lane) - 1u))] = k[u];
      base += __popc(ball);
    }
    __syncwarp();
  }
  return base;
}

// Bits k (value k = 2 nb + e of a lane's row group: column 8 nb + 2 t4 + e of
// the tile) whose column j is a real column (j < nB) other than the row i
// itself when rows and columns are one set (self); a row past nA has none.
__device__ __forceinline__ uint32_t valid_cols(uint32_t i, uint32_t tile, uint32_t nA, uint32_t nB, bool self,
                                               int t4) {
  if (i >= nA) return 0u;
  const uint32_t j0 = tile * kTileCols;
  uint32_t v = 0xffffu;
  if (j0 + kTileCols > nB || (self && (i >> 6) == tile)) {
    v = 0u;
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const uint32_t j = j0 + (uint32_t)((k >> 1) * 8 + 2 * t4 + (k & 1));
      if (j < nB && !(self && j == i)) v |= 1u << k;
    }
  }
  return v;
}

__device__ __forceinline__ int pow2_at_least(int x) {
  int p = 32;
  while (p < x) p <<= 1;
  return p;
}

// One launch: rows QA[0, nA) against columns QB[0, nB) (both in the padded,
// swizzled bf16 layout); biasf holds the columns' biases as floats (exact:
// |bias| <= 2^23), zero-padded to a multiple of kTileCols entries.  self:
// rows and columns are one set, and row i skips column i.
// With splits > 1, CTA (x, y) sweeps only the column tiles [y * tps, (y +
// 1) * tps) and writes its rows' C best keys, sorted, to part (a merge
// kernel then takes each row's C best of its splits' lists).
struct DotArgs {
  const __nv_bfloat16* QA;
  const __nv_bfloat16* QB;
  const float* biasf;
  uint32_t nA, nB, C;
  bool self;
  uint32_t splits, tps;
  uint64_t* buf;   // (nA x splits) x kCap keys
  uint64_t* part;  // (nA x splits) x C keys when splits > 1
  uint32_t* out_idx;
  int32_t* out_val;
  uint32_t* err;
  long long wait_cycles;  // bound of every pipeline wait (SM clock cycles)
  uint32_t withhold;      // debug: a column tile never issued (UINT32_MAX: none)
};

template <bool kSplit, bool kSelf>
__global__ void __launch_bounds__(kThreads, kCtasPerSm) dot_topk_kernel(const DotArgs P) {
  const float* __restrict__ biasf = P.biasf;
  const uint32_t C = P.C;
  uint64_t* __restrict__ buf = P.buf;
  uint32_t* __restrict__ out_idx = P.out_idx;
  int32_t* __restrict__ out_val = P.out_val;
  uint32_t* __restrict__ err = P.err;
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* sB = smem;
  float* sBias = reinterpret_cast<float*>(smem + kOffBias);
  uint64_t* sSort = reinterpret_cast<uint64_t*>(smem + kOffSort);
  unsigned* sHist = reinterpret_cast<unsigned*>(smem + kOffHist);
  int* sCnt = reinterpret_cast<int*>(smem + kOffCnt);
  float* sThr = reinterpret_cast<float*>(smem + kOffThr);

  const uint32_t barFull = smem_u32(smem + kOffBars), barEmpty = barFull + 8 * kStages;
  uint32_t* sNext = reinterpret_cast<uint32_t*>(smem + kOffBars + 16 * kStages);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t row0 = blockIdx.x * (uint32_t)kRowsPerCta;
  const unsigned char* Qa = reinterpret_cast<const unsigned char*>(P.QA);
  const unsigned char* Qb = reinterpret_cast<const unsigned char*>(P.QB);
  // this CTA's column tiles: global tiles tlo + [0, ntiles)
  const uint32_t ys = kSplit ? blockIdx.y : 0u;
  const uint32_t tall = (P.nB + kTileCols - 1) / kTileCols;
  const uint32_t tlo = kSplit ? min(tall, ys * P.tps) : 0u;
  const uint32_t ntiles = kSplit ? min(tall - tlo, P.tps) : tall;
  // row i's append buffer
  auto row_buf = [&](uint32_t i) { return buf + (kSplit ? (size_t)i * P.splits + ys : (size_t)i) * kCap; };
  const uint32_t npadA = (P.nA + kTileCols - 1) / kTileCols * kTileCols;

  // column tile u into ring stage u % kStages: its rows (already swizzled and
  // zero-padded in global memory) and biases, counted on the stage's full barrier
  auto issue = [&](uint32_t u) {
    if (u == P.withhold) return;  // debug: its waits run out with nothing in flight
    const uint32_t st = u % kStages;
    mbar_expect_tx(barFull + 8 * st, kTileBytes + kTileBiasBytes);
    bulk_g2s(smem_u32(sB + st * kTileBytes), Qb + (size_t)(tlo + u) * kTileBytes, kTileBytes, barFull + 8 * st);
    bulk_g2s(smem_u32(sBias + st * kTileCols), biasf + (size_t)(tlo + u) * kTileCols, kTileBiasBytes,
             barFull + 8 * st);
  };

  // stage the CTA's 256 rows (zero past the padded rows) into the sort area
  unsigned char* sA = reinterpret_cast<unsigned char*>(sSort);
  for (int x = tid; x < kRowsPerCta * 8; x += kThreads) {
    const uint32_t g = row0 + (uint32_t)(x >> 3);
    cp_async16(smem_u32(sA + x * 16), Qa + (size_t)(g < npadA ? g : 0) * kRowBytes + (x & 7) * 16, g < npadA);
  }
  cp_async_commit();
  for (int r = tid; r < kRowsPerCta; r += kThreads) {
    sCnt[r] = 0;
    sThr[r] = -FLT_MAX;
  }
  if (tid == 0) {
    for (int st = 0; st < kStages; ++st) {
      mbar_init(barFull + 8 * st, 1);
      mbar_init(barEmpty + 8 * st, kWarps);
    }
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    const uint32_t first = min(ntiles, (uint32_t)kStages);
    for (uint32_t u = 0; u < first; ++u) issue(u);
    *sNext = first;
  }
  cp_async_wait<0>();
  __syncthreads();

  // A fragments: slab s (16 rows), k-step ks
  uint32_t afr[kSlabs][4][4];
#pragma unroll
  for (int s = 0; s < kSlabs; ++s)
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const int r = warp * kRowsPerWarp + s * 16 + (lane & 15);
      const int c = 2 * ks + (lane >> 4);
      ldmatrix_x4(smem_u32(sA + swz(r, c)), afr[s][ks][0], afr[s][ks][1], afr[s][ks][2], afr[s][ks][3]);
    }
  __syncthreads();  // the sort area is free from here on

  const int g = lane >> 2, t4 = lane & 3;
  float thr[kSlabs][2];
  int cnt[kSlabs][2];  // keys in the row's buffer (same in the row's four lanes)
#pragma unroll
  for (int s = 0; s < kSlabs; ++s)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      thr[s][h] = -FLT_MAX;
      cnt[s][h] = 0;
    }

  uint64_t* sMine = sSort + warp * kSel;
  unsigned* hMine = sHist + warp * 256;
  const int trigger = min(kCap - kTileCols, 2 * (int)C);
  const unsigned keep_limit = (C + (unsigned)trigger) / 2;  // a compaction frees at least this much
  // Warps sweep the ring at their own pace.  A stage is released by each
  // warp once its products are taken, and refilled by whichever warp finds it
  // free first (the next tile to issue is claimed with a compare-and-swap), so
  // a warp may run up to kStages tiles ahead of the CTA's slowest.
  for (uint32_t tile = 0; tile < ntiles; ++tile) {
    const int b = (int)(tile % kStages);
    if (lane == 0) {
      for (;;) {
        const uint32_t u = *reinterpret_cast<volatile uint32_t*>(sNext);
        if (u >= ntiles || u >= tile + kStages) break;
        // stage u % kStages last held tile u - kStages: free once every warp released it
        if (!mbar_test(barEmpty + 8 * (u % kStages), ((u / kStages) + 1) & 1)) break;
        if (atomicCAS(sNext, u, u + 1) == u) issue(u);
      }
    }
    const bool landed = mbar_wait(barFull + 8 * b, (tile / kStages) & 1, P.wait_cycles);
    if (__any_sync(0xffffffffu, !landed)) {
      if (lane == 0) atomicOr(err, kErrWait);
      break;
    }

    const unsigned char* tB = sB + b * (kTileCols * kRowBytes);
    const float* tBias = sBias + b * kTileCols;
    float acc[kSlabs][8][4];
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
#pragma unroll
      for (int nb = 0; nb < 8; nb += 2) {
        const int r = 8 * (nb + (lane >> 4)) + (lane & 7);
        const int c = 2 * ks + ((lane >> 3) & 1);
        uint32_t b0, b1, b2, b3;
        ldmatrix_x4(smem_u32(tB + swz(r, c)), b0, b1, b2, b3);
        if (ks == 0) {
          const float2 c0 = *reinterpret_cast<const float2*>(tBias + nb * 8 + 2 * t4);
          const float2 c1 = *reinterpret_cast<const float2*>(tBias + (nb + 1) * 8 + 2 * t4);
#pragma unroll
          for (int s = 0; s < kSlabs; ++s) {
            mma_bf16_init(acc[s][nb], afr[s][0], b0, b1, c0.x, c0.y);
            mma_bf16_init(acc[s][nb + 1], afr[s][0], b2, b3, c1.x, c1.y);
          }
        } else {
#pragma unroll
          for (int s = 0; s < kSlabs; ++s) {
            mma_bf16(acc[s][nb], afr[s][ks], b0, b1);
            mma_bf16(acc[s][nb + 1], afr[s][ks], b2, b3);
          }
        }
      }
    }

    __syncwarp();
    if (lane == 0) mbar_arrive(barEmpty + 8 * b);

    // epilogue: the maximum of each (slab, half) row group against its row's
    // threshold; only groups that beat it look at their values one by one
    bool gh[kSlabs][2];
#pragma unroll
    for (int s = 0; s < kSlabs; ++s)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float m[8];  // a tree of maxima: depth 4 instead of a chain of 15
#pragma unroll
        for (int nb = 0; nb < 8; ++nb) m[nb] = fmaxf(acc[s][nb][2 * h], acc[s][nb][2 * h + 1]);
#pragma unroll
        for (int w = 4; w > 0; w >>= 1)
#pragma unroll
          for (int x = 0; x < w; ++x) m[x] = fmaxf(m[x], m[x + w]);
        gh[s][h] = m[0] > thr[s][h];
      }
    bool any_hit = false;
#pragma unroll
    for (int s = 0; s < kSlabs; ++s) any_hit |= gh[s][0] | gh[s][1];
    if (__any_sync(0xffffffffu, any_hit)) {
      // A row's 16 x 4 values of this tile sit in the four lanes of one quad,
      // and no other warp appends to it: the quad's lanes take consecutive
      // slots by a prefix sum of their hit counts, with no atomics.  Hits are
      // found as a bit mask, then read back from this lane's staging slots.
      float* stage = reinterpret_cast<float*>(sMine) + lane * 32;
#pragma unroll
      for (int s = 0; s < kSlabs; ++s) {
        uint32_t m[2] = {0u, 0u};
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (gh[s][h]) {
            uint32_t part[4] = {0u, 0u, 0u, 0u};  // independent partial masks
#pragma unroll
            for (int nb = 0; nb < 8; ++nb)
#pragma unroll
              for (int e = 0; e < 2; ++e)
                if (acc[s][nb][2 * h + e] > thr[s][h]) part[nb & 3] |= 1u << (2 * nb + e);
            m[h] = (part[0] | part[1]) | (part[2] | part[3]);
            const uint32_t i = row0 + (uint32_t)(warp * kRowsPerWarp + s * 16 + h * 8 + g);
            if (m[h] != 0u) m[h] &= valid_cols(i, tlo + tile, P.nA, P.nB, kSelf, t4);
          }
        }
        uint32_t pos[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int hc = __popc(m[h]);
          int incl = hc;
#pragma unroll
          for (int o = 1; o < 4; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o, 4);
            if (t4 >= o) incl += t;
          }
          pos[h] = (uint32_t)(cnt[s][h] + incl - hc);
          cnt[s][h] += __shfl_sync(0xffffffffu, incl, 3, 4);
        }
        if ((m[0] | m[1]) != 0u) {
#pragma unroll
          for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int nb = 0; nb < 8; ++nb)
              *reinterpret_cast<float2*>(stage + h * 16 + 2 * nb) =
                  make_float2(acc[s][nb][2 * h], acc[s][nb][2 * h + 1]);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const uint32_t i = row0 + (uint32_t)(warp * kRowsPerWarp + s * 16 + h * 8 + g);
            uint64_t* rb = row_buf(i);
            uint32_t mm = m[h], slot = pos[h];
            while (mm != 0u) {
              const int k = __ffs(mm) - 1;
              mm &= mm - 1u;
              const uint32_t j = (tlo + tile) * kTileCols + (uint32_t)((k >> 1) * 8 + 2 * t4 + (k & 1));
              rb[slot++] = make_key((int)stage[h * 16 + k], j);
            }
          }
        }
      }
    }
    __syncwarp();

    // rows of this warp holding more than `trigger` keys: compacting at 2C
    // (or when the buffer could overflow during the next tile) keeps the
    // thresholds close to the running C-th best value
    bool over = false;
#pragma unroll
    for (int s = 0; s < kSlabs; ++s) over |= (cnt[s][0] > trigger) | (cnt[s][1] > trigger);
    if (__any_sync(0xffffffffu, over)) {
      if (t4 == 0) {
#pragma unroll
        for (int s = 0; s < kSlabs; ++s)
#pragma unroll
          for (int h = 0; h < 2; ++h) sCnt[warp * kRowsPerWarp + s * 16 + h * 8 + g] = cnt[s][h];
      }
      __syncwarp();
      unsigned full = __ballot_sync(0xffffffffu, lane < kRowsPerWarp && sCnt[warp * kRowsPerWarp + lane] > trigger);
      while (full) {
        const int l = __ffs(full) - 1;
        full &= full - 1;
        const int lr = warp * kRowsPerWarp + l;
        uint64_t* rb = row_buf(row0 + (uint32_t)lr);
        const int c = sCnt[lr];
        // A threshold t at or below the C-th best value is enough here (the
        // final pass selects exactly): t is the lower edge of the 256-bin
        // value-histogram bin holding the C-th best key, and the keys with
        // value >= t stay.  A later value that can still enter the row's top
        // C beats the C-th best key now, hence t.  A crowded bin falls back
        // to the exact C-th key.
        int lo, hi;
        warp_value_range(rb, c, lane, lo, hi);
        const unsigned span = (unsigned)(hi - lo);
        const int sh = span < 256u ? 0 : 24 - __clz((int)span);
        warp_value_hist(rb, c, lo, sh, hMine, lane);
        int bin;
        unsigned above;
        hist_find_desc(hMine, C, lane, bin, above);
        const unsigned keep = above + hMine[bin];
        __syncwarp();
        int kept, t;
        if (keep <= keep_limit) {
          t = lo + (bin << sh);
          kept = warp_keep_value_ge(rb, c, t, lane);  // == keep
        } else {
          const uint64_t kth = warp_select_kth(rb, c, (int)C, hMine, lane);
          kept = warp_gather_ge(rb, c, kth, sMine, lane);  // == C
          for (int x = lane; x < kept; x += 32) rb[x] = sMine[x];
          t = key_val(kth);
        }
        if (lane == 0) {
          sCnt[lr] = kept;
          sThr[lr] = (float)t;
        }
        __syncwarp();
      }
#pragma unroll
      for (int s = 0; s < kSlabs; ++s)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          thr[s][h] = sThr[warp * kRowsPerWarp + s * 16 + h * 8 + g];
          cnt[s][h] = sCnt[warp * kRowsPerWarp + s * 16 + h * 8 + g];
        }
      __syncwarp();
    }
  }
  if (t4 == 0) {
#pragma unroll
    for (int s = 0; s < kSlabs; ++s)
#pragma unroll
      for (int h = 0; h < 2; ++h) sCnt[warp * kRowsPerWarp + s * 16 + h * 8 + g] = cnt[s][h];
  }
  __syncwarp();

  // final lists: the C best keys of each row, sorted
  for (int l = 0; l < kRowsPerWarp; ++l) {
    const int lr = warp * kRowsPerWarp + l;
    const uint32_t i = row0 + (uint32_t)lr;
    if (i >= P.nA) break;
    const int cnt = sCnt[lr];
    const uint64_t* rb = row_buf(i);
    const uint64_t kmin = cnt > (int)C ? warp_select_kth(rb, cnt, (int)C, hMine, lane) : 1ull;
    const int kept = warp_gather_ge(rb, cnt, kmin, sMine, lane);
    const int size = pow2_at_least(kept);
    for (int x = kept + lane; x < size; x += 32) sMine[x] = 0ull;
    __syncwarp();
    warp_bitonic_desc(sMine, size, lane);
    if (kSplit) {
      uint64_t* dst = P.part + ((size_t)i * P.splits + ys) * C;
      for (uint32_t x = lane; x < C; x += 32) dst[x] = (int)x < kept ? sMine[x] : 0ull;
    } else {
      for (uint32_t x = lane; x < C; x += 32) {
        const bool have = (int)x < kept;
        out_idx[(size_t)i * C + x] = have ? key_idx(sMine[x]) : 0xffffffffu;
        out_val[(size_t)i * C + x] = have ? key_val(sMine[x]) : INT32_MIN;
      }
    }
    __syncwarp();
  }

  // every issued copy has landed before the CTA's shared memory is released
  // (all of them were consumed, unless a wait ran out); each wait is bounded
  __syncthreads();
  if (tid == 0) {
    const uint32_t issued = *sNext;
    for (uint32_t u = issued > (uint32_t)kStages ? issued - kStages : 0u; u < issued; ++u) {
      if (u == P.withhold) continue;
      if (!mbar_wait(barFull + 8 * (u % kStages), (u / kStages) & 1, P.wait_cycles)) {
        atomicOr(err, kErrWait);
        break;
      }
    }
  }
}

// one warp per row: the C best of the row's splits' sorted lists (S x C
// keys, 0 for missing) by the exact select, then sorted
constexpr int kMergeWarps = 8;
__global__ void __launch_bounds__(kMergeWarps * 32)
    merge_splits_kernel(const uint64_t* __restrict__ part, uint32_t nA, uint32_t S, uint32_t C,
                        uint32_t* __restrict__ out_idx, int32_t* __restrict__ out_val) {
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
  const int size = pow2_at_least(kept);
  for (int x = kept + lane; x < size; x += 32) keep[warp][x] = 0ull;
  __syncwarp();
  warp_bitonic_desc(keep[warp], size, lane);
  for (uint32_t x = lane; x < C; x += 32) {
    const bool have = (int)x < kept;
    out_idx[(size_t)i * C + x] = have ? key_idx(keep[warp][x]) : 0xffffffffu;
    out_val[(size_t)i * C + x] = have ? key_val(keep[warp][x]) : INT32_MIN;
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

// Element (r, c) of the bf16 rows the candidate kernel reads: rows padded
// with zeros to a whole number of column tiles, and the 16-byte chunks of row
// r permuted by r & 7, the shared-memory swizzle its tiles are copied into.
__device__ __forceinline__ size_t swz_index(size_t r, int c) {
  return r * kDim + (size_t)((((c >> 3) ^ (int)(r & 7)) << 3) | (c & 7));
}

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
  if (qb) qb[swz_index(r, c)] = __float2bfloat16_rn(v);
}

__global__ void widen_kernel(const int8_t* __restrict__ q, uint32_t n, uint32_t npad, __nv_bfloat16* qb) {
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (size_t)npad * kDim) return;
  const size_t r = x / kDim;
  qb[swz_index(r, (int)(x - r * kDim))] = __float2bfloat16_rn(r < n ? (float)q[x] : 0.f);
}

__global__ void bias_float_kernel(const int32_t* __restrict__ bias, uint32_t n, uint32_t npad, float* biasf) {
  const uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x < npad) biasf[x] = (bias && x < n) ? (float)bias[x] : 0.f;
}

size_t bias_pad(uint32_t n) { return ((size_t)n + kTileCols - 1) / kTileCols * kTileCols; }

}  // namespace

size_t dot_topk_qb_bytes(uint32_t n) { return bias_pad(n) * kRowBytes; }

// column splits of a launch over nA rows and nB columns on the current
// device: enough CTAs for kCtasPerSm per SM when the row blocks alone are
// fewer, each split at least 8 tiles of 64 columns
uint32_t dot_topk_splits(uint32_t nA, uint32_t nB) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                   cudaSuccess || sms <= 0) {
    cudaGetLastError();
    sms = 152;
  }
  const uint32_t blocks = (nA + kRowsPerCta - 1) / kRowsPerCta;
  const uint32_t tiles = (nB + kTileCols - 1) / kTileCols;
  const uint32_t slots = (uint32_t)kCtasPerSm * (uint32_t)sms;
  const uint32_t want = (slots + blocks - 1) / std::max(blocks, 1u);
  return std::max(1u, std::min(want, tiles / 8));
}

size_t dot_topk_buffer_bytes(uint32_t nA, uint32_t nB, uint32_t C) {
  const size_t S = dot_topk_splits(nA, nB);
  return (size_t)nA * S * kCap * sizeof(uint64_t) + bias_pad(nB) * sizeof(float) + 16 +
         (S > 1 ? (size_t)nA * S * C * sizeof(uint64_t) : 0);
}

uint32_t* dot_topk_err_word(uint64_t* buf, uint32_t nA, uint32_t nB) {
  const size_t S = dot_topk_splits(nA, nB);
  return reinterpret_cast<uint32_t*>(reinterpret_cast<float*>(buf + (size_t)nA * S * kCap) + bias_pad(nB));
}

cudaError_t dot_topk_rect(const __nv_bfloat16* QA, uint32_t nA, const __nv_bfloat16* QB, const int32_t* biasB,
                          uint32_t nB, uint32_t C, bool self, uint64_t* buf, uint32_t* idx, int32_t* val,
                          uint32_t* err, cudaStream_t s, DotDebug dbg) {
  if (nA == 0) return cudaSuccess;
  const uint32_t S = dot_topk_splits(nA, nB);
  const auto kernel = S > 1 ? (self ? dot_topk_kernel<true, true> : dot_topk_kernel<true, false>)
                             : (self ? dot_topk_kernel<false, true> : dot_topk_kernel<false, false>);
  cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotal);
  if (e != cudaSuccess) return e;
  const uint32_t tiles = (nB + kTileCols - 1) / kTileCols;
  DotArgs P;
  P.QA = QA;
  P.QB = QB;
  P.biasf = reinterpret_cast<float*>(buf + (size_t)nA * S * kCap);  // after the append buffers (16-byte aligned)
  P.nA = nA;
  P.nB = nB;
  P.C = C;
  P.self = self;
  P.splits = S;
  P.tps = (tiles + S - 1) / S;
  P.buf = buf;
  // the split lists follow the buffer's own error-word slot (err itself may live elsewhere)
  P.part = S > 1 ? reinterpret_cast<uint64_t*>(reinterpret_cast<char*>(dot_topk_err_word(buf, nA, nB)) + 16) : nullptr;
  P.out_idx = idx;
  P.out_val = val;
  P.err = err;
  P.wait_cycles = dbg.wait_cycles >= 0 ? dbg.wait_cycles : kWaitCycles;
  P.withhold = dbg.withhold;
  const uint32_t npad = (uint32_t)bias_pad(nB);
  bias_float_kernel<<<(npad + 255) / 256 + (npad == 0), 256, 0, s>>>(biasB, nB, npad, const_cast<float*>(P.biasf));
  const dim3 grid((nA + kRowsPerCta - 1) / kRowsPerCta, S);
  kernel<<<grid, kThreads, kSmemTotal, s>>>(P);
  if (S > 1)
    merge_splits_kernel<<<(nA + kMergeWarps - 1) / kMergeWarps, kMergeWarps * 32, 0, s>>>(P.part, nA, S, C, idx, val);
  return cudaGetLastError();
}

cudaError_t dot_topk(const __nv_bfloat16* Qb, const int32_t* bias, uint32_t n, uint32_t C, uint64_t* buf,
                     uint32_t* idx, int32_t* val, uint32_t* err, cudaStream_t s, DotDebug dbg) {
  return dot_topk_rect(Qb, n, Qb, bias, n, C, true, buf, idx, val, err, s, dbg);
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

cudaError_t widen(const int8_t* q, uint32_t n, __nv_bfloat16* qb, cudaStream_t s) {
  const size_t count = (size_t)bias_pad(n) * kDim;
  if (!count) return cudaSuccess;
  widen_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(q, n, (uint32_t)bias_pad(n), qb);
  return cudaGetLastError();
}

}  // namespace prop
}  // namespace nw
