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
// and no branch).  When a row holds more than 4C keys (or its buffer could
// overflow during the next tile), its warp finds the row's C-th best key by
// an 8-pass radix select (8 bits per pass), keeps the C keys at or above it
// and raises the threshold to that key's value.  Later columns
// have higher indices, so a later value equal to the threshold never
// displaces a kept key: the comparison is strict and the lists are exact.
#include <cuda_bf16.h>
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
constexpr int kRowsPerWarp = 32;
constexpr int kWarps = 8;
constexpr int kRowsPerCta = kRowsPerWarp * kWarps;  // 256
constexpr int kTileCols = 64;
constexpr int kThreads = kWarps * 32;
constexpr int kSel = NW_MAX_CANDIDATES;  // per-warp gather/sort area (keys)

// dynamic shared memory layout (bytes)
constexpr int kStages = 3;                              // B tiles in flight (one barrier per tile)
constexpr int kSmemB = kStages * kTileCols * kRowBytes; // 24 KiB
constexpr int kSmemBias = kStages * kTileCols * 4;      // their biases (float)
constexpr int kSmemSort = kWarps * kSel * 8;            // 32 KiB (A staging at start)
constexpr int kSmemHist = kWarps * 256 * 4;             // radix histograms
constexpr int kSmemCnt = kRowsPerCta * 4;
constexpr int kSmemThr = kRowsPerCta * 4;
constexpr int kOffBias = kSmemB;
constexpr int kOffSort = kOffBias + kSmemBias;
constexpr int kOffHist = kOffSort + kSmemSort;
constexpr int kOffCnt = kOffHist + kSmemHist;
constexpr int kOffThr = kOffCnt + kSmemCnt;
constexpr int kSmemTotal = kOffThr + kSmemThr;
static_assert(kRowsPerCta * kRowBytes <= kSmemSort, "A staging fits the sort area");
static_assert(kCap - kTileCols > NW_MAX_CANDIDATES, "a compaction leaves room for a tile");

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
    for (int i = lane; i < cnt; i += 32) {
      const uint64_t k = buf[i];
      if ((k & hmask) == prefix) atomicAdd(&hist[(uint32_t)(k >> sh) & 255u], 1u);
    }
    __syncwarp();
    // lane l holds bins 255 - 8l .. 248 - 8l (descending digit order)
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
    int bin = 0;
    unsigned before = 0;
    if (mine) {
      unsigned acc = excl;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (acc + c[q] >= need) {
          bin = 255 - 8 * lane - q;
          before = acc;
          break;
        }
        acc += c[q];
      }
    }
    bin = __shfl_sync(0xffffffffu, bin, src);
    before = __shfl_sync(0xffffffffu, before, src);
    prefix |= (uint64_t)bin << sh;
    need -= before;
    __syncwarp();
  }
  return prefix;
}

// Copies the keys >= kmin of buf[0, cnt) into s (in any order); returns how many.
__device__ int warp_gather_ge(const uint64_t* buf, int cnt, uint64_t kmin, uint64_t* s, int lane) {
  int base = 0;
  for (int i0 = 0; i0 < cnt; i0 += 32) {
    const int i = i0 + lane;
    const uint64_t k = i < cnt ? buf[i] : 0ull;
    const bool keep = i < cnt && k >= kmin;
    const unsigned ball = __ballot_sync(0xffffffffu, keep);
    if (keep) s[base + __popc(ball & ((1u << lane) - 1u))] = k;
    base += __popc(ball);
  }
  __syncwarp();
  return base;
}

__device__ __forceinline__ int pow2_at_least(int x) {
  int p = 32;
  while (p < x) p <<= 1;
  return p;
}

// biasf: the columns' biases as floats (exact: |bias| <= 2^23), zero-padded to
// a multiple of kTileCols entries
__global__ void __launch_bounds__(kThreads, 2)
    dot_topk_kernel(const __nv_bfloat16* __restrict__ Q, const float* __restrict__ biasf, uint32_t n, uint32_t C,
                    uint64_t* __restrict__ buf, uint32_t* __restrict__ out_idx, int32_t* __restrict__ out_val) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* sB = smem;
  float* sBias = reinterpret_cast<float*>(smem + kOffBias);
  uint64_t* sSort = reinterpret_cast<uint64_t*>(smem + kOffSort);
  unsigned* sHist = reinterpret_cast<unsigned*>(smem + kOffHist);
  int* sCnt = reinterpret_cast<int*>(smem + kOffCnt);
  float* sThr = reinterpret_cast<float*>(smem + kOffThr);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t row0 = blockIdx.x * (uint32_t)kRowsPerCta;
  const unsigned char* Qb = reinterpret_cast<const unsigned char*>(Q);

  // stage the CTA's 256 rows (zero past n) into the sort area, swizzled
  unsigned char* sA = reinterpret_cast<unsigned char*>(sSort);
  for (int x = tid; x < kRowsPerCta * 8; x += kThreads) {
    const int r = x >> 3, c = x & 7;
    const uint32_t g = row0 + (uint32_t)r;
    cp_async16(smem_u32(sA + swz(r, c)), Qb + (size_t)(g < n ? g : 0) * kRowBytes + c * 16, g < n);
  }
  cp_async_commit();
  for (int r = tid; r < kRowsPerCta; r += kThreads) {
    sCnt[r] = 0;
    sThr[r] = -FLT_MAX;
  }
  cp_async_wait<0>();
  __syncthreads();

  // A fragments: slab s (16 rows), k-step ks
  uint32_t afr[2][4][4];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
      const int r = warp * kRowsPerWarp + s * 16 + (lane & 15);
      const int c = 2 * ks + (lane >> 4);
      ldmatrix_x4(smem_u32(sA + swz(r, c)), afr[s][ks][0], afr[s][ks][1], afr[s][ks][2], afr[s][ks][3]);
    }
  __syncthreads();  // the sort area is free from here on

  const int g = lane >> 2, t4 = lane & 3;
  float thr[2][2];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int h = 0; h < 2; ++h) thr[s][h] = -FLT_MAX;

  const uint32_t ntiles = (n + kTileCols - 1) / kTileCols;
  auto load_tile = [&](uint32_t tile, int b) {
    unsigned char* dst = sB + b * (kTileCols * kRowBytes);
    for (int x = tid; x < kTileCols * 8; x += kThreads) {
      const int r = x >> 3, c = x & 7;
      const uint32_t j = tile * kTileCols + (uint32_t)r;
      cp_async16(smem_u32(dst + swz(r, c)), Qb + (size_t)(j < n ? j : 0) * kRowBytes + c * 16, j < n);
    }
    if (tid < kTileCols / 4)
      cp_async16(smem_u32(sBias + b * kTileCols + tid * 4), biasf + (size_t)tile * kTileCols + tid * 4, true);
  };
#pragma unroll
  for (int st = 0; st < kStages - 1; ++st) {
    if ((uint32_t)st < ntiles) load_tile((uint32_t)st, st);
    cp_async_commit();
  }

  uint64_t* sMine = sSort + warp * kSel;
  unsigned* hMine = sHist + warp * 256;
  const int trigger = min(kCap - kTileCols, 4 * (int)C);
  for (uint32_t tile = 0; tile < ntiles; ++tile) {
    const int b = (int)(tile % kStages);
    cp_async_wait<kStages - 2>();  // this tile's group has landed
    __syncthreads();               // ... for every thread; and every warp is done with tile - 1
    if (tile + kStages - 1 < ntiles) load_tile(tile + kStages - 1, (int)((tile + kStages - 1) % kStages));
    cp_async_commit();

    const unsigned char* tB = sB + b * (kTileCols * kRowBytes);
    const float* tBias = sBias + b * kTileCols;
    float acc[2][8][4];
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
          for (int s = 0; s < 2; ++s) {
            mma_bf16_init(acc[s][nb], afr[s][0], b0, b1, c0.x, c0.y);
            mma_bf16_init(acc[s][nb + 1], afr[s][0], b2, b3, c1.x, c1.y);
          }
        } else {
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            mma_bf16(acc[s][nb], afr[s][ks], b0, b1);
            mma_bf16(acc[s][nb + 1], afr[s][ks], b2, b3);
          }
        }
      }
    }

    // epilogue: the maximum of each (slab, half) row group against its row's
    // threshold; only groups that beat it look at their values one by one
    bool gh[2][2];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        float m = fmaxf(acc[s][0][2 * h], acc[s][0][2 * h + 1]);
#pragma unroll
        for (int nb = 1; nb < 8; ++nb) m = fmaxf(m, fmaxf(acc[s][nb][2 * h], acc[s][nb][2 * h + 1]));
        gh[s][h] = m > thr[s][h];
      }
    if (__any_sync(0xffffffffu, gh[0][0] | gh[0][1] | gh[1][0] | gh[1][1])) {
      const uint32_t j0 = tile * kTileCols + 2u * (uint32_t)t4;
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (!gh[s][h]) continue;
          const int lr = warp * kRowsPerWarp + s * 16 + h * 8 + g;
          const uint32_t i = row0 + (uint32_t)lr;
#pragma unroll
          for (int nb = 0; nb < 8; ++nb)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const float v = acc[s][nb][2 * h + e];
              if (v > thr[s][h]) {
                const uint32_t j = j0 + (uint32_t)(nb * 8 + e);
                if (i < n && j < n && j != i) {
                  const int slot = atomicAdd(&sCnt[lr], 1);
                  buf[(size_t)i * kCap + slot] = make_key((int)v, j);
                }
              }
            }
        }
    }
    __syncwarp();

    // rows of this warp holding more than `trigger` keys: compacting at 4C
    // (or when the buffer could overflow during the next tile) keeps the
    // thresholds close to the running C-th best value
    unsigned full = __ballot_sync(0xffffffffu, sCnt[warp * kRowsPerWarp + lane] > trigger);
    if (full) {
      while (full) {
        const int l = __ffs(full) - 1;
        full &= full - 1;
        const int lr = warp * kRowsPerWarp + l;
        uint64_t* rb = buf + (size_t)(row0 + (uint32_t)lr) * kCap;
        const uint64_t kth = warp_select_kth(rb, sCnt[lr], (int)C, hMine, lane);
        const int kept = warp_gather_ge(rb, sCnt[lr], kth, sMine, lane);  // == C
        for (int x = lane; x < kept; x += 32) rb[x] = sMine[x];
        if (lane == 0) {
          sCnt[lr] = kept;
          sThr[lr] = (float)key_val(kth);
        }
        __syncwarp();
      }
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int h = 0; h < 2; ++h) thr[s][h] = sThr[warp * kRowsPerWarp + s * 16 + h * 8 + g];
    }
  }
  cp_async_wait<0>();

  // final lists: the C best keys of each row, sorted
  for (int l = 0; l < kRowsPerWarp; ++l) {
    const int lr = warp * kRowsPerWarp + l;
    const uint32_t i = row0 + (uint32_t)lr;
    if (i >= n) break;
    const int cnt = sCnt[lr];
    const uint64_t* rb = buf + (size_t)i * kCap;
    const uint64_t kmin = cnt > (int)C ? warp_select_kth(rb, cnt, (int)C, hMine, lane) : 1ull;
    const int kept = warp_gather_ge(rb, cnt, kmin, sMine, lane);
    const int size = pow2_at_least(kept);
    for (int x = kept + lane; x < size; x += 32) sMine[x] = 0ull;
    __syncwarp();
    warp_bitonic_desc(sMine, size, lane);
    for (uint32_t x = lane; x < C; x += 32) {
      const bool have = (int)x < kept;
      out_idx[(size_t)i * C + x] = have ? key_idx(sMine[x]) : 0xffffffffu;
      out_val[(size_t)i * C + x] = have ? key_val(sMine[x]) : INT32_MIN;
    }
    __syncwarp();
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

__global__ void quantize_kernel(const float* __restrict__ E, uint32_t n, const unsigned int* amax_bits, int8_t* q,
                                __nv_bfloat16* qb, int32_t* bias, float* scale_out) {
  const float scale = __uint_as_float(*amax_bits) / 127.0f;
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x == 0 && scale_out) *scale_out = scale;
  if (x >= (size_t)n * kDim) return;
  const size_t r = x / kDim;
  const int c = (int)(x - r * kDim);
  float v = 0.f;
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
  if (qb) qb[x] = __float2bfloat16_rn(v);
}

__global__ void widen_kernel(const int8_t* __restrict__ q, size_t count, __nv_bfloat16* qb) {
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < count) qb[x] = __float2bfloat16_rn((float)q[x]);
}

__global__ void bias_float_kernel(const int32_t* __restrict__ bias, uint32_t n, uint32_t npad, float* biasf) {
  const uint32_t x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x < npad) biasf[x] = (bias && x < n) ? (float)bias[x] : 0.f;
}

size_t bias_pad(uint32_t n) { return ((size_t)n + kTileCols - 1) / kTileCols * kTileCols; }

}  // namespace

size_t dot_topk_buffer_bytes(uint32_t n) { return (size_t)n * kCap * sizeof(uint64_t) + bias_pad(n) * sizeof(float); }

cudaError_t dot_topk(const __nv_bfloat16* Qb, const int32_t* bias, uint32_t n, uint32_t C, uint64_t* buf,
                     uint32_t* idx, int32_t* val, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(dot_topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotal);
  if (e != cudaSuccess) return e;
  float* biasf = reinterpret_cast<float*>(buf + (size_t)n * kCap);  // after the append buffers
  const uint32_t npad = (uint32_t)bias_pad(n);
  bias_float_kernel<<<(npad + 255) / 256, 256, 0, s>>>(bias, n, npad, biasf);
  const unsigned grid = (n + kRowsPerCta - 1) / kRowsPerCta;
  dot_topk_kernel<<<grid, kThreads, kSmemTotal, s>>>(Qb, biasf, n, C, buf, idx, val);
  return cudaGetLastError();
}

cudaError_t quantize(const float* E, uint32_t n, unsigned int* amax_bits, int8_t* q, __nv_bfloat16* qb,
                     int32_t* bias, float* scale, cudaStream_t s) {
  const size_t count = (size_t)n * kDim;
  cudaError_t e = cudaMemsetAsync(amax_bits, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  if (count) absmax_kernel<<<1024, 256, 0, s>>>(E, n, amax_bits);
  quantize_kernel<<<(unsigned)((count + 255) / 256 + (count == 0)), 256, 0, s>>>(E, n, amax_bits, q, qb, bias,
                                                                                   scale);
  return cudaGetLastError();
}

cudaError_t widen(const int8_t* q, uint32_t n, __nv_bfloat16* qb, cudaStream_t s) {
  const size_t count = (size_t)n * kDim;
  if (!count) return cudaSuccess;
  widen_kernel<<<(unsigned)((count + 255) / 256), 256, 0, s>>>(q, count, qb);
  return cudaGetLastError();
}

}  // namespace prop
}  // namespace nw
