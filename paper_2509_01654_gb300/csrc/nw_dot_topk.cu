// nw_dot_topk.cu -- candidate proposal by dot product of quantised embeddings.
//
// Embeddings are quantised to integers in [-127, 127] and stored as bf16,
// which holds them exactly; products of two are at most 16,129 and a sum of
// 64 at most 1,032,256 < 2^24, so the tensor cores' float32 accumulation
// gives the exact integer dot product in any order.  The top-C selection is
// then an exact, deterministic function of the integers (ties: lower index).
//
// dot_topk_kernel: a CTA owns 256 rows (8 warps x 32 rows, A fragments held
// in registers for the whole sweep) and sweeps every column in tiles of 64
// (double-buffered cp.async into swizzled shared memory, ldmatrix, bf16
// m16n8k16 mma.sync with float32 accumulators).  Each row keeps an append
// buffer of kCap keys in global memory and a threshold: a value enters when it
// beats the threshold; when a row's buffer could overflow in the next tile its
// warp sorts it (bitonic, in shared memory), keeps the C best and raises the
// threshold to the C-th value.  Later columns have higher indices, so a later
// value equal to the threshold can never displace a kept one: the comparison
// is strict and the final lists are exact.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <float.h>
#include <stdint.h>

#include "nw_internal.cuh"
#include "nw_proposal_internal.h"

namespace nw {
namespace prop {
namespace {

constexpr int kDim = 64;                 // embedding values per row (bf16)
constexpr int kRowBytes = kDim * 2;      // 128
constexpr int kRowsPerWarp = 32;
constexpr int kWarps = 8;
constexpr int kRowsPerCta = kRowsPerWarp * kWarps;  // 256
constexpr int kTileCols = 64;
constexpr int kThreads = kWarps * 32;
constexpr int kSortSlots = kCap;         // per-warp sort area (keys)

// dynamic shared memory layout (bytes)
constexpr int kSmemB = 2 * kTileCols * kRowBytes;                   // 16 KiB, two B tiles
constexpr int kSmemSort = kWarps * kSortSlots * 8;                  // 64 KiB (A staging at start)
constexpr int kSmemCnt = kRowsPerCta * 4;
constexpr int kSmemThr = kRowsPerCta * 4;
constexpr int kSmemTotal = kSmemB + kSmemSort + kSmemCnt + kSmemThr;
static_assert(kRowsPerCta * kRowBytes <= kSmemSort, "A staging fits the sort area");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

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

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// key: higher dot first, then lower index; 0 sorts below every real key
__device__ __forceinline__ uint64_t make_key(int dot, uint32_t j) {
  return ((uint64_t)(uint32_t)(dot + 0x80000000) << 32) | (uint64_t)(0xffffffffu - j);
}
__device__ __forceinline__ int key_dot(uint64_t k) { return (int)((uint32_t)(k >> 32) - 0x80000000u); }
__device__ __forceinline__ uint32_t key_idx(uint64_t k) { return 0xffffffffu - (uint32_t)k; }

// Sorts s[0, size) descending (size a power of two, <= kSortSlots) with the warp.
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

__device__ __forceinline__ int pow2_at_least(int x) {
  int p = 32;
  while (p < x) p <<= 1;
  return p;
}

// Loads a row's buffer into the warp's sort area and sorts it; returns the padded size.
__device__ int load_sort(const uint64_t* buf, int cnt, uint64_t* s, int lane) {
  const int size = pow2_at_least(cnt);
  for (int i = lane; i < size; i += 32) s[i] = i < cnt ? buf[i] : 0ull;
  __syncwarp();
  warp_bitonic_desc(s, size, lane);
  return size;
}

__global__ void __launch_bounds__(kThreads, 2)
    dot_topk_kernel(const __nv_bfloat16* __restrict__ Q, uint32_t n, uint32_t C, uint64_t* __restrict__ buf,
                    uint32_t* __restrict__ out_idx, int32_t* __restrict__ out_dot) {
  extern __shared__ __align__(128) unsigned char smem[];
  unsigned char* sB = smem;
  uint64_t* sSort = reinterpret_cast<uint64_t*>(smem + kSmemB);
  int* sCnt = reinterpret_cast<int*>(smem + kSmemB + kSmemSort);
  float* sThr = reinterpret_cast<float*>(smem + kSmemB + kSmemSort + kSmemCnt);

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
  // rows of this lane's accumulator values: slab s, half h -> local row
  int lrow[2][2];
#pragma unroll
  for (int s = 0; s < 2; ++s)
#pragma unroll
    for (int h = 0; h < 2; ++h) lrow[s][h] = warp * kRowsPerWarp + s * 16 + h * 8 + g;
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
  };
  if (ntiles) load_tile(0, 0);
  cp_async_commit();

  uint64_t* sMine = sSort + warp * kSortSlots;
  for (uint32_t tile = 0; tile < ntiles; ++tile) {
    const int b = tile & 1;
    if (tile + 1 < ntiles) load_tile(tile + 1, b ^ 1);
    cp_async_commit();
    cp_async_wait<1>();
    __syncthreads();

    const unsigned char* tB = sB + b * (kTileCols * kRowBytes);
    float acc[2][8][4];
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int nb = 0; nb < 8; ++nb)
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[s][nb][q] = 0.f;
#pragma unroll
    for (int ks = 0; ks < 4; ++ks) {
#pragma unroll
      for (int nb = 0; nb < 8; nb += 2) {
        const int r = 8 * (nb + (lane >> 4)) + (lane & 7);
        const int c = 2 * ks + ((lane >> 3) & 1);
        uint32_t b0, b1, b2, b3;
        ldmatrix_x4(smem_u32(tB + swz(r, c)), b0, b1, b2, b3);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          mma_bf16(acc[s][nb], afr[s][ks], b0, b1);
          mma_bf16(acc[s][nb + 1], afr[s][ks], b2, b3);
        }
      }
    }

    // epilogue: one compare per value; the rare winners take the slow path
    bool any = false;
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int nb = 0; nb < 8; ++nb)
#pragma unroll
        for (int q = 0; q < 4; ++q) any |= acc[s][nb][q] > thr[s][q >> 1];
    if (__any_sync(0xffffffffu, any)) {
      const uint32_t j0 = tile * kTileCols;
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int lr = lrow[s][h];
          const uint32_t i = row0 + (uint32_t)lr;
          if (i >= n) continue;
#pragma unroll
          for (int nb = 0; nb < 8; ++nb)
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const float v = acc[s][nb][2 * h + e];
              const uint32_t j = j0 + (uint32_t)(nb * 8 + 2 * t4 + e);
              if (v > thr[s][h] && j < n && j != i) {
                const int slot = atomicAdd(&sCnt[lr], 1);
                buf[(size_t)i * kCap + slot] = make_key((int)v, j);
              }
            }
        }
    }
    __syncwarp();

    // rows of this warp whose buffers could overflow during the next tile
    const int myrow = warp * kRowsPerWarp + lane;
    unsigned full = __ballot_sync(0xffffffffu, sCnt[myrow] > kCap - kTileCols);
    if (full) {
      while (full) {
        const int l = __ffs(full) - 1;
        full &= full - 1;
        const int lr = warp * kRowsPerWarp + l;
        const uint32_t i = row0 + (uint32_t)lr;
        uint64_t* rb = buf + (size_t)i * kCap;
        load_sort(rb, sCnt[lr], sMine, lane);
        for (uint32_t x = lane; x < C; x += 32) rb[x] = sMine[x];
        if (lane == 0) {
          sCnt[lr] = (int)C;
          sThr[lr] = (float)key_dot(sMine[C - 1]);
        }
        __syncwarp();
      }
#pragma unroll
      for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int h = 0; h < 2; ++h) thr[s][h] = sThr[lrow[s][h]];
    }
    __syncthreads();  // the B buffer of this tile is reloaded next
  }

  // final lists: sort each row's buffer and write its C best
  for (int l = 0; l < kRowsPerWarp; ++l) {
    const int lr = warp * kRowsPerWarp + l;
    const uint32_t i = row0 + (uint32_t)lr;
    if (i >= n) break;
    const int cnt = sCnt[lr];
    load_sort(buf + (size_t)i * kCap, cnt, sMine, lane);
    for (uint32_t x = lane; x < C; x += 32) {
      const bool have = (int)x < cnt;
      out_idx[(size_t)i * C + x] = have ? key_idx(sMine[x]) : 0xffffffffu;
      out_dot[(size_t)i * C + x] = have ? key_dot(sMine[x]) : INT32_MIN;
    }
    __syncwarp();
  }
}

__global__ void absmax_kernel(const float* __restrict__ E, size_t count, unsigned int* amax_bits) {
  float m = 0.f;
  for (size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x; x < count; x += (size_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(E[x]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(amax_bits, __float_as_uint(m));  // non-negative floats order as integers
}

__global__ void quantize_kernel(const float* __restrict__ E, size_t count, const unsigned int* amax_bits,
                                int8_t* q, __nv_bfloat16* qb, float* scale_out) {
  const float scale = __uint_as_float(*amax_bits) / 127.0f;
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x == 0 && scale_out) *scale_out = scale;
  if (x >= count) return;
  float v = 0.f;
  if (scale > 0.f) v = fminf(fmaxf(rintf(E[x] / scale), -127.f), 127.f);
  if (q) q[x] = (int8_t)v;
  if (qb) qb[x] = __float2bfloat16_rn(v);
}

__global__ void widen_kernel(const int8_t* __restrict__ q, size_t count, __nv_bfloat16* qb) {
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x < count) qb[x] = __float2bfloat16_rn((float)q[x]);
}

}  // namespace

size_t dot_topk_buffer_bytes(uint32_t n) { return (size_t)n * kCap * sizeof(uint64_t); }

cudaError_t dot_topk(const __nv_bfloat16* Qb, uint32_t n, uint32_t C, uint64_t* buf, uint32_t* idx, int32_t* dot,
                     cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(dot_topk_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemTotal);
  if (e != cudaSuccess) return e;
  const unsigned grid = (n + kRowsPerCta - 1) / kRowsPerCta;
  dot_topk_kernel<<<grid, kThreads, kSmemTotal, s>>>(Qb, n, C, buf, idx, dot);
  return cudaGetLastError();
}

cudaError_t quantize(const float* E, uint32_t n, unsigned int* amax_bits, int8_t* q, __nv_bfloat16* qb,
                     float* scale, cudaStream_t s) {
  const size_t count = (size_t)n * kDim;
  cudaError_t e = cudaMemsetAsync(amax_bits, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  if (count) absmax_kernel<<<1024, 256, 0, s>>>(E, count, amax_bits);
  quantize_kernel<<<(unsigned)((count + 255) / 256 + (count == 0)), 256, 0, s>>>(E, count, amax_bits, q, qb, scale);
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
