// nw_cnn.cu -- kernels of the proposal network: bf16 tensor-core matrix
// products (float32 accumulation) whose operand loaders gather convolution windows directly from the packed
// activations (no im2col buffer, no padding rows), and the elementwise steps
// around them.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "nw_cnn.h"
#include "nw_internal.cuh"
#include "nw_tc.cuh"

namespace nw {
namespace cnn {
namespace {

// ---------------------------------------------------------------------------
// operand views: element (r, c) of a logical matrix, read four at a time
// along the view's contiguous axis: kColFast views give (r, c .. c + 3),
// the others (r .. r + 3, c).  Contiguous extents are multiples of four and
// rows start 16-byte aligned; channel counts are powers of two.

struct Dense {  // row-major
  const float* p;
  int ld;
  static constexpr bool kColFast = true;
  __device__ __forceinline__ float4 vec4(int r, int c) const {
    return __ldg(reinterpret_cast<const float4*>(p + (size_t)r * ld + c));
  }
  // the same, with the row's table entry read ahead (none for a dense view)
  __device__ __forceinline__ int row_info(int) const { return 0; }
  __device__ __forceinline__ float4 vec4r(int r, int c, int) const { return vec4(r, c); }
};

struct DenseT {  // transpose of a row-major matrix
  const float* p;
  int ld;
  static constexpr bool kColFast = false;
  __device__ __forceinline__ float4 vec4(int r, int c) const {
    return __ldg(reinterpret_cast<const float4*>(p + (size_t)c * ld + r));
  }
};

// im2col of packed X[T][Ci]: (t, tap * Ci + ch) = X[t + tap - 1][ch] when
// position pos(t) + tap - 1 lies inside t's word (rinfo: (pos << 8) | len)
struct Im2col {
  const float* X;
  const int* rinfo;
  int lg;  // log2 Ci
  static constexpr bool kColFast = true;
  __device__ __forceinline__ float4 vec4(int t, int k) const { return vec4r(t, k, row_info(t)); }
  // the same with row t's table entry given (a kernel that keeps its rows' entries at hand)
  __device__ __forceinline__ int row_info(int t) const { return __ldg(rinfo + t); }
  __device__ __forceinline__ float4 vec4r(int t, int k, int info) const {
    const int tap = k >> lg;
    const int pos = (info >> 8) + tap - 1;
    if (pos < 0 || pos >= (info & 255)) return make_float4(0.f, 0.f, 0.f, 0.f);
    return __ldg(reinterpret_cast<const float4*>(X + ((size_t)(t + tap - 1) << lg) + (k & ((1 << lg) - 1))));
  }
};

// shifted output gradient: (t, tap * Co + o) = dY[t - tap + 1][o] when
// position pos(t) - tap + 1 lies inside t's word
struct Shift {
  const float* dY;
  const int* rinfo;
  int lg;  // log2 Co
  static constexpr bool kColFast = true;
  __device__ __forceinline__ float4 vec4(int t, int k) const {
    const int tap = k >> lg;
    const int info = __ldg(rinfo + t);
    const int pos = (info >> 8) - tap + 1;
    if (pos < 0 || pos >= (info & 255)) return make_float4(0.f, 0.f, 0.f, 0.f);
    return __ldg(reinterpret_cast<const float4*>(dY + ((size_t)(t - tap + 1) << lg) + (k & ((1 << lg) - 1))));
  }
};

// W[Co][3][Ci] read as the (tap * Co + o, ch) matrix of the input gradient
struct WTap {
  const float* W;
  int lgCo, Ci;
  static constexpr bool kColFast = true;
  __device__ __forceinline__ float4 vec4(int k, int ch) const {
    const int tap = k >> lgCo, o = k & ((1 << lgCo) - 1);
    return __ldg(reinterpret_cast<const float4*>(W + ((size_t)o * 3 + tap) * Ci + ch));
  }
};

// bf16 tensor-core tiles: 128 x 128 outputs per block of 8 warps (2 x 4,
// 64 x 32 each, m16n8k16 products with float32 accumulation), K in steps of
// 32 through two shared buffers.  Each operand tile is staged in its
// memory's orientation -- [m][k] / [n][k] when K is the contiguous axis,
// [k][m] / [k][n] otherwise (read back with ldmatrix .trans) -- by 16-byte
// loads rounded to bf16 (nearest even).  Shared rows are padded (40 or 136
// values) so that the eight 16-byte rows of an ldmatrix fall in distinct
// banks.
constexpr int BM = 128, BN = 128, BK = 32, NT = 256;
constexpr int LDK = BK + 8;    // row of a [m][k] tile
constexpr int LDM = BM + 8;    // row of a [k][m] tile
constexpr int kTileHalfs = BM * LDK > BK * LDM ? BM * LDK : BK * LDM;

__device__ __forceinline__ uint2 pack4_bf16(float4 v) {
  const __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
  return make_uint2(*reinterpret_cast<const uint32_t*>(&lo), *reinterpret_cast<const uint32_t*>(&hi));
}

__device__ __forceinline__ void ldsm_x4(const void* p, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}
__device__ __forceinline__ void ldsm_x4_t(const void* p, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3) {
  const uint32_t a = (uint32_t)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0, %1, %2, %3}, [%4];\n"
               : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
               : "r"(a));
}

__device__ __forceinline__ void mma_bf16(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// One operand's 128 x 32 tile (outer index o over 128, k over 32).  KFast:
// the memory is contiguous along k (vectors (o, k .. k + 3)), staged [o][k];
// else along o (vectors (o .. o + 3, k)), staged [k][o].  Thread tid holds
// vectors tid + 256 q, q < 4.  at(o, k) is the view's vec4 at logical
// (outer, k) for A, (k, outer) for B.
template <bool KFast>
struct TileMap {
  __device__ __forceinline__ static void pos(int x, int& o, int& k) {
    if (KFast) {
      o = x >> 3;
      k = (x & 7) * 4;
    } else {
      k = x >> 5;
      o = (x & 31) * 4;
    }
  }
  __device__ __forceinline__ static int off(int o, int k) { return KFast ? o * LDK + k : k * LDM + o; }
};

// C[M][N] = A[M][K] . B[K][N] over the K range of blockIdx.z.  Mlim / Klim
// (device, may be null) lower M / K below the launch's bounds.
template <class AV, class BV>
__global__ void __launch_bounds__(NT, 2) gemm_kernel(AV A, BV B, int M, int N, int K, int kchunk, float* C, int ldc,
                                                  Epi e, const int* Mlim, const int* Klim) {
  constexpr bool kAK = AV::kColFast;   // A contiguous along k
  constexpr bool kBK = !BV::kColFast;  // B contiguous along k
  using MA = TileMap<kAK>;
  using MB = TileMap<kBK>;
  __shared__ __align__(16) __nv_bfloat16 As[2][kTileHalfs];
  __shared__ __align__(16) __nv_bfloat16 Bs[2][kTileHalfs];
  if (Mlim) M = min(M, *Mlim);
  if (Klim) K = min(K, *Klim);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp >> 2, wn = warp & 3, g = lane >> 2, t4 = lane & 3;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kb = blockIdx.z * kchunk;
  const int ke = min(K, kb + kchunk);
  if (m0 >= M || (e.atomic && kb >= ke)) return;  // block-uniform
  float acc[4][4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int x = 0; x < 4; ++x) acc[i][j][x] = 0.f;

  float4 ra[4], rb[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int o, k;
      MA::pos(tid + q * NT, o, k);
      ra[q] = (m0 + o < M && k0 + k < ke) ? A.vec4(m0 + o, k0 + k) : make_float4(0.f, 0.f, 0.f, 0.f);
      MB::pos(tid + q * NT, o, k);
      rb[q] = (n0 + o < N && k0 + k < ke) ? B.vec4(k0 + k, n0 + o) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto stage = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      int o, k;
      MA::pos(tid + q * NT, o, k);
      *reinterpret_cast<uint2*>(&As[buf][MA::off(o, k)]) = pack4_bf16(ra[q]);
      MB::pos(tid + q * NT, o, k);
      *reinterpret_cast<uint2*>(&Bs[buf][MB::off(o, k)]) = pack4_bf16(rb[q]);
    }
  };
  load(kb);
  stage(0);
  __syncthreads();
  int buf = 0;
  const int q8 = lane >> 3, r8 = lane & 7;
  for (int k0 = kb; k0 < ke; k0 += BK) {
    const bool more = k0 + BK < ke;
    if (more) load(k0 + BK);
#pragma unroll
    for (int ks = 0; ks < 2; ++ks) {
      uint32_t af[4][4], bfr[4][2];
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) {
        const int mb = wm * 64 + mi * 16;
        if (kAK)
          ldsm_x4(&As[buf][MA::off(mb + (lane & 15), ks * 16 + (lane >> 4) * 8)], af[mi][0], af[mi][1], af[mi][2],
                  af[mi][3]);
        else
          ldsm_x4_t(&As[buf][MA::off(mb + ((q8 & 1) << 3), ks * 16 + r8 + ((q8 >> 1) << 3))], af[mi][0], af[mi][1],
                    af[mi][2], af[mi][3]);
      }
#pragma unroll
      for (int np = 0; np < 2; ++np) {
        const int nb = wn * 32 + np * 16;
        if (kBK)
          ldsm_x4(&Bs[buf][MB::off(nb + (lane >> 4) * 8 + r8, ks * 16 + ((lane >> 3) & 1) * 8)], bfr[2 * np][0],
                  bfr[2 * np][1], bfr[2 * np + 1][0], bfr[2 * np + 1][1]);
        else
          ldsm_x4_t(&Bs[buf][MB::off(nb + ((q8 >> 1) << 3), ks * 16 + r8 + ((q8 & 1) << 3))], bfr[2 * np][0],
                    bfr[2 * np][1], bfr[2 * np + 1][0], bfr[2 * np + 1][1]);
      }
#pragma unroll
      for (int mi = 0; mi < 4; ++mi)
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_bf16(acc[mi][ni], af[mi], bfr[ni][0], bfr[ni][1]);
    }
    if (more) stage(buf ^ 1);
    __syncthreads();
    buf ^= 1;
  }

#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int rr = 0; rr < 2; ++rr) {
      const int m = m0 + wm * 64 + mi * 16 + g + 8 * rr;
      if (m >= M) continue;
#pragma unroll
      for (int ni = 0; ni < 4; ++ni)
#pragma unroll
        for (int ee = 0; ee < 2; ++ee) {
          const int n = n0 + wn * 32 + ni * 8 + 2 * t4 + ee;
          if (n >= N) continue;
          float* dst = C + (size_t)m * ldc + n;
          float v = acc[mi][ni][2 * rr + ee];
          if (e.atomic) {
            atomicAdd(dst, v);
            continue;
          }
          if (e.bias) v += __ldg(e.bias + n);
          if (e.relu) v = fmaxf(v, 0.f);
          if (e.gate && !(__ldg(e.gate + (size_t)m * ldc + n) > 0.f)) v = 0.f;
          *dst = v;
        }
    }
}

// ---- the same products on the fifth-generation tensor cores, for operands
// that are both contiguous along K (the forward convolutions and the linear
// layer).  One CTA of 256 threads computes a 128 x 128 output tile into a
// 128-column tensor-memory accumulator.  K advances 32 at a time through two
// shared stages in the canonical K-major layout (8-row x 16-byte core
// matrices, no swizzle): each thread loads its four 16-byte vectors of each
// operand for the next stage while the tensor cores multiply the current
// one, and stores them (rounded to bf16) once the products that last read
// that stage have completed, which its mbarrier tells.  Thread 0 issues the
// two K = 16 products of a stage and commits them to the stage's barrier.
// Epilogue: warp w reads tensor-memory lanes 32 (w % 4) .. 32 (w % 4) + 31
// (one output row per thread) and columns 64 (w / 4) .. + 63 with
// tcgen05.ld.  Every wait is bounded: on a timeout the CTA sets kErrWait,
// waits (bounded) for the products it issued, frees its tensor memory and
// writes nothing.
constexpr int kTcK = 32;
constexpr int kTcTileBytes = BM * kTcK * 2;  // one operand's stage: 8 KiB
constexpr uint32_t kTcIdesc = tc::idesc_bf16(BM, BN);
constexpr long long kTcWaitCycles = 2000000000ll;  // about a second

template <class AV, class BV>
__global__ void __launch_bounds__(NT, 4) gemm_tc_kernel(AV A, BV B, int M, int N, int K, float* C, int ldc, Epi e,
                                                     const int* Mlim) {
  static_assert(AV::kColFast && !BV::kColFast, "both operands contiguous along K");
  __shared__ __align__(1024) unsigned char sm[2][2][kTcTileBytes];  // [stage][A, B]
  __shared__ __align__(8) unsigned long long bars[2];
  __shared__ uint32_t tmem_base;
  __shared__ int rows_info[BM];  // the A view's table entries of the tile's rows, read once
  if (Mlim) M = min(M, *Mlim);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  if (m0 >= M) return;  // block-uniform, before any barrier or allocation
  const uint32_t bar0 = tc::smem_u32(&bars[0]), bar1 = tc::smem_u32(&bars[1]);
  if (tid == 0) {
    tc::mbar_init(bar0, 1);
    tc::mbar_init(bar1, 1);
    tc::mbar_init_fence();
  }
  if (warp == 0) tc::tmem_alloc(tc::smem_u32(&tmem_base), BN);
  if (tid < BM) rows_info[tid] = m0 + tid < M ? A.row_info(m0 + tid) : 0;
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tbase = tmem_base;
  int info[4];  // this thread's four A rows (fixed for the whole K loop)
#pragma unroll
  for (int q = 0; q < 4; ++q) info[q] = rows_info[(tid + q * NT) >> 3];

  float4 ra[4], rb[4];
  auto load = [&](int k0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int x = tid + q * NT, o = x >> 3, k = (x & 7) * 4;
      ra[q] = (m0 + o < M && k0 + k < K) ? A.vec4r(m0 + o, k0 + k, info[q]) : make_float4(0.f, 0.f, 0.f, 0.f);
      rb[q] = (n0 + o < N && k0 + k < K) ? B.vec4(k0 + k, n0 + o) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  auto stage = [&](int buf) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int x = tid + q * NT, o = x >> 3, k = (x & 7) * 4;
      const uint32_t off = tc::kmajor_offset((uint32_t)o, (uint32_t)k, kTcK);
      *reinterpret_cast<uint2*>(&sm[buf][0][off]) = pack4_bf16(ra[q]);
      *reinterpret_cast<uint2*>(&sm[buf][1][off]) = pack4_bf16(rb[q]);
    }
  };
  const int nk = (K + kTcK - 1) / kTcK;
  uint32_t parity = 0u;  // bit b: parity of stage b's barrier's next completion
  int last = -1;         // stage of the last committed products
  bool ok = true;
  load(0);
  for (int kt = 0; kt < nk; ++kt) {
    const int buf = kt & 1;
    if (kt >= 2) {  // the products of stage kt - 2 read this buffer
      const bool got = tc::mbar_wait(buf ? bar1 : bar0, (parity >> buf) & 1u, kTcWaitCycles);
      parity ^= 1u << buf;
      if (!__syncthreads_and(got)) {
        ok = false;
        break;
      }
    }
    stage(buf);
    tc::fence_proxy_async();  // the stores, for the tensor cores
    __syncthreads();
    if (tid == 0) {
      tc::fence_after();
      const uint32_t a = tc::smem_u32(&sm[buf][0][0]), b = tc::smem_u32(&sm[buf][1][0]);
#pragma unroll
      for (uint32_t ks = 0; ks < (uint32_t)(kTcK / 16); ++ks)
        tc::mma(tbase, tc::smem_desc(a + 256u * ks, 128u, 16u * kTcK, 0u),
                tc::smem_desc(b + 256u * ks, 128u, 16u * kTcK, 0u), kTcIdesc, (kt > 0 || ks > 0) ? 1u : 0u);
      tc::commit(buf ? bar1 : bar0);
    }
    last = buf;
    if (kt + 1 < nk) load((kt + 1) * kTcK);  // in flight while the products run
  }
  // every product issued has completed before the accumulator is read or freed
  // (the last commit covers all earlier products of thread 0)
  if (last >= 0) {
    const bool got = tc::mbar_wait(last ? bar1 : bar0, (parity >> last) & 1u, kTcWaitCycles);
    ok = __syncthreads_and(got && ok) != 0;
  }
  tc::fence_after();
  if (ok) {
    const int lq = warp & 3, half = warp >> 2;
    const int m = m0 + lq * 32 + lane;
    const uint32_t taddr = tbase + ((uint32_t)(lq * 32) << 16) + (uint32_t)(half * 64);
#pragma unroll
    for (int c = 0; c < 64; c += 32) {
      uint32_t v[32];
      tc::tmem_ld32(taddr + (uint32_t)c, v);
      tc::tmem_wait(v);
      if (m < M) {
        const int nb = n0 + half * 64 + c;
#pragma unroll
        for (int j = 0; j < 32; j += 4) {
          const int n = nb + j;
          if (n >= N) break;
          float4 r = make_float4(__uint_as_float(v[j]), __uint_as_float(v[j + 1]), __uint_as_float(v[j + 2]),
                                 __uint_as_float(v[j + 3]));
          if (e.bias) {
            r.x += __ldg(e.bias + n);
            r.y += __ldg(e.bias + min(n + 1, N - 1));
            r.z += __ldg(e.bias + min(n + 2, N - 1));
            r.w += __ldg(e.bias + min(n + 3, N - 1));
          }
          if (e.relu) {
            r.x = fmaxf(r.x, 0.f);
            r.y = fmaxf(r.y, 0.f);
            r.z = fmaxf(r.z, 0.f);
            r.w = fmaxf(r.w, 0.f);
          }
          if (e.gate) {
            const float* gp = e.gate + (size_t)m * ldc;
            if (!(__ldg(gp + n) > 0.f)) r.x = 0.f;
            if (!(__ldg(gp + min(n + 1, N - 1)) > 0.f)) r.y = 0.f;
            if (!(__ldg(gp + min(n + 2, N - 1)) > 0.f)) r.z = 0.f;
            if (!(__ldg(gp + min(n + 3, N - 1)) > 0.f)) r.w = 0.f;
          }
          float* dst = C + (size_t)m * ldc + n;
          if (n + 4 <= N) {
            *reinterpret_cast<float4*>(dst) = r;
          } else {  // N is a multiple of four: not reached, kept for safety
            dst[0] = r.x;
            if (n + 1 < N) dst[1] = r.y;
            if (n + 2 < N) dst[2] = r.z;
          }
        }
      }
    }
  } else if (tid == 0) {
    if (e.err) atomicOr(e.err, kErrWait);
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tbase, BN);
}

template <class AV, class BV>
cudaError_t run_gemm(AV A, BV B, int M, int N, int K, float* C, int ldc, const Epi& e, int splits, cudaStream_t s,
                     const int* Mlim = nullptr, const int* Klim = nullptr) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  // the operands are read in 16-byte vectors along their contiguous axes
  if ((AV::kColFast ? K : M) % 4 != 0 || (BV::kColFast ? N : K) % 4 != 0) return cudaErrorInvalidValue;
  const int gx = (N + BN - 1) / BN, gy = (M + BM - 1) / BM;
  int kchunk = K;
  int gz = 1;
  if (splits > 1 && K > BK) {
    kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + BK - 1) / BK * BK;
    gz = (K + kchunk - 1) / kchunk;
  }
  if (K <= 0) gz = 1;
  if constexpr (AV::kColFast && !BV::kColFast) {
    // both operands contiguous along K: the tcgen05 kernel, when nothing is split or accumulated
    if (gz == 1 && !e.atomic && !Klim && K > 0 && ldc % 4 == 0) {
      gemm_tc_kernel<AV, BV><<<dim3(gx, gy), NT, 0, s>>>(A, B, M, N, K, C, ldc, e, Mlim);
      return cudaGetLastError();
    }
  }
  gemm_kernel<AV, BV><<<dim3(gx, gy, gz), NT, 0, s>>>(A, B, M, N, K, kchunk, C, ldc, e, Mlim, Klim);
  return cudaGetLastError();
}

// split count giving about two waves of 128 x 128 tiles
int splits_for(int M, int N, int K, int nsm) {
  const int tiles = ((N + BN - 1) / BN) * ((M + BM - 1) / BM);
  int z = (2 * nsm + tiles - 1) / tiles;
  const int maxz = (K + 255) / 256;  // at least 256 of K per split
  return z < 1 ? 1 : (z > maxz ? (maxz < 1 ? 1 : maxz) : z);
}

// ---------------------------------------------------------------------------
// elementwise steps

__global__ void word_len_kernel(WordSrc src, int Bw, int* len, uint32_t* err) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= Bw) return;
  const uint32_t i = src.widx[w];
  if (i >= src.n) {
    atomicOr(err, kErrInput);
    len[w] = 0;
    return;
  }
  len[w] = __ldg(src.slen + __ldg(src.rank + i));
}

constexpr int kScanThreads = 1024;

// off = exclusive prefix sum of len (one block), T = the total (at most Tmax)
__global__ void __launch_bounds__(kScanThreads) scan_kernel(const int* len, int Bw, int* off, int* T, int Tmax,
                                                            uint32_t* err) {
  __shared__ int warp_sum[kScanThreads / 32];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (Bw + kScanThreads - 1) / kScanThreads;
  const int w0 = min(Bw, tid * per), w1 = min(Bw, w0 + per);
  int local = 0;
  for (int w = w0; w < w1; ++w) local += len[w];
  int incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_sum[warp] = incl;
  __syncthreads();
  if (warp == 0) {
    int ws = warp_sum[lane];
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, ws, o);
      if (lane >= o) ws += t;
    }
    warp_sum[lane] = ws;  // inclusive over warps
  }
  __syncthreads();
  int run = incl - local + (warp ? warp_sum[warp - 1] : 0);
  for (int w = w0; w < w1; ++w) {
    off[w] = run;
    run += len[w];
  }
  if (tid == kScanThreads - 1) {
    const int total = warp_sum[kScanThreads / 32 - 1];
    if (total > Tmax) atomicOr(err, kErrInput);
    *T = min(total, Tmax);
  }
}

// per-row tables: thread per word (rows past Tmax are dropped)
__global__ void fill_rows_kernel(const int* len, const int* off, int Bw, int Tmax, int* rinfo, int* rword) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= Bw) return;
  const int L = len[w], o = off[w];
  for (int t = 0; t < L && o + t < Tmax; ++t) {
    rinfo[o + t] = (t << 8) | L;
    rword[o + t] = w;
  }
}

// one warp per packed row: lane = embedding channel
__global__ void gather_kernel(WordSrc src, const int* Tdev, int Tmax, const float* __restrict__ emb, const int* rinfo,
                              const int* rword, int32_t* codes, float* X0, uint32_t* err, uint32_t alphabet) {
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= min(Tmax, *Tdev)) return;
  const int w = rword[row], t = rinfo[row] >> 8;
  const uint32_t pos = __ldg(src.rank + src.widx[w]);
  const uint32_t v = __ldg(src.a_enc + __ldg(src.aoff + pos) + t);
  int code = (int)((v & 0xffffu) >> src.shift);
  if ((uint32_t)code >= alphabet) {
    if (lane == 0) atomicOr(err, kErrInput);
    code = -1;
  }
  if (lane == 0) codes[row] = code;
  X0[(size_t)row * kEmb + lane] = code >= 0 ? __ldg(emb + (size_t)code * kEmb + lane) : 0.f;
}

// P[w] = mean of word w's rows (0 for an empty word)
__global__ void pool_kernel(const float* __restrict__ Y, const int* len, const int* off, int Bw, int Tmax, float* P) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= Bw * kCh) return;
  const int w = x / kCh, ch = x - w * kCh;
  const int o = off[w];
  const int L = min(len[w], max(0, Tmax - o));  // rows past Tmax were never filled (an error already raised)
  float acc = 0.f;
  for (int t = 0; t < L; ++t) acc += Y[((size_t)o + t) * kCh + ch];
  P[x] = L > 0 ? acc / (float)L : 0.f;
}

__global__ void pool_bwd_kernel(const float* __restrict__ dP, const float* __restrict__ Y, const int* len,
                                const int* rword, const int* Tdev, int Tmax, float* dY) {
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (size_t)min(Tmax, *Tdev) * kCh) return;
  const int row = (int)(x / kCh), ch = (int)(x - (size_t)row * kCh);
  const int w = rword[row];
  dY[x] = Y[x] > 0.f ? dP[(size_t)w * kCh + ch] / (float)len[w] : 0.f;
}

// one warp per pair: lanes hold dimensions lane and lane + 32.  The 64
// outputs are 63 features and a bias (the last): pred = phi_a . phi_b + beta_a + beta_b
__global__ void pair_loss_kernel(const float* __restrict__ E, const float* __restrict__ target, int m, float* dE,
                                 float* loss_acc) {
  const int p = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (p >= m) return;
  const float* a = E + (size_t)(2 * p) * kOut;
  const float* b = E + (size_t)(2 * p + 1) * kOut;
  const float a0 = a[lane], a1 = a[lane + 32], b0 = b[lane], b1 = b[lane + 32];
  const bool bias_lane = lane == 31;  // holds output 63 as its second value
  float d = a0 * b0 + (bias_lane ? a1 + b1 : a1 * b1);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  const float diff = d - target[p];
  const float g = 2.f * diff / (float)m;
  float* da = dE + (size_t)(2 * p) * kOut;
  float* db = dE + (size_t)(2 * p + 1) * kOut;
  da[lane] = g * b0;
  da[lane + 32] = bias_lane ? g : g * b1;
  db[lane] = g * a0;
  db[lane + 32] = bias_lane ? g : g * a1;
  if (lane == 0 && loss_acc) atomicAdd(loss_acc, diff * diff / (float)m);
}

constexpr int kColSumRows = 256;

__global__ void col_sum_kernel(const float* __restrict__ Y, int rows, const int* rows_dev, int cols, float* out) {
  const int c = threadIdx.x;
  if (rows_dev) rows = min(rows, *rows_dev);
  const int r0 = blockIdx.x * kColSumRows;
  const int r1 = min(rows, r0 + kColSumRows);
  if (c >= cols || r0 >= r1) return;
  float acc = 0.f;
  for (int r = r0; r < r1; ++r) acc += Y[(size_t)r * cols + c];
  atomicAdd(out + c, acc);
}

__global__ void emb_scatter_kernel(const float* __restrict__ dX0, const int32_t* codes, const int* Tdev, int Tmax,
                                   float* demb) {
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (size_t)min(Tmax, *Tdev) * kEmb) return;
  const int row = (int)(x / kEmb), ch = (int)(x - (size_t)row * kEmb);
  const int code = codes[row];
  if (code >= 0) atomicAdd(demb + (size_t)code * kEmb + ch, dX0[x]);
}

// Adam with bias correction; the gradient is scaled by min(1, clip / |g|)
// when clip > 0 (|g|^2 in *sumsq), and the rate falls linearly from lr to
// lr_final over the steps [step0, step0 + nsteps).
__global__ void adam_kernel(float* theta, const float* __restrict__ g, float* m, float* v, uint64_t n,
                            const uint32_t* step, AdamCfg c) {
  const uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  const uint32_t st = *step;
  const float t = (float)st;
  const float frac = c.nsteps ? fminf(1.f, (float)(st - 1u - c.step0) / (float)c.nsteps) : 0.f;
  const float lr = c.lr + (c.lr_final - c.lr) * frac;
  const float b1 = c.b1, b2 = c.b2, eps = c.eps;
  float gscale = 1.f;
  if (c.clip > 0.f) {
    const float norm = sqrtf(*c.sumsq);
    if (norm > c.clip) gscale = c.clip / norm;
  }
  const float gx = g[x] * gscale;
  const float mx = b1 * m[x] + (1.f - b1) * gx;
  const float vx = b2 * v[x] + (1.f - b2) * gx * gx;
  m[x] = mx;
  v[x] = vx;
  const float mhat = mx / (1.f - powf(b1, t));
  const float vhat = vx / (1.f - powf(b2, t));
  theta[x] -= lr * mhat / (sqrtf(vhat) + eps);
}

__global__ void bump_kernel(uint32_t* step) { *step += 1u; }

__global__ void sumsq_kernel(const float* __restrict__ g, uint64_t n, float* out) {
  float acc = 0.f;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += (uint64_t)gridDim.x * blockDim.x)
    acc += g[x] * g[x];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, acc);
}

__global__ void record_loss_kernel(float* cur, float* losses, const uint32_t* step, uint32_t step0,
                                   uint32_t nsteps) {
  const uint32_t x = *step - 1u - step0;
  if (x < nsteps) losses[x] = *cur;
  *cur = 0.f;
}

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

__global__ void draw_pairs_kernel(PairDraw d, uint32_t* pi, uint32_t* pj, uint32_t* widx) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= d.m) return;
  const uint64_t ctr = ((uint64_t)*d.step << 32) | p;
  const uint64_t u1 = splitmix64(d.seed ^ splitmix64(2 * ctr));
  const uint64_t u2 = splitmix64(d.seed ^ splitmix64(2 * ctr + 1));
  uint32_t i = (uint32_t)(u1 % d.n);
  if (d.nlong && (uint32_t)((u2 >> 44) & 0xfffffu) < d.long_thresh)
    i = __ldg(d.perm + d.long0 + (uint32_t)((u1 >> 1) % d.nlong));
  uint32_t j = 0xffffffffu;
  if (d.nbr && p < d.n_nbr && d.knb) {
    j = __ldg(d.nbr + (size_t)i * d.knb + (uint32_t)(u2 % d.knb));
    if (j >= d.n || j == i) j = 0xffffffffu;
  }
  if (j == 0xffffffffu) j = (uint32_t)((i + 1u + (uint32_t)((u2 >> 20) % (uint64_t)(d.n - 1))) % d.n);
  pi[p] = i;
  pj[p] = j;
  widx[2 * p] = i;
  widx[2 * p + 1] = j;
}

__global__ void targets_kernel(const int16_t* score, const uint32_t* pi, const uint32_t* pj, const uint32_t* rank,
                               const uint8_t* slen, int m, float raw_scale, float* target) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m) return;
  if (raw_scale > 0.f) {
    target[p] = (float)score[p] * raw_scale;
    return;
  }
  int L = max((int)slen[rank[pi[p]]], (int)slen[rank[pj[p]]]);
  L = L > 0 ? L : 1;
  target[p] = (float)score[p] / (float)L;
}

__global__ void interleave_kernel(const uint32_t* pi, const uint32_t* pj, int m, uint32_t* widx) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m) return;
  widx[2 * p] = pi[p];
  widx[2 * p + 1] = pj[p];
}

__global__ void take_kernel(const uint32_t* src, uint32_t base, int count, uint32_t* out) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x < count) out[x] = src[base + (uint32_t)x];
}

__global__ void scatter_rows_kernel(const float* __restrict__ E, const uint32_t* widx, int Bw, float* dst) {
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (size_t)Bw * kOut) return;
  const size_t w = x / kOut;
  dst[(size_t)widx[w] * kOut + (x - w * kOut)] = E[x];
}

inline unsigned blocks_for(size_t n, unsigned b) { return (unsigned)((n + b - 1) / b); }

// log2 of a channel count (32 or 128: the views index taps by shifts)
inline int log2_ch(int c) {
  int l = 0;
  while ((1 << l) < c) ++l;
  return l;
}

}  // namespace

cudaError_t conv_fwd(const float* X, int Ci, const float* W, int Co, const Packed& pk, float* Y, const Epi& e,
                     cudaStream_t s) {
  return run_gemm(Im2col{X, pk.rinfo, log2_ch(Ci)}, DenseT{W, 3 * Ci}, pk.Tmax, Co, 3 * Ci, Y, Co, e, 1, s, pk.T);
}

cudaError_t conv_dw(const float* dY, int Co, const float* X, int Ci, const Packed& pk, float* dW, int nsm,
                    cudaStream_t s) {
  Epi e;
  e.atomic = true;
  return run_gemm(DenseT{dY, Co}, Im2col{X, pk.rinfo, log2_ch(Ci)}, Co, 3 * Ci, pk.Tmax, dW, 3 * Ci, e,
                  splits_for(Co, 3 * Ci, pk.Tmax, nsm), s, nullptr, pk.T);
}

cudaError_t conv_dx(const float* dY, int Co, const float* W, int Ci, const Packed& pk, float* dX, const Epi& e,
                    cudaStream_t s) {
  return run_gemm(Shift{dY, pk.rinfo, log2_ch(Co)}, WTap{W, log2_ch(Co), Ci}, pk.Tmax, Ci, 3 * Co, dX, Ci, e, 1, s,
                  pk.T);
}

cudaError_t lin_fwd(const float* P, int Ci, const float* Wl, int Co, int B, float* E, const Epi& e, cudaStream_t s) {
  return run_gemm(Dense{P, Ci}, DenseT{Wl, Ci}, B, Co, Ci, E, Co, e, 1, s);
}

cudaError_t lin_dw(const float* dE, int Co, const float* P, int Ci, int B, float* dWl, int nsm, cudaStream_t s) {
  Epi e;
  e.atomic = true;
  return run_gemm(DenseT{dE, Co}, Dense{P, Ci}, Co, Ci, B, dWl, Ci, e, splits_for(Co, Ci, B, nsm), s);
}

cudaError_t lin_dx(const float* dE, int Co, const float* Wl, int Ci, int B, float* dP, cudaStream_t s) {
  return run_gemm(Dense{dE, Co}, Dense{Wl, Ci}, B, Ci, Co, dP, Ci, Epi{}, 1, s);
}

cudaError_t pack_words(const WordSrc& src, int Bw, int Tmax, const float* emb, const PackBufs& b, float* X0,
                       uint32_t* err, uint32_t alphabet, cudaStream_t s) {
  if (Bw <= 0) return cudaMemsetAsync(b.T, 0, sizeof(int), s);
  word_len_kernel<<<blocks_for(Bw, 256), 256, 0, s>>>(src, Bw, b.len, err);
  scan_kernel<<<1, kScanThreads, 0, s>>>(b.len, Bw, b.off, b.T, Tmax, err);
  fill_rows_kernel<<<blocks_for(Bw, 256), 256, 0, s>>>(b.len, b.off, Bw, Tmax, b.rinfo, b.rword);
  gather_kernel<<<blocks_for((size_t)Tmax, 8), 256, 0, s>>>(src, b.T, Tmax, emb, b.rinfo, b.rword, b.codes, X0, err,
                                                             alphabet);
  return cudaGetLastError();
}

cudaError_t mean_pool(const float* Y, const Packed& pk, float* P, cudaStream_t s) {
  if (pk.Bw <= 0) return cudaSuccess;
  pool_kernel<<<blocks_for((size_t)pk.Bw * kCh, 256), 256, 0, s>>>(Y, pk.len, pk.off, pk.Bw, pk.Tmax, P);
  return cudaGetLastError();
}

cudaError_t mean_pool_bwd(const float* dP, const float* Y, const Packed& pk, float* dY, cudaStream_t s) {
  if (pk.Tmax <= 0) return cudaSuccess;
  pool_bwd_kernel<<<blocks_for((size_t)pk.Tmax * kCh, 256), 256, 0, s>>>(dP, Y, pk.len, pk.rword, pk.T, pk.Tmax, dY);
  return cudaGetLastError();
}

cudaError_t pair_loss(const float* E, const float* target, int m, float* dE, float* loss_acc, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  pair_loss_kernel<<<blocks_for(m, 8), 256, 0, s>>>(E, target, m, dE, loss_acc);
  return cudaGetLastError();
}

cudaError_t col_sum(const float* Y, int rows, const int* rows_dev, int cols, float* out, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  col_sum_kernel<<<blocks_for(rows, kColSumRows), cols <= 64 ? 64 : 128, 0, s>>>(Y, rows, rows_dev, cols, out);
  return cudaGetLastError();
}

cudaError_t emb_scatter(const float* dX0, const int32_t* codes, const Packed& pk, float* demb, cudaStream_t s) {
  if (pk.Tmax <= 0) return cudaSuccess;
  emb_scatter_kernel<<<blocks_for((size_t)pk.Tmax * kEmb, 256), 256, 0, s>>>(dX0, codes, pk.T, pk.Tmax, demb);
  return cudaGetLastError();
}

cudaError_t adam(float* theta, const float* g, float* m, float* v, uint64_t n, const uint32_t* step,
                 const AdamCfg& c, cudaStream_t s) {
  if (c.clip > 0.f) {
    cudaError_t e = cudaMemsetAsync(c.sumsq, 0, sizeof(float), s);
    if (e != cudaSuccess) return e;
    sumsq_kernel<<<256, 256, 0, s>>>(g, n, c.sumsq);
  }
  adam_kernel<<<blocks_for(n, 256), 256, 0, s>>>(theta, g, m, v, n, step, c);
  return cudaGetLastError();
}

cudaError_t bump_step(uint32_t* step, cudaStream_t s) {
  bump_kernel<<<1, 1, 0, s>>>(step);
  return cudaGetLastError();
}

cudaError_t record_loss(float* cur, float* losses, const uint32_t* step, uint32_t step0, uint32_t nsteps,
                        cudaStream_t s) {
  record_loss_kernel<<<1, 1, 0, s>>>(cur, losses, step, step0, nsteps);
  return cudaGetLastError();
}

cudaError_t draw_pairs(const PairDraw& d, uint32_t* pi, uint32_t* pj, uint32_t* widx, cudaStream_t s) {
  if (d.m == 0) return cudaSuccess;
  draw_pairs_kernel<<<blocks_for(d.m, 256), 256, 0, s>>>(d, pi, pj, widx);
  return cudaGetLastError();
}

cudaError_t pair_targets(const int16_t* score, const uint32_t* pi, const uint32_t* pj, const uint32_t* rank,
                         const uint8_t* slen, int m, float raw_scale, float* target, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  targets_kernel<<<blocks_for(m, 256), 256, 0, s>>>(score, pi, pj, rank, slen, m, raw_scale, target);
  return cudaGetLastError();
}

cudaError_t interleave_pairs(const uint32_t* pi, const uint32_t* pj, int m, uint32_t* widx, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  interleave_kernel<<<blocks_for(m, 256), 256, 0, s>>>(pi, pj, m, widx);
  return cudaGetLastError();
}

cudaError_t take(const uint32_t* src, uint32_t base, int count, uint32_t* out, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  take_kernel<<<blocks_for(count, 256), 256, 0, s>>>(src, base, count, out);
  return cudaGetLastError();
}

cudaError_t scatter_rows(const float* E, const uint32_t* widx, int Bw, float* dst, cudaStream_t s) {
  if (Bw <= 0) return cudaSuccess;
  scatter_rows_kernel<<<blocks_for((size_t)Bw * kOut, 256), 256, 0, s>>>(E, widx, Bw, dst);
  return cudaGetLastError();
}

}  // namespace cnn
}  // namespace nw
