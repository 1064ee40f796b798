// nw_cnn.cu -- kernels of the proposal network: tiled float32 matrix products
// whose operand loaders gather convolution windows directly from the padded
// activations (no im2col buffer), and the elementwise steps around them.
#include <cuda_runtime.h>
#include <stdint.h>

#include "nw_cnn.h"
#include "nw_internal.cuh"

namespace nw {
namespace cnn {
namespace {

// ---------------------------------------------------------------------------
// operand views: element (r, c) of a logical matrix.  kColFast: consecutive
// c are adjacent in memory (the tile loader then walks c fastest).

struct Dense {  // row-major
  const float* p;
  int ld;
  static constexpr bool kColFast = true;
  __device__ __forceinline__ float at(int r, int c) const { return __ldg(p + (size_t)r * ld + c); }
};

struct DenseT {  // transpose of a row-major matrix
  const float* p;
  int ld;
  static constexpr bool kColFast = false;
  __device__ __forceinline__ float at(int r, int c) const { return __ldg(p + (size_t)c * ld + r); }
};

// im2col of padded X[T][Ci]: (t, tap * Ci + ch) = X[t + tap - 1][ch] within t's word block
struct Im2col {
  const float* X;
  int Ci, Lp;
  static constexpr bool kColFast = true;
  __device__ __forceinline__ float at(int t, int k) const {
    const int tap = k / Ci, ch = k - tap * Ci;
    const int pos = t % Lp + tap - 1;
    if (pos < 0 || pos >= Lp) return 0.f;
    return __ldg(X + (size_t)(t + tap - 1) * Ci + ch);
  }
};

// shifted output gradient: (t, tap * Co + o) = dY[t - tap + 1][o] within t's word block
struct Shift {
  const float* dY;
  int Co, Lp;
  static constexpr bool kColFast = true;
  __device__ __forceinline__ float at(int t, int k) const {
    const int tap = k / Co, o = k - tap * Co;
    const int pos = t % Lp - tap + 1;
    if (pos < 0 || pos >= Lp) return 0.f;
    return __ldg(dY + (size_t)(t - tap + 1) * Co + o);
  }
};

// W[Co][3][Ci] read as the (tap * Co + o, ch) matrix of the input gradient
struct WTap {
  const float* W;
  int Co, Ci;
  static constexpr bool kColFast = true;
  __device__ __forceinline__ float at(int k, int ch) const {
    const int tap = k / Co, o = k - tap * Co;
    return __ldg(W + ((size_t)o * 3 + tap) * Ci + ch);
  }
};

constexpr int BM = 128, BN = 128, BK = 8, NT = 256;

// C[M][N] = A[M][K] . B[K][N] over the K range of blockIdx.z: 128 x 128 tiles,
// 8 x 8 outputs per thread (two 4 x 4 blocks 64 apart in each direction).
template <class AV, class BV>
__global__ void __launch_bounds__(NT) gemm_kernel(AV A, BV B, int M, int N, int K, int kchunk, float* C, int ldc,
                                                  Epi e) {
  __shared__ __align__(16) float As[BK][BM];
  __shared__ __align__(16) float Bs[BK][BN];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kb = blockIdx.z * kchunk;
  const int ke = min(K, kb + kchunk);
  float acc[8][8];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;

  for (int k0 = kb; k0 < ke; k0 += BK) {
#pragma unroll
    for (int q = 0; q < (BM * BK) / NT; ++q) {
      const int x = tid + q * NT;
      int mm, kk;
      if constexpr (AV::kColFast) { mm = x / BK; kk = x % BK; } else { kk = x / BM; mm = x % BM; }
      const int gm = m0 + mm, gk = k0 + kk;
      As[kk][mm] = (gm < M && gk < ke) ? A.at(gm, gk) : 0.f;
    }
#pragma unroll
    for (int q = 0; q < (BN * BK) / NT; ++q) {
      const int x = tid + q * NT;
      int kk, nn;
      if constexpr (BV::kColFast) { kk = x / BN; nn = x % BN; } else { nn = x / BK; kk = x % BK; }
      const int gk = k0 + kk, gn = n0 + nn;
      Bs[kk][nn] = (gk < ke && gn < N) ? B.at(gk, gn) : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(&As[kk][ty * 4]);
      const float4 a1 = *reinterpret_cast<const float4*>(&As[kk][ty * 4 + 64]);
      const float4 b0 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4]);
      const float4 b1 = *reinterpret_cast<const float4*>(&Bs[kk][tx * 4 + 64]);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }

#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int m = m0 + ty * 4 + (i & 3) + (i >> 2) * 64;
    if (m >= M) continue;
    const bool rowok = !e.rowlen || (m % e.Lp) < __ldg(e.rowlen + m / e.Lp);
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int n = n0 + tx * 4 + (j & 3) + (j >> 2) * 64;
      if (n >= N) continue;
      float* dst = C + (size_t)m * ldc + n;
      float v = acc[i][j];
      if (e.atomic) {
        atomicAdd(dst, v);
        continue;
      }
      if (e.bias) v += __ldg(e.bias + n);
      if (e.relu) v = fmaxf(v, 0.f);
      if (e.gate && !(__ldg(e.gate + (size_t)m * ldc + n) > 0.f)) v = 0.f;
      if (!rowok) v = 0.f;
      *dst = v;
    }
  }
}

template <class AV, class BV>
cudaError_t run_gemm(AV A, BV B, int M, int N, int K, float* C, int ldc, const Epi& e, int splits, cudaStream_t s) {
  if (M <= 0 || N <= 0) return cudaSuccess;
  const int gx = (N + BN - 1) / BN, gy = (M + BM - 1) / BM;
  int kchunk = K;
  int gz = 1;
  if (splits > 1 && K > BK) {
    kchunk = (K + splits - 1) / splits;
    kchunk = (kchunk + BK - 1) / BK * BK;
    gz = (K + kchunk - 1) / kchunk;
  }
  if (K <= 0) gz = 1;
  gemm_kernel<AV, BV><<<dim3(gx, gy, gz), NT, 0, s>>>(A, B, M, N, K, kchunk, C, ldc, e);
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

__global__ void word_len_kernel(WordSrc src, int Bw, int* rowlen, uint32_t* err) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= Bw) return;
  const uint32_t i = src.widx[w];
  if (i >= src.n) {
    atomicOr(err, kErrInput);
    rowlen[w] = 0;
    return;
  }
  rowlen[w] = __ldg(src.slen + __ldg(src.rank + i));
}

// one warp per padded position: lane = embedding channel
__global__ void gather_kernel(WordSrc src, int Bw, int Lp, const float* __restrict__ emb, const int* rowlen,
                              int32_t* codes, float* X0, uint32_t* err, uint32_t alphabet) {
  const int row = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (row >= Bw * Lp) return;
  const int w = row / Lp, t = row - w * Lp;
  int code = -1;
  if (t < rowlen[w]) {
    const uint32_t pos = __ldg(src.rank + src.widx[w]);
    const uint32_t v = __ldg(src.a_enc + __ldg(src.aoff + pos) + t);
    code = (int)((v & 0xffffu) >> src.shift);
    if ((uint32_t)code >= alphabet) {
      if (lane == 0) atomicOr(err, kErrInput);
      code = -1;
    }
  }
  if (lane == 0) codes[row] = code;
  X0[(size_t)row * kEmb + lane] = code >= 0 ? __ldg(emb + (size_t)code * kEmb + lane) : 0.f;
}

__global__ void pool_kernel(const float* __restrict__ Y, const int* rowlen, int Bw, int Lp, float* P) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= Bw * kCh) return;
  const int w = x / kCh, ch = x - w * kCh;
  const int L = rowlen[w];
  float acc = 0.f;
  for (int t = 0; t < L; ++t) acc += Y[((size_t)w * Lp + t) * kCh + ch];
  P[x] = L > 0 ? acc / (float)L : 0.f;
}

__global__ void pool_bwd_kernel(const float* __restrict__ dP, const float* __restrict__ Y, const int* rowlen,
                                int Bw, int Lp, float* dY) {
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (size_t)Bw * Lp * kCh) return;
  const int row = (int)(x / kCh), ch = (int)(x - (size_t)row * kCh);
  const int w = row / Lp, t = row - w * Lp;
  const int L = rowlen[w];
  dY[x] = (t < L && Y[x] > 0.f) ? dP[(size_t)w * kCh + ch] / (float)L : 0.f;
}

// one warp per pair: lanes hold dimensions lane and lane + 32
__global__ void pair_loss_kernel(const float* __restrict__ E, const float* __restrict__ target, int m, float* dE,
                                 float* loss_acc) {
  const int p = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (p >= m) return;
  const float* a = E + (size_t)(2 * p) * kOut;
  const float* b = E + (size_t)(2 * p + 1) * kOut;
  const float a0 = a[lane], a1 = a[lane + 32], b0 = b[lane], b1 = b[lane + 32];
  float d = a0 * b0 + a1 * b1;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
  const float diff = d - target[p];
  const float g = 2.f * diff / (float)m;
  float* da = dE + (size_t)(2 * p) * kOut;
  float* db = dE + (size_t)(2 * p + 1) * kOut;
  da[lane] = g * b0;
  da[lane + 32] = g * b1;
  db[lane] = g * a0;
  db[lane + 32] = g * a1;
  if (lane == 0 && loss_acc) atomicAdd(loss_acc, diff * diff / (float)m);
}

constexpr int kColSumRows = 256;

__global__ void col_sum_kernel(const float* __restrict__ Y, int rows, int cols, float* out) {
  const int c = threadIdx.x;
  const int r0 = blockIdx.x * kColSumRows;
  const int r1 = min(rows, r0 + kColSumRows);
  if (c >= cols) return;
  float acc = 0.f;
  for (int r = r0; r < r1; ++r) acc += Y[(size_t)r * cols + c];
  atomicAdd(out + c, acc);
}

__global__ void emb_scatter_kernel(const float* __restrict__ dX0, const int32_t* codes, int T, float* demb) {
  const size_t x = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= (size_t)T * kEmb) return;
  const int row = (int)(x / kEmb), ch = (int)(x - (size_t)row * kEmb);
  const int code = codes[row];
  if (code >= 0) atomicAdd(demb + (size_t)code * kEmb + ch, dX0[x]);
}

__global__ void adam_kernel(float* theta, const float* __restrict__ g, float* m, float* v, uint64_t n,
                            const uint32_t* step, float lr, float b1, float b2, float eps) {
  const uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= n) return;
  const float t = (float)*step;
  const float gx = g[x];
  const float mx = b1 * m[x] + (1.f - b1) * gx;
  const float vx = b2 * v[x] + (1.f - b2) * gx * gx;
  m[x] = mx;
  v[x] = vx;
  const float mhat = mx / (1.f - powf(b1, t));
  const float vhat = vx / (1.f - powf(b2, t));
  theta[x] -= lr * mhat / (sqrtf(vhat) + eps);
}

__global__ void bump_kernel(uint32_t* step) { *step += 1u; }

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
  const uint32_t i = (uint32_t)(u1 % d.n);
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
                               const uint8_t* slen, int m, float* target) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= m) return;
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

__global__ void iota_kernel(uint32_t* out, uint32_t base, int count) {
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x < count) out[x] = base + (uint32_t)x;
}

inline unsigned blocks_for(size_t n, unsigned b) { return (unsigned)((n + b - 1) / b); }

}  // namespace

cudaError_t conv_fwd(const float* X, int Ci, const float* W, int Co, int T, int Lp, float* Y, const Epi& e,
                     cudaStream_t s) {
  return run_gemm(Im2col{X, Ci, Lp}, DenseT{W, 3 * Ci}, T, Co, 3 * Ci, Y, Co, e, 1, s);
}

cudaError_t conv_dw(const float* dY, int Co, const float* X, int Ci, int T, int Lp, float* dW, int nsm,
                    cudaStream_t s) {
  Epi e;
  e.atomic = true;
  return run_gemm(DenseT{dY, Co}, Im2col{X, Ci, Lp}, Co, 3 * Ci, T, dW, 3 * Ci, e, splits_for(Co, 3 * Ci, T, nsm),
                  s);
}

cudaError_t conv_dx(const float* dY, int Co, const float* W, int Ci, int T, int Lp, float* dX, const Epi& e,
                    cudaStream_t s) {
  return run_gemm(Shift{dY, Co, Lp}, WTap{W, Co, Ci}, T, Ci, 3 * Co, dX, Ci, e, 1, s);
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

cudaError_t gather_words(const WordSrc& src, int Bw, int Lp, const float* emb, int* rowlen, int32_t* codes,
                         float* X0, uint32_t* err, uint32_t alphabet, cudaStream_t s) {
  if (Bw <= 0) return cudaSuccess;
  word_len_kernel<<<blocks_for(Bw, 256), 256, 0, s>>>(src, Bw, rowlen, err);
  gather_kernel<<<blocks_for((size_t)Bw * Lp, 8), 256, 0, s>>>(src, Bw, Lp, emb, rowlen, codes, X0, err, alphabet);
  return cudaGetLastError();
}

cudaError_t mean_pool(const float* Y, const int* rowlen, int Bw, int Lp, float* P, cudaStream_t s) {
  if (Bw <= 0) return cudaSuccess;
  pool_kernel<<<blocks_for((size_t)Bw * kCh, 256), 256, 0, s>>>(Y, rowlen, Bw, Lp, P);
  return cudaGetLastError();
}

cudaError_t mean_pool_bwd(const float* dP, const float* Y, const int* rowlen, int Bw, int Lp, float* dY,
                          cudaStream_t s) {
  if (Bw <= 0) return cudaSuccess;
  pool_bwd_kernel<<<blocks_for((size_t)Bw * Lp * kCh, 256), 256, 0, s>>>(dP, Y, rowlen, Bw, Lp, dY);
  return cudaGetLastError();
}

cudaError_t pair_loss(const float* E, const float* target, int m, float* dE, float* loss_acc, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  pair_loss_kernel<<<blocks_for(m, 8), 256, 0, s>>>(E, target, m, dE, loss_acc);
  return cudaGetLastError();
}

cudaError_t col_sum(const float* Y, int rows, int cols, float* out, cudaStream_t s) {
  if (rows <= 0) return cudaSuccess;
  col_sum_kernel<<<blocks_for(rows, kColSumRows), cols <= 64 ? 64 : 128, 0, s>>>(Y, rows, cols, out);
  return cudaGetLastError();
}

cudaError_t emb_scatter(const float* dX0, const int32_t* codes, int T, float* demb, cudaStream_t s) {
  if (T <= 0) return cudaSuccess;
  emb_scatter_kernel<<<blocks_for((size_t)T * kEmb, 256), 256, 0, s>>>(dX0, codes, T, demb);
  return cudaGetLastError();
}

cudaError_t adam(float* theta, const float* g, float* m, float* v, uint64_t n, const uint32_t* step, float lr,
                 float b1, float b2, float eps, cudaStream_t s) {
  adam_kernel<<<blocks_for(n, 256), 256, 0, s>>>(theta, g, m, v, n, step, lr, b1, b2, eps);
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
                         const uint8_t* slen, int m, float* target, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  targets_kernel<<<blocks_for(m, 256), 256, 0, s>>>(score, pi, pj, rank, slen, m, target);
  return cudaGetLastError();
}

cudaError_t interleave_pairs(const uint32_t* pi, const uint32_t* pj, int m, uint32_t* widx, cudaStream_t s) {
  if (m <= 0) return cudaSuccess;
  interleave_kernel<<<blocks_for(m, 256), 256, 0, s>>>(pi, pj, m, widx);
  return cudaGetLastError();
}

cudaError_t iota(uint32_t* out, uint32_t base, int count, cudaStream_t s) {
  if (count <= 0) return cudaSuccess;
  iota_kernel<<<blocks_for(count, 256), 256, 0, s>>>(out, base, count);
  return cudaGetLastError();
}

}  // namespace cnn
}  // namespace nw
