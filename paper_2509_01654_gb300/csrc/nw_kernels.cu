// nw_kernels.cu -- ingest (stable length bucketing and encoding), list
// finalisation and the integer-rate microbenchmarks.
#include <cuda_runtime.h>
#include <limits.h>
#include <stdint.h>

#include "nw_dp.cuh"
#include "nw_launch.h"

namespace nw {

// ---------------------------------------------------------------------------
// ingest.  Words arrive in CSR form (codes, offsets).  Sorting is a stable
// counting sort by length: per-block counts, a scan over blocks per length,
// then a scatter that ranks equal lengths inside a block warp by warp.

__global__ void ingest_count_kernel(const uint8_t* __restrict__ codes,
                                    const uint32_t* __restrict__ offsets, uint32_t n,
                                    uint32_t alphabet, uint32_t* __restrict__ block_counts,
                                    uint32_t* err) {
  __shared__ uint32_t cnt[kBuckets];
  for (int t = threadIdx.x; t < kBuckets; t += blockDim.x) cnt[t] = 0u;
  __syncthreads();
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const uint32_t o0 = offsets[i], o1 = offsets[i + 1];
    bool bad = (i == 0 && o0 != 0u) || o1 < o0 || o1 - o0 > (uint32_t)kMaxLen;
    if (!bad) {
      for (uint32_t s = o0; s < o1; ++s) bad |= codes[s] >= alphabet;
      atomicAdd(&cnt[o1 - o0], 1u);
    }
    if (bad) atomicOr(err, kErrInput);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < kBuckets; t += blockDim.x)
    block_counts[(size_t)blockIdx.x * kBuckets + t] = cnt[t];
}

__global__ void ingest_scan_kernel(uint32_t* __restrict__ block_counts, uint32_t nblk,
                                   uint32_t* __restrict__ bucket_count) {
  const int L = threadIdx.x;
  if (L >= kBuckets) return;
  uint32_t run = 0;
  for (uint32_t b = 0; b < nblk; ++b) {
    const uint32_t c = block_counts[(size_t)b * kBuckets + L];
    block_counts[(size_t)b * kBuckets + L] = run;
    run += c;
  }
  bucket_count[L] = run;
}

__global__ void ingest_scatter_kernel(const uint32_t* __restrict__ offsets, uint32_t n,
                                      const uint32_t* __restrict__ block_base, const Buckets bk,
                                      uint32_t* __restrict__ perm, uint32_t* __restrict__ rank,
                                      uint8_t* __restrict__ slen) {
  __shared__ uint32_t wcnt[kIngestBlock / 32][kBuckets];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < (int)(kIngestBlock / 32) * kBuckets; t += blockDim.x)
    (&wcnt[0][0])[t] = 0u;
  __syncthreads();
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  const uint32_t L = i < n ? offsets[i + 1] - offsets[i] : 0xffu;  // lengths were validated
  const uint32_t peers = __match_any_sync(0xffffffffu, L);
  const uint32_t below = peers & ((1u << lane) - 1u);
  if (below == 0u && L <= (uint32_t)kMaxLen) wcnt[w][L] = __popc(peers);
  __syncthreads();
  if (i < n) {
    uint32_t pos = bk.start[L] + block_base[(size_t)blockIdx.x * kBuckets + L] + __popc(below);
    for (int v = 0; v < w; ++v) pos += wcnt[v][L];
    perm[pos] = i;
    rank[i] = pos;
    slen[pos] = (uint8_t)L;
  }
}

__global__ void ingest_encode_kernel(const uint8_t* __restrict__ codes,
                                     const uint32_t* __restrict__ offsets, uint32_t n,
                                     const uint32_t* __restrict__ perm,
                                     const uint8_t* __restrict__ slen, const Buckets bk,
                                     uint32_t shift, uint32_t* __restrict__ a_enc,
                                     uint32_t* __restrict__ aoff, uint32_t* __restrict__ b_rec,
                                     uint32_t* __restrict__ brec_w) {
  const uint32_t p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const uint32_t L = slen[p];
  const uint32_t i = perm[p];
  const uint32_t o = offsets[i];
  const uint32_t r = p - bk.start[L];
  const uint32_t ao = bk.aenc_base[L] + r * L;
  const uint32_t bw = bk.brec_word_base[L] + (r >> 1) * (uint32_t)ceil4((int)L);
  const uint32_t half = r & 1u;
  aoff[p] = ao;
  brec_w[p] = bw | half;  // records start at multiples of 4 words: bit 0 carries the half
  uint16_t* b16 = reinterpret_cast<uint16_t*>(b_rec);
  for (uint32_t s = 0; s < L; ++s) {
    const uint32_t e = (uint32_t)codes[o + s] << shift;
    a_enc[ao + s] = e | (e << 16);
    b16[(size_t)(bw + s) * 2 + half] = (uint16_t)(~e & 0xffffu);
  }
}

cudaError_t launch_ingest_count(const uint8_t* codes, const uint32_t* offsets, uint32_t n,
                                uint32_t alphabet, uint32_t* block_counts, uint32_t* err,
                                cudaStream_t s) {
  const uint32_t nblk = (n + kIngestBlock - 1) / kIngestBlock;
  ingest_count_kernel<<<nblk, kIngestBlock, 0, s>>>(codes, offsets, n, alphabet, block_counts, err);
  return cudaGetLastError();
}

cudaError_t launch_ingest_scan(uint32_t* block_counts, uint32_t nblk, uint32_t* bucket_count,
                               cudaStream_t s) {
  ingest_scan_kernel<<<1, 64, 0, s>>>(block_counts, nblk, bucket_count);
  return cudaGetLastError();
}

cudaError_t launch_ingest_scatter(const uint32_t* offsets, uint32_t n, const uint32_t* block_base,
                                  const Buckets& bk, uint32_t* perm, uint32_t* rank, uint8_t* slen,
                                  cudaStream_t s) {
  const uint32_t nblk = (n + kIngestBlock - 1) / kIngestBlock;
  ingest_scatter_kernel<<<nblk, kIngestBlock, 0, s>>>(offsets, n, block_base, bk, perm, rank, slen);
  return cudaGetLastError();
}

cudaError_t launch_ingest_encode(const uint8_t* codes, const uint32_t* offsets, uint32_t n,
                                 const uint32_t* perm, const uint8_t* slen, const Buckets& bk,
                                 uint32_t shift, uint32_t* a_enc, uint32_t* aoff,
                                 uint32_t* b_rec, uint32_t* brec_w, cudaStream_t s) {
  const uint32_t nblk = (n + kIngestBlock - 1) / kIngestBlock;
  ingest_encode_kernel<<<nblk, kIngestBlock, 0, s>>>(codes, offsets, n, perm, slen, bk, shift,
                                                     a_enc, aoff, b_rec, brec_w);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// finalisation: each list's k slots, sorted by decreasing key, decoded.

__global__ void finalize_kernel(const uint32_t* __restrict__ slots, uint32_t nlists, uint32_t k,
                                const uint32_t* __restrict__ perm, uint32_t ib, uint32_t imask,
                                int32_t key_lo, uint32_t* __restrict__ out_idx,
                                int16_t* __restrict__ out_score, const int16_t* __restrict__ norm_frac,
                                const uint8_t* __restrict__ slen, const uint32_t* __restrict__ rank) {
  const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= nlists) return;
  uint32_t keys[NW_MAX_K];
  const uint32_t* row = slots + (size_t)w * k;
  for (uint32_t r = 0; r < k; ++r) {
    const uint32_t v = row[r];
    uint32_t q = r;
    while (q > 0 && keys[q - 1] < v) { keys[q] = keys[q - 1]; --q; }
    keys[q] = v;
  }
  const size_t o = (size_t)perm[w] * k;
  for (uint32_t r = 0; r < k; ++r) {
    const uint32_t key = keys[r];
    if (key == 0u) {
      out_idx[o + r] = 0xffffffffu;
      out_score[o + r] = INT16_MIN;
    } else {
      const uint32_t partner = imask - (key & imask);
      out_idx[o + r] = partner;
      if (norm_frac) {
        const uint32_t q = (key >> ib) - 1u;
        uint32_t m = slen[w];
        const uint32_t mp = slen[rank[partner]];
        m = m > mp ? m : mp;
        m = m > 0u ? m : 1u;
        out_score[o + r] = (int16_t)(norm_frac[2 * q] * (int32_t)(m / (uint32_t)norm_frac[2 * q + 1]));
      } else {
        out_score[o + r] = (int16_t)((int32_t)(key >> ib) + key_lo);
      }
    }
  }
}

cudaError_t launch_finalize(const uint32_t* slots, uint32_t nlists, uint32_t k, const uint32_t* perm,
                            uint32_t ib, uint32_t imask, int32_t key_lo, uint32_t* out_idx,
                            int16_t* out_score, cudaStream_t s, const int16_t* norm_frac, const uint8_t* slen,
                            const uint32_t* rank) {
  if (nlists == 0) return cudaSuccess;
  const uint32_t blk = 128;
  finalize_kernel<<<(nlists + blk - 1) / blk, blk, 0, s>>>(slots, nlists, k, perm, ib, imask, key_lo,
                                                           out_idx, out_score, norm_frac, slen, rank);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// integer-rate microbenchmarks: 8 chains per thread, each step of chain u
// reading chain u+1 of the previous step so no step can be folded away.

template <int OP>
__device__ __forceinline__ uint32_t rate_op(uint32_t x, uint32_t y, uint32_t c) {
  if constexpr (OP == kRateViaddmax) return __viaddmax_s16x2(x, y, c);
  else if constexpr (OP == kRateVimax3) return __vimax3_s16x2(x, y, c);
  else if constexpr (OP == kRateVimaxRelu) return __vimax_s16x2_relu(x, y);
  else if constexpr (OP == kRateIadd3) return x + y + c;
  else return (x & y) ^ c;
}

template <int OP>
__global__ void __launch_bounds__(kRateBlock) rate_kernel(const uint32_t* __restrict__ in,
                                                          uint32_t* __restrict__ out, int iters,
                                                          unsigned long long* cycles) {
  const uint32_t c = in[0] + blockIdx.x;
  uint32_t x[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) x[u] = in[1 + u] ^ (threadIdx.x * 0x9e3779b9u + u);
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
    uint32_t y[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) y[u] = rate_op<OP>(x[u], x[(u + 1) & 7], c);
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = y[u];
  }
  const long long t1 = clock64();
  uint32_t acc = 0;
#pragma unroll
  for (int u = 0; u < 8; ++u) acc ^= x[u];
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
  if (threadIdx.x == 0) atomicAdd(cycles, (unsigned long long)(t1 - t0));
}

// The alignment core alone (the kernel's dp_row, rows two at a time): each
// thread aligns an 8-symbol word from shared memory against two 16-symbol
// words held in registers, repeatedly.
__global__ void __launch_bounds__(kRateBlock) rate_cell_kernel(const uint32_t* __restrict__ in,
                                                               uint32_t* __restrict__ out, int iters,
                                                               unsigned long long* cycles) {
  constexpr int LB = 16, LA = 8;
  __shared__ uint32_t sa[LA * 4];
  if (threadIdx.x < LA * 4) sa[threadIdx.x] = (in[threadIdx.x & 15] & 0x001f001fu) << 1;
  __syncthreads();
  BRow<LB> b;
#pragma unroll
  for (int j = 0; j < LB; ++j) b.v[j] = ~((in[(j + threadIdx.x) & 15] & 0x001f001fu) << 1);
  const uint32_t C1 = 0x00040004u, C2 = 0x00010001u;  // scoring (+1, -1, -1)
  uint32_t acc = 0;
  const long long t0 = clock64();
  for (int it = 0; it < iters; ++it) {
    uint32_t G[LB];
#pragma unroll
    for (int j = 0; j < LB; ++j) G[j] = acc & 1u;
    const uint32_t* arow = sa + (it & 3) * LA;
#pragma unroll 1
    for (int i = 0; i < LA; i += 2) {
      dp_row<LB>(G, arow[i], b, C1, C2);
      dp_row<LB>(G, arow[i + 1], b, C1, C2);
    }
    acc += G[LB - 1];
  }
  const long long t1 = clock64();
  out[blockIdx.x * blockDim.x + threadIdx.x] = acc;
  if (threadIdx.x == 0) atomicAdd(cycles, (unsigned long long)(t1 - t0));
}

double rate_ops_per_iter(int op) { return op == kRateCell ? 8.0 * 16.0 : 8.0; }

int rate_blocks_per_sm(int op) {
  const void* fn = nullptr;
  switch (op) {
    case kRateViaddmax: fn = reinterpret_cast<const void*>(&rate_kernel<kRateViaddmax>); break;
    case kRateVimax3: fn = reinterpret_cast<const void*>(&rate_kernel<kRateVimax3>); break;
    case kRateVimaxRelu: fn = reinterpret_cast<const void*>(&rate_kernel<kRateVimaxRelu>); break;
    case kRateIadd3: fn = reinterpret_cast<const void*>(&rate_kernel<kRateIadd3>); break;
    case kRateLop3: fn = reinterpret_cast<const void*>(&rate_kernel<kRateLop3>); break;
    default: fn = reinterpret_cast<const void*>(&rate_cell_kernel); break;
  }
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kRateBlock, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return nb > 0 ? nb : 1;
}

cudaError_t launch_rate(int op, int blocks, int iters, const uint32_t* in, uint32_t* out,
                        unsigned long long* cycles, cudaStream_t s) {
  switch (op) {
    case kRateViaddmax: rate_kernel<kRateViaddmax><<<blocks, kRateBlock, 0, s>>>(in, out, iters, cycles); break;
    case kRateVimax3: rate_kernel<kRateVimax3><<<blocks, kRateBlock, 0, s>>>(in, out, iters, cycles); break;
    case kRateVimaxRelu: rate_kernel<kRateVimaxRelu><<<blocks, kRateBlock, 0, s>>>(in, out, iters, cycles); break;
    case kRateIadd3: rate_kernel<kRateIadd3><<<blocks, kRateBlock, 0, s>>>(in, out, iters, cycles); break;
    case kRateLop3: rate_kernel<kRateLop3><<<blocks, kRateBlock, 0, s>>>(in, out, iters, cycles); break;
    case kRateCell: rate_cell_kernel<<<blocks, kRateBlock, 0, s>>>(in, out, iters, cycles); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

namespace {
__global__ void topk_merge_kernel(uint32_t n, uint32_t k, uint32_t nparts, const uint32_t* __restrict__ idx_parts,
                                  const int16_t* __restrict__ score_parts, uint32_t* __restrict__ idx_out,
                                  int16_t* __restrict__ score_out) {
  const uint32_t w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= n) return;
  const size_t row = (size_t)w * k, part = (size_t)n * k;
  merge_ranked_row(
      nparts, k,
      [&](uint32_t p, uint32_t r, uint32_t& j, int32_t& s) {
        j = __ldg(idx_parts + p * part + row + r);
        s = __ldg(score_parts + p * part + row + r);
      },
      idx_out + row, score_out + row);
}
}  // namespace

cudaError_t launch_topk_merge(uint32_t n, uint32_t k, uint32_t nparts, const uint32_t* idx_parts,
                              const int16_t* score_parts, uint32_t* idx_out, int16_t* score_out, cudaStream_t s) {
  topk_merge_kernel<<<(n + 127) / 128, 128, 0, s>>>(n, k, nparts, idx_parts, score_parts, idx_out, score_out);
  return cudaGetLastError();
}

}  // namespace nw
