// nw_cnn.h -- kernels of the proposal network (see include/nw_proposal.h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace nw {
namespace cnn {

constexpr int kEmb = 32;
constexpr int kCh = 128;
constexpr int kOut = 64;
constexpr int kTaps = 3;

// Offsets of the parameter blocks in the flat vector for `alphabet` codes.
struct Layout {
  uint64_t emb, W1, b1, W2, b2, W3, b3, Wl, bl, total;
};
inline Layout layout(uint32_t alphabet) {
  Layout L{};
  uint64_t o = 0;
  L.emb = o; o += (uint64_t)alphabet * kEmb;
  L.W1 = o; o += (uint64_t)kCh * kTaps * kEmb;
  L.b1 = o; o += kCh;
  L.W2 = o; o += (uint64_t)kCh * kTaps * kCh;
  L.b2 = o; o += kCh;
  L.W3 = o; o += (uint64_t)kCh * kTaps * kCh;
  L.b3 = o; o += kCh;
  L.Wl = o; o += (uint64_t)kOut * kCh;
  L.bl = o; o += kOut;
  L.total = o;
  return L;
}

// Per-word inputs of a batch, gathered from a dictionary's device arrays.
struct WordSrc {
  const uint32_t* widx;   // Bw original indices
  const uint32_t* rank;   // original -> sorted position
  const uint8_t* slen;    // sorted position -> length
  const uint32_t* aoff;   // sorted position -> a_enc offset
  const uint32_t* a_enc;  // encoded symbols: code = (v & 0xffff) >> shift
  uint32_t shift;
  uint32_t n;             // words of the dictionary (bound of widx)
};

// A batch of Bw words in the packed layout: word w owns rows
// [off[w], off[w] + len[w]) of every activation matrix, row off[w] + t
// holding position t.  Grids are sized for Tmax rows; the actual row count T
// lives in device memory (kernels stop there), so a step whose words are
// drawn on the device can still be captured in a graph.
struct Packed {
  const int* len;    // Bw word lengths
  const int* off;    // Bw first rows
  const int* T;      // device: rows in use
  const int* rinfo;  // per row: (position << 8) | word length
  const int* rword;  // per row: word
  int Bw, Tmax;
};

// GEMM epilogue: out = acc (+ bias[n]) (ReLU) (x (gate[m][n] > 0)), or
// atomicAdd of acc (split-K accumulation into a zeroed C).
struct Epi {
  const float* bias = nullptr;
  bool relu = false;
  const float* gate = nullptr;   // same layout as C
  bool atomic = false;
  uint32_t* err = nullptr;       // receives kErrWait if a tensor-core pipeline wait runs out (may be null)
};

// The network's matrix products: bf16 tensor-core tiles, operands rounded
// to bf16 (nearest even) as they are loaded, float32 accumulation.  W is
// [Co][3][Ci], Wl is [Co][Ci]; Ci and Co of a convolution are powers of
// two; activations of a packed batch have pk.T rows.
//   conv_fwd: Y[T][Co]  = im2col(X[T][Ci]) . W^T            (epilogue e)
//   conv_dw:  dW[Co][3Ci] += dY^T . im2col(X)               (split over rows, atomic)
//   conv_dx:  dX[T][Ci] = sum_tap shift_tap(dY) . W[.][tap]  (col2im folded in; epilogue e)
//   lin_fwd:  E[B][Co]  = P[B][Ci] . Wl^T                   (epilogue e)
//   lin_dw:   dWl[Co][Ci] += dE^T . P                       (split over B, atomic)
//   lin_dx:   dP[B][Ci] = dE[B][Co] . Wl
// im2col(X) row t, column tap * Ci + c, is X[t + tap - 1][c] when position
// pos(t) + tap - 1 lies inside t's word, else 0 (the zero padding).
cudaError_t conv_fwd(const float* X, int Ci, const float* W, int Co, const Packed& pk, float* Y, const Epi& e,
                     cudaStream_t s);
cudaError_t conv_dw(const float* dY, int Co, const float* X, int Ci, const Packed& pk, float* dW, int nsm,
                    cudaStream_t s);
cudaError_t conv_dx(const float* dY, int Co, const float* W, int Ci, const Packed& pk, float* dX, const Epi& e,
                    cudaStream_t s);
cudaError_t lin_fwd(const float* P, int Ci, const float* Wl, int Co, int B, float* E, const Epi& e, cudaStream_t s);
cudaError_t lin_dw(const float* dE, int Co, const float* P, int Ci, int B, float* dWl, int nsm, cudaStream_t s);
cudaError_t lin_dx(const float* dE, int Co, const float* Wl, int Ci, int B, float* dP, cudaStream_t s);

// word lengths, row offsets and T of widx's words, the per-row tables, the
// codes and the embedded input X0 (rows past Tmax raise kErrInput)
struct PackBufs {
  int* len;
  int* off;
  int* T;
  int* rinfo;
  int* rword;
  int32_t* codes;
};
cudaError_t pack_words(const WordSrc& src, int Bw, int Tmax, const float* emb, const PackBufs& b, float* X0,
                       uint32_t* err, uint32_t alphabet, cudaStream_t s);
cudaError_t mean_pool(const float* Y, const Packed& pk, float* P, cudaStream_t s);
cudaError_t mean_pool_bwd(const float* dP, const float* Y, const Packed& pk, float* dY, cudaStream_t s);
// pairs are word slots (2p, 2p + 1), pred = phi . phi + beta + beta (outputs
// 0..62 features, 63 bias); loss_acc += sum (pred - y)^2 / m (if non-null)
cudaError_t pair_loss(const float* E, const float* target, int m, float* dE, float* loss_acc, cudaStream_t s);
// out += column sums of Y's first rows (rows: a host count, or the device count *rows_dev when non-null)
cudaError_t col_sum(const float* Y, int rows, const int* rows_dev, int cols, float* out, cudaStream_t s);
cudaError_t emb_scatter(const float* dX0, const int32_t* codes, const Packed& pk, float* demb, cudaStream_t s);
struct AdamCfg {
  float lr, lr_final, b1, b2, eps;
  float clip;        // > 0: scale the gradient to norm <= clip
  float* sumsq;      // device scratch for |g|^2
  uint32_t step0, nsteps;  // the rate falls linearly over steps step0 + 1 .. step0 + nsteps
};
cudaError_t adam(float* theta, const float* g, float* m, float* v, uint64_t n, const uint32_t* step,
                 const AdamCfg& c, cudaStream_t s);
cudaError_t bump_step(uint32_t* step, cudaStream_t s);
// losses[*step - 1 - step0] = *cur (when inside [0, nsteps)), then *cur = 0
cudaError_t record_loss(float* cur, float* losses, const uint32_t* step, uint32_t step0, uint32_t nsteps,
                        cudaStream_t s);

// training pairs of one step: pi/pj, word slots widx[2p], widx[2p + 1]
struct PairDraw {
  uint64_t seed;
  const uint32_t* step;   // device step counter (graph replays read it)
  uint32_t n, m;
  const uint32_t* nbr;    // n x knb or null
  uint32_t knb;
  uint32_t n_nbr;         // pairs [0, n_nbr) come from the lists
  const uint32_t* perm;   // sorted position -> original index (long-word draws)
  uint32_t long0, nlong;  // the long words' sorted positions [long0, long0 + nlong)
  uint32_t long_thresh;   // a pair's i is a long word when 20 bits of its draw are below this
};
cudaError_t draw_pairs(const PairDraw& d, uint32_t* pi, uint32_t* pj, uint32_t* widx, cudaStream_t s);
// target[p] = score[p] * raw_scale (raw_scale > 0), else score[p] / max(len_i, len_j, 1)
cudaError_t pair_targets(const int16_t* score, const uint32_t* pi, const uint32_t* pj, const uint32_t* rank,
                         const uint8_t* slen, int m, float raw_scale, float* target, cudaStream_t s);
cudaError_t interleave_pairs(const uint32_t* pi, const uint32_t* pj, int m, uint32_t* widx, cudaStream_t s);
// out[x] = src[base + x]
cudaError_t take(const uint32_t* src, uint32_t base, int count, uint32_t* out, cudaStream_t s);
// dst[widx[w] * 64 + d] = E[w * 64 + d]
cudaError_t scatter_rows(const float* E, const uint32_t* widx, int Bw, float* dst, cudaStream_t s);

}  // namespace cnn
}  // namespace nw
