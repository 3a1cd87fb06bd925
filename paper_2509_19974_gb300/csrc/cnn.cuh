// cnn.cuh -- the learned lag proposal: a small 1-D CNN over decimated
// quantized signals whose feature correlation proposes lag windows for the
// exact integer correlation (cnn.cu).
#pragma once

#include <climits>

#include "common.cuh"

// Architecture (shared by both signals of a pair):
//   input  d[i] = (sum of 16 consecutive levels) / 4,  length Ld = n / 16
//   4 x [conv1d kernel 9, padding 4, 32 output channels, + bias, ReLU,
//        max-pool 2]   ->  features f[32][Lf],  Lf = Ld / 16 = n / 256
//   score[l] = alpha * sum_c sum_i fx[c][i] fy[c][i + l],  l in [-(Lf-1), Lf-1]
//   bin l covers lags tau in [256 l - 128, 256 l + 128] (width 257).
constexpr int kCnnC = 32, kCnnK = 9, kCnnLayers = 4, kCnnDec = 16, kCnnBin = 256;
constexpr int kCnnTopK = 8, kCnnWin = 257;
constexpr int kCnnFusedMaxLf = 256;  // longest features of the one-launch proposal

// Parameter layout (FP32 master copy, BF16 copy for the forward pass):
// per layer l: W_l[32][cin_l][9] then b_l[32] (cin_1 = 1, else 32); then alpha.
__host__ __device__ constexpr int cnn_cin(int l) { return l == 0 ? 1 : kCnnC; }
__host__ __device__ constexpr int cnn_woff(int l) {
  return l == 0 ? 0 : cnn_woff(l - 1) + kCnnC * cnn_cin(l - 1) * kCnnK + kCnnC;
}
__host__ __device__ constexpr int cnn_boff(int l) { return cnn_woff(l) + kCnnC * cnn_cin(l) * kCnnK; }
constexpr int kCnnAlpha = cnn_woff(kCnnLayers);
constexpr int kCnnParams = kCnnAlpha + 1;

struct CnnLayerIO {
  const float* in;  // [S][cin][L]
  float* pre;       // [S][32][L] post-ReLU before pooling (training), or nullptr
  float* out;       // [S][32][L/2]
  int L;
};

// Decimate: q [S][n] int8 -> d [S][n/16] float (block sums / 4).
cudaError_t launch_cnn_decimate(const int8_t* q, int64_t n, int nsig, float* d, cudaStream_t st);
// One layer for S signals with the BF16 weights of layer l.
cudaError_t launch_cnn_layer(const CnnLayerIO& io, int l, int nsig, const uint16_t* wbf,
                             const float* params, cudaStream_t st);
// Inference forward (decimate + 4 layers) with BF16 activations between
// layers: act[l] holds layer l's output, nsig x cnn_eo_elems((n/16) >> (l+1))
// BF16 in the layout above; feat receives the FP32 features [nsig][n/256][32]
// (position-major);
// qe (nullable, nsig x n bytes) the levels as E4M3 bytes.  n a multiple of
// 2048.
cudaError_t launch_cnn_infer(const int8_t* q, int64_t n, int nsig, const uint16_t* wbf,
                             const float* params, uint16_t* const act[kCnnLayers - 1], float* feat,
                             uint8_t* qe, uint32_t* d_status, cudaStream_t st);
// Inference activations between conv layers: a layer's input of length L
// is, per signal, 8 arrays (position parity x 8-channel chunk, parity-major)
// of cnn_eo_rows(L) rows of 8 BF16 channels; row r holds position 2r - 4
// (even array) or 2r - 3 (odd array) and is zero outside [0, L).  The rows
// cover whole 128-output tiles plus a 4-row halo.
__host__ __device__ constexpr int cnn_eo_rows(int L) { return (L / 2 + 127) / 128 * 128 + 4; }
__host__ __device__ constexpr int64_t cnn_eo_elems(int L) { return (int64_t)8 * cnn_eo_rows(L) * 8; }

// One 32 -> 32 channel layer of the inference forward on the tensor cores
// (mma.cu): in = that layer's input (length L, layout above); out = the next
// layer's input (length L/2, same layout, zero rows included) or (last) FP32
// features [nsig][L/2][32] (position-major); wbf / bias = that layer's BF16 weights
// [32][32][9] and FP32 bias.  L a multiple of 4.  Time-outs set
// TDE_ST_TIMEOUT.
cudaError_t launch_cnn_conv_tc(const uint16_t* in, void* out, int L, int nsig, const uint16_t* wbf,
                               const float* bias, bool last, uint32_t* d_status, cudaStream_t st);
// Layers 1 and 2 of the inference forward in one kernel (mma.cu): decimation
// of q [nsig][n] int8, conv 1 -> 32 (weights w1bf [32][1][9], bias1), whose
// output (layer 2's input) stays in shared memory, then conv 32 -> 32 (w2bf,
// bias2); out = the third layer's input (length n/64, parity arrays with
// their zero rows); qe (nullable, nsig x n bytes) receives the levels as E4M3
// bytes, for levels in {-1, 0, 1} (the learned path's b <= 2; other levels
// give other bytes).  n/16 a multiple of 8.  Time-outs set TDE_ST_TIMEOUT.
cudaError_t launch_cnn_conv12_tc(const int8_t* q, int64_t n, int nsig, const uint16_t* w1bf, const float* bias1,
                                 const uint16_t* w2bf, const float* bias2, uint16_t* out, uint8_t* qe,
                                 uint32_t* d_status, cudaStream_t st);
// score[p][l + Lf - 1] for npairs pairs (features of pair p: signals 2p, 2p+1;
// channel-major [S][32][Lf], or position-major [S][Lf][32] with pos_major).
// Channel-major features (the training forward) are scored in FP32 FMA;
// position-major ones (inference) up to Lf = kCnnFusedMaxLf on the tensor
// cores (the Gram matrix of the pair's features in split BF16, its diagonal
// sums in a fixed order), a time-out there setting TDE_ST_TIMEOUT in status
// (nullable).
cudaError_t launch_cnn_scores(const float* feat, int npairs, int Lf, const float* params,
                              float* scores, cudaStream_t st, bool pos_major = false,
                              uint32_t* status = nullptr);
// Top-8 bins per pair -> window centres in samples (256 l), softmax mass of
// the top 8 (margin).
cudaError_t launch_cnn_topk(const float* scores, int npairs, int Lf, int32_t* centres,
                            float* margin, cudaStream_t st);

// ---- training
// Softmax cross-entropy against label bins round(tau / 256); loss[p],
// dscore[p][.] = (softmax - onehot) / npairs.
cudaError_t launch_cnn_softmax_ce(const float* scores, const int64_t* labels, int npairs, int Lf,
                                  float* loss, float* dscores, cudaStream_t st);
// d features and per-pair d alpha from d scores.
cudaError_t launch_cnn_scores_bwd(const float* feat, const float* dscores, int npairs, int Lf,
                                  const float* params, float* dfeat, float* dalpha_pp,
                                  cudaStream_t st);
// Through max-pool and ReLU: dout [S][32][L/2] -> dz [S][32][L].
cudaError_t launch_cnn_pool_relu_bwd(const float* pre, const float* dout, int nsig, int L,
                                     float* dz, cudaStream_t st);
// din [S][32][L] = conv^T(dz) with layer l's weights (l >= 1).
cudaError_t launch_cnn_dgrad(const float* dz, int nsig, int L, int l, const uint16_t* wbf,
                             float* din, cudaStream_t st);
// Per-signal weight/bias gradient partials [S][32*cin*9 + 32].
cudaError_t launch_cnn_wgrad(const float* dz, const float* in, int nsig, int L, int l,
                             float* partial, cudaStream_t st);
// grad[off + i] = sum over signals of partial[s][i] (fixed order).
cudaError_t launch_cnn_reduce(const float* partial, int nsig, int count, float* grad,
                              cudaStream_t st);
// AdamW on all parameters; refreshes the BF16 copy.
cudaError_t launch_cnn_adamw(float* params, const float* grad, float* m, float* v, uint16_t* wbf,
                             int64_t step, float lr, float beta1, float beta2, float eps,
                             float wd, cudaStream_t st);
cudaError_t launch_cnn_to_bf16(const float* params, uint16_t* wbf, cudaStream_t st);

// ---- windows of the exact correlation and their argmax
struct WinJob {
  int64_t lag_lo, lag_hi;  // window, clipped to the overlap range (lag_hi - lag_lo <= 256)
  int32_t* c;              // lag lag_lo + i at c[i], i <= lag_hi - lag_lo
};
#ifdef __CUDACC__
// The window of 257 lags around centre c (samples), clipped to the lags of two
// signals of length n; its correlations go to cbuf_i (lag c - 128 + i at
// cbuf_i[i]).  An empty window (hi < lo) writes nothing; its pointer stays in
// range.
__device__ __forceinline__ WinJob win_job_of(int64_t c, int64_t n, int32_t* cbuf_i) {
  int64_t lo = c - kCnnBin / 2, hi = c + kCnnBin / 2;
  const int64_t first = lo;
  if (lo < -(n - 1)) lo = -(n - 1);
  if (hi > n - 1) hi = n - 1;
  return WinJob{lo, hi, cbuf_i + (hi >= lo ? lo - first : 0)};
}

// The windows' 128-lag blocks in the polyphase windows kernel (winpp.cu):
// window [lo, hi] needs blocks floor(lo / 128) .. floor((hi + 127) / 128),
// a[w] .. b[w] here (INT_MAX for an empty window, hi < lo), sorted by a.
__device__ __forceinline__ int64_t win_fdiv128(int64_t v) { return v >= 0 ? v / 128 : -((-v + 127) / 128); }
__device__ __forceinline__ void win_blocks(const int64_t (&lo)[kCnnTopK], const int64_t (&hi)[kCnnTopK],
                                           int (&a)[kCnnTopK], int (&b)[kCnnTopK]) {
#pragma unroll
  for (int w = 0; w < kCnnTopK; ++w) {
    const bool empty = hi[w] < lo[w];
    a[w] = empty ? INT_MAX : (int)win_fdiv128(lo[w]);
    b[w] = empty ? INT_MAX : (int)win_fdiv128(hi[w] + 127);
  }
#pragma unroll
  for (int pass = 0; pass < kCnnTopK; ++pass)  // odd-even transposition sort
#pragma unroll
    for (int i = pass & 1; i + 1 < kCnnTopK; i += 2)
      if (a[i] > a[i + 1]) {
        const int ta = a[i], tb = b[i];
        a[i] = a[i + 1], b[i] = b[i + 1];
        a[i + 1] = ta, b[i + 1] = tb;
      }
}
// Its jobs for those sorted ranges: overlapping or adjacent ranges join into
// runs, and a run of L blocks is ceil(L / 2) jobs of one or two blocks.
__device__ __forceinline__ int win_jobs(const int (&a)[kCnnTopK], const int (&b)[kCnnTopK]) {
  if (a[0] == INT_MAX) return 0;
  int n = 0, r0 = a[0], r1 = b[0];
#pragma unroll
  for (int i = 1; i < kCnnTopK; ++i) {
    if (a[i] == INT_MAX) break;
    if (a[i] <= r1 + 1) {
      r1 = b[i] > r1 ? b[i] : r1;
    } else {
      n += (r1 - r0 + 2) / 2;
      r0 = a[i], r1 = b[i];
    }
  }
  return n + (r1 - r0 + 2) / 2;
}
#endif
// The learned step's proposal in one launch, for Lf <= kCnnFusedMaxLf (else
// cudaErrorNotSupported): the scores of launch_cnn_scores (position-major
// features, tensor cores), then per pair the centres and margin of launch_cnn_topk
// (identical arithmetic, so identical values) and its 8 window jobs for
// signals of length n (window w of pair p writes cbuf + (8 p + w) * 257),
// with those 8 * 257 correlations zeroed, and njobs[p] = the pair's job
// count in the polyphase windows kernel (win_jobs).
cudaError_t launch_cnn_scores_propose(const float* feat, int npairs, int Lf, const float* params,
                                      float* scores, int32_t* centres, float* margin, WinJob* jobs,
                                      int32_t* cbuf, int64_t n, int32_t* njobs, cudaStream_t st,
                                      uint32_t* status = nullptr);
// Per pair: tie-ruled argmax over its 8 windows -> lag, value.
cudaError_t launch_window_argmax(const WinJob* d_jobs, int npairs, int64_t* lag, int64_t* val,
                                 cudaStream_t st);
