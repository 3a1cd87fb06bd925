// cnn.cu -- learned lag proposal kernels (inference and training) and the
// windowed exact correlation that checks its proposals.
//
// The proposal only decides WHERE the exact integer correlation of
// Algorithm 1's correlation step (arXiv 2509.19974) is evaluated: the lag returned is
// always the tie-ruled maximiser of exact integer values, either inside the
// proposed windows or, when the proposal's confidence (softmax mass of its top
// 8 bins) is below a threshold, over the full lag range.
//
// The windows' exact correlation runs on the tensor cores
// (launch_xcorr_win_pp in winpp.cu); this file holds their argmax.
//
// Weights are BF16-rounded everywhere and every sum is FP32.  Inference runs
// its four conv layers on tcgen05 (mma.cu: k_conv12_tc, k_conv_tc) with BF16
// activations between layers; the training forward keeps FP32 activations
// (the first layer in FP32 FMA, the 32-channel layers as mma.sync BF16 tiles
// with FP32 accumulation), and the backward pass is deterministic (per-signal
// partial sums reduced in a fixed order, no float atomics).  Training shapes:
// conv layers tile 128 output positions x 32 channels per CTA; a warp's 32
// lanes are the 32 output channels (forward) or input channels (data
// gradient), so shared-memory weight reads are contiguous and activation
// reads are broadcasts.
#include <cstring>

#include "cnn.cuh"
#include "tc.cuh"

namespace {

constexpr int kT = 128;  // positions per conv CTA
constexpr int kThreads = 256;

__device__ __forceinline__ float bf16_to_f(uint16_t b) { return __uint_as_float((uint32_t)b << 16); }

// FP32 -> BF16, round to nearest even (NaN-free inputs).
__host__ __device__ __forceinline__ uint16_t f_to_bf16(float f) {
#ifdef __CUDA_ARCH__
  const uint32_t u = __float_as_uint(f);
#else
  uint32_t u;
  memcpy(&u, &f, 4);
#endif
  return (uint16_t)((u + 0x7FFFu + ((u >> 16) & 1u)) >> 16);
}

__global__ void k_decimate(const int8_t* __restrict__ q, int64_t n, int nsig, float* __restrict__ d) {
  const int64_t ld = n / kCnnDec;
  const int64_t total = (int64_t)nsig * ld;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = i / ld, j = i % ld;
    const int8_t* src = q + s * n + j * kCnnDec;
    int acc = 0;
#pragma unroll
    for (int k = 0; k < kCnnDec; ++k) acc += src[k];
    d[i] = 0.25f * (float)acc;
  }
}

// conv (kernel 9, pad 4) + bias + ReLU (+ store) + max-pool 2.  A thread owns
// 4 output channels x 16 positions (64 accumulators); a CTA covers 512
// positions; weights are read as float4 (4 channels) per (ci, k).
constexpr int kTP = 512;  // positions per forward CTA

template <int CIN>
__global__ void __launch_bounds__(kThreads) k_conv_fwd(const float* __restrict__ in,
                                                       float* __restrict__ pre,
                                                       float* __restrict__ out, int L,
                                                       const uint16_t* __restrict__ wbf,
                                                       const float* __restrict__ bias) {
  extern __shared__ float csm[];
  float* in_s = csm;                          // [CIN][kTP + 8]
  float* w_s = csm + CIN * (kTP + 8);         // [ci*9 + k][32 co]
  const int s = blockIdx.y, p0 = blockIdx.x * kTP;
  const float* src = in + (int64_t)s * CIN * L;
  for (int idx = threadIdx.x; idx < CIN * (kTP + 8); idx += kThreads) {
    const int ci = idx / (kTP + 8), j = idx % (kTP + 8);
    const int pos = p0 - 4 + j;
    in_s[idx] = (pos >= 0 && pos < L) ? src[(int64_t)ci * L + pos] : 0.f;
  }
  for (int idx = threadIdx.x; idx < kCnnC * CIN * kCnnK; idx += kThreads) {
    const int co = idx / (CIN * kCnnK), r = idx % (CIN * kCnnK);
    w_s[r * kCnnC + co] = bf16_to_f(wbf[idx]);
  }
  __syncthreads();
  const int cg = threadIdx.x & 7, pg = threadIdx.x >> 3;  // 8 channel groups x 32 position groups
  const int co0 = cg * 4;
  if (p0 + pg * 16 >= L) return;  // short layers (L < 512): idle position groups
  float acc[4][16];
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    const float b = bias[co0 + c];
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[c][j] = b;
  }
  for (int ci = 0; ci < CIN; ++ci) {
    float xr[24];
    const float* row = in_s + ci * (kTP + 8) + pg * 16;
#pragma unroll
    for (int j = 0; j < 24; ++j) xr[j] = row[j];
#pragma unroll
    for (int k = 0; k < kCnnK; ++k) {
      const float4 w = *reinterpret_cast<const float4*>(w_s + (ci * kCnnK + k) * kCnnC + co0);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float xv = xr[j + k];
        acc[0][j] = fmaf(w.x, xv, acc[0][j]);
        acc[1][j] = fmaf(w.y, xv, acc[1][j]);
        acc[2][j] = fmaf(w.z, xv, acc[2][j]);
        acc[3][j] = fmaf(w.w, xv, acc[3][j]);
      }
    }
  }
  const int pbase = p0 + pg * 16;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
#pragma unroll
    for (int j = 0; j < 16; ++j) acc[c][j] = fmaxf(acc[c][j], 0.f);
    if (pre) {
      float* dp = pre + ((int64_t)s * kCnnC + co0 + c) * L + pbase;
#pragma unroll
      for (int j = 0; j < 16; j += 4)
        *reinterpret_cast<float4*>(dp + j) =
            make_float4(acc[c][j], acc[c][j + 1], acc[c][j + 2], acc[c][j + 3]);
    }
    float* dst = out + ((int64_t)s * kCnnC + co0 + c) * (L / 2) + pbase / 2;
#pragma unroll
    for (int j = 0; j < 16; j += 8)
      *reinterpret_cast<float4*>(dst + j / 2) =
          make_float4(fmaxf(acc[c][j], acc[c][j + 1]), fmaxf(acc[c][j + 2], acc[c][j + 3]),
                      fmaxf(acc[c][j + 4], acc[c][j + 5]), fmaxf(acc[c][j + 6], acc[c][j + 7]));
  }
}

// Inference form of the 32 -> 32 conv layers on the tensor cores
// (mma.sync m16n8k16, BF16 operands, FP32 accumulation): for each tap k,
// Y[p][co] += sum_ci X[p + k - 4][ci] W[co][ci][k], a 16-position x 32-channel
// tile per warp step.  Activations are rounded to BF16 when staged; the
// training forward keeps FP32 activations (k_conv_fwd).
constexpr int kXR = 40;  // padded BF16 row (32 channels + 8): conflict-free fragment loads

__device__ __forceinline__ uint32_t pack_bf16x2(float lo, float hi) {
  return (uint32_t)f_to_bf16(lo) | ((uint32_t)f_to_bf16(hi) << 16);
}

__device__ __forceinline__ void mma_bf16_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                               uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, "
      "{%8, %9}, {%0, %1, %2, %3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__global__ void __launch_bounds__(kThreads) k_conv_fwd_tc(const float* __restrict__ in,
                                                          float* __restrict__ out, int L,
                                                          const uint16_t* __restrict__ wbf,
                                                          const float* __restrict__ bias) {
  extern __shared__ uint32_t tsm[];
  uint16_t* xs = reinterpret_cast<uint16_t*>(tsm);                 // [kTP + 8][kXR]
  uint16_t* ws = xs + (kTP + 8) * kXR;                             // [9][32 co][kXR]
  const int s = blockIdx.y, p0 = blockIdx.x * kTP;
  const float* src = in + (int64_t)s * kCnnC * L;
  // X rows r <-> position p0 - 4 + r; two channels per 32-bit word
  for (int idx = threadIdx.x; idx < (kTP + 8) * (kCnnC / 2); idx += kThreads) {
    const int r = idx % (kTP + 8), cp = idx / (kTP + 8);
    const int pos = p0 - 4 + r;
    float v0 = 0.f, v1 = 0.f;
    if (pos >= 0 && pos < L) {
      v0 = src[(int64_t)(2 * cp) * L + pos];
      v1 = src[(int64_t)(2 * cp + 1) * L + pos];
    }
    *reinterpret_cast<uint32_t*>(xs + r * kXR + 2 * cp) = pack_bf16x2(v0, v1);
  }
  for (int idx = threadIdx.x; idx < kCnnC * kCnnC * kCnnK; idx += kThreads) {
    const int co = idx / (kCnnC * kCnnK), r = idx % (kCnnC * kCnnK);
    const int ci = r / kCnnK, k = r % kCnnK;
    ws[(k * kCnnC + co) * kXR + ci] = wbf[idx];
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, t = lane & 3;
  const int nmt = (L - p0) < kTP ? (L - p0) / 16 : kTP / 16;  // m-tiles of this CTA
  float acc[4][4][4];  // [m-tile of the warp][n-tile][frag]
#pragma unroll
  for (int mi = 0; mi < 4; ++mi)
#pragma unroll
    for (int ni = 0; ni < 4; ++ni)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[mi][ni][e] = 0.f;
#pragma unroll 1
  for (int k = 0; k < kCnnK; ++k) {
#pragma unroll
    for (int ks = 0; ks < kCnnC; ks += 16) {
      uint32_t b[4][2];
#pragma unroll
      for (int ni = 0; ni < 4; ++ni) {
        const uint16_t* wr = ws + (k * kCnnC + ni * 8 + g) * kXR + ks + 2 * t;
        b[ni][0] = *reinterpret_cast<const uint32_t*>(wr);
        b[ni][1] = *reinterpret_cast<const uint32_t*>(wr + 8);
      }
#pragma unroll
      for (int mi = 0; mi < 4; ++mi) {
        const int mt = warp + 8 * mi;
        if (mt >= nmt) continue;
        const uint16_t* xr = xs + (mt * 16 + g + k) * kXR + ks + 2 * t;
        uint32_t a[4];
        a[0] = *reinterpret_cast<const uint32_t*>(xr);
        a[1] = *reinterpret_cast<const uint32_t*>(xr + 8 * kXR);
        a[2] = *reinterpret_cast<const uint32_t*>(xr + 8);
        a[3] = *reinterpret_cast<const uint32_t*>(xr + 8 * kXR + 8);
#pragma unroll
        for (int ni = 0; ni < 4; ++ni) mma_bf16_16816(acc[mi][ni], a, b[ni][0], b[ni][1]);
      }
    }
  }
  // epilogue: bias, ReLU, max-pool rows (g, g^1) via a lane shuffle (lane ^ 4)
#pragma unroll
  for (int mi = 0; mi < 4; ++mi) {
    const int mt = warp + 8 * mi;
    if (mt >= nmt) continue;  // warp-uniform
#pragma unroll
    for (int ni = 0; ni < 4; ++ni) {
      const int co = ni * 8 + 2 * t;
      const float b0 = bias[co], b1 = bias[co + 1];
      float v[4] = {fmaxf(acc[mi][ni][0] + b0, 0.f), fmaxf(acc[mi][ni][1] + b1, 0.f),
                    fmaxf(acc[mi][ni][2] + b0, 0.f), fmaxf(acc[mi][ni][3] + b1, 0.f)};
      float o[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) o[e] = fmaxf(v[e], __shfl_xor_sync(0xffffffffu, v[e], 4));
      if ((g & 1) == 0) {
        const int prow = p0 + mt * 16 + g;  // even position; rows g and g + 8
        float* d0 = out + ((int64_t)s * kCnnC + co) * (L / 2);
        float* d1 = d0 + (L / 2);
        d0[prow / 2] = o[0];
        d1[prow / 2] = o[1];
        d0[prow / 2 + 4] = o[2];
        d1[prow / 2 + 4] = o[3];
      }
    }
  }
}

// ---- inference chain with BF16 activations
// Inference keeps the activations between layers as BF16 parity arrays (the
// layout in cnn.cuh): every layer runs on the tensor cores (tcgen05, in
// mma.cu), which take BF16 operands anyway, so the values are those of the
// FP32 chain rounded where the tensor cores read them, at half the traffic.
// The last layer writes FP32 features [signal][Lf][32] for the scores.


// Scores: score[l] = alpha * sum_c sum_i fx[c][i] fy[c][i + l].  A CTA
// takes 128 consecutive bins of one pair, a warp 16 of them, a lane one
// channel; the positions stream through shared memory in tiles of 128 (both
// features transposed to [position][channel], rows padded to 33 floats so
// the transposing stores and the lane-per-channel loads are conflict-free,
// zeros outside [0, Lf)).  Each warp walks only the positions where its bins
// overlap, in blocks of 16 (a block that runs past the overlap multiplies
// zeros), keeps a 31-value sliding window of fy in registers (16 FMAs per
// shared-memory load pair) and reduces its 16 per-channel sums across the
// lanes at the end.  Any Lf: shared memory does not grow with it.
constexpr int kScWarps = 8;                     // warps per CTA
constexpr int kScG = 16;                        // bins per warp
constexpr int kScBins = kScWarps * kScG;        // bins per CTA (128)
constexpr int kScT = 128;                       // positions per tile
constexpr int kScRow = kCnnC + 1;               // padded row
constexpr int kScYRows = kScT + kScBins + kScG; // fy rows per tile (272)
constexpr int kScSmem = (kScT + kScYRows) * kScRow * 4;

template <bool kPosMajor>
__global__ void __launch_bounds__(kScWarps * 32) k_scores(const float* __restrict__ feat, int Lf,
                                                          const float* __restrict__ params,
                                                          float* __restrict__ scores) {
  extern __shared__ __align__(16) float sm[];
  float* xs = sm;                    // [kScT][kScRow]: fx at position i0 + r
  float* ys = sm + kScT * kScRow;    // [kScYRows][kScRow]: fy at position i0 + l_lo + r
  const int p = blockIdx.y;
  const int nb = 2 * Lf - 1;
  const int b_lo = blockIdx.x * kScBins;
  const int l_lo = b_lo - (Lf - 1);  // lag of the CTA's first bin
  const float* gx = feat + (int64_t)(2 * p) * kCnnC * Lf;
  const float* gy = feat + (int64_t)(2 * p + 1) * kCnnC * Lf;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lg = l_lo + kScG * warp;  // lag of the warp's first bin
  // positions where some bin of the warp (of the CTA) overlaps, rounded out to 16
  const int wlo = max(0, -(lg + kScG - 1)) & ~(kScG - 1);
  const int whi = (min(Lf, Lf - lg) + kScG - 1) & ~(kScG - 1);
  const int clo = max(0, -(l_lo + kScBins - 1)) & ~(kScG - 1);
  const int chi = min(Lf, Lf - l_lo);
  float acc[kScG];
#pragma unroll
  for (int t = 0; t < kScG; ++t) acc[t] = 0.f;
  for (int i0 = clo; i0 < chi; i0 += kScT) {
    if (kPosMajor) {  // [position][channel]: coalesced rows of 32 channels
      for (int idx = threadIdx.x; idx < kCnnC * kScT; idx += kScWarps * 32) {
        const int r = idx >> 5, c = idx & 31, i = i0 + r;
        xs[r * kScRow + c] = i < Lf ? __ldg(gx + (int64_t)i * kCnnC + c) : 0.f;
      }
      for (int idx = threadIdx.x; idx < kCnnC * kScYRows; idx += kScWarps * 32) {
        const int r = idx >> 5, c = idx & 31, j = i0 + l_lo + r;
        ys[r * kScRow + c] = (j >= 0 && j < Lf) ? __ldg(gy + (int64_t)j * kCnnC + c) : 0.f;
      }
    } else {
      for (int idx = threadIdx.x; idx < kCnnC * kScT; idx += kScWarps * 32) {
        const int c = idx / kScT, r = idx % kScT, i = i0 + r;
        xs[r * kScRow + c] = i < Lf ? __ldg(gx + (int64_t)c * Lf + i) : 0.f;
      }
      for (int idx = threadIdx.x; idx < kCnnC * kScYRows; idx += kScWarps * 32) {
        const int c = idx / kScYRows, r = idx % kScYRows, j = i0 + l_lo + r;
        ys[r * kScRow + c] = (j >= 0 && j < Lf) ? __ldg(gy + (int64_t)c * Lf + j) : 0.f;
      }
    }
    __syncthreads();
    const int blo = max(wlo, i0), bhi = min(whi, i0 + kScT);  // warp-uniform
    if (blo < bhi) {
      const float* xr = xs + (blo - i0) * kScRow + lane;
      const float* yr = ys + (blo - i0 + kScG * warp) * kScRow + lane;
      float yv[2 * kScG - 1];
#pragma unroll
      for (int t = 0; t < kScG - 1; ++t) yv[t] = yr[t * kScRow];
      for (int ib = blo; ib < bhi; ib += kScG) {
        float xv[kScG];
#pragma unroll
        for (int s2 = 0; s2 < kScG; ++s2) xv[s2] = xr[s2 * kScRow];
#pragma unroll
        for (int t = kScG - 1; t < 2 * kScG - 1; ++t) yv[t] = yr[t * kScRow];
#pragma unroll
        for (int s2 = 0; s2 < kScG; ++s2)
#pragma unroll
          for (int t = 0; t < kScG; ++t) acc[t] = fmaf(xv[s2], yv[s2 + t], acc[t]);
#pragma unroll
        for (int t = 0; t < kScG - 1; ++t) yv[t] = yv[t + kScG];
        xr += kScG * kScRow;
        yr += kScG * kScRow;
      }
    }
    __syncthreads();
  }
  // sum over the 32 lanes (channels): each step halves the values a lane
  // keeps (the step with mask m keeps the upper half when lane & m), so
  // afterwards the lane holds bin (lane >> 1) & 15 summed over all lanes.
#pragma unroll
  for (int half = kScG / 2, m = 16; half >= 1; half >>= 1, m >>= 1) {
    const bool hi = (lane & m) != 0;
#pragma unroll
    for (int j = 0; j < half; ++j) {
      const float send = hi ? acc[j] : acc[j + half];
      const float keep = hi ? acc[j + half] : acc[j];
      acc[j] = keep + __shfl_xor_sync(0xffffffffu, send, m);
    }
  }
  acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
  const int bin = b_lo + kScG * warp + ((lane >> 1) & (kScG - 1));
  if ((lane & 1) == 0 && bin < nb) scores[(int64_t)p * nb + bin] = params[kCnnAlpha] * acc[0];
}

// lag rank of bin l: smaller |l| first, then negative first (the estimator's
// tie order), used to break exact score ties deterministically.
__device__ __forceinline__ bool better(float s, int l, float bs, int bl) {
  if (s != bs) return s > bs;
  const int a = l < 0 ? -l : l, ab = bl < 0 ? -bl : bl;
  return a != ab ? a < ab : l < bl;
}

// Top-8 of one pair's nb = 2 Lf - 1 bin scores, warp-wide.  v[i] is the
// score of bin lane + 32 i (-inf past nb).  Softmax over all bins; eight
// rounds of a register scan plus one warp reduction, a taken bin marked by a
// flag bit.  Lane r < 8 receives the r-th centre in samples (256 l, best
// first, exact ties by the lag order of `better`); every lane the softmax
// mass of the eight (the margin).
template <int PER>
__device__ __forceinline__ void topk_warp(const float (&v)[PER], int nb, int Lf, int lane,
                                          int32_t& centre, float& margin) {
  uint32_t taken = 0;
  float mx = -INFINITY;
#pragma unroll
  for (int i = 0; i < PER; ++i) mx = fmaxf(mx, v[i]);
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  float sum = 0.f;
#pragma unroll
  for (int i = 0; i < PER; ++i)
    if (lane + 32 * i < nb) sum += __expf(v[i] - mx);
  for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  float top = 0.f;
  centre = 0;
  for (int r = 0; r < kCnnTopK; ++r) {
    float bs = -INFINITY;
    int bl = 1 << 30, bi = -1;
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int b = lane + 32 * i;
      const int l = b - (Lf - 1);
      if (b < nb && !(taken >> i & 1u) && (bl == (1 << 30) || better(v[i], l, bs, bl))) {
        bs = v[i];
        bl = l;
        bi = i;
      }
    }
    int owner = lane;
    for (int o = 16; o; o >>= 1) {
      const float os = __shfl_xor_sync(0xffffffffu, bs, o);
      const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
      const int ow = __shfl_xor_sync(0xffffffffu, owner, o);
      if (ol != (1 << 30) && (bl == (1 << 30) || better(os, ol, bs, bl))) {
        bs = os;
        bl = ol;
        owner = ow;
      }
    }
    if (lane == owner && bi >= 0) taken |= 1u << bi;
    top += __expf(bs - mx);
    if (lane == r) centre = kCnnBin * bl;
  }
  margin = top / sum;
}

// Short features (Lf <= 256) in FP32 FMA (the training forward's
// channel-major features): one CTA per pair with both features whole in
// shared memory (32 zero rows padding y on both sides), 16 warps, warp w
// taking the bin groups w and w + ngroups/2: their overlaps add up to about
// Lf, so every warp does the same work and the grid is one wave.  The inner
// loop and the lane reduction are those of k_scores.
constexpr int kSpWarps = 16;
constexpr int kSpMaxLf = kCnnFusedMaxLf;
constexpr int kSpPad = 32;
constexpr int kSpSmem = ((kSpMaxLf + 16) + (kSpMaxLf + 2 * kSpPad)) * kScRow * 4;

struct TopOut {
  int32_t* centres;  // [P][8]
  float* margin;     // [P]
  WinJob* jobs;      // [P][8]
  int32_t* cbuf;     // window w of pair p at cbuf + (8 p + w) * 257
  int64_t n;         // signal length (lag range of the windows)
  int32_t* njobs;    // [P]: jobs of the polyphase windows kernel
};

template <bool kPosMajor>
__global__ void __launch_bounds__(kSpWarps * 32, 2) k_scores_pair(const float* __restrict__ feat, int Lf,
                                                                  const float* __restrict__ params,
                                                                  float* __restrict__ scores) {
  extern __shared__ __align__(16) float sm[];
  float* xs = sm;                               // [Lf + 16][kScRow]: fx at row i
  float* ys = sm + (kSpMaxLf + 16) * kScRow;    // [Lf + 64][kScRow]: fy at row i + kSpPad
  const int p = blockIdx.x;
  const int nb = 2 * Lf - 1;
  const float* gx = feat + (int64_t)(2 * p) * kCnnC * Lf;
  const float* gy = feat + (int64_t)(2 * p + 1) * kCnnC * Lf;
  for (int idx = threadIdx.x; idx < kCnnC * (Lf + 16); idx += kSpWarps * 32) {
    const int r = kPosMajor ? idx >> 5 : idx % (Lf + 16), c = kPosMajor ? idx & 31 : idx / (Lf + 16);
    xs[r * kScRow + c] = r < Lf ? __ldg(kPosMajor ? gx + (int64_t)r * kCnnC + c : gx + (int64_t)c * Lf + r) : 0.f;
  }
  for (int idx = threadIdx.x; idx < kCnnC * (Lf + 2 * kSpPad); idx += kSpWarps * 32) {
    const int r = kPosMajor ? idx >> 5 : idx % (Lf + 2 * kSpPad), c = kPosMajor ? idx & 31 : idx / (Lf + 2 * kSpPad);
    const int j = r - kSpPad;
    ys[r * kScRow + c] =
        (j >= 0 && j < Lf) ? __ldg(kPosMajor ? gy + (int64_t)j * kCnnC + c : gy + (int64_t)c * Lf + j) : 0.f;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int ngroups = (nb + kScG - 1) / kScG, half = (ngroups + 1) / 2;
  const float alpha = params[kCnnAlpha];
  for (int gi = 0; gi < 2; ++gi) {
    const int g = warp + gi * half;
    if (warp >= half || g >= ngroups) continue;  // warp-uniform
    const int lg = kScG * g - (Lf - 1);          // lag of the group's first bin
    const int wlo = max(0, -(lg + kScG - 1)) & ~(kScG - 1);
    const int whi = (min(Lf, Lf - lg) + kScG - 1) & ~(kScG - 1);
    float acc[kScG];
#pragma unroll
    for (int t = 0; t < kScG; ++t) acc[t] = 0.f;
    if (wlo < whi) {
      const float* xr = xs + wlo * kScRow + lane;
      const float* yr = ys + (wlo + lg + kSpPad) * kScRow + lane;
      float yv[2 * kScG - 1];
#pragma unroll
      for (int t = 0; t < kScG - 1; ++t) yv[t] = yr[t * kScRow];
      for (int ib = wlo; ib < whi; ib += kScG) {
        float xv[kScG];
#pragma unroll
        for (int s2 = 0; s2 < kScG; ++s2) xv[s2] = xr[s2 * kScRow];
#pragma unroll
        for (int t = kScG - 1; t < 2 * kScG - 1; ++t) yv[t] = yr[t * kScRow];
#pragma unroll
        for (int s2 = 0; s2 < kScG; ++s2)
#pragma unroll
          for (int t = 0; t < kScG; ++t) acc[t] = fmaf(xv[s2], yv[s2 + t], acc[t]);
#pragma unroll
        for (int t = 0; t < kScG - 1; ++t) yv[t] = yv[t + kScG];
        xr += kScG * kScRow;
        yr += kScG * kScRow;
      }
    }
#pragma unroll
    for (int hf = kScG / 2, m = 16; hf >= 1; hf >>= 1, m >>= 1) {
      const bool hi = (lane & m) != 0;
#pragma unroll
      for (int j = 0; j < hf; ++j) {
        const float send = hi ? acc[j] : acc[j + hf];
        const float keep = hi ? acc[j + hf] : acc[j];
        acc[j] = keep + __shfl_xor_sync(0xffffffffu, send, m);
      }
    }
    acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], 1);
    const int bin = kScG * g + ((lane >> 1) & (kScG - 1));
    if ((lane & 1) == 0 && bin < nb) scores[(int64_t)p * nb + bin] = alpha * acc[0];
  }
}


// Short features (Lf <= 256, position-major) on the tensor cores: per pair the
// Gram matrix G[i][j] = sum_c fx[i][c] fy[j][c] (rows past Lf zero; two M = 128
// tiles of N = 256, K = 32, FP32 in tensor memory) and the scores as its
// diagonal sums, score[l] = alpha sum_i G[i][i + l].  Each FP32 feature is
// split as f = hi + lo (hi = BF16(f), lo = BF16(f - hi)) and G accumulates
// hi.hi + hi.lo + lo.hi (kind::f16, BF16 operands): what is left out, lo.lo
// and the rounding of lo, is below 2^-16 of each product, whose terms are all
// non-negative (ReLU features), so the scores keep about 16 bits -- the FP32
// sums they replace keep about as many over 8192 terms.  The diagonal sums are
// deterministic: warp w reads its 32 x 32 blocks of G (TMEM lanes of quadrant
// w % 4, columns of half w / 4) in a fixed order, sums each block's 63
// diagonals through a skewed shared-memory copy (row stride 33: the writes
// and the diagonal reads are conflict-free) into its own row of partial
// scores, and the eight rows are added in warp order.  Operands: per part
// (x hi, x lo, y hi, y lo) four 8-channel chunks of 256 rows of 16 bytes,
// K-major without swizzle (core matrices of 8 rows at 128 bytes, the next
// chunk 4096 bytes on).  The skew copies reuse the operands' space once the
// MMAs are done.  With kTop the CTA then takes the pair's top 8 and writes
// its centres, margin and window jobs (the learned step's proposal in one
// launch).
constexpr int kStWarps = 8;
constexpr int kStRows = 256;                       // rows of an operand (Lf padded with zeros)
constexpr int kStChunk = kStRows * 16;             // one 8-channel chunk (4096 bytes)
constexpr int kStOp = 4 * kStChunk;                // one part: 256 rows x 32 channels BF16
constexpr int kStPart = 512;                       // partial scores per warp (lag + 255)
constexpr int kStSkew = 32 * 33;                   // floats of a warp's skew copy
constexpr int kStSmem = 4 * kStOp + kStWarps * kStPart * 4 + 2 * kSpMaxLf * 4 + 16 + 16 + 128;
static_assert(kStWarps * kStSkew * 4 <= 4 * kStOp, "skew copies fit the operands' space");
static_assert(kSpMaxLf <= kStRows, "features fit an operand");
// kind::f16: D F32 (bit 4), A and B BF16 (bits 7, 10), both K-major, N = 256
// (N >> 3 at bits 17-22), M = 128 (M >> 4 at bits 24-28).
constexpr uint32_t kStIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(256 >> 3) << 17) |
                              ((uint32_t)(128 >> 4) << 24);

__device__ __forceinline__ void st_mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kStIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ uint32_t st_pack_bf16x2(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

// Ordering key of a bin: the score's bits mapped to an unsigned order (-0
// taken as +0), then 2 |l| + (l > 0) inverted, so that the larger key is the
// better bin of `better` (higher score, then smaller |l|, then negative l).
// Never 0 for a bin, so 0 marks "none".
__device__ __forceinline__ unsigned long long st_key(float s, int l) {
  uint32_t u = __float_as_uint(s == 0.f ? 0.f : s);
  u = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
  const uint32_t a = (uint32_t)(l < 0 ? -l : l);
  const uint32_t rank = 2u * a + (l > 0 ? 1u : 0u);
  return ((unsigned long long)u << 32) | (0xFFFFFFFFu - rank);
}
__device__ __forceinline__ float st_key_score(unsigned long long k) {
  const uint32_t u = (uint32_t)(k >> 32);
  return __uint_as_float((u & 0x80000000u) ? (u ^ 0x80000000u) : ~u);
}
__device__ __forceinline__ int st_key_lag(unsigned long long k) {
  const uint32_t rank = 0xFFFFFFFFu - (uint32_t)(k & 0xFFFFFFFFull);
  const int a = (int)(rank >> 1);
  return (rank & 1u) ? a : -a;
}

template <bool kTop>
__global__ void __launch_bounds__(kStWarps * 32, 2) k_scores_tc(const float* __restrict__ feat, int Lf,
                                                                const float* __restrict__ params,
                                                                float* __restrict__ scores, TopOut top,
                                                                uint32_t* __restrict__ status) {
  extern __shared__ uint8_t st_raw[];
  const uint32_t raw = smem_u32(st_raw);
  const uint32_t base = (raw + 127u) & ~127u;
  uint8_t* sb = st_raw + (base - raw);
  float* part = reinterpret_cast<float*>(sb + 4 * kStOp);           // [8][512]
  float* ss = part + kStWarps * kStPart;                              // kTop: [2 Lf - 1]
  const uint32_t bar = base + 4 * kStOp + kStWarps * kStPart * 4 + 2 * kSpMaxLf * 4;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sb + 4 * kStOp + kStWarps * kStPart * 4 + 2 * kSpMaxLf * 4 + 16);
  const int p = blockIdx.x, nb = 2 * Lf - 1;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float* gx = feat + (int64_t)(2 * p) * kCnnC * Lf;
  const float* gy = feat + (int64_t)(2 * p + 1) * kCnnC * Lf;
  // operands: item (signal, chunk c, row r) -> 8 channels split into hi, lo
  for (int it = threadIdx.x; it < 2 * 4 * kStRows; it += kStWarps * 32) {
    const int r = it & (kStRows - 1), c = (it >> 8) & 3, sg = it >> 10;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a;
    if (r < Lf) {
      const float4* src = reinterpret_cast<const float4*>((sg ? gy : gx) + (int64_t)r * kCnnC + 8 * c);
      a = __ldg(src);
      b = __ldg(src + 1);
    }
    const float f[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
    uint32_t h[4], l[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      h[e] = st_pack_bf16x2(f[2 * e], f[2 * e + 1]);
      const float h0 = __uint_as_float(h[e] << 16), h1 = __uint_as_float(h[e] & 0xFFFF0000u);
      l[e] = st_pack_bf16x2(f[2 * e] - h0, f[2 * e + 1] - h1);
    }
    const uint32_t off = (uint32_t)(c * kStChunk + r * 16);
    st_shared_v4(base + (uint32_t)((2 * sg) * kStOp) + off, h[0], h[1], h[2], h[3]);
    st_shared_v4(base + (uint32_t)((2 * sg + 1) * kStOp) + off, l[0], l[1], l[2], l[3]);
  }
  for (int i = threadIdx.x; i < kStWarps * kStPart; i += kStWarps * 32) part[i] = 0.f;
  if (kTop) {
    int32_t* cz = top.cbuf + (int64_t)p * kCnnTopK * kCnnWin;
    for (int i = threadIdx.x; i < kCnnTopK * kCnnWin; i += kStWarps * 32) cz[i] = 0;
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    mbar_init(bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  if (threadIdx.x == 0) {
    const uint32_t xh = base, xl = base + kStOp, yh = base + 2 * kStOp, yl = base + 3 * kStOp;
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
      const uint32_t d = tmem + 256u * (uint32_t)mt;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const uint32_t ko = (uint32_t)(2 * k * kStChunk), mo = (uint32_t)(mt * 128 * 16);
        const uint64_t ah = sdesc(xh + ko + mo, kStChunk, 128, 0, 0), al = sdesc(xl + ko + mo, kStChunk, 128, 0, 0);
        const uint64_t bh = sdesc(yh + ko, kStChunk, 128, 0, 0), bl = sdesc(yl + ko, kStChunk, 128, 0, 0);
        st_mma_bf16(d, ah, bh, k > 0 ? 1u : 0u);
        st_mma_bf16(d, ah, bl, 1u);
        st_mma_bf16(d, al, bh, 1u);
      }
    }
    mma_commit(bar);
  }
  const bool ok = __syncthreads_and(warp_wait(bar, 0));
  if (ok) {
    tc_fence_after();
    // each warp: its 8 blocks of 32 x 32 in a fixed order
    const int q = warp & 3, half = warp >> 2;
    float* S = reinterpret_cast<float*>(sb) + warp * kStSkew;
    float* pw = part + warp * kStPart;
#pragma unroll 1
    for (int mt = 0; mt < 2; ++mt) {
#pragma unroll 1
      for (int cb = 0; cb < 4; ++cb) {
        const int j0 = 128 * half + 32 * cb, i0 = 128 * mt + 32 * q;
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(256 * mt + j0), v);
#pragma unroll
        for (int c = 0; c < 32; ++c) S[lane * 33 + c] = __uint_as_float(v[c]);
        __syncwarp();
        // diagonals d1 = lane - 31 (rows 31 - lane .. 31) and d2 = lane + 1
        // (rows 0 .. 30 - lane), rows in ascending order
        float s1 = 0.f, s2 = 0.f;
#pragma unroll
        for (int r = 0; r < 32; ++r) {
          if (r >= 31 - lane) s1 += S[r * 33 + r + lane - 31];
          if (r <= 30 - lane) s2 += S[r * 33 + r + lane + 1];
        }
        pw[j0 - i0 + lane - 31 + 255] += s1;
        if (lane < 31) pw[j0 - i0 + lane + 1 + 255] += s2;
        __syncwarp();
      }
    }
  } else if (threadIdx.x == 0 && status) {
    atomicOr(status, TDE_ST_TIMEOUT);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
  const float alpha = params[kCnnAlpha];
  for (int b = threadIdx.x; b < nb; b += kStWarps * 32) {
    const int li = b - (Lf - 1) + 255;
    float t = 0.f;
#pragma unroll
    for (int w = 0; w < kStWarps; ++w) t += part[w * kStPart + li];
    scores[(int64_t)p * nb + b] = alpha * t;
    if (kTop) ss[b] = alpha * t;
  }
  if (kTop) {
    // softmax max and sum over the bins, then the top 8 as the largest keys
    // (st_key: score, then the lag order of `better`): each warp keeps the 8
    // best of its 64 bins, warp 0 takes the 8 best of those 64
    __shared__ float red_s[kStWarps];
    __shared__ unsigned long long cand_s[kStWarps * kCnnTopK];
    __syncthreads();
    const int b0 = threadIdx.x, b1 = threadIdx.x + kStWarps * 32;
    const float s0 = b0 < nb ? ss[b0] : -INFINITY, s1 = b1 < nb ? ss[b1] : -INFINITY;
    float mx = fmaxf(s0, s1);
    for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) red_s[warp] = mx;
    __syncthreads();
    mx = red_s[0];
#pragma unroll
    for (int w = 1; w < kStWarps; ++w) mx = fmaxf(mx, red_s[w]);
    float e = (b0 < nb ? __expf(s0 - mx) : 0.f) + (b1 < nb ? __expf(s1 - mx) : 0.f);
    for (int o = 16; o; o >>= 1) e += __shfl_xor_sync(0xffffffffu, e, o);
    __syncthreads();  // every thread has read red_s
    if (lane == 0) red_s[warp] = e;
    unsigned long long k0 = b0 < nb ? st_key(s0, b0 - (Lf - 1)) : 0ull;
    unsigned long long k1 = b1 < nb ? st_key(s1, b1 - (Lf - 1)) : 0ull;
#pragma unroll 1
    for (int r = 0; r < kCnnTopK; ++r) {
      unsigned long long bk = k0 > k1 ? k0 : k1;
      for (int o = 16; o; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, bk, o);
        bk = t > bk ? t : bk;
      }
      if (lane == 0) cand_s[warp * kCnnTopK + r] = bk;
      if (k0 == bk) k0 = 0ull;  // keys are distinct (one per lag)
      if (k1 == bk) k1 = 0ull;
    }
    __syncthreads();
    if (warp != 0) return;
    float sum = 0.f;
#pragma unroll
    for (int w = 0; w < kStWarps; ++w) sum += red_s[w];
    k0 = cand_s[lane], k1 = cand_s[lane + 32];
    float topm = 0.f;
    int32_t centre = 0;
#pragma unroll 1
    for (int r = 0; r < kCnnTopK; ++r) {
      unsigned long long bk = k0 > k1 ? k0 : k1;
      for (int o = 16; o; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, bk, o);
        bk = t > bk ? t : bk;
      }
      if (k0 == bk) k0 = 0ull;
      if (k1 == bk) k1 = 0ull;
      if (bk == 0ull) continue;  // fewer than 8 bins
      topm += __expf(st_key_score(bk) - mx);
      if (lane == r) centre = kCnnBin * st_key_lag(bk);
    }
    const float margin = topm / sum;
    const int64_t i = (int64_t)p * kCnnTopK + lane;
    const WinJob J = win_job_of(centre, top.n, top.cbuf + i * kCnnWin);
    if (lane < kCnnTopK) {
      top.centres[i] = centre;
      top.jobs[i] = J;
    }
    int64_t lo[kCnnTopK], hi[kCnnTopK];
#pragma unroll
    for (int w = 0; w < kCnnTopK; ++w) {
      lo[w] = __shfl_sync(0xffffffffu, J.lag_lo, w);
      hi[w] = __shfl_sync(0xffffffffu, J.lag_hi, w);
    }
    if (lane == 0) {
      int a[kCnnTopK], b[kCnnTopK];
      win_blocks(lo, hi, a, b);
      top.njobs[p] = win_jobs(a, b);
      top.margin[p] = margin;
    }
  }
}

// Any length: the bins are re-read from global memory every round.
__global__ void k_topk_any(const float* __restrict__ scores, int npairs, int Lf,
                           int32_t* __restrict__ centres, float* __restrict__ margin) {
  const int p = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (p >= npairs) return;
  const int nb = 2 * Lf - 1;
  const float* sc = scores + (int64_t)p * nb;
  float mx = -INFINITY;
  for (int b = lane; b < nb; b += 32) mx = fmaxf(mx, sc[b]);
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  float sum = 0.f;
  for (int b = lane; b < nb; b += 32) sum += __expf(sc[b] - mx);
  for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  float top = 0.f;
  int taken[kCnnTopK];
  for (int r = 0; r < kCnnTopK; ++r) {
    float bs = -INFINITY;
    int bl = 1 << 30;
    for (int b = lane; b < nb; b += 32) {
      const int l = b - (Lf - 1);
      bool used = false;
      for (int t = 0; t < r; ++t) used |= taken[t] == l;
      if (!used && (bl == (1 << 30) || better(sc[b], l, bs, bl))) {
        bs = sc[b];
        bl = l;
      }
    }
    for (int o = 16; o; o >>= 1) {
      const float os = __shfl_xor_sync(0xffffffffu, bs, o);
      const int ol = __shfl_xor_sync(0xffffffffu, bl, o);
      if (ol != (1 << 30) && (bl == (1 << 30) || better(os, ol, bs, bl))) {
        bs = os;
        bl = ol;
      }
    }
    taken[r] = bl;
    top += __expf(bs - mx);
    if (lane == 0) centres[(int64_t)p * kCnnTopK + r] = kCnnBin * bl;
  }
  if (lane == 0) margin[p] = top / sum;
}

// One warp per pair: softmax, top-8 bins, margin.  Each lane keeps its bins'
// scores in registers (bins lane, lane + 32, ...); a taken bin is marked by a
// flag bit, so every round is a register scan plus one warp reduction.
constexpr int kTopPer = 32;  // bins per lane held in registers (nb <= 1024)

template <int PER>  // bins per lane (nb <= 32 PER)
__global__ void k_topk(const float* __restrict__ scores, int npairs, int Lf,
                       int32_t* __restrict__ centres, float* __restrict__ margin) {
  const int p = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (p >= npairs) return;
  const int nb = 2 * Lf - 1;
  const float* sc = scores + (int64_t)p * nb;
  float v[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int b = lane + 32 * i;
    v[i] = b < nb ? sc[b] : -INFINITY;
  }
  int32_t centre;
  float mg;
  topk_warp(v, nb, Lf, lane, centre, mg);
  if (lane < kCnnTopK) centres[(int64_t)p * kCnnTopK + lane] = centre;
  if (lane == 0) margin[p] = mg;
}

// ---------------------------------------------------------------- training

__global__ void k_softmax_ce(const float* __restrict__ scores, const int64_t* __restrict__ labels,
                             int npairs, int Lf, float* __restrict__ loss,
                             float* __restrict__ dscores) {
  const int p = blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  const int lane = threadIdx.x & 31;
  if (p >= npairs) return;
  const int nb = 2 * Lf - 1;
  const float* sc = scores + (int64_t)p * nb;
  // label bin: the window [256 l - 128, 256 l + 128] holding the lag
  int64_t l = labels[p] + kCnnBin / 2;
  l = l >= 0 ? l / kCnnBin : -((-l + kCnnBin - 1) / kCnnBin);
  if (l < -(Lf - 1)) l = -(Lf - 1);
  if (l > Lf - 1) l = Lf - 1;
  const int t = (int)l + Lf - 1;
  float mx = -INFINITY;
  for (int b = lane; b < nb; b += 32) mx = fmaxf(mx, sc[b]);
  for (int o = 16; o; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  float sum = 0.f;
  for (int b = lane; b < nb; b += 32) sum += expf(sc[b] - mx);
  for (int o = 16; o; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
  const float inv = 1.f / sum, scale = 1.f / (float)npairs;
  for (int b = lane; b < nb; b += 32)
    dscores[(int64_t)p * nb + b] = (expf(sc[b] - mx) * inv - (b == t ? 1.f : 0.f)) * scale;
  if (lane == 0) loss[p] = logf(sum) + mx - sc[t];
}

// d features of one pair; d alpha partial = sum_b dS[b] * score[b] / alpha.
__global__ void __launch_bounds__(kThreads) k_scores_bwd(const float* __restrict__ feat,
                                                         const float* __restrict__ dscores,
                                                         int Lf, const float* __restrict__ params,
                                                         float* __restrict__ dfeat,
                                                         float* __restrict__ dalpha_pp) {
  extern __shared__ float sm[];
  const int nb = 2 * Lf - 1;
  float* fx = sm;                  // [32][3 Lf] padded
  float* fy = sm + kCnnC * 3 * Lf; // [32][3 Lf] padded
  float* ds = fy + kCnnC * 3 * Lf; // [nb]
  __shared__ float red[kThreads / 32];
  const int p = blockIdx.x;
  const float* gx = feat + (int64_t)(2 * p) * kCnnC * Lf;
  const float* gy = feat + (int64_t)(2 * p + 1) * kCnnC * Lf;
  for (int i = threadIdx.x; i < kCnnC * 3 * Lf; i += kThreads) {
    const int c = i / (3 * Lf), j = i % (3 * Lf) - Lf;
    fx[i] = (j >= 0 && j < Lf) ? gx[c * Lf + j] : 0.f;
    fy[i] = (j >= 0 && j < Lf) ? gy[c * Lf + j] : 0.f;
  }
  for (int b = threadIdx.x; b < nb; b += kThreads) ds[b] = dscores[(int64_t)p * nb + b];
  __syncthreads();
  const float alpha = params[kCnnAlpha];
  float* dx = dfeat + (int64_t)(2 * p) * kCnnC * Lf;
  float* dy = dfeat + (int64_t)(2 * p + 1) * kCnnC * Lf;
  // dfx[c][i] = alpha sum_l dS[l] fy[c][i + l];  dfy[c][j] = alpha sum_l dS[l] fx[c][j - l]
  float da = 0.f;
  for (int e = threadIdx.x; e < kCnnC * Lf; e += kThreads) {
    const int c = e / Lf, i = e % Lf;
    const float* yrow = fy + c * 3 * Lf + Lf + i - (Lf - 1);   // index by b: fy[i + l]
    const float* xrow = fx + c * 3 * Lf + Lf + i + (Lf - 1);   // fx[i - l] = xrow[-b]
    float ax = 0.f, ay = 0.f;
    for (int b = 0; b < nb; ++b) {
      ax = fmaf(ds[b], yrow[b], ax);
      ay = fmaf(ds[b], xrow[-b], ay);
    }
    dx[e] = alpha * ax;
    dy[e] = alpha * ay;
    // sum_b dS[b] raw[b] = sum_c sum_i fx[c][i] * (sum_b dS[b] fy[c][i + l_b])
    da = fmaf(fx[c * 3 * Lf + Lf + i], ax, da);
  }
  for (int o = 16; o; o >>= 1) da += __shfl_xor_sync(0xffffffffu, da, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = da;
  __syncthreads();
  if (threadIdx.x == 0) {
    float t = 0.f;
    for (int w = 0; w < kThreads / 32; ++w) t += red[w];
    dalpha_pp[p] = t;
  }
}

__global__ void k_pool_relu_bwd(const float* __restrict__ pre, const float* __restrict__ dout,
                                int64_t total_out, float* __restrict__ dz) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total_out;
       i += (int64_t)gridDim.x * blockDim.x) {
    const float a0 = pre[2 * i], a1 = pre[2 * i + 1];
    const float g = dout[i];
    const bool second = a1 > a0;
    const float gm = (second ? a1 : a0) > 0.f ? g : 0.f;
    dz[2 * i] = second ? 0.f : gm;
    dz[2 * i + 1] = second ? gm : 0.f;
  }
}

// din[ci][p] = sum_co sum_k dz[co][p + 4 - k] W[co][ci][k]  (32 -> 32 layers)
__global__ void __launch_bounds__(kThreads) k_conv_dgrad(const float* __restrict__ dz, int L,
                                                         const uint16_t* __restrict__ wbf,
                                                         float* __restrict__ din) {
  extern __shared__ float csm[];
  float (*dz_s)[kT + 8] = reinterpret_cast<float (*)[kT + 8]>(csm);                  // [co][kT+8]
  float (*w_s)[kCnnC] = reinterpret_cast<float (*)[kCnnC]>(csm + kCnnC * (kT + 8));  // [co*9+k][ci]
  const int s = blockIdx.y, p0 = blockIdx.x * kT;
  const float* src = dz + (int64_t)s * kCnnC * L;
  for (int idx = threadIdx.x; idx < kCnnC * (kT + 8); idx += kThreads) {
    const int co = idx / (kT + 8), j = idx % (kT + 8);
    const int pos = p0 - 4 + j;
    dz_s[co][j] = (pos >= 0 && pos < L) ? src[(int64_t)co * L + pos] : 0.f;
  }
  for (int idx = threadIdx.x; idx < kCnnC * kCnnC * kCnnK; idx += kThreads) {
    const int co = idx / (kCnnC * kCnnK), r = idx % (kCnnC * kCnnK);
    const int ci = r / kCnnK, k = r % kCnnK;
    w_s[co * kCnnK + k][ci] = bf16_to_f(wbf[idx]);
  }
  __syncthreads();
  const int ci = threadIdx.x & 31, pg = threadIdx.x >> 5;
  float acc[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) acc[j] = 0.f;
  for (int co = 0; co < kCnnC; ++co) {
    float g[24];
#pragma unroll
    for (int j = 0; j < 24; ++j) g[j] = dz_s[co][pg * 16 + j];
#pragma unroll
    for (int k = 0; k < kCnnK; ++k) {
      const float w = w_s[co * kCnnK + k][ci];
      // dz[p + 4 - k] sits at dz_s[.][p - p0 + 8 - k]
#pragma unroll
      for (int j = 0; j < 16; ++j) acc[j] = fmaf(w, g[j + 8 - k], acc[j]);
    }
  }
  float* dst = din + ((int64_t)s * kCnnC + ci) * L + p0 + pg * 16;
#pragma unroll
  for (int j = 0; j < 16; j += 4)
    *reinterpret_cast<float4*>(dst + j) = make_float4(acc[j], acc[j + 1], acc[j + 2], acc[j + 3]);
}

// Per-signal partials: dW[co][ci][k] = sum_p dz[co][p] in[ci][p + k - 4],
// db[co] = sum_p dz[co][p].  One CTA per signal.
template <int CIN>
__global__ void __launch_bounds__(kThreads) k_conv_wgrad(const float* __restrict__ dz,
                                                         const float* __restrict__ in, int L,
                                                         float* __restrict__ partial) {
  __shared__ float dz_s[kCnnC][kT];
  __shared__ float in_s[CIN][kT + 8];
  constexpr int kOut = kCnnC * CIN * kCnnK;
  constexpr int kPer = (kOut + kThreads - 1) / kThreads;
  const int s = blockIdx.x;
  const float* gz = dz + (int64_t)s * kCnnC * L;
  const float* gi = in + (int64_t)s * CIN * L;
  float acc[kPer];
#pragma unroll
  for (int r = 0; r < kPer; ++r) acc[r] = 0.f;
  float accb = 0.f;
  for (int p0 = 0; p0 < L; p0 += kT) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < kCnnC * kT; idx += kThreads)
      dz_s[idx / kT][idx % kT] = gz[(int64_t)(idx / kT) * L + p0 + idx % kT];
    for (int idx = threadIdx.x; idx < CIN * (kT + 8); idx += kThreads) {
      const int ci = idx / (kT + 8), j = idx % (kT + 8);
      const int pos = p0 - 4 + j;
      in_s[ci][j] = (pos >= 0 && pos < L) ? gi[(int64_t)ci * L + pos] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int o = threadIdx.x + r * kThreads;
      if (o < kOut) {
        const int co = o / (CIN * kCnnK), ci = (o / kCnnK) % CIN, k = o % kCnnK;
        float a = acc[r];
        for (int p = 0; p < kT; ++p) a = fmaf(dz_s[co][p], in_s[ci][p + k], a);
        acc[r] = a;
      }
    }
    if (threadIdx.x < kCnnC)
      for (int p = 0; p < kT; ++p) accb += dz_s[threadIdx.x][p];
  }
  float* dst = partial + (int64_t)s * (kOut + kCnnC);
#pragma unroll
  for (int r = 0; r < kPer; ++r) {
    const int o = threadIdx.x + r * kThreads;
    if (o < kOut) dst[o] = acc[r];
  }
  if (threadIdx.x < kCnnC) dst[kOut + threadIdx.x] = accb;
}

__global__ void k_reduce(const float* __restrict__ partial, int nsig, int count,
                         float* __restrict__ grad) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= count) return;
  float a = 0.f;
  for (int s = 0; s < nsig; ++s) a += partial[(int64_t)s * count + i];
  grad[i] = a;
}

__global__ void k_adamw(float* __restrict__ params, const float* __restrict__ grad,
                        float* __restrict__ m, float* __restrict__ v, uint16_t* __restrict__ wbf,
                        float c1, float c2, float lr, float beta1, float beta2, float eps,
                        float wd) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kCnnParams) return;
  const float g = grad[i];
  const float mi = beta1 * m[i] + (1.f - beta1) * g;
  const float vi = beta2 * v[i] + (1.f - beta2) * g * g;
  m[i] = mi;
  v[i] = vi;
  // decoupled weight decay on conv weights only (not biases or alpha)
  bool is_w = false;
  for (int l = 0; l < kCnnLayers; ++l) is_w |= (i >= cnn_woff(l) && i < cnn_boff(l));
  float p = params[i];
  p -= lr * ((mi / c1) / (sqrtf(vi / c2) + eps) + (is_w ? wd * p : 0.f));
  params[i] = p;
  wbf[i] = f_to_bf16(p);
}

__global__ void k_to_bf16(const float* __restrict__ params, uint16_t* __restrict__ wbf) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < kCnnParams) wbf[i] = f_to_bf16(params[i]);
}

// ------------------------------------------------ argmax over the windows

__device__ __forceinline__ unsigned long long pack_key(int32_t v, int64_t tau) {
  const uint64_t a = (uint64_t)(tau < 0 ? -tau : tau);
  const uint32_t rank = (uint32_t)(2 * a + (tau > 0 ? 1 : 0));
  return ((unsigned long long)((uint32_t)v ^ 0x80000000u) << 32) | (0xFFFFFFFFu - rank);
}

// The pair's 8 window descriptors are staged in shared memory first, so that
// every thread's loads of window values are independent (flat index f over
// the 8 x 257 slots: window f / 257, lag lag_lo + f % 257 when inside it).
__global__ void __launch_bounds__(kThreads) k_window_argmax(const WinJob* __restrict__ jobs,
                                                            int64_t* __restrict__ lag,
                                                            int64_t* __restrict__ val) {
  __shared__ unsigned long long red[kThreads / 32];
  __shared__ WinJob js[kCnnTopK];
  const int p = blockIdx.x;
  if (threadIdx.x < kCnnTopK) js[threadIdx.x] = jobs[(int64_t)p * kCnnTopK + threadIdx.x];
  __syncthreads();
  constexpr int kPer = (kCnnTopK * kCnnWin + kThreads - 1) / kThreads;
  int32_t v[kPer];
  int64_t tau[kPer];
  bool in[kPer];
#pragma unroll
  for (int r = 0; r < kPer; ++r) {
    const int f = threadIdx.x + r * kThreads, w = f / kCnnWin, i = f - w * kCnnWin;
    in[r] = false;
    if (w < kCnnTopK) {
      const WinJob& J = js[w];
      in[r] = i <= J.lag_hi - J.lag_lo;
      tau[r] = J.lag_lo + i;
      if (in[r]) v[r] = J.c[i];
    }
  }
  unsigned long long best = 0;
#pragma unroll
  for (int r = 0; r < kPer; ++r)
    if (in[r]) {
      const unsigned long long k = pack_key(v[r], tau[r]);
      best = k > best ? k : best;
    }
  for (int o = 16; o; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, best, o);
    best = t > best ? t : best;
  }
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = best;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kThreads / 32; ++w) best = red[w] > best ? red[w] : best;
    best = red[0] > best ? red[0] : best;
    const uint64_t rank = 0xFFFFFFFFull - (best & 0xFFFFFFFFull);
    const int64_t a = (int64_t)(rank >> 1);
    lag[p] = (rank & 1) ? a : -a;
    val[p] = (int64_t)(int32_t)((uint32_t)(best >> 32) ^ 0x80000000u);
  }
}

unsigned grid1(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (unsigned)(g < 1 ? 1 : (g > 65535 ? 65535 : g));
}

}  // namespace

cudaError_t launch_cnn_decimate(const int8_t* q, int64_t n, int nsig, float* d, cudaStream_t st) {
  k_decimate<<<grid1((int64_t)nsig * n / kCnnDec), 256, 0, st>>>(q, n, nsig, d);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

constexpr int conv_smem(int cin) { return (cin * (kT + 8) + cin * kCnnK * kCnnC) * 4; }
constexpr int fwd_smem(int cin) { return (cin * (kTP + 8) + cin * kCnnK * kCnnC) * 4; }

cudaError_t launch_cnn_layer(const CnnLayerIO& io, int l, int nsig, const uint16_t* wbf,
                             const float* params, cudaStream_t st) {
  dim3 grid((io.L + kTP - 1) / kTP, nsig);
  if (l == 0) {
    k_conv_fwd<1><<<grid, kThreads, fwd_smem(1), st>>>(io.in, io.pre, io.out, io.L,
                                                       wbf + cnn_woff(0), params + cnn_boff(0));
  } else if (io.pre == nullptr && io.L % 16 == 0) {
    // inference: tensor cores, BF16 activations
    const int smem = ((kTP + 8) * kXR + kCnnK * kCnnC * kXR) * 2;
    cudaFuncSetAttribute(k_conv_fwd_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    k_conv_fwd_tc<<<grid, kThreads, smem, st>>>(io.in, io.out, io.L, wbf + cnn_woff(l),
                                                params + cnn_boff(l));
  } else {
    cudaFuncSetAttribute(k_conv_fwd<kCnnC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         fwd_smem(kCnnC));
    k_conv_fwd<kCnnC><<<grid, kThreads, fwd_smem(kCnnC), st>>>(
        io.in, io.pre, io.out, io.L, wbf + cnn_woff(l), params + cnn_boff(l));
  }
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_cnn_infer(const int8_t* q, int64_t n, int nsig, const uint16_t* wbf,
                             const float* params, uint16_t* const act[kCnnLayers - 1], float* feat,
                             uint8_t* qe, uint32_t* d_status, cudaStream_t st) {
  const int Ld = (int)(n / kCnnDec);
  if (Ld % 128 != 0) return cudaErrorInvalidValue;  // every layer's length a multiple of 16
  // layers 1 and 2 in one kernel (layer 2's input stays on chip; act[0] is
  // not used), then layers 3 and 4
  cudaError_t e = launch_cnn_conv12_tc(q, n, nsig, wbf + cnn_woff(0), params + cnn_boff(0), wbf + cnn_woff(1),
                                       params + cnn_boff(1), act[1], qe, d_status, st);
  for (int l = 2; l < kCnnLayers && e == cudaSuccess; ++l) {
    const bool last = l == kCnnLayers - 1;
    e = launch_cnn_conv_tc(act[l - 1], last ? static_cast<void*>(feat) : static_cast<void*>(act[l]),
                           Ld >> l, nsig, wbf + cnn_woff(l), params + cnn_boff(l), last, d_status, st);
  }
  return e;
}

cudaError_t launch_cnn_scores(const float* feat, int npairs, int Lf, const float* params,
                              float* scores, cudaStream_t st, bool pos_major, uint32_t* status) {
  if (Lf < 1 || npairs <= 0) return npairs <= 0 ? cudaSuccess : cudaErrorInvalidValue;
  if (pos_major && Lf <= kSpMaxLf) {  // inference: the tensor cores
    cudaFuncSetAttribute(k_scores_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStSmem);
    k_scores_tc<false><<<npairs, kStWarps * 32, kStSmem, st>>>(feat, Lf, params, scores, TopOut{}, status);
    TDE_COUNT_LAUNCH(1);
    return cudaGetLastError();
  }
  if (Lf <= kSpMaxLf) {
    cudaFuncSetAttribute(k_scores_pair<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kSpSmem);
    k_scores_pair<false><<<npairs, kSpWarps * 32, kSpSmem, st>>>(feat, Lf, params, scores);
    TDE_COUNT_LAUNCH(1);
    return cudaGetLastError();
  }
  auto kern = pos_major ? k_scores<true> : k_scores<false>;
  cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kScSmem);
  const int nb = 2 * Lf - 1;
  kern<<<dim3((nb + kScBins - 1) / kScBins, npairs), kScWarps * 32, kScSmem, st>>>(feat, Lf, params, scores);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_cnn_scores_propose(const float* feat, int npairs, int Lf, const float* params,
                                      float* scores, int32_t* centres, float* margin, WinJob* jobs,
                                      int32_t* cbuf, int64_t n, int32_t* njobs, cudaStream_t st,
                                      uint32_t* status) {
  if (npairs <= 0) return cudaSuccess;
  if (Lf < 1 || Lf > kSpMaxLf) return cudaErrorNotSupported;
  cudaFuncSetAttribute(k_scores_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kStSmem);
  k_scores_tc<true><<<npairs, kStWarps * 32, kStSmem, st>>>(
      feat, Lf, params, scores, TopOut{centres, margin, jobs, cbuf, n, njobs}, status);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_cnn_topk(const float* scores, int npairs, int Lf, int32_t* centres,
                            float* margin, cudaStream_t st) {
  if (2 * Lf - 1 > 32 * kTopPer)
    k_topk_any<<<(npairs + 3) / 4, 128, 0, st>>>(scores, npairs, Lf, centres, margin);
  else if (2 * Lf - 1 <= 32 * 16)
    k_topk<16><<<(npairs + 1) / 2, 64, 0, st>>>(scores, npairs, Lf, centres, margin);
  else
    k_topk<kTopPer><<<(npairs + 1) / 2, 64, 0, st>>>(scores, npairs, Lf, centres, margin);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_cnn_softmax_ce(const float* scores, const int64_t* labels, int npairs, int Lf,
                                  float* loss, float* dscores, cudaStream_t st) {
  k_softmax_ce<<<(npairs + 3) / 4, 128, 0, st>>>(scores, labels, npairs, Lf, loss, dscores);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_cnn_scores_bwd(const float* feat, const float* dscores, int npairs, int Lf,
                                  const float* params, float* dfeat, float* dalpha_pp,
                                  cudaStream_t st) {
  const int smem = (2 * kCnnC * 3 * Lf + 2 * Lf) * 4;
  cudaFuncSetAttribute(k_scores_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  k_scores_bwd<<<npairs, kThreads, smem, st>>>(feat, dscores, Lf, params, dfeat, dalpha_pp);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_cnn_pool_relu_bwd(const float* pre, const float* dout, int nsig, int L,
                                     float* dz, cudaStream_t st) {
  const int64_t total = (int64_t)nsig * kCnnC * (L / 2);
  k_pool_relu_bwd<<<grid1(total), 256, 0, st>>>(pre, dout, total, dz);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_cnn_dgrad(const float* dz, int nsig, int L, int l, const uint16_t* wbf,
                             float* din, cudaStream_t st) {
  cudaFuncSetAttribute(k_conv_dgrad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       conv_smem(kCnnC));
  k_conv_dgrad<<<dim3(L / kT, nsig), kThreads, conv_smem(kCnnC), st>>>(dz, L, wbf + cnn_woff(l),
                                                                        din);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_cnn_wgrad(const float* dz, const float* in, int nsig, int L, int l,
                             float* partial, cudaStream_t st) {
  if (l == 0)
    k_conv_wgrad<1><<<nsig, kThreads, 0, st>>>(dz, in, L, partial);
  else
    k_conv_wgrad<kCnnC><<<nsig, kThreads, 0, st>>>(dz, in, L, partial);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_cnn_reduce(const float* partial, int nsig, int count, float* grad,
                              cudaStream_t st) {
  k_reduce<<<(count + 255) / 256, 256, 0, st>>>(partial, nsig, count, grad);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_cnn_adamw(float* params, const float* grad, float* m, float* v, uint16_t* wbf,
                             int64_t step, float lr, float beta1, float beta2, float eps,
                             float wd, cudaStream_t st) {
  const float c1 = 1.f - powf(beta1, (float)step), c2 = 1.f - powf(beta2, (float)step);
  k_adamw<<<(kCnnParams + 255) / 256, 256, 0, st>>>(params, grad, m, v, wbf, c1, c2, lr, beta1,
                                                    beta2, eps, wd);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_cnn_to_bf16(const float* params, uint16_t* wbf, cudaStream_t st) {
  k_to_bf16<<<(kCnnParams + 255) / 256, 256, 0, st>>>(params, wbf);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_window_argmax(const WinJob* d_jobs, int npairs, int64_t* lag, int64_t* val,
                                 cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  k_window_argmax<<<npairs, kThreads, 0, st>>>(d_jobs, lag, val);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}
