// quantize.cu -- Algorithm 1's quantization step (arXiv 2509.19974, Sec. 3.2): the
// monotone integer maps phi, psi with phi(0) = psi(0) = 0.
//
//  bits = 1: q = sign(x), sign(0) = 0 (the quantizer of Sec. 4.2).  One pass.
//  bits = 2, 4: sign-magnitude rank quantizer, L = 2^bits - 1 levels.  The
//    thresholds t_m are order statistics of |x| (ranks floor((2m-1) n / L),
//    clamped to n-1).  They are found exactly by a radix select on the FP32
//    bit patterns of |x| (for finite non-negative floats the unsigned bit
//    pattern orders like the value; -0.0 maps to +0.0): three histogram passes
//    over digits of 11, 11 and 9 bits, each followed by a one-block select.
//    q = sign(x) * #{m : |x| >= t_m} is then one elementwise pass.
// All passes are HBM-streaming; the batch dimension is blockIdx.y.
#include "common.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kBins = 2048;

__device__ __forceinline__ uint32_t abs_bits(float v) { return __float_as_uint(v) & 0x7FFFFFFFu; }
__device__ __forceinline__ int sign_of(float v) { return (v > 0.0f) - (v < 0.0f); }

__global__ void __launch_bounds__(kThreads) k_sign(const QSig* __restrict__ sigs,
                                                   uint32_t* __restrict__ status) {
  const QSig s = sigs[blockIdx.y];
  int bad = 0;
  const int64_t stride = (int64_t)gridDim.x * kThreads * 4;
  // Four samples per thread per step; scalar loads keep any alignment legal.
  for (int64_t i0 = ((int64_t)blockIdx.x * kThreads + threadIdx.x) * 4; i0 < s.n; i0 += stride) {
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      int64_t i = i0 + k;
      if (i < s.n) {
        float v = s.x[i];
        bad |= abs_bits(v) >= 0x7F800000u;
        s.q[i] = (int8_t)sign_of(v);
      }
    }
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, TDE_ST_NONFINITE);
}

// Ranks of the thresholds: r_m = min(n-1, floor((2m-1) n / L)), m = 1..M.
__global__ void k_rank_init(const QSig* __restrict__ sigs, RankState* __restrict__ state, int M,
                            int L) {
  const int sig = blockIdx.x;
  if (threadIdx.x < 7) {
    int m = threadIdx.x;
    int64_t n = sigs[sig].n;
    uint32_t r = 0;
    if (m < M) {
      int64_t idx = ((2 * (int64_t)(m + 1) - 1) * n) / L;
      r = (uint32_t)(idx > n - 1 ? n - 1 : idx);
    }
    state[sig].rank[m] = r;
    state[sig].prefix[m] = 0;
  }
}

// Histogram of one digit of |x| over the elements whose higher bits equal the
// prefix found so far, one histogram per threshold (pass 0 shares one).
template <int PASS>
__global__ void __launch_bounds__(kThreads) k_rank_hist(const QSig* __restrict__ sigs,
                                                        const RankState* __restrict__ state,
                                                        uint32_t* __restrict__ hist, int M,
                                                        uint32_t* __restrict__ status) {
  extern __shared__ uint32_t sh[];
  constexpr int kShift = PASS == 0 ? 20 : (PASS == 1 ? 9 : 0);
  constexpr uint32_t kMask = PASS == 2 ? 511u : 2047u;
  constexpr int kHiShift = PASS == 1 ? 20 : 9;  // bits above the digit (PASS > 0)
  const int sig = blockIdx.y;
  const QSig s = sigs[sig];
  const int hcount = PASS == 0 ? 1 : M;
  for (int i = threadIdx.x; i < hcount * kBins; i += kThreads) sh[i] = 0;
  uint32_t pre[7];
#pragma unroll
  for (int m = 0; m < 7; ++m) pre[m] = state[sig].prefix[m];
  __syncthreads();
  int bad = 0;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < s.n; i += stride) {
    uint32_t u = abs_bits(s.x[i]);
    if (PASS == 0) {
      bad |= u >= 0x7F800000u;
      atomicAdd(&sh[u >> kShift], 1u);
    } else {
      uint32_t hi = u >> kHiShift;
      uint32_t d = (u >> kShift) & kMask;
#pragma unroll
      for (int m = 0; m < 7; ++m)
        if (m < M && hi == pre[m]) atomicAdd(&sh[m * kBins + d], 1u);
    }
  }
  __syncthreads();
  uint32_t* gh = hist + (size_t)sig * 7 * kBins;
  for (int i = threadIdx.x; i < hcount * kBins; i += kThreads)
    if (sh[i]) atomicAdd(&gh[i], sh[i]);
  if (PASS == 0 && __syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, TDE_ST_NONFINITE);
}

// Block-wide exclusive scan of one value per thread (kThreads threads).
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* warp_tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) warp_tot[warp] = incl;
  __syncthreads();
  uint32_t base = 0;
  for (int w = 0; w < warp; ++w) base += warp_tot[w];
  __syncthreads();
  return base + incl - v;
}

// Finds, for every threshold, the bin holding its residual rank; appends the
// bin to the prefix, subtracts the elements below it, and clears the
// histogram for the next pass.
template <int PASS>
__global__ void __launch_bounds__(kThreads) k_rank_select(RankState* __restrict__ state,
                                                          uint32_t* __restrict__ hist, int M) {
  __shared__ uint32_t warp_tot[kThreads / 32];
  constexpr int kNBins = PASS == 2 ? 512 : 2048;
  constexpr int kPer = kNBins / kThreads;  // bins per thread
  constexpr int kWidth = PASS == 2 ? 9 : 11;
  const int sig = blockIdx.x;
  uint32_t* gh = hist + (size_t)sig * 7 * kBins;
  for (int m = 0; m < M; ++m) {
    const uint32_t* h = gh + (PASS == 0 ? 0 : m) * kBins;
    // Every thread reads the residual rank before the scan's barriers: the
    // one thread whose bins hold it rewrites it after them.
    const uint32_t r = state[sig].rank[m];
    uint32_t cnt[kPer];
    uint32_t local = 0;
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
      cnt[k] = h[threadIdx.x * kPer + k];
      local += cnt[k];
    }
    uint32_t before = block_exclusive_scan(local, warp_tot);
    if (r >= before && r < before + local) {
      uint32_t acc = before;
#pragma unroll
      for (int k = 0; k < kPer; ++k) {
        if (r >= acc && r < acc + cnt[k]) {
          uint32_t bin = threadIdx.x * kPer + k;
          state[sig].prefix[m] = (state[sig].prefix[m] << kWidth) | bin;
          state[sig].rank[m] = r - acc;
        }
        acc += cnt[k];
      }
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < 7 * kBins; i += kThreads) gh[i] = 0;
}

__global__ void __launch_bounds__(kThreads) k_rank_apply(const QSig* __restrict__ sigs,
                                                         const RankState* __restrict__ state,
                                                         int M) {
  const int sig = blockIdx.y;
  const QSig s = sigs[sig];
  uint32_t t[7];
#pragma unroll
  for (int m = 0; m < 7; ++m) t[m] = m < M ? state[sig].prefix[m] : 0xFFFFFFFFu;
  const int64_t stride = (int64_t)gridDim.x * kThreads;
  for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < s.n; i += stride) {
    float v = s.x[i];
    uint32_t u = abs_bits(v);
    int level = 0;
#pragma unroll
    for (int m = 0; m < 7; ++m) level += (u >= t[m]) ? 1 : 0;
    s.q[i] = (int8_t)(sign_of(v) * level);
  }
}

int grid_x_for(int64_t max_n, int per_block) {
  int64_t g = ceil_div64(max_n, per_block);
  if (g < 1) g = 1;
  if (g > 1184) g = 1184;  // 8 CTAs per SM on 148-152 SMs; grid-stride beyond
  return (int)g;
}

}  // namespace

cudaError_t launch_quantize_sign(const QSig* d_sigs, int nsig, int64_t max_n, uint32_t* d_status,
                                 cudaStream_t st) {
  dim3 grid(grid_x_for(max_n, kThreads * 4), nsig);
  k_sign<<<grid, kThreads, 0, st>>>(d_sigs, d_status);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_quantize_rank(const QSig* d_sigs, int nsig, int64_t max_n, int bits,
                                 RankState* d_state, uint32_t* d_hist, uint32_t* d_status,
                                 cudaStream_t st) {
  const int M = (1 << (bits - 1)) - 1;
  const int L = (1 << bits) - 1;
  cudaFuncSetAttribute(k_rank_hist<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 7 * kBins * 4);
  cudaFuncSetAttribute(k_rank_hist<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, 7 * kBins * 4);
  cudaError_t e = cudaMemsetAsync(d_hist, 0, (size_t)nsig * 7 * kBins * 4, st);
  if (e != cudaSuccess) return e;
  k_rank_init<<<nsig, 32, 0, st>>>(d_sigs, d_state, M, L);
  TDE_COUNT_LAUNCH(1);
  dim3 grid(grid_x_for(max_n, kThreads * 16), nsig);
  k_rank_hist<0><<<grid, kThreads, kBins * 4, st>>>(d_sigs, d_state, d_hist, M, d_status);
  TDE_COUNT_LAUNCH(1);
  k_rank_select<0><<<nsig, kThreads, 0, st>>>(d_state, d_hist, M);
  TDE_COUNT_LAUNCH(1);
  k_rank_hist<1><<<grid, kThreads, M * kBins * 4, st>>>(d_sigs, d_state, d_hist, M, d_status);
  TDE_COUNT_LAUNCH(1);
  k_rank_select<1><<<nsig, kThreads, 0, st>>>(d_state, d_hist, M);
  TDE_COUNT_LAUNCH(1);
  k_rank_hist<2><<<grid, kThreads, M * kBins * 4, st>>>(d_sigs, d_state, d_hist, M, d_status);
  TDE_COUNT_LAUNCH(1);
  k_rank_select<2><<<nsig, kThreads, 0, st>>>(d_state, d_hist, M);
  TDE_COUNT_LAUNCH(1);
  dim3 grid_a(grid_x_for(max_n, kThreads * 4), nsig);
  k_rank_apply<<<grid_a, kThreads, 0, st>>>(d_sigs, d_state, M);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}
