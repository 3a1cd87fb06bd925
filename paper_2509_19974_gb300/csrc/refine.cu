// refine.cu -- the last steps of Algorithm 1 (arXiv 2509.19974, Sec. 3.3):
// the set of lags where the integer correlation is maximal and, when it holds
// several, its subset where the real cross-correlation (x * y)[tau] of the
// original FP32 signals (Eq. (1) without quantization) is maximal; plus a
// parabolic sub-sample offset of the real cross-correlation at the set's
// representative (smallest |tau|, then tau).
//
//   k_ref_collect  the lags whose correlation equals the maximum (device list);
//   k_ref_dots     the real cross-correlation at each listed lag: FP64 sums of
//                  the exact FP32 x FP32 products, one CTA per lag, a fixed
//                  reduction order (deterministic);
//   k_ref_pick     one CTA: the maximum over the list, the re-ranked set's
//                  bounds, size and representative, the neighbours' values
//                  and the parabola's vertex.
#include "refine.cuh"

namespace {

constexpr int kRT = 256;

// FP64 block sum (kRT threads); the result is valid in every thread.
__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();  // sh reusable
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double t = 0.0;
#pragma unroll
  for (int w = 0; w < kRT / 32; ++w) t += sh[w];
  return t;
}

// (x * y)[tau] over the overlap, FP64, in a fixed order.
__device__ double real_ccf(const float* __restrict__ x, int64_t nx, const float* __restrict__ y,
                           int64_t ny, int64_t tau, double* sh) {
  const int64_t lo = tau < 0 ? -tau : 0;
  const int64_t hi = nx < ny - tau ? nx : ny - tau;
  double acc = 0.0;
  for (int64_t n = lo + threadIdx.x; n < hi; n += kRT) acc = fma((double)x[n], (double)y[n + tau], acc);
  return block_sum(acc, sh);
}

template <typename T>
__global__ void k_ref_collect(const T* __restrict__ c, int64_t count, int64_t lag_min,
                              const int64_t* __restrict__ vmax, int64_t* __restrict__ list,
                              unsigned long long* __restrict__ n) {
  const int64_t v = *vmax;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    if ((int64_t)c[i] == v) list[atomicAdd(n, 1ull)] = lag_min + i;
}

__global__ void __launch_bounds__(kRT) k_ref_dots(const float* __restrict__ x, int64_t nx,
                                                  const float* __restrict__ y, int64_t ny,
                                                  const int64_t* __restrict__ list,
                                                  const unsigned long long* __restrict__ n,
                                                  double* __restrict__ r) {
  __shared__ double sh[kRT / 32];
  const unsigned long long nn = *n;
  if (nn < 2) return;  // a single maximum needs no re-ranking
  for (unsigned long long t = blockIdx.x; t < nn; t += gridDim.x) {
    const double v = real_ccf(x, nx, y, ny, list[t], sh);
    if (threadIdx.x == 0) r[t] = v;
  }
}

__device__ __forceinline__ unsigned long long tie_rank(int64_t lag) {
  return 2ull * (unsigned long long)(lag < 0 ? -lag : lag) + (lag > 0 ? 1ull : 0ull);
}

__global__ void __launch_bounds__(kRT) k_ref_pick(const float* __restrict__ x, int64_t nx,
                                                  const float* __restrict__ y, int64_t ny,
                                                  const int64_t* __restrict__ list,
                                                  const unsigned long long* __restrict__ n,
                                                  const double* __restrict__ r,
                                                  const int64_t* __restrict__ vmax,
                                                  tde_refined* __restrict__ out) {
  __shared__ double sh[kRT / 32];
  __shared__ double s_w[kRT / 32];
  __shared__ double s_rmax;
  __shared__ unsigned long long s_rank, s_cnt;
  __shared__ long long s_lo, s_hi;
  const unsigned long long nn = *n;
  if (threadIdx.x == 0) {
    s_rank = ~0ull;
    s_cnt = 0;
    s_lo = LLONG_MAX;
    s_hi = LLONG_MIN;
  }
  // the real maximum over the tied lags (not needed when there is one)
  double m = -INFINITY;
  if (nn > 1)
    for (unsigned long long t = threadIdx.x; t < nn; t += kRT) m = fmax(m, r[t]);
  for (int o = 16; o; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) s_w[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double mm = -INFINITY;
    for (int w = 0; w < kRT / 32; ++w) mm = fmax(mm, s_w[w]);
    s_rmax = mm;
  }
  __syncthreads();
  const double rmax = s_rmax;
  for (unsigned long long t = threadIdx.x; t < nn; t += kRT) {
    if (nn > 1 && r[t] != rmax) continue;
    const long long lag = (long long)list[t];
    atomicMin(&s_rank, tie_rank(lag));
    atomicMin(&s_lo, lag);
    atomicMax(&s_hi, lag);
    atomicAdd(&s_cnt, 1ull);
  }
  __syncthreads();
  const unsigned long long rk = s_rank;
  const int64_t rep = (rk & 1ull) ? (int64_t)(rk >> 1) : -(int64_t)(rk >> 1);
  const double r0 = real_ccf(x, nx, y, ny, rep, sh);
  double frac = 0.0;
  if (-(nx - 1) <= rep - 1 && rep + 1 <= ny - 1) {
    const double rm = real_ccf(x, nx, y, ny, rep - 1, sh);
    const double rp = real_ccf(x, nx, y, ny, rep + 1, sh);
    const double den = rm - 2.0 * r0 + rp;
    if (den < 0.0 && r0 >= rm && r0 >= rp) frac = fmin(0.5, fmax(-0.5, 0.5 * (rm - rp) / den));
  }
  if (threadIdx.x == 0) {
    out->lag = rep;
    out->value = *vmax;
    out->lag_lo = s_lo;
    out->lag_hi = s_hi;
    out->n_int_ties = (int64_t)nn;
    out->n_ties = (int64_t)s_cnt;
    out->r = r0;
    out->frac = frac;
  }
}

}  // namespace

cudaError_t launch_refine(const float* x, int64_t nx, const float* y, int64_t ny, const void* c, bool c64,
                          int64_t lag_min, int64_t count, const int64_t* d_vmax, int64_t* d_list,
                          double* d_r, unsigned long long* d_n, tde_refined* d_out, int sms,
                          cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(d_n, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return e;
  int64_t g = (count + 255) / 256;
  if (g > 8 * (int64_t)sms) g = 8 * (int64_t)sms;
  if (g < 1) g = 1;
  if (c64)
    k_ref_collect<long long><<<(unsigned)g, 256, 0, st>>>(static_cast<const long long*>(c), count, lag_min,
                                                          d_vmax, d_list, d_n);
  else
    k_ref_collect<int><<<(unsigned)g, 256, 0, st>>>(static_cast<const int*>(c), count, lag_min, d_vmax,
                                                    d_list, d_n);
  k_ref_dots<<<2 * sms, kRT, 0, st>>>(x, nx, y, ny, d_list, d_n, d_r);
  k_ref_pick<<<1, kRT, 0, st>>>(x, nx, y, ny, d_list, d_n, d_r, d_vmax, d_out);
  TDE_COUNT_LAUNCH(3);
  return cudaGetLastError();
}
