// fftcmp.cu -- the FP32 FFT correlation comparator (the "Real-FFT" baseline of
// arXiv 2509.19974, Sec. 2.3 / 4.1, run on the GPU): zero-pad both signals to
// a power of two L >= nx + ny - 1, c = IDFT( conj(DFT x) * DFT y ) / L, so that
// c[tau] = sum_n x[n] y[n + tau] sits at index tau mod L.  It is not exact and
// not on the estimator's path; it exists to be compared against the exact
// integer correlation.  cuFFT does the transforms (called as a library); the
// padding, the spectral product and the lag extraction are kernels here.
#include <cufft.h>

#include "common.cuh"
#include "fftcmp.cuh"

namespace {

__global__ void k_fft_load(const void* __restrict__ src, int in_i8, int64_t n, int64_t L,
                           float* __restrict__ dst) {
  const int p = blockIdx.y;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < L; i += stride) {
    float v = 0.f;
    if (i < n)
      v = in_i8 ? (float)static_cast<const int8_t*>(src)[(int64_t)p * n + i]
                : static_cast<const float*>(src)[(int64_t)p * n + i];
    dst[(int64_t)p * L + i] = v;
  }
}

// Y <- conj(X) * Y / L, elementwise over npairs spectra of L/2 + 1 bins.
__global__ void k_fft_mul(const float2* __restrict__ X, float2* __restrict__ Y, int64_t bins,
                          float inv_l) {
  const int p = blockIdx.y;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < bins; i += stride) {
    const float2 a = X[(int64_t)p * bins + i], b = Y[(int64_t)p * bins + i];
    Y[(int64_t)p * bins + i] =
        make_float2((a.x * b.x + a.y * b.y) * inv_l, (a.x * b.y - a.y * b.x) * inv_l);
  }
}

__global__ void k_fft_extract(const float* __restrict__ r, int64_t L, int64_t lag_min,
                              int64_t count, float* __restrict__ out) {
  const int p = blockIdx.y;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    int64_t t = (lag_min + i) % L;
    if (t < 0) t += L;
    out[(int64_t)p * count + i] = r[(int64_t)p * L + t];
  }
}

int64_t grid_for(int64_t n) {
  int64_t g = (n + 255) / 256;
  return g < 1 ? 1 : (g > 4096 ? 4096 : g);
}

}  // namespace

int64_t fft_length(int64_t nx, int64_t ny) {
  int64_t L = 1;
  while (L < nx + ny - 1) L <<= 1;
  return L;
}

int fft_plan(FftPlan* plan, int64_t L, int npairs) {
  if (plan->fwd && plan->L == L && plan->npairs == npairs) return 0;
  fft_plan_destroy(plan);
  int n[1] = {(int)L};
  cufftHandle f, b;
  if (cufftPlanMany(&f, 1, n, nullptr, 1, (int)L, nullptr, 1, (int)(L / 2 + 1), CUFFT_R2C,
                    npairs) != CUFFT_SUCCESS)
    return -1;
  if (cufftPlanMany(&b, 1, n, nullptr, 1, (int)(L / 2 + 1), nullptr, 1, (int)L, CUFFT_C2R,
                    npairs) != CUFFT_SUCCESS) {
    cufftDestroy(f);
    return -1;
  }
  plan->fwd = (int)f;
  plan->inv = (int)b;
  plan->L = L;
  plan->npairs = npairs;
  return 0;
}

void fft_plan_destroy(FftPlan* plan) {
  if (plan->fwd) cufftDestroy((cufftHandle)plan->fwd);
  if (plan->inv) cufftDestroy((cufftHandle)plan->inv);
  *plan = FftPlan{};
}

int fft_xcorr(const FftPlan& plan, const void* x, const void* y, int in_i8, int64_t nx,
              int64_t ny, int64_t lag_min, int64_t count, float* c_out, float* rx, float* ry,
              float2* sx, float2* sy, cudaStream_t st) {
  const int64_t L = plan.L, bins = L / 2 + 1;
  const int np = plan.npairs;
  cufftHandle f = (cufftHandle)plan.fwd, b = (cufftHandle)plan.inv;
  if (cufftSetStream(f, st) != CUFFT_SUCCESS || cufftSetStream(b, st) != CUFFT_SUCCESS) return -1;
  k_fft_load<<<dim3((unsigned)grid_for(L), np), 256, 0, st>>>(x, in_i8, nx, L, rx);
  k_fft_load<<<dim3((unsigned)grid_for(L), np), 256, 0, st>>>(y, in_i8, ny, L, ry);
  TDE_COUNT_LAUNCH(2);
  if (cufftExecR2C(f, rx, reinterpret_cast<cufftComplex*>(sx)) != CUFFT_SUCCESS) return -1;
  if (cufftExecR2C(f, ry, reinterpret_cast<cufftComplex*>(sy)) != CUFFT_SUCCESS) return -1;
  k_fft_mul<<<dim3((unsigned)grid_for(bins), np), 256, 0, st>>>(sx, sy, bins, 1.0f / (float)L);
  TDE_COUNT_LAUNCH(1);
  if (cufftExecC2R(b, reinterpret_cast<cufftComplex*>(sy), rx) != CUFFT_SUCCESS) return -1;
  k_fft_extract<<<dim3((unsigned)grid_for(count), np), 256, 0, st>>>(rx, L, lag_min, count, c_out);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError() == cudaSuccess ? 0 : -1;
}
