// fftcmp.cuh -- the FP32 FFT correlation comparator (fftcmp.cu).
#pragma once

#include "common.cuh"

struct FftPlan {
  int fwd = 0, inv = 0;  // cufftHandle values (0: none)
  int64_t L = 0;
  int npairs = 0;
};

// Power-of-two transform length >= nx + ny - 1.
int64_t fft_length(int64_t nx, int64_t ny);
// (Re)creates batched R2C / C2R plans for npairs transforms of length L; 0 on success.
int fft_plan(FftPlan* plan, int64_t L, int npairs);
void fft_plan_destroy(FftPlan* plan);
// c_out[p][i] = correlation at lag lag_min + i of pair p (x: npairs * nx,
// y: npairs * ny, float or int8).  rx, ry: npairs * L floats; sx, sy:
// npairs * (L/2 + 1) complex.  0 on success.
int fft_xcorr(const FftPlan& plan, const void* x, const void* y, int in_i8, int64_t nx,
              int64_t ny, int64_t lag_min, int64_t count, float* c_out, float* rx, float* ry,
              float2* sx, float2* sy, cudaStream_t st);
