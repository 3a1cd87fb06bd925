// refine.cuh -- Algorithm 1's last steps on the device (refine.cu).
#pragma once

#include "common.cuh"

// c (int32 or int64, lags lag_min ..) has its maximum at *d_vmax (device);
// d_list / d_r: room for count lags / values, d_n one counter; d_out receives
// the result.  x, y: the original FP32 signals (device).
cudaError_t launch_refine(const float* x, int64_t nx, const float* y, int64_t ny, const void* c, bool c64,
                          int64_t lag_min, int64_t count, const int64_t* d_vmax, int64_t* d_list,
                          double* d_r, unsigned long long* d_n, tde_refined* d_out, int sms,
                          cudaStream_t st);
