// mma.cuh -- host/device interface of the tensor-core (tcgen05) correlation
// engine in mma.cu.
#pragma once

#include "cnn.cuh"
#include "common.cuh"

// Lags per CTA tile (128 TMEM lanes x 256 columns) and samples of the sum per
// CTA (a K segment); a tile whose overlap is longer is split over several
// CTAs whose partial sums are added with integer atomics.
constexpr int kMmaTileLags = 32768;
constexpr int kMmaKs = 24576;
// Samples per K chunk; tile starts T0 and segment bounds are multiples of it.
constexpr int kMmaChunk = 128;

struct MmaPair {
  const int8_t* qx;
  const int8_t* qy;
  int64_t nx, ny, lag_min, lag_max;
  void* c;
  int c64;         // 1: int64 output
  int zero_first;  // 1: some tile is split, so the output is zeroed first
};

// One CTA: lags T0 + (127 - m) + 128 n, sum over k in [ks, ke).
struct MmaItem {
  int32_t pair;
  int32_t single;  // 1: this CTA covers the tile's whole sum (plain stores)
  int64_t T0;
  int64_t ks, ke;
};

int mma_smem_bytes();
// Zeroes the outputs of pairs with zero_first set (of the first *d_count
// pairs when d_count, a device count, is given).
cudaError_t launch_mma_zero(const MmaPair* d_pairs, int npairs, int64_t max_count, cudaStream_t st,
                            const int* d_count = nullptr);
// Persistent launch: `grid` CTAs (two per SM fit) take items from *d_counter
// (zeroed here) in array order; sort items longest first.  d_nitems (device,
// nullable) overrides the item count when the items are made on the device
// (nitems is then an upper bound).
cudaError_t launch_xcorr_mma(const MmaPair* d_pairs, const MmaItem* d_items, int nitems,
                             int* d_counter, int grid, uint32_t* d_status, cudaStream_t st,
                             const int* d_nitems = nullptr);

// The same over items planned for 128-column tiles (16384 lags: tau = T0 +
// (127 - m) + 128 n, n < 128) on packed E2M1 operands; levels must lie in
// {-1, 0, 1} (bits 1, 2), one outside flags TDE_ST_INTERNAL.
constexpr int kMmaTileLags4 = 16384;
// Samples of the sum per CTA on E2M1 operands: exact for any K < 2^24 (|level|
// <= 1); bounded by the shared memory that stages a segment.
#ifndef TDE_M4_KS
#define TDE_M4_KS 24576
#endif
constexpr int kMmaKs4 = TDE_M4_KS;
cudaError_t launch_xcorr_mma4(const MmaPair* d_pairs, const MmaItem* d_items, int nitems,
                              int* d_counter, int grid, uint32_t* d_status, cudaStream_t st,
                              const int* d_nitems = nullptr);

// The learned proposal's windows on the tensor cores, in polyphase form
// (winpp.cu): per pair the 128 x 128 blocks
// D_u[b][j] = sum_a x[128 a + b] y[128 (a + u) + j] that the windows need, as
// MN-major E4M3 GEMMs over the 128-sample rows a, and each window lag as a
// sum of block diagonals.  d_qe: the levels as E4M3 bytes, signal stride n_pad
// (a multiple of 128, zeros in [n, n_pad), 16-byte aligned); pair p is
// x = signal 2 p, y = signal 2 p + 1 (n levels each, |level| <= 7; a block
// sums at most 512 rows, exact in FP32); its 8 windows d_jobs[8 p + w]
// (lag_lo, lag_hi <= lag_lo + 256, c) receive c[i] += sum_n x[n] y[n + lag_lo
// + i] for lag_lo + i <= lag_hi: the c buffers must be zeroed first, and the
// caller checks n * 4^(bits-1) < 2^31 for the int32 c.  d_njobs[p] = win_jobs
// of pair p's windows (device).  One CTA per SM.
cudaError_t launch_xcorr_win_pp(const uint8_t* d_qe, int64_t n, int64_t n_pad, int npairs, const WinJob* d_jobs,
                                const int32_t* d_njobs, uint32_t* d_status, cudaStream_t st);
// One CTA whose bounded waits (the kernels' own) run out on a barrier
// nothing arrives on: TDE_ST_TIMEOUT in d_status after about 4 s.
cudaError_t launch_wait_selftest(uint32_t* d_status, cudaStream_t st);
// Levels [nsig][n] -> E4M3 bytes [nsig][n_pad] (zeros past n); n_pad % 4 == 0.
// A level outside the bits' range (|q| > 1, or > 7 for bits 4) flags
// TDE_ST_INTERNAL in d_status.
cudaError_t launch_to_e4m3(const int8_t* d_q, int64_t n, int64_t n_pad, int nsig, int bits, uint8_t* d_qe,
                           uint32_t* d_status, cudaStream_t st);
