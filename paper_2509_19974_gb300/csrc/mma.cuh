// mma.cuh -- host/device interface of the tensor-core (tcgen05) correlation
// engine in mma.cu.
#pragma once

#include "common.cuh"

// Lags per CTA tile (128 TMEM lanes x 256 columns) and samples of the sum per
// CTA (a K segment); a tile whose overlap is longer is split over several
// CTAs whose partial sums are added with integer atomics.
constexpr int kMmaTileLags = 32768;
constexpr int kMmaKs = 12288;

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
// Zeroes the outputs of pairs with zero_first set.
cudaError_t launch_mma_zero(const MmaPair* d_pairs, int npairs, int64_t max_count, cudaStream_t st);
// Persistent launch: `grid` CTAs (two per SM fit) take items from *d_counter
// (zeroed here) in array order; sort items longest first.
cudaError_t launch_xcorr_mma(const MmaPair* d_pairs, const MmaItem* d_items, int nitems,
                             int* d_counter, int grid, uint32_t* d_status, cudaStream_t st);
