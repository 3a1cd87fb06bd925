// argmax.cu -- Algorithm 1's argmax step (arXiv 2509.19974): the maximiser of the
// integer correlation, collapsed to one lag by a fixed rule: largest value,
// then smallest |tau|, then smallest tau.
//
// Lag priority: rank(tau) = 2|tau| + (tau > 0) orders exactly that way
// (0, -1, 1, -2, 2, ...).  int32 correlations are reduced in one pass with a
// packed key  ((v ^ 0x80000000) << 32) | (0xFFFFFFFF - rank)  and a 64-bit
// atomicMax per pair: a larger key is a larger value, then a smaller rank.
// int64 correlations take two passes: the maximum value, then the smallest
// rank among the lags holding it.  Reads are HBM-streaming, grid-strided.
#include "common.cuh"

namespace {

constexpr int kThreads = 256;

__device__ __forceinline__ uint32_t lag_rank(int64_t tau) {
  const uint64_t a = (uint64_t)(tau < 0 ? -tau : tau);
  return (uint32_t)(2 * a + (tau > 0 ? 1 : 0));
}

__device__ __forceinline__ unsigned long long pack32(int32_t v, int64_t tau) {
  return ((unsigned long long)((uint32_t)v ^ 0x80000000u) << 32) |
         (unsigned long long)(0xFFFFFFFFu - lag_rank(tau));
}

template <typename T, typename Op>
__device__ T block_reduce(T v, Op op) {
  __shared__ T part[kThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_down_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    v = threadIdx.x < kThreads / 32 ? part[threadIdx.x] : part[0];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = op(v, __shfl_down_sync(0xffffffffu, v, o));
  }
  return v;
}

struct MaxU64 {
  __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const {
    return a > b ? a : b;
  }
};
struct MaxI64 {
  __device__ long long operator()(long long a, long long b) const { return a > b ? a : b; }
};
struct MinU64 {
  __device__ unsigned long long operator()(unsigned long long a, unsigned long long b) const {
    return a < b ? a : b;
  }
};

// Pairs y = blockIdx.y, + gridDim.y, ... below the pair count (a device count
// when the pairs were made on the device: the grid is then small).
__device__ __forceinline__ int pair_limit(int npairs, const int* d_count) {
  if (!d_count) return npairs;
  const int c = *d_count;
  return c < npairs ? c : npairs;
}

__global__ void __launch_bounds__(kThreads) k_argmax32(const ArgPair* __restrict__ pairs,
                                                       unsigned long long* __restrict__ keys, int npairs,
                                                       const int* __restrict__ d_count) {
  const int lim = pair_limit(npairs, d_count);
  const int64_t tid = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const int64_t nthr = (int64_t)gridDim.x * kThreads;
  for (int y = blockIdx.y; y < lim; y += gridDim.y) {
    const ArgPair P = pairs[y];
    const int32_t* c = static_cast<const int32_t*>(P.c);
    const int64_t n = P.count;
    // c is 4-byte aligned: `head` scalars up to the first 16-byte boundary,
    // then nv int4 vectors (four per thread per step, all loaded before the
    // compares), then the scalar tail
    int64_t head = (int64_t)(((16u - ((uint32_t)reinterpret_cast<uintptr_t>(c) & 15u)) & 15u) >> 2);
    if (head > n) head = n;
    const int64_t nv = (n - head) >> 2;
    const int64_t tail0 = head + 4 * nv;
    unsigned long long best = 0;
    auto take = [&](int32_t v, int64_t i) {
      const unsigned long long k = pack32(v, P.lag_min + i);
      best = k > best ? k : best;
    };
    if (tid < head) take(c[tid], tid);
    if (tid < n - tail0) take(c[tail0 + tid], tail0 + tid);
    const int4* cv = reinterpret_cast<const int4*>(c + head);
    for (int64_t v0 = tid; v0 < nv; v0 += 4 * nthr) {
      int4 a[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int64_t v = v0 + k * nthr;
        a[k] = v < nv ? cv[v] : make_int4(0, 0, 0, 0);
      }
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int64_t v = v0 + k * nthr;
        if (v < nv) {
          const int64_t i = head + 4 * v;
          take(a[k].x, i), take(a[k].y, i + 1), take(a[k].z, i + 2), take(a[k].w, i + 3);
        }
      }
    }
    best = block_reduce(best, MaxU64());
    if (threadIdx.x == 0) atomicMax(&keys[2 * y], best);
  }
}

__global__ void __launch_bounds__(kThreads) k_argmax64_value(const ArgPair* __restrict__ pairs,
                                                             unsigned long long* __restrict__ keys, int npairs,
                                                             const int* __restrict__ d_count) {
  const int lim = pair_limit(npairs, d_count);
  for (int y = blockIdx.y; y < lim; y += gridDim.y) {
    const ArgPair P = pairs[y];
    const long long* c = static_cast<const long long*>(P.c);
    long long best = LLONG_MIN;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < P.count; i += stride)
      best = c[i] > best ? c[i] : best;
    best = block_reduce(best, MaxI64());
    if (threadIdx.x == 0) atomicMax(reinterpret_cast<long long*>(&keys[2 * y]), best);
  }
}

__global__ void __launch_bounds__(kThreads) k_argmax64_lag(const ArgPair* __restrict__ pairs,
                                                           unsigned long long* __restrict__ keys, int npairs,
                                                           const int* __restrict__ d_count) {
  const int lim = pair_limit(npairs, d_count);
  for (int y = blockIdx.y; y < lim; y += gridDim.y) {
    const ArgPair P = pairs[y];
    const long long* c = static_cast<const long long*>(P.c);
    const long long vmax = static_cast<long long>(keys[2 * y]);
    unsigned long long best = ~0ull;
    const int64_t stride = (int64_t)gridDim.x * kThreads;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < P.count; i += stride)
      if (c[i] == vmax) {
        unsigned long long r = lag_rank(P.lag_min + i);
        best = r < best ? r : best;
      }
    best = block_reduce(best, MinU64());
    if (threadIdx.x == 0 && best != ~0ull) atomicMin(&keys[2 * y + 1], best);
  }
}

__global__ void k_argmax_init(unsigned long long* keys, int npairs, int c64,
                              const int* __restrict__ d_count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (d_count && p >= *d_count) return;
  if (p < npairs) {
    keys[2 * p] = c64 ? (unsigned long long)LLONG_MIN : 0ull;
    keys[2 * p + 1] = ~0ull;
  }
}

__device__ __forceinline__ int64_t rank_to_lag(uint64_t rank) {
  const int64_t a = (int64_t)(rank >> 1);
  return (rank & 1) ? a : -a;
}

__global__ void k_argmax_finalize(const ArgPair* __restrict__ pairs,
                                  const unsigned long long* __restrict__ keys, int npairs,
                                  int c64, const int* __restrict__ d_count) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (d_count && p >= *d_count) return;
  if (p >= npairs) return;
  const ArgPair P = pairs[p];
  if (c64) {
    P.val_out[0] = static_cast<int64_t>(keys[2 * p]);
    P.lag_out[0] = rank_to_lag(keys[2 * p + 1]);
  } else {
    const unsigned long long k = keys[2 * p];
    P.val_out[0] = (int64_t)(int32_t)((uint32_t)(k >> 32) ^ 0x80000000u);
    P.lag_out[0] = rank_to_lag(0xFFFFFFFFull - (k & 0xFFFFFFFFull));
  }
}

}  // namespace

cudaError_t launch_argmax(const ArgPair* d_pairs, int npairs, int64_t max_count, int c64,
                          unsigned long long* d_keys, cudaStream_t st, const int* d_count) {
  if (npairs <= 0) return cudaSuccess;
  const int blocks_p = (npairs + 127) / 128;
  k_argmax_init<<<blocks_p, 128, 0, st>>>(d_keys, npairs, c64, d_count);
  TDE_COUNT_LAUNCH(1);
  int64_t gx = ceil_div64(max_count, (int64_t)kThreads * 16);
  if (gx < 1) gx = 1;
  if (gx > 1024) gx = 1024;
  // counted pairs (made on the device): a small grid loops over them
  dim3 grid((unsigned)gx, d_count ? (npairs < 8 ? npairs : 8) : npairs);
  if (c64) {
    k_argmax64_value<<<grid, kThreads, 0, st>>>(d_pairs, d_keys, npairs, d_count);
    TDE_COUNT_LAUNCH(1);
    k_argmax64_lag<<<grid, kThreads, 0, st>>>(d_pairs, d_keys, npairs, d_count);
    TDE_COUNT_LAUNCH(1);
  } else {
    k_argmax32<<<grid, kThreads, 0, st>>>(d_pairs, d_keys, npairs, d_count);
    TDE_COUNT_LAUNCH(1);
  }
  k_argmax_finalize<<<blocks_p, 128, 0, st>>>(d_pairs, d_keys, npairs, c64, d_count);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}
