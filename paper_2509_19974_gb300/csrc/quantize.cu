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
//
// Fused form (k_rank_fused, signals up to 262144 samples, bits 2 and 4): a
// thread-block cluster of C CTAs holds one signal on chip -- each CTA keeps
// its slice's FP32 bit patterns in shared memory -- and runs the same three
// radix passes there.  After each pass every CTA sums the cluster's
// histograms through distributed shared memory and makes the same selection,
// so all CTAs agree on the thresholds without touching HBM.  One read of x,
// one write of q (and, on request, the bit planes of the popc kernels, by
// warp ballots) instead of four reads.
#include <cooperative_groups.h>

#include "common.cuh"

namespace cg = cooperative_groups;

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

// ---------------------------------------------------------------- fused form

constexpr int kFT = 256;                 // threads per fused CTA
constexpr int kFusedChunkTarget = 8192;  // samples per CTA when the cluster allows
constexpr int kFusedChunkMax = 32768;
constexpr int kFusedClusterMax = 8;
constexpr int kCand = 1024;            // pass-1 candidate list per CTA

// Per-CTA selection state in shared memory, one entry per threshold.
struct FusedSel {
  uint32_t pre[8];    // digits of t_m fixed so far
  uint32_t rank[8];   // rank of t_m among the keys that share pre[m]
  int owner[8];       // first threshold with the same prefix (shares its histogram)
};

// merged[m] = sum over the cluster's CTAs of their hist[m], for every owner
// m < M (nbins bins each).  All remote loads of a vector are issued before
// they are summed.
__device__ __forceinline__ void cluster_merge(cg::cluster_group& cl, const uint32_t* hist,
                                              uint32_t* merged, const FusedSel& sel, int M,
                                              int nbins) {
  const int C = (int)cl.num_blocks();
  const int nvec = nbins >> 2;
  for (int idx = threadIdx.x; idx < M * nvec; idx += kFT) {
    const int m = idx / nvec, v = idx - m * nvec;
    if (sel.owner[m] != m) continue;
    const uint4* src = reinterpret_cast<const uint4*>(hist + m * kBins) + v;
    uint4 t[kFusedClusterMax];
#pragma unroll
    for (int r = 0; r < kFusedClusterMax; ++r)
      if (r < C) t[r] = *cl.map_shared_rank(src, r);
    uint4 acc = make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int r = 0; r < kFusedClusterMax; ++r)
      if (r < C) acc.x += t[r].x, acc.y += t[r].y, acc.z += t[r].z, acc.w += t[r].w;
    reinterpret_cast<uint4*>(merged + m * kBins)[v] = acc;
  }
}

// Warp-wide selection for threshold m over histogram h (nbins = 2048 or
// 512): appends the bin holding rank[m] to pre[m] and leaves the rank within
// it.  Every lane reads rank[m] before the shuffles; one lane writes after.
__device__ __forceinline__ void warp_select(const uint32_t* h, int nbins, int width, FusedSel& sel,
                                            int m) {
  const int lane = threadIdx.x & 31;
  const int per = nbins >> 5;  // 64 or 16 bins per lane
  const uint32_t* hh = h + lane * per;
  const uint32_t r = sel.rank[m];
  uint32_t local = 0;
  for (int k = 0; k < per; k += 4) {
    const uint4 v = *reinterpret_cast<const uint4*>(hh + k);
    local += v.x + v.y + v.z + v.w;
  }
  uint32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  const uint32_t before = incl - local;
  if (r >= before && r < incl) {
    uint32_t acc = before;
    for (int k = 0; k < per; ++k) {
      const uint32_t c = hh[k];
      if (r < acc + c) {
        sel.pre[m] = (sel.pre[m] << width) | (uint32_t)(lane * per + k);
        sel.rank[m] = r - acc;
        break;
      }
      acc += c;
    }
  }
}

// One cluster per signal (blockIdx.x / C); CTA rank r holds samples
// [r * chunk, (r + 1) * chunk).  chunk is a multiple of 32, so bit-plane
// words never straddle CTAs.  No CTA returns early: all take part in every
// cluster barrier.  M = number of thresholds (1 for bits 2, 7 for bits 4).
// Pass 1 also collects its matching keys (a few percent of the slice) in a
// candidate list, so pass 2 scans that list instead of the whole slice
// (unless it overflowed).
template <int M>
__global__ void __launch_bounds__(kFT, M == 1 ? 4 : 1)
    k_rank_fused(const QSig* __restrict__ sigs, const QPlanes* __restrict__ planes, int chunk,
                 uint32_t* __restrict__ status) {
  constexpr int kBitsT = M == 1 ? 2 : 4;
  constexpr int L = 2 * M + 1;
  cg::cluster_group cl = cg::this_cluster();
  const int C = (int)cl.num_blocks();
  const int crank = (int)cl.block_rank();
  const int sig = blockIdx.x / C;
  extern __shared__ __align__(16) uint32_t smf[];
  uint32_t* keys = smf;                    // [chunk] raw FP32 bits
  uint32_t* hist = smf + chunk;            // [M][kBins] this CTA's histograms
  uint32_t* merged = hist + M * kBins;     // [M][kBins] the cluster's sums
  uint32_t* cand = merged + M * kBins;     // [kCand] pass-1 keys for pass 2
  __shared__ FusedSel sel;
  __shared__ int ncand;
  const QSig s = sigs[sig];
  const int64_t base = (int64_t)crank * chunk;
  const int64_t rem = s.n - base;
  const int cnt = rem <= 0 ? 0 : (rem < chunk ? (int)rem : chunk);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;

  for (int i = threadIdx.x; i < kBins; i += kFT) hist[i] = 0;
  if (threadIdx.x < 8) {
    const int m = threadIdx.x;
    const int64_t idx = ((2 * (int64_t)m + 1) * s.n) / L;
    sel.rank[m] = (uint32_t)(idx > s.n - 1 ? s.n - 1 : idx);
    sel.pre[m] = 0;
    sel.owner[m] = 0;  // pass 0: one histogram for all thresholds
  }
  __syncthreads();
  // load + pass 0 (digit = bits 30..20 of |x|)
  int bad = 0;
  const float* xs = s.x + base;
  const bool vec = (reinterpret_cast<uintptr_t>(xs) & 15) == 0;
  const int n4 = vec ? cnt >> 2 : 0;
  {
    const float4* x4 = reinterpret_cast<const float4*>(xs);
    // four independent 16-byte loads in flight per thread before any atomic
    for (int i0 = threadIdx.x; i0 < n4; i0 += 4 * kFT) {
      float4 v[4];
#pragma unroll
      for (int k = 0; k < 4; ++k)
        if (i0 + k * kFT < n4) v[k] = x4[i0 + k * kFT];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int i = i0 + k * kFT;
        if (i >= n4) break;
        const uint4 w = make_uint4(__float_as_uint(v[k].x), __float_as_uint(v[k].y),
                                   __float_as_uint(v[k].z), __float_as_uint(v[k].w));
        reinterpret_cast<uint4*>(keys)[i] = w;
        const uint32_t u0 = w.x & 0x7FFFFFFFu, u1 = w.y & 0x7FFFFFFFu, u2 = w.z & 0x7FFFFFFFu,
                       u3 = w.w & 0x7FFFFFFFu;
        bad |= max(max(u0, u1), max(u2, u3)) >= 0x7F800000u;
        atomicAdd(&hist[u0 >> 20], 1u);
        atomicAdd(&hist[u1 >> 20], 1u);
        atomicAdd(&hist[u2 >> 20], 1u);
        atomicAdd(&hist[u3 >> 20], 1u);
      }
    }
  }
  for (int i = (n4 << 2) + threadIdx.x; i < cnt; i += kFT) {
    const uint32_t w = __float_as_uint(xs[i]);
    keys[i] = w;
    const uint32_t u = w & 0x7FFFFFFFu;
    bad |= u >= 0x7F800000u;
    atomicAdd(&hist[u >> 20], 1u);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, TDE_ST_NONFINITE);
  cl.sync();
  cluster_merge(cl, hist, merged, sel, 1, kBins);
  __syncthreads();
  if (warp < M) warp_select(merged, kBins, 11, sel, warp);
  __syncthreads();

  // ---- pass 1 (bits 19..9) over the whole slice; collect candidates
  uint32_t pre[M];
#pragma unroll
  for (int m = 0; m < M; ++m) pre[m] = sel.pre[m];
  cl.sync();  // the peers have finished reading the pass-0 histograms
  if (threadIdx.x < 8) {
    const int m = threadIdx.x;
    int o = m;
    for (int k = m - 1; k >= 0; --k)
      if (sel.pre[k] == sel.pre[m]) o = k;
    sel.owner[m] = o;
  }
  if (threadIdx.x == 0) ncand = 0;
  for (int i = threadIdx.x; i < M * kBins; i += kFT) hist[i] = 0;
  __syncthreads();
  const int cnt4 = cnt >> 2;
  for (int j0 = warp * 32; j0 < ((cnt + 3) >> 2); j0 += kFT) {
    const int i = j0 + lane;  // keys 4i .. 4i+3
    uint4 w = make_uint4(0u, 0u, 0u, 0u);
    int nk = 0;
    if (i < cnt4) {
      w = reinterpret_cast<const uint4*>(keys)[i];
      nk = 4;
    } else if (4 * i < cnt) {
      nk = cnt - 4 * i;
      w.x = keys[4 * i];
      if (nk > 1) w.y = keys[4 * i + 1];
      if (nk > 2) w.z = keys[4 * i + 2];
    }
    const uint32_t wk[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const uint32_t u = wk[k] & 0x7FFFFFFFu;
      const uint32_t hi = u >> 20;
      int mm = -1;
#pragma unroll
      for (int m = M - 1; m >= 0; --m)
        if (hi == pre[m]) mm = m;
      const bool hit = k < nk && mm >= 0;
      if (hit) atomicAdd(&hist[mm * kBins + ((u >> 9) & 2047u)], 1u);
      const uint32_t hits = __ballot_sync(0xffffffffu, hit);
      if (hits) {
        int slot0 = 0;
        if (lane == __ffs(hits) - 1) slot0 = atomicAdd(&ncand, __popc(hits));
        slot0 = __shfl_sync(0xffffffffu, slot0, __ffs(hits) - 1);
        const int slot = slot0 + __popc(hits & ((1u << lane) - 1u));
        if (hit && slot < kCand) cand[slot] = u;
      }
    }
  }
  cl.sync();
  cluster_merge(cl, hist, merged, sel, M, kBins);
  __syncthreads();
  if (warp < M) warp_select(merged + sel.owner[warp] * kBins, kBins, 11, sel, warp);
  __syncthreads();

  // ---- pass 2 (bits 8..0) over the candidates
#pragma unroll
  for (int m = 0; m < M; ++m) pre[m] = sel.pre[m];
  cl.sync();  // the peers have finished reading the pass-1 histograms
  if (threadIdx.x < 8) {
    const int m = threadIdx.x;
    int o = m;
    for (int k = m - 1; k >= 0; --k)
      if (sel.pre[k] == sel.pre[m]) o = k;
    sel.owner[m] = o;
  }
  for (int i = threadIdx.x; i < M * kBins; i += kFT) hist[i] = 0;
  __syncthreads();
  const bool from_cand = ncand <= kCand;
  const int n2 = from_cand ? ncand : cnt;
  for (int i = threadIdx.x; i < n2; i += kFT) {
    const uint32_t u = (from_cand ? cand[i] : keys[i]) & 0x7FFFFFFFu;
    const uint32_t hi = u >> 9;
    int mm = -1;
#pragma unroll
    for (int m = M - 1; m >= 0; --m)
      if (hi == pre[m]) mm = m;
    if (mm >= 0) atomicAdd(&hist[mm * kBins + (u & 511u)], 1u);
  }
  cl.sync();
  cluster_merge(cl, hist, merged, sel, M, 512);
  __syncthreads();
  if (warp < M) warp_select(merged + sel.owner[warp] * kBins, 512, 9, sel, warp);
  __syncthreads();
  cl.sync();  // last remote reads of this CTA's histograms are done

  // ---- apply: q = sign(x) * #{m : |x| >= t_m}; optional planes by ballots
  uint32_t t[M];
#pragma unroll
  for (int m = 0; m < M; ++m) t[m] = sel.pre[m];
  const QPlanes pl = planes ? planes[sig] : QPlanes{nullptr, 0};
  int8_t* qo = s.q + base;
  if (!pl.planes && (reinterpret_cast<uintptr_t>(qo) & 3) == 0) {
    // four levels per 32-bit store
    for (int i = threadIdx.x; i < cnt4; i += kFT) {
      const uint4 w = reinterpret_cast<const uint4*>(keys)[i];
      const uint32_t wk[4] = {w.x, w.y, w.z, w.w};
      uint32_t packed = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint32_t u = wk[k] & 0x7FFFFFFFu;
        int level = 0;
#pragma unroll
        for (int m = 0; m < M; ++m) level += u >= t[m];
        const int q = sign_of(__uint_as_float(wk[k])) * level;
        packed |= ((uint32_t)q & 0xFFu) << (8 * k);
      }
      reinterpret_cast<uint32_t*>(qo)[i] = packed;
    }
    for (int j = (cnt4 << 2) + threadIdx.x; j < cnt; j += kFT) {
      const uint32_t w = keys[j];
      const uint32_t u = w & 0x7FFFFFFFu;
      int level = 0;
#pragma unroll
      for (int m = 0; m < M; ++m) level += u >= t[m];
      qo[j] = (int8_t)(sign_of(__uint_as_float(w)) * level);
    }
    return;
  }
  for (int j0 = warp * 32; j0 < cnt; j0 += kFT) {
    const int j = j0 + lane;
    const bool valid = j < cnt;
    const uint32_t w = valid ? keys[j] : 0u;
    const uint32_t u = w & 0x7FFFFFFFu;
    int level = 0;
#pragma unroll
    for (int m = 0; m < M; ++m) level += u >= t[m];
    const int q = sign_of(__uint_as_float(w)) * level;
    if (valid) qo[j] = (int8_t)q;
    if (pl.planes) {
      const int64_t word = (base + j0) >> 5;
      const uint32_t b0 = __ballot_sync(0xffffffffu, q < 0);
      if (kBitsT <= 2) {
        const uint32_t b1 = __ballot_sync(0xffffffffu, q != 0);
        if (lane == 0) pl.planes[word] = b0, pl.planes[pl.words + word] = b1;
      } else {
        const int a = q < 0 ? -q : q;
        const uint32_t b1 = __ballot_sync(0xffffffffu, a & 1);
        const uint32_t b2 = __ballot_sync(0xffffffffu, a & 2);
        const uint32_t b3 = __ballot_sync(0xffffffffu, a & 4);
        if (lane == 0) {
          pl.planes[word] = b0;
          pl.planes[pl.words + word] = b1;
          pl.planes[2 * pl.words + word] = b2;
          pl.planes[3 * pl.words + word] = b3;
        }
      }
    }
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

// Largest slice one CTA can hold: keys, 2 M histograms and the candidate
// list within the 227 KB a CTA may use (1 KB kept for static shared memory).
int fused_chunk_max(int bits) {
  const int M = (1 << (bits - 1)) - 1;
  const int fit = (232448 - 1024 - 2 * M * kBins * 4 - kCand * 4) / 4;
  const int c = fit < kFusedChunkMax ? fit : kFusedChunkMax;
  return c & ~31;
}

bool quantize_fused_ok(int bits, int64_t max_n) {
  return (bits == 2 || bits == 4) && max_n >= 1 &&
         max_n <= (int64_t)kFusedClusterMax * fused_chunk_max(bits);
}

template <int M>
cudaError_t launch_fused_m(const QSig* d_sigs, const QPlanes* d_planes, int nsig, int C, int chunk,
                           uint32_t* d_status, cudaStream_t st) {
  const size_t smem = (size_t)chunk * 4 + (size_t)2 * M * kBins * 4 + kCand * 4;
  cudaError_t e = cudaFuncSetAttribute(k_rank_fused<M>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nsig * C));
  cfg.blockDim = dim3(kFT);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, k_rank_fused<M>, d_sigs, d_planes, chunk, d_status);
  TDE_COUNT_LAUNCH(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_quantize_fused(const QSig* d_sigs, const QPlanes* d_planes, int nsig,
                                  int64_t max_n, int bits, uint32_t* d_status, cudaStream_t st) {
  if (!quantize_fused_ok(bits, max_n)) return cudaErrorInvalidValue;
  int C = 1;
  while (C < kFusedClusterMax && ceil_div64(max_n, C) > kFusedChunkTarget) C *= 2;
  const int chunk = (int)(ceil_div64(ceil_div64(max_n, C), 32) * 32);
  return bits == 2 ? launch_fused_m<1>(d_sigs, d_planes, nsig, C, chunk, d_status, st)
                   : launch_fused_m<7>(d_sigs, d_planes, nsig, C, chunk, d_status, st);
}
