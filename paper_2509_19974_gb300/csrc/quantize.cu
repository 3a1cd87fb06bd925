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
// Streaming form (k_q*, used by every caller with a workspace; the
// multi-pass kernels above serve the allocation-free entry point):
//   k_qhist   histogram of the top 12 bits of |x| per signal (one read of x);
//   k_qsel1   per signal: the bin of each threshold's rank;
//   k_qcand   the keys in those bins (a few percent) appended to the
//             signal's candidate list (one read of x);
//   k_qsel2 (signals up to 2^18 samples) or k_qchist/k_qcsel (longer: each
//             pass a grid of histogram CTAs per signal and a one-CTA select):
//             two radix passes (10 + 9 bits) over the candidates give the
//             exact order statistics;
//   k_qfix    the candidates' levels: k_qcand already wrote every other
//             sample's level (its first digit decides it), so x is read twice
//             (for signals up to 2^18 samples k_qsel2 does this itself);
//   k_qapply  (only when the popc kernels' bit planes are wanted)
//             q = sign(x) * #{m : |x| >= t_m} and the planes (a third read).
//   k_qone    signals up to 2^18 samples, no planes: all of the above in one
//             launch, one CTA per signal, x read from HBM once (its second
//             read comes from L2).
// The candidate list has room for the whole signal (keys, then index and
// sign), so no input (ties, constant signals) needs another path.
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

// ------------------------------------------------------------ streaming form

constexpr int kQB = 4096;            // first digit: bits 30..19 of |x|
constexpr int kQC = 7 * 1024;        // candidate-histogram words per signal
constexpr int kQT = 256;             // threads per streaming CTA
constexpr int kQPer = 8192;          // samples per streaming CTA and step

__device__ __forceinline__ void q_bad(uint32_t u, int& bad) { bad |= u >= 0x7F800000u; }

// Histogram of the first digit; each CTA adds its non-zero bins.  (Having
// the last CTA of each signal run k_qsel1's step here measured slower: every
// CTA then waits on a fence for its atomics before it exits.)
__global__ void __launch_bounds__(kQT) k_qhist(const QSig* __restrict__ sigs, QWork w,
                                               uint32_t* __restrict__ status) {
  __shared__ uint32_t sh[kQB];
  const int sig = blockIdx.y;
  const QSig s = sigs[sig];
  for (int i = threadIdx.x; i < kQB; i += kQT) sh[i] = 0;
  __syncthreads();
  int bad = 0;
  const bool vec = (reinterpret_cast<uintptr_t>(s.x) & 15) == 0;
  const int64_t n4 = vec ? s.n >> 2 : 0;
  const float4* x4 = reinterpret_cast<const float4*>(s.x);
  for (int64_t i0 = (int64_t)blockIdx.x * (kQPer / 4) + threadIdx.x; i0 < n4;
       i0 += (int64_t)gridDim.x * (kQPer / 4)) {
    float4 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t i = i0 + k * kQT;
      if (i < n4) v[k] = x4[i];
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t i = i0 + k * kQT;
      if (i < n4) {
        const uint32_t u0 = __float_as_uint(v[k].x) & 0x7FFFFFFFu, u1 = __float_as_uint(v[k].y) & 0x7FFFFFFFu;
        const uint32_t u2 = __float_as_uint(v[k].z) & 0x7FFFFFFFu, u3 = __float_as_uint(v[k].w) & 0x7FFFFFFFu;
        q_bad(u0, bad), q_bad(u1, bad), q_bad(u2, bad), q_bad(u3, bad);
        atomicAdd(&sh[u0 >> 19], 1u);
        atomicAdd(&sh[u1 >> 19], 1u);
        atomicAdd(&sh[u2 >> 19], 1u);
        atomicAdd(&sh[u3 >> 19], 1u);
      }
    }
  }
  // the tail (or every sample, when x is not 16-byte aligned)
  for (int64_t i = (n4 << 2) + (int64_t)blockIdx.x * kQT + threadIdx.x; i < s.n;
       i += (int64_t)gridDim.x * kQT) {
    const uint32_t u = __float_as_uint(s.x[i]) & 0x7FFFFFFFu;
    q_bad(u, bad);
    atomicAdd(&sh[u >> 19], 1u);
  }
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(status, TDE_ST_NONFINITE);
  uint32_t* gh = w.hist + (size_t)sig * kQB;
  for (int i = threadIdx.x; i < kQB; i += kQT)
    if (sh[i]) atomicAdd(&gh[i], sh[i]);
}

// Warp-wide: the bin of h (nbins = 512, 1024 or 4096) holding rank r, in two
// levels (lanes own nbins/32 bins; then the owning lane's bins are split over
// the warp).  Every lane returns the bin and the rank left within it.
__device__ __noinline__ void warp_find(const uint32_t* h, int nbins, uint32_t r, uint32_t& bin,
                                       uint32_t& rest) {
  const int lane = threadIdx.x & 31;
  const int per = nbins >> 5;  // 16, 32 or 128
  uint32_t local = 0;
  {
    const uint4* hv = reinterpret_cast<const uint4*>(h + lane * per);
    for (int k = 0; k < (per >> 2); ++k) {
      const uint4 v = hv[k];
      local += (v.x + v.y) + (v.z + v.w);
    }
  }
  uint32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  const uint32_t own = __ballot_sync(0xffffffffu, r >= incl - local && r < incl);
  const int L1 = own ? __ffs(own) - 1 : 0;
  const uint32_t r1 = r - __shfl_sync(0xffffffffu, incl - local, L1);
  // second level: bins L1*per .. + per - 1, `sub` per lane
  const int sub = per >= 32 ? per >> 5 : 1;
  const int base = L1 * per + lane * sub;
  uint32_t c[4] = {0u, 0u, 0u, 0u};
  uint32_t loc2 = 0;
  if (lane * sub < per)
    for (int k = 0; k < sub; ++k) c[k] = h[base + k], loc2 += c[k];
  uint32_t inc2 = loc2;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc2, o);
    if (lane >= o) inc2 += t;
  }
  const bool mine = lane * sub < per && r1 >= inc2 - loc2 && r1 < inc2;
  uint32_t fb = 0, fr = 0;
  if (mine) {
    uint32_t acc = inc2 - loc2;
    for (int k = 0; k < sub; ++k) {
      if (r1 < acc + c[k]) {
        fb = (uint32_t)(base + k);
        fr = r1 - acc;
        break;
      }
      acc += c[k];
    }
  }
  const uint32_t who = __ballot_sync(0xffffffffu, mine);
  const int src = who ? __ffs(who) - 1 : 0;
  bin = __shfl_sync(0xffffffffu, fb, src);
  rest = __shfl_sync(0xffffffffu, fr, src);
}

// warp_find for a bin count fixed at compile time (NB = 4096, 1024 or 512),
// everything in registers: lane l sums bins [l NB/32, (l + 1) NB/32), reading
// its 16-byte words in a lane-rotated order so that the warp's loads spread
// over eight bank groups instead of one; the owning lane's bins are then split
// over the warp.  Every lane returns the bin holding rank r and the rank left
// within it (bin 0, rank 0 when r is not below the total).
template <int NB>
__device__ __noinline__ void warp_find_t(const uint32_t* h, uint32_t r, uint32_t& bin, uint32_t& rest) {
  constexpr int kPer = NB / 32;                 // bins per lane: 128, 32, 16
  constexpr int kV = kPer / 4;                  // 16-byte words per lane
  constexpr int kSub = kPer >= 32 ? kPer / 32 : 1;  // second-level bins per lane
  static_assert(kSub == 1 || kSub == 4, "second level");
  const int lane = threadIdx.x & 31;
  const uint4* hv = reinterpret_cast<const uint4*>(h + lane * kPer);
  uint32_t local = 0;
#pragma unroll
  for (int k = 0; k < kV; ++k) {
    const uint4 v = hv[(k + lane) & (kV - 1)];
    local += (v.x + v.y) + (v.z + v.w);
  }
  uint32_t incl = local;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  const uint32_t own = __ballot_sync(0xffffffffu, r >= incl - local && r < incl);
  const int L1 = own ? __ffs(own) - 1 : 0;
  const uint32_t r1 = r - __shfl_sync(0xffffffffu, incl - local, L1);
  const bool act = lane * kSub < kPer;
  const int base = L1 * kPer + lane * kSub;
  uint32_t c[kSub];
  if (kSub == 4) {
    const uint4 v = act ? *reinterpret_cast<const uint4*>(h + base) : make_uint4(0, 0, 0, 0);
    c[0] = v.x, c[kSub > 1 ? 1 : 0] = v.y, c[kSub > 2 ? 2 : 0] = v.z, c[kSub > 3 ? 3 : 0] = v.w;
  } else {
    c[0] = act ? h[base] : 0u;
  }
  uint32_t loc2 = 0;
#pragma unroll
  for (int k = 0; k < kSub; ++k) loc2 += c[k];
  uint32_t inc2 = loc2;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t t = __shfl_up_sync(0xffffffffu, inc2, o);
    if (lane >= o) inc2 += t;
  }
  const bool mine = act && r1 >= inc2 - loc2 && r1 < inc2;
  uint32_t fb = 0, fr = 0, acc = inc2 - loc2;
  bool found = false;
#pragma unroll
  for (int k = 0; k < kSub; ++k) {
    if (!found && r1 < acc + c[k]) fb = (uint32_t)(base + k), fr = r1 - acc, found = true;
    acc += c[k];
  }
  const uint32_t who = __ballot_sync(0xffffffffu, mine);
  const int src = who ? __ffs(who) - 1 : 0;
  bin = __shfl_sync(0xffffffffu, fb, src);
  rest = __shfl_sync(0xffffffffu, fr, src);
}

// Per signal: first digit of every threshold (warp m for threshold m).
__global__ void __launch_bounds__(kQT) k_qsel1(const QSig* __restrict__ sigs, QWork w, int M, int L) {
  __shared__ __align__(16) uint32_t sh[kQB];
  const int sig = blockIdx.x;
  const int64_t n = sigs[sig].n;
  const uint32_t* gh = w.hist + (size_t)sig * kQB;
  for (int i = threadIdx.x; i < kQB / 4; i += kQT)
    reinterpret_cast<uint4*>(sh)[i] = reinterpret_cast<const uint4*>(gh)[i];
  __syncthreads();
  const int warp = threadIdx.x >> 5;
  QState* st = w.state + sig;
  if (warp < M) {
    const int64_t idx = ((2 * (int64_t)warp + 1) * n) / L;
    const uint32_t r = (uint32_t)(idx > n - 1 ? n - 1 : idx);
    uint32_t bin, rest;
    warp_find(sh, kQB, r, bin, rest);
    if ((threadIdx.x & 31) == 0) st->pre[warp] = bin, st->rank[warp] = rest;
  }
  if (threadIdx.x == 0) st->ncand = 0;
  uint32_t* ch = w.chist + (size_t)sig * kQC;
  for (int i = threadIdx.x; i < M * 1024; i += kQT) ch[i] = 0;
}

// Keys whose first digit is a threshold's -> the signal's candidate list.
// Each thread counts its hits and reserves room for them with one shared
// atomic; the CTA gathers them in shared memory and adds them to the list with
// one global atomic (hits that do not fit in the buffer go straight to the
// list).
constexpr int kCandBuf = 4096;

// kApply: the keys' levels are written as well wherever the first digit
// decides them (q = sign(x) * #{m : digit > digit of t_m}); a candidate's
// level waits for the exact thresholds (k_qfix), so its index and sign go to
// the second half of the list, cidx[i] = index | (x < 0) << 31.
template <int M, bool kApply>
__global__ void __launch_bounds__(kQT) k_qcand(const QSig* __restrict__ sigs, QWork w) {
  __shared__ uint32_t buf[kCandBuf];
  __shared__ uint32_t bufi[kApply ? kCandBuf : 1];
  __shared__ uint32_t nbuf, gbase;
  const int sig = blockIdx.y;
  const QSig s = sigs[sig];
  QState* st = w.state + sig;
  uint32_t pre[M];
#pragma unroll
  for (int m = 0; m < M; ++m) pre[m] = st->pre[m];
  uint32_t* cand = w.cand[sig];
  uint32_t* cidx = cand + s.n;
  auto match = [&](uint32_t u) {
    const uint32_t hi = u >> 19;
    bool h = false;
#pragma unroll
    for (int m = 0; m < M; ++m) h |= hi == pre[m];
    return h;
  };
  // level of a non-candidate from its first digit (signed, sign(0) = 0)
  auto level_of = [&](float f) {
    const uint32_t hi = (__float_as_uint(f) & 0x7FFFFFFFu) >> 19;
    int lv = 0;
#pragma unroll
    for (int m = 0; m < M; ++m) lv += hi > pre[m];
    return sign_of(f) * lv;
  };
  auto put = [&](uint32_t slot, uint32_t u, uint32_t ix) {
    if (slot < kCandBuf) {
      buf[slot] = u;
      if (kApply) bufi[slot] = ix;
    } else {
      const uint32_t g = atomicAdd(&st->ncand, 1u);
      cand[g] = u;
      if (kApply) cidx[g] = ix;
    }
  };
  if (threadIdx.x == 0) nbuf = 0;
  __syncthreads();
  const bool vec = (reinterpret_cast<uintptr_t>(s.x) & 15) == 0 &&
                   (!kApply || (reinterpret_cast<uintptr_t>(s.q) & 3) == 0);
  const int64_t n4 = vec ? s.n >> 2 : 0;
  const float4* x4 = reinterpret_cast<const float4*>(s.x);
  for (int64_t c0 = (int64_t)blockIdx.x * (kQPer / 4); c0 < n4; c0 += (int64_t)gridDim.x * (kQPer / 4)) {
    const bool full = c0 + kQPer / 4 <= n4;  // uniform: no per-load bounds in the common case
    float4 v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int64_t i = c0 + k * kQT + threadIdx.x;
      v[k] = (full || i < n4) ? x4[i] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
    uint32_t hits = 0;  // bit 4k + e: element e of load k
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      if (!full && c0 + k * kQT + threadIdx.x >= n4) continue;
      const uint32_t b[4] = {__float_as_uint(v[k].x), __float_as_uint(v[k].y), __float_as_uint(v[k].z),
                             __float_as_uint(v[k].w)};
      uint32_t packed = 0;
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        // bucket test and (for non-candidates) the level, integer-only: the
        // sign bit picks +-level; +-0 has level 0.  A candidate's byte is a
        // placeholder that k_qfix overwrites.
        const uint32_t hi = (b[e] & 0x7FFFFFFFu) >> 19;
        bool c = false;
        int lv = 0;
#pragma unroll
        for (int m = 0; m < M; ++m) c |= hi == pre[m], lv += hi > pre[m];
        hits |= (uint32_t)c << (4 * k + e);
        if (kApply) packed |= ((uint32_t)((b[e] >> 31) ? -lv : lv) & 0xFFu) << (8 * e);
      }
      if (kApply) reinterpret_cast<uint32_t*>(s.q)[c0 + k * kQT + threadIdx.x] = packed;
    }
    if (hits) {
      uint32_t slot = atomicAdd(&nbuf, (uint32_t)__popc(hits));
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const float f[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
        const uint32_t i4 = (uint32_t)(4 * (c0 + k * kQT + threadIdx.x));
#pragma unroll
        for (int e = 0; e < 4; ++e)
          if (hits >> (4 * k + e) & 1u)
            put(slot++, __float_as_uint(f[e]) & 0x7FFFFFFFu, (i4 + e) | (f[e] < 0.f ? 0x80000000u : 0u));
      }
    }
  }
  // the tail (or every sample, when x is not 16-byte aligned)
  for (int64_t j = (n4 << 2) + (int64_t)blockIdx.x * kQT + threadIdx.x; j < s.n;
       j += (int64_t)gridDim.x * kQT) {
    const float f = s.x[j];
    const uint32_t u = __float_as_uint(f) & 0x7FFFFFFFu;
    if (match(u))
      put(atomicAdd(&nbuf, 1u), u, (uint32_t)j | (f < 0.f ? 0x80000000u : 0u));
    else if (kApply)
      s.q[j] = (int8_t)level_of(f);
  }
  __syncthreads();
  const uint32_t nb = nbuf < (uint32_t)kCandBuf ? nbuf : (uint32_t)kCandBuf;
  if (threadIdx.x == 0) gbase = nb ? atomicAdd(&st->ncand, nb) : 0u;
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < nb; i += kQT) {
    cand[gbase + i] = buf[i];
    if (kApply) cidx[gbase + i] = bufi[i];
  }
}

// The candidates' levels, from the exact thresholds: q[idx] = sign * #{m :
// key >= t_m} (sign(0) = 0).
template <int M>
__global__ void __launch_bounds__(kQT) k_qfix(const QSig* __restrict__ sigs, QWork w) {
  const int sig = blockIdx.y;
  const QSig s = sigs[sig];
  const QState* st = w.state + sig;
  uint32_t t[M];
#pragma unroll
  for (int m = 0; m < M; ++m) t[m] = st->thr[m];
  const uint32_t nc = st->ncand;
  const uint32_t* cand = w.cand[sig];
  const uint32_t* cidx = cand + s.n;
  for (uint32_t i = blockIdx.x * kQT + threadIdx.x; i < nc; i += gridDim.x * kQT) {
    const uint32_t u = cand[i], c = cidx[i];
    int lv = 0;
#pragma unroll
    for (int m = 0; m < M; ++m) lv += u >= t[m];
    s.q[c & 0x7FFFFFFFu] = (int8_t)(u == 0 ? 0 : ((c >> 31) ? -lv : lv));
  }
}

// Short signals (few candidates): both candidate passes in one CTA per
// signal -- digits 18..9 then 8..0, one histogram per distinct prefix, one
// warp per threshold.  kFix: then the candidates' levels, as k_qfix.
template <bool kFix>
__global__ void __launch_bounds__(kQT) k_qsel2(const QSig* __restrict__ sigs, QWork w, int M) {
  __shared__ __align__(16) uint32_t sh[7 * 1024];
  __shared__ uint32_t pre_s[7], rank_s[7];
  __shared__ int owner_s[7];
  const int sig = blockIdx.x;
  QState* st = w.state + sig;
  const uint32_t* cand = w.cand[sig];
  const uint32_t nc = st->ncand;
  if (threadIdx.x < 7) {
    const int m = threadIdx.x;
    pre_s[m] = m < M ? st->pre[m] : 0xFFFFFFFFu;
    rank_s[m] = m < M ? st->rank[m] : 0u;
  }
  const int warp = threadIdx.x >> 5;
#pragma unroll 1
  for (int pass = 0; pass < 2; ++pass) {
    const int nbins = pass == 0 ? 1024 : 512, shift = pass == 0 ? 9 : 0, hs = pass == 0 ? 19 : 9;
    const uint32_t mask = pass == 0 ? 1023u : 511u;
    __syncthreads();  // pre_s as the previous pass (or the load above) left it
    // thresholds with equal prefixes so far share the first one's histogram
    if (threadIdx.x < 7) {
      const int m = threadIdx.x;
      int o = m;
      for (int k = m - 1; k >= 0; --k)
        if (pre_s[k] == pre_s[m]) o = k;
      owner_s[m] = o;
    }
    for (int i = threadIdx.x; i < M * 1024; i += kQT) sh[i] = 0;
    __syncthreads();
    uint32_t pre[7];
    int own[7];
#pragma unroll
    for (int m = 0; m < 7; ++m) pre[m] = pre_s[m], own[m] = owner_s[m];
    for (uint32_t i = threadIdx.x; i < nc; i += kQT) {
      const uint32_t u = cand[i];
      const uint32_t hi = u >> hs;
      int mm = -1;
#pragma unroll
      for (int m = 6; m >= 0; --m)
        if (m < M && hi == pre[m]) mm = own[m];
      if (mm >= 0) atomicAdd(&sh[mm * 1024 + ((u >> shift) & mask)], 1u);
    }
    __syncthreads();
    if (warp < M) {
      uint32_t bin, rest;
      warp_find(sh + owner_s[warp] * 1024, nbins, rank_s[warp], bin, rest);
      if ((threadIdx.x & 31) == 0) {
        pre_s[warp] = (pre_s[warp] << (pass == 0 ? 10 : 9)) | bin;
        rank_s[warp] = rest;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < 7) st->thr[threadIdx.x] = threadIdx.x < M ? pre_s[threadIdx.x] : 0xFFFFFFFFu;
  if (kFix) {
    // pre_s holds the exact thresholds (the pass loop ends in a barrier)
    const QSig s = sigs[sig];
    const uint32_t* cidx = cand + s.n;
    uint32_t t[7];
#pragma unroll
    for (int m = 0; m < 7; ++m) t[m] = m < M ? pre_s[m] : 0xFFFFFFFFu;
    // batches of kFixB candidates per thread, loaded before any store (the
    // byte stores could alias the list, so loads after a store would wait)
    constexpr int kFixB = 16;
    for (uint32_t i0 = threadIdx.x; i0 < nc; i0 += kFixB * kQT) {
      uint32_t u[kFixB], c[kFixB];
#pragma unroll
      for (int k = 0; k < kFixB; ++k) {
        const uint32_t i = i0 + k * kQT;
        u[k] = i < nc ? cand[i] : 0u;
        c[k] = i < nc ? cidx[i] : 0u;
      }
#pragma unroll
      for (int k = 0; k < kFixB; ++k) {
        if (i0 + k * kQT >= nc) break;
        int lv = 0;
#pragma unroll
        for (int m = 0; m < 7; ++m) lv += u[k] >= t[m];
        s.q[c[k] & 0x7FFFFFFFu] = (int8_t)(u[k] == 0 ? 0 : ((c[k] >> 31) ? -lv : lv));
      }
    }
  }
}

// One CTA per signal (persistent over the signals), for signals up to
// kQOneMax samples when no bit planes are wanted: the streaming form's steps
// in one launch, with x read from HBM once --
//   1. the first-digit histogram in shared memory (x from HBM); a non-finite
//      sample lands in the top 16 bins (bit patterns from 0x7F800000 up);
//   2. each threshold's bin and rank within it (all threads: a scan of the
//      bins' 16-bin sums);
//   3. the level table: for every 13-bit key (sign, first digit) the signed
//      level its first digit decides, or kQMark where the digit is a
//      threshold's (the sample is a candidate);
//   4. x again (still in L2, read last chunk first so the lines the CTA read
//      most recently come first): each sample's level, candidates to the
//      signal's list (key, then index | sign) -- at b = 2 (about 1 % of the
//      samples) each thread appends to its own column, so no step of the
//      pass waits on another thread; at b = 4 (about 10 %) the list is
//      filled densely, one shared atomic per warp and chunk;
//   5. two radix passes over the candidates (digits 18..9, 8..0, one
//      histogram per distinct prefix) give the exact thresholds;
//   6. the candidates' levels.
// Steps 5 and 6 read the list as columns: entry i * kQOC + t is thread t's.
// It has qone_rows(n) rows (no thread sees more samples than that): keys in
// the first kQOC * rows words, their index | sign in the next.
// Four CTAs per SM, so that a batch of up to 4 x #SM signals is resident at
// once; each thread holds two chunks of loads in flight (the next chunk's
// loads are issued before the current one is processed).  No grid-wide
// step: a signal's chain is the CTA's own.
constexpr int kQOneMax = 1 << 18;
constexpr int kQOC = 256;                  // threads of k_qone
constexpr int kQOV = 4;                    // float4 per thread and chunk
constexpr uint32_t kQOChunk = kQOV * kQOC; // float4 per chunk (16 KB)
constexpr int kQOLV = 4;                   // float4 per thread and chunk of step 4
constexpr int kQTE = kQB / kQOC;           // table entries per thread and sign
constexpr uint32_t kQMark = 0x80u;         // level byte of a candidate (levels are -7..7)
constexpr int kQOneRound = 4;              // CTAs per SM in one round of signals
static_assert(kQTE % 4 == 0, "table words per thread");

// Rows of k_qone's column-major candidate list: a consumer thread sees at
// most 4 ceil(n4 / kQOC) + ceil((n - 4 n4) / kQOC) <= n / kQOC + 5 samples.
__host__ __device__ constexpr uint32_t qone_rows(uint32_t n) { return n / kQOC + 8; }
static_assert(kQOC * 8 <= kQCandSlack, "the columns fit a list of n + kQCandSlack entries");

__device__ __forceinline__ void qone_bar() { __syncthreads(); }

// The level table of step 3 for first digits [kQTE * t, kQTE * (t + 1)):
// bytes 0..4095 for x >= 0, 4096..8191 for x < 0 (index = bits >> 19).
template <int M>
__device__ __forceinline__ void qone_table(uint8_t* tab, const uint32_t* pre) {
  const uint32_t h0 = (uint32_t)(kQTE * threadIdx.x);
  uint32_t lv0 = 0;
#pragma unroll
  for (int m = 0; m < M; ++m) lv0 += pre[m] < h0 ? 1u : 0u;
  uint32_t w[kQTE / 4], cm = 0;  // levels (bytes) and candidate entries (bits)
#pragma unroll
  for (int k = 0; k < kQTE / 4; ++k) w[k] = lv0 * 0x01010101u;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const uint32_t d = pre[m] - h0;
    if (d < (uint32_t)kQTE) {  // a threshold digit in this thread's range
      cm |= 1u << d;
#pragma unroll
      for (int j = 0; j < kQTE; ++j)
        if ((uint32_t)j > d) w[j >> 2] += 1u << (8 * (j & 3));
    }
  }
#pragma unroll
  for (int k = 0; k < kQTE / 4; ++k) {
    uint32_t mk = 0;  // 0xFF in each candidate byte
#pragma unroll
    for (int e = 0; e < 4; ++e) mk |= ((cm >> (4 * k + e)) & 1u) ? 0xFFu << (8 * e) : 0u;
    // -l per byte without borrows across bytes: (0x80 - l) ^ 0x80 for l <= 7
    const uint32_t neg = (0x80808080u - w[k]) ^ 0x80808080u;
    reinterpret_cast<uint32_t*>(tab)[kQTE / 4 * threadIdx.x + k] = (w[k] & ~mk) | (0x80808080u & mk);
    reinterpret_cast<uint32_t*>(tab + kQB)[kQTE / 4 * threadIdx.x + k] = (neg & ~mk) | (0x80808080u & mk);
  }
}

// 0x80 in each byte of p that is kQMark (bit 7 set, bit 6 clear: negative
// levels are 0xF9..0xFF, positive ones 0..7).
__device__ __forceinline__ uint32_t qone_marks(uint32_t p) { return p & ~(p << 1) & 0x80808080u; }

// The level byte of one sample (FP32 bits b): a lookup of its sign and first
// digit.
__device__ __forceinline__ uint32_t qone_level(uint32_t b, const uint8_t* tab) { return tab[b >> 19]; }

// L2 eviction priorities.  At b = 2 x is kept (evict_last) from the
// histogram pass to the level pass, whose loads then give it up
// (evict_first): measured 4 us faster on a 512 x 65536 batch.  At b = 4 the
// candidate traffic is ten times larger and the hints measured slower, so
// both passes load with the normal priority there.
__device__ __forceinline__ uint64_t l2_policy_keep() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_drop() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ uint64_t l2_policy_normal() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ float4 ld_policy(const float4* a, uint64_t pol) {
  float4 v;
  asm("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
      : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
      : "l"(a), "l"(pol));
  return v;
}

__device__ __forceinline__ void qone_load(float4 (&v)[kQOV], const float4* x4, uint32_t c0, uint32_t n4,
                                          uint64_t pol) {
#pragma unroll
  for (int k = 0; k < kQOV; ++k) {
    const uint32_t i = c0 + k * kQOC + threadIdx.x;
    v[k] = i < n4 ? ld_policy(x4 + i, pol) : make_float4(0.f, 0.f, 0.f, 0.f);
  }
}

__device__ __forceinline__ void qone_hist(const float4 (&v)[kQOV], uint32_t* h, uint32_t c0, uint32_t n4) {
#pragma unroll
  for (int k = 0; k < kQOV; ++k) {
    if (c0 + k * kQOC + threadIdx.x >= n4) continue;
    atomicAdd(&h[(__float_as_uint(v[k].x) & 0x7FFFFFFFu) >> 19], 1u);
    atomicAdd(&h[(__float_as_uint(v[k].y) & 0x7FFFFFFFu) >> 19], 1u);
    atomicAdd(&h[(__float_as_uint(v[k].z) & 0x7FFFFFFFu) >> 19], 1u);
    atomicAdd(&h[(__float_as_uint(v[k].w) & 0x7FFFFFFFu) >> 19], 1u);
  }
}

// Step 4 on one chunk: levels stored four to a word, candidates appended.
// kCols (b = 2, about 1 % candidates): each thread appends to its own column
// (cnt: the entries it holds), so no step waits on another thread.  Else
// (b = 4, about 10 %): the list is filled densely from entry 0, each warp
// reserving its room with one shared atomic (ncand).
template <int V, bool kCols>
__device__ __forceinline__ void qone_levels(const float4 (&v)[V], uint32_t c0, uint32_t n4, const uint8_t* tab,
                                            uint32_t* q4, uint32_t* cand, uint32_t* cidx, uint32_t& cnt,
                                            uint32_t* ncand) {
  uint32_t mk[V], any = 0;
#pragma unroll
  for (int k = 0; k < V; ++k) {
    const uint32_t i = c0 + k * kQOC + threadIdx.x;
    const uint32_t l0 = qone_level(__float_as_uint(v[k].x), tab), l1 = qone_level(__float_as_uint(v[k].y), tab);
    const uint32_t l2 = qone_level(__float_as_uint(v[k].z), tab), l3 = qone_level(__float_as_uint(v[k].w), tab);
    const uint32_t p = __byte_perm(__byte_perm(l0, l1, 0x0040), __byte_perm(l2, l3, 0x0040), 0x5410);
    mk[k] = i < n4 ? qone_marks(p) : 0u;
    any |= mk[k];
    if (i < n4) __stcs(q4 + i, p);  // a candidate's byte is rewritten in step 6
  }
  uint32_t slot;
  if (kCols) {
    if (any == 0) return;
    slot = cnt;
  } else {
    if (__ballot_sync(0xffffffffu, any != 0) == 0) return;
    const uint32_t lane = threadIdx.x & 31;
    uint32_t c = 0;
#pragma unroll
    for (int k = 0; k < V; ++k) c += __popc(mk[k]);
    uint32_t incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    uint32_t base = 0;
    if (lane == 31) base = atomicAdd(ncand, incl);
    slot = __shfl_sync(0xffffffffu, base, 31) + incl - c;
    if (c == 0) return;
  }
#pragma unroll
  for (int k = 0; k < V; ++k) {
    if (mk[k] == 0) continue;
    const uint32_t b[4] = {__float_as_uint(v[k].x), __float_as_uint(v[k].y), __float_as_uint(v[k].z),
                           __float_as_uint(v[k].w)};
    const uint32_t i4 = 4 * (c0 + k * kQOC + threadIdx.x);
#pragma unroll
    for (int e = 0; e < 4; ++e)
      if ((mk[k] >> (8 * e + 7)) & 1u) {
        const uint32_t a = kCols ? slot * kQOC + threadIdx.x : slot;
        cand[a] = b[e] & 0x7FFFFFFFu;
        cidx[a] = (i4 + e) | (b[e] & 0x80000000u);
        ++slot;
      }
  }
  if (kCols) cnt = slot;
}

template <int M>
__global__ void __launch_bounds__(kQOC, kQOneRound) k_qone(const QSig* __restrict__ sigs, int nsig, QWork w,
                                                             int L, uint32_t* __restrict__ status) {
  extern __shared__ __align__(16) uint32_t qs[];  // max(kQB, M * 1024) words
  __shared__ uint32_t pre_s[7], rank_s[7], r_s[7], wsum_s[kQOC / 32], ncand_s;
  __shared__ int owner_s[7];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t tid = threadIdx.x;
  const uint64_t keep = M == 1 ? l2_policy_keep() : l2_policy_normal();
  const uint64_t drop = M == 1 ? l2_policy_drop() : keep;
  for (int sig = blockIdx.x; sig < nsig; sig += gridDim.x) {
    const QSig s = sigs[sig];
    const uint32_t n = (uint32_t)s.n;
    uint32_t* cand = w.cand[sig];
    uint32_t* cidx = cand + kQOC * qone_rows(n);
    // ---- 1. first-digit histogram
    for (uint32_t i = tid; i < (uint32_t)kQB / 4; i += kQOC) reinterpret_cast<uint4*>(qs)[i] = make_uint4(0, 0, 0, 0);
    if (tid < (uint32_t)M) {
      const int64_t idx = ((2 * (int64_t)tid + 1) * s.n) / L;
      r_s[tid] = (uint32_t)(idx > s.n - 1 ? s.n - 1 : idx);
      pre_s[tid] = 0, rank_s[tid] = 0;
    }
    if (tid == 0) ncand_s = 0;
    qone_bar();
    const bool vec = (reinterpret_cast<uintptr_t>(s.x) & 15) == 0 && (reinterpret_cast<uintptr_t>(s.q) & 3) == 0;
    const uint32_t n4 = vec ? n >> 2 : 0;
    const float4* x4 = reinterpret_cast<const float4*>(s.x);
    const uint32_t nc4 = (n4 + kQOChunk - 1) / kQOChunk;  // chunks of the float4 passes
    {
      float4 va[kQOV], vb[kQOV];
      if (nc4 > 0) qone_load(va, x4, 0, n4, keep);
      for (uint32_t c = 0; c < nc4; c += 2) {
        if (c + 1 < nc4) qone_load(vb, x4, (c + 1) * kQOChunk, n4, keep);
        qone_hist(va, qs, c * kQOChunk, n4);
        if (c + 1 < nc4) {
          if (c + 2 < nc4) qone_load(va, x4, (c + 2) * kQOChunk, n4, keep);
          qone_hist(vb, qs, (c + 1) * kQOChunk, n4);
        }
      }
    }
    for (uint32_t j = 4 * n4 + tid; j < n; j += kQOC) atomicAdd(&qs[(__float_as_uint(s.x[j]) & 0x7FFFFFFFu) >> 19], 1u);
    qone_bar();
    if (tid < 16 && qs[kQB - 16 + tid] != 0) atomicOr(status, TDE_ST_NONFINITE);
    // ---- 2. each threshold's bin: thread t sums bins [16 t, 16 t + 16)
    // (words read in a lane-rotated order: eight bank groups per warp)
    {
      const uint4* hv = reinterpret_cast<const uint4*>(qs + 16 * tid);
      uint32_t loc = 0;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const uint4 v = hv[(k + lane) & 3];
        loc += (v.x + v.y) + (v.z + v.w);
      }
      uint32_t incl = loc;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
      }
      if (lane == 31) wsum_s[warp] = incl;
      qone_bar();
      uint32_t before = 0;
      for (int k = 0; k < warp; ++k) before += wsum_s[k];
      const uint32_t P = before + incl - loc;
#pragma unroll
      for (int m = 0; m < M; ++m) {
        const uint32_t r = r_s[m];
        if (r >= P && r - P < loc) {  // this thread's bins hold rank r
          uint32_t acc = P;
          for (int j = 0; j < 16; ++j) {
            const uint32_t c = qs[16 * tid + j];
            if (r < acc + c) {
              pre_s[m] = 16 * tid + j, rank_s[m] = r - acc;
              break;
            }
            acc += c;
          }
        }
      }
    }
    qone_bar();
    // ---- 3. the level table (over the histogram, no longer needed)
    uint8_t* tab = reinterpret_cast<uint8_t*>(qs);
    {
      uint32_t pre[M];
#pragma unroll
      for (int m = 0; m < M; ++m) pre[m] = pre_s[m];
      qone_table<M>(tab, pre);
    }
    qone_bar();
    // ---- 4. levels; candidates to the list (last chunk first)
    constexpr bool kCols = M == 1;
    uint32_t cnt = 0;
    {
      uint32_t* q4 = reinterpret_cast<uint32_t*>(s.q);
      // one chunk of loads in flight: the candidate appends keep a chunk's
      // samples live, and two chunks would not fit the CTA's registers
      constexpr int V2 = kQOLV;
      const uint32_t ncl = (n4 + V2 * kQOC - 1) / (V2 * kQOC);
      for (uint32_t c = ncl; c-- > 0;) {
        float4 v[V2];
#pragma unroll
        for (int k = 0; k < V2; ++k) {
          const uint32_t i = c * V2 * kQOC + k * kQOC + tid;
          v[k] = i < n4 ? ld_policy(x4 + i, drop) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        qone_levels<V2, kCols>(v, c * V2 * kQOC, n4, tab, q4, cand, cidx, cnt, &ncand_s);
      }
      for (uint32_t j = 4 * n4 + tid; j < n; j += kQOC) {
        const uint32_t b = __float_as_uint(s.x[j]);
        const uint32_t l = qone_level(b, tab);
        if (l == kQMark) {
          const uint32_t a = kCols ? cnt++ * kQOC + tid : atomicAdd(&ncand_s, 1u);
          cand[a] = b & 0x7FFFFFFFu;
          cidx[a] = j | (b & 0x80000000u);
        } else {
          s.q[j] = (int8_t)l;
        }
      }
    }
    qone_bar();  // the table is read no more (step 5 reuses its words)
    if (!kCols) {  // the dense list read as columns: entry i * kQOC + t is thread t's
      const uint32_t nc = ncand_s;
      cnt = nc > tid ? (nc - tid + kQOC - 1) / kQOC : 0u;
    }
    // ---- 5. exact thresholds from the candidates
#pragma unroll 1
    for (int pass = 0; pass < 2; ++pass) {
      const int shift = pass == 0 ? 9 : 0, hs = pass == 0 ? 19 : 9;
      const uint32_t mask = pass == 0 ? 1023u : 511u;
      if (tid < 7) {  // thresholds with equal prefixes share the first one's histogram
        const int m = tid;
        int o = m;
        if (m < M)
          for (int k = m - 1; k >= 0; --k)
            if (pre_s[k] == pre_s[m]) o = k;
        owner_s[m] = o;
      }
      for (uint32_t i = tid; i < (uint32_t)M * 1024 / 4; i += kQOC)
        reinterpret_cast<uint4*>(qs)[i] = make_uint4(0, 0, 0, 0);
      qone_bar();
      uint32_t pre[M];
      int own[M];
#pragma unroll
      for (int m = 0; m < M; ++m) pre[m] = pre_s[m], own[m] = owner_s[m];
      for (uint32_t i0 = 0; i0 < cnt; i0 += 8) {  // the thread's own column
        uint32_t u[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) u[k] = i0 + k < cnt ? cand[(i0 + k) * kQOC + tid] : 0u;
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          if (i0 + k >= cnt) break;
          const uint32_t hi = u[k] >> hs;
          int mm = -1;
#pragma unroll
          for (int m = M - 1; m >= 0; --m)
            if (hi == pre[m]) mm = own[m];
          if (mm >= 0) atomicAdd(&qs[mm * 1024 + ((u[k] >> shift) & mask)], 1u);
        }
      }
      qone_bar();
      if (warp < M) {
        uint32_t bin, rest;
        if (pass == 0)
          warp_find_t<1024>(qs + owner_s[warp] * 1024, rank_s[warp], bin, rest);
        else
          warp_find_t<512>(qs + owner_s[warp] * 1024, rank_s[warp], bin, rest);
        if (lane == 0) {
          pre_s[warp] = (pre_s[warp] << (pass == 0 ? 10 : 9)) | bin;
          rank_s[warp] = rest;
        }
      }
      qone_bar();
    }
    // ---- 6. the candidates' levels (loads batched ahead of the byte stores,
    // which could alias the list)
    {
      uint32_t t[M];
#pragma unroll
      for (int m = 0; m < M; ++m) t[m] = pre_s[m];
      constexpr int kFixB = 8;
      for (uint32_t i0 = 0; i0 < cnt; i0 += kFixB) {
        uint32_t u[kFixB], c[kFixB];
#pragma unroll
        for (int k = 0; k < kFixB; ++k) {
          const uint32_t i = i0 + k;
          u[k] = i < cnt ? cand[i * kQOC + tid] : 0u;
          c[k] = i < cnt ? cidx[i * kQOC + tid] : 0u;
        }
#pragma unroll
        for (int k = 0; k < kFixB; ++k) {
          if (i0 + k >= cnt) break;
          int lv = 0;
#pragma unroll
          for (int m = 0; m < M; ++m) lv += u[k] >= t[m];
          s.q[c[k] & 0x7FFFFFFFu] = (int8_t)(u[k] == 0 ? 0 : ((c[k] >> 31) ? -lv : lv));
        }
      }
    }
    qone_bar();  // shared state is reused by the next signal
  }
}

// The exact thresholds from the candidates: digits 18..9 then 8..0.  Each
// pass is a grid of CTAs per signal that histograms a share of the candidates
// (one histogram per distinct prefix, in shared memory, non-zero bins added to
// the signal's global histogram) and a one-CTA select per signal (one warp per
// threshold) that also zeroes the global histogram for the next use.
template <int PASS>
__global__ void __launch_bounds__(kQT) k_qchist(QWork w, int M) {
  __shared__ uint32_t sh[kQC];
  const int sig = blockIdx.y;
  const QState* st = w.state + sig;
  const uint32_t nc = st->ncand;
  const uint32_t* cand = w.cand[sig];
  constexpr int hs = PASS == 0 ? 19 : 9, shift = PASS == 0 ? 9 : 0;
  constexpr uint32_t mask = PASS == 0 ? 1023u : 511u;
  uint32_t pre[7];
  int own[7];
#pragma unroll
  for (int m = 0; m < 7; ++m) pre[m] = m < M ? st->pre[m] : 0xFFFFFFFFu, own[m] = st->owner[m];
  if ((uint32_t)blockIdx.x * kQT >= nc) return;  // no candidates for this CTA (uniform)
  for (int i = threadIdx.x; i < M * 1024; i += kQT) sh[i] = 0;
  __syncthreads();
  for (uint32_t i = blockIdx.x * kQT + threadIdx.x; i < nc; i += gridDim.x * kQT) {
    const uint32_t u = cand[i];
    const uint32_t hi = u >> hs;
    int mm = -1;
#pragma unroll
    for (int m = 6; m >= 0; --m)
      if (m < M && hi == pre[m]) mm = own[m];
    if (mm >= 0) atomicAdd(&sh[mm * 1024 + ((u >> shift) & mask)], 1u);
  }
  __syncthreads();
  uint32_t* gh = w.chist + (size_t)sig * kQC;
  for (int i = threadIdx.x; i < M * 1024; i += kQT)
    if (sh[i]) atomicAdd(&gh[i], sh[i]);
}

// PASS 0 / 1: select the next digit (10 / 9 bits).  PASS -1 (after k_qsel1):
// only prepare the owners for pass 0.
template <int PASS>
__global__ void __launch_bounds__(kQT) k_qcsel(QWork w, int M) {
  __shared__ uint32_t pre_s[7];
  const int sig = blockIdx.x;
  QState* st = w.state + sig;
  uint32_t* gh = w.chist + (size_t)sig * kQC;
  const int warp = threadIdx.x >> 5;
  if (threadIdx.x < 7) pre_s[threadIdx.x] = threadIdx.x < M ? st->pre[threadIdx.x] : 0xFFFFFFFFu;
  __syncthreads();
  if (PASS >= 0 && warp < M) {
    const int o = st->owner[warp];
    uint32_t bin, rest;
    warp_find(gh + o * 1024, PASS == 0 ? 1024 : 512, st->rank[warp], bin, rest);
    if ((threadIdx.x & 31) == 0) {
      pre_s[warp] = (pre_s[warp] << (PASS == 0 ? 10 : 9)) | bin;
      st->rank[warp] = rest;
    }
  }
  __syncthreads();
  if (threadIdx.x < 7) {
    const int m = threadIdx.x;
    st->pre[m] = pre_s[m];
    int o = m;
    for (int k = m - 1; k >= 0; --k)
      if (pre_s[k] == pre_s[m]) o = k;
    st->owner[m] = o;  // thresholds with equal prefixes share the first one's histogram
    if (PASS == 1) st->thr[m] = m < M ? pre_s[m] : 0xFFFFFFFFu;
  }
  if (PASS >= 0)
    for (int i = threadIdx.x; i < M * 1024; i += kQT) gh[i] = 0;
}

// q = sign(x) * #{m : |x| >= t_m}; bit planes by warp ballots when asked.
template <int M>
__global__ void __launch_bounds__(kQT) k_qapply(const QSig* __restrict__ sigs,
                                                const QPlanes* __restrict__ planes, QWork w) {
  const int sig = blockIdx.y;
  const QSig s = sigs[sig];
  uint32_t t[M];
#pragma unroll
  for (int m = 0; m < M; ++m) t[m] = w.state[sig].thr[m];
  const QPlanes pl = planes ? planes[sig] : QPlanes{nullptr, 0};
  const int lane = threadIdx.x & 31;
  const bool vec = !pl.planes && (reinterpret_cast<uintptr_t>(s.x) & 15) == 0 &&
                   (reinterpret_cast<uintptr_t>(s.q) & 3) == 0;
  if (vec) {
    const int64_t n4 = s.n >> 2;
    const float4* x4 = reinterpret_cast<const float4*>(s.x);
    uint32_t* q4 = reinterpret_cast<uint32_t*>(s.q);
    for (int64_t i0 = (int64_t)blockIdx.x * (kQPer / 4) + threadIdx.x; i0 < n4;
         i0 += (int64_t)gridDim.x * (kQPer / 4)) {
      float4 v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k)
        if (i0 + k * kQT < n4) v[k] = x4[i0 + k * kQT];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        if (i0 + k * kQT >= n4) break;
        const float f[4] = {v[k].x, v[k].y, v[k].z, v[k].w};
        uint32_t packed = 0;
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const uint32_t u = __float_as_uint(f[e]) & 0x7FFFFFFFu;
          int level = 0;
#pragma unroll
          for (int m = 0; m < M; ++m) level += u >= t[m];
          packed |= ((uint32_t)(sign_of(f[e]) * level) & 0xFFu) << (8 * e);
        }
        q4[i0 + k * kQT] = packed;
      }
    }
    for (int64_t j = (n4 << 2) + (int64_t)blockIdx.x * kQT + threadIdx.x; j < s.n;
         j += (int64_t)gridDim.x * kQT) {
      const float f = s.x[j];
      const uint32_t u = __float_as_uint(f) & 0x7FFFFFFFu;
      int level = 0;
#pragma unroll
      for (int m = 0; m < M; ++m) level += u >= t[m];
      s.q[j] = (int8_t)(sign_of(f) * level);
    }
    return;
  }
  // one sample per lane, 32 consecutive samples per warp (plane words)
  for (int64_t c0 = (int64_t)blockIdx.x * kQPer; c0 < s.n; c0 += (int64_t)gridDim.x * kQPer) {
    const int64_t c1 = c0 + kQPer < s.n ? c0 + kQPer : s.n;
    for (int64_t j0 = c0 + (threadIdx.x & ~31); j0 < c1; j0 += kQT) {
      const int64_t j = j0 + lane;
      const bool valid = j < c1;
      const float f = valid ? s.x[j] : 0.f;
      const uint32_t u = __float_as_uint(f) & 0x7FFFFFFFu;
      int level = 0;
#pragma unroll
      for (int m = 0; m < M; ++m) level += u >= t[m];
      const int q = sign_of(f) * level;
      if (valid) s.q[j] = (int8_t)q;
      if (pl.planes) {
        const int64_t word = j0 >> 5;
        const uint32_t b0 = __ballot_sync(0xffffffffu, q < 0);
        if (M == 1) {
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

cudaError_t launch_quantize_stream(const QSig* d_sigs, const QPlanes* d_planes, int nsig,
                                   int64_t max_n, int bits, QWork w, uint32_t* d_status,
                                   cudaStream_t st) {
  if (bits != 2 && bits != 4) return cudaErrorInvalidValue;
  const int M = (1 << (bits - 1)) - 1, L = (1 << bits) - 1;
  if (d_planes == nullptr && max_n <= kQOneMax) {
    // one CTA per signal, x read from HBM once: kQOneRound CTAs per SM, the
    // signals dealt in equal rounds, so that the signals in flight (one per
    // CTA) stay within L2 until their second read
    const size_t smem = sizeof(uint32_t) * (M == 1 ? kQB : 7 * 1024);
    auto kern = M == 1 ? k_qone<1> : k_qone<7>;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t cap = kQOneRound * (int64_t)sms;
    const int64_t rounds = ceil_div64(nsig, cap);
    const int grid = (int)ceil_div64(nsig, rounds);
    kern<<<grid, kQOC, smem, st>>>(d_sigs, nsig, w, L, d_status);
    TDE_COUNT_LAUNCH(1);
    return cudaGetLastError();
  }
  int64_t gx = ceil_div64(max_n, kQPer);
  if (gx < 1) gx = 1;
  if (gx > 65535) gx = 65535;
  const dim3 grid((unsigned)gx, (unsigned)nsig);
  cudaError_t e = cudaMemsetAsync(w.hist, 0, sizeof(uint32_t) * (size_t)nsig * kQB, st);
  if (e != cudaSuccess) return e;
  k_qhist<<<grid, kQT, 0, st>>>(d_sigs, w, d_status);
  k_qsel1<<<nsig, kQT, 0, st>>>(d_sigs, w, M, L);
  const bool fused = d_planes == nullptr;  // levels written by k_qcand + k_qfix
  if (M == 1)
    fused ? k_qcand<1, true><<<grid, kQT, 0, st>>>(d_sigs, w) : k_qcand<1, false><<<grid, kQT, 0, st>>>(d_sigs, w);
  else
    fused ? k_qcand<7, true><<<grid, kQT, 0, st>>>(d_sigs, w) : k_qcand<7, false><<<grid, kQT, 0, st>>>(d_sigs, w);
  const bool short_sig = max_n <= (1 << 18);
  if (short_sig) {
    fused ? k_qsel2<true><<<nsig, kQT, 0, st>>>(d_sigs, w, M)  // + k_qfix's step
          : k_qsel2<false><<<nsig, kQT, 0, st>>>(d_sigs, w, M);
    TDE_COUNT_LAUNCH(1);
  } else {
    int64_t gc = ceil_div64(max_n, 32768);  // candidate-histogram CTAs per signal
    if (gc > 256) gc = 256;
    const dim3 cgrid((unsigned)gc, (unsigned)nsig);
    k_qcsel<-1><<<nsig, kQT, 0, st>>>(w, M);
    k_qchist<0><<<cgrid, kQT, 0, st>>>(w, M);
    k_qcsel<0><<<nsig, kQT, 0, st>>>(w, M);
    k_qchist<1><<<cgrid, kQT, 0, st>>>(w, M);
    k_qcsel<1><<<nsig, kQT, 0, st>>>(w, M);
    TDE_COUNT_LAUNCH(5);
  }
  if (fused && !short_sig) {
    int64_t gf = ceil_div64(max_n, 16 * kQT);  // candidates are a few percent of a signal
    if (gf < 1) gf = 1;
    if (gf > 65535) gf = 65535;
    const dim3 fgrid((unsigned)gf, (unsigned)nsig);
    if (M == 1)
      k_qfix<1><<<fgrid, kQT, 0, st>>>(d_sigs, w);
    else
      k_qfix<7><<<fgrid, kQT, 0, st>>>(d_sigs, w);
    TDE_COUNT_LAUNCH(1);
  } else if (!fused) {
    if (M == 1)
      k_qapply<1><<<grid, kQT, 0, st>>>(d_sigs, d_planes, w);
    else
      k_qapply<7><<<grid, kQT, 0, st>>>(d_sigs, d_planes, w);
    TDE_COUNT_LAUNCH(1);
  }
  TDE_COUNT_LAUNCH(3);  // k_qhist, k_qsel1, k_qcand
  return cudaGetLastError();
}
