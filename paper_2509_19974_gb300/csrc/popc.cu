// popc.cu -- direct integer cross-correlation on bit planes (Algorithm 1's
// correlation step; Eq. (1) of arXiv 2509.19974), exact, for short signals and for the
// windowed/edge cases where a GEMM tile would be mostly empty.
//
// Representation: q = s * m with s = (-1)^sign and m = |q| given by bit planes
// (bits <= 2: one plane "q != 0"; bits = 4: three planes of |q| bits).  For
// 32 samples at once,
//   sum_i qx_i qy_i = sum_{p,r} 2^(p+r) [ popc(Mxp & Myr)
//                                        - 2 popc(Mxp & Myr & (Sx ^ Sy)) ].
// Lag tau = 32 a + r (floor division): lane r of a warp funnel-shifts the
// y words (w + a, w + a + 1) right by r, so the 32 lanes of a warp cover 32
// consecutive lags with one broadcast shared-memory load per word.  Each warp
// owns 8 consecutive values of a, each CTA 64 (2048 lags).  The POPC pipe
// (quarter rate) bounds it: 2 POPC per 32 ternary MACs.
#include "common.cuh"

namespace {

constexpr int kWarps = 8;
constexpr int kAW = 8;                  // a-values per warp
constexpr int kACta = kWarps * kAW;     // 64 a-values = 2048 lags per CTA
constexpr int kWC = 1024;               // x words per shared-memory chunk
static_assert(kACta * 32 == kPopcLagsPerCta, "lag tile");

__global__ void __launch_bounds__(256) k_pack(const PlaneSig* __restrict__ sigs, int bits,
                                              uint32_t* __restrict__ status) {
  const PlaneSig s = sigs[blockIdx.y];
  const int lane = threadIdx.x & 31;
  const int64_t w = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (w >= s.words) return;
  const int64_t i = w * 32 + lane;
  const int v = i < s.n ? (int)s.q[i] : 0;
  const int a = v < 0 ? -v : v;
  const int lim = bits == 4 ? 7 : 1;
  const uint32_t bad = __ballot_sync(0xffffffffu, a > lim);
  const uint32_t sgn = __ballot_sync(0xffffffffu, v < 0);
  if (bits == 4) {
    const uint32_t m0 = __ballot_sync(0xffffffffu, a & 1);
    const uint32_t m1 = __ballot_sync(0xffffffffu, a & 2);
    const uint32_t m2 = __ballot_sync(0xffffffffu, a & 4);
    if (lane == 0) {
      s.planes[w] = sgn;
      s.planes[s.words + w] = m0;
      s.planes[2 * s.words + w] = m1;
      s.planes[3 * s.words + w] = m2;
    }
  } else {
    const uint32_t nz = __ballot_sync(0xffffffffu, a != 0);
    if (lane == 0) {
      s.planes[w] = sgn;
      s.planes[s.words + w] = nz;
    }
  }
  if (lane == 0 && bad) atomicOr(status, TDE_ST_INTERNAL);
}

// PL = planes per signal: 2 (bits <= 2) or 4 (bits = 4).
template <int PL>
__global__ void __launch_bounds__(256) k_xcorr_popc(const XcPair* __restrict__ pairs,
                                                    const PopcItem* __restrict__ items) {
  __shared__ uint32_t xs[PL][kWC];
  __shared__ uint32_t ys[PL][kWC + kACta + 1];
  const PopcItem it = items[blockIdx.x];
  const XcPair P = pairs[it.pair];
  const int warp = threadIdx.x >> 5, r = threadIdx.x & 31;
  const int64_t a_lo = it.a0, a_hi = it.a0 + kACta - 1;
  // x word w meets y words w + a, w + a + 1 inside [0, wy) for some a in the tile
  int64_t w_begin = -a_hi - 1;
  if (w_begin < 0) w_begin = 0;
  int64_t w_end = P.wy - a_lo;
  if (w_end > P.wx) w_end = P.wx;

  int acc[kAW];
  int acc2[kAW];
#pragma unroll
  for (int i = 0; i < kAW; ++i) acc[i] = acc2[i] = 0;

  for (int64_t wc = w_begin; wc < w_end; wc += kWC) {
    const int cnt = (int)((w_end - wc) < kWC ? (w_end - wc) : kWC);
    __syncthreads();
    for (int p = 0; p < PL; ++p) {
      for (int i = threadIdx.x; i < cnt; i += 256) xs[p][i] = P.px[(int64_t)p * P.wx + wc + i];
      for (int j = threadIdx.x; j < cnt + kACta; j += 256) {
        const int64_t yw = wc + a_lo + j;
        ys[p][j] = (yw >= 0 && yw < P.wy) ? P.py[(int64_t)p * P.wy + yw] : 0u;
      }
    }
    __syncthreads();
    const int jb = warp * kAW;
    for (int w = 0; w < cnt; ++w) {
      if (PL == 2) {
        const uint32_t sx = xs[0][w], zx = xs[1][w];
#pragma unroll
        for (int i = 0; i < kAW; ++i) {
          const int j = w + jb + i;
          const uint32_t sy = __funnelshift_r(ys[0][j], ys[0][j + 1], r);
          const uint32_t zy = __funnelshift_r(ys[1][j], ys[1][j + 1], r);
          const uint32_t m = zx & zy;
          acc[i] += __popc(m);
          acc2[i] += __popc(m & (sx ^ sy));
        }
      } else {
        const uint32_t sx = xs[0][w];
        const uint32_t mx0 = xs[1][w], mx1 = xs[2][w], mx2 = xs[3][w];
#pragma unroll
        for (int i = 0; i < kAW; ++i) {
          const int j = w + jb + i;
          const uint32_t sxy = sx ^ __funnelshift_r(ys[0][j], ys[0][j + 1], r);
          const uint32_t my0 = __funnelshift_r(ys[1][j], ys[1][j + 1], r);
          const uint32_t my1 = __funnelshift_r(ys[2][j], ys[2][j + 1], r);
          const uint32_t my2 = __funnelshift_r(ys[3][j], ys[3][j + 1], r);
          int v = 0;
          uint32_t m;
          m = mx0 & my0; v += (__popc(m) - 2 * __popc(m & sxy));
          m = mx0 & my1; v += (__popc(m) - 2 * __popc(m & sxy)) << 1;
          m = mx1 & my0; v += (__popc(m) - 2 * __popc(m & sxy)) << 1;
          m = mx0 & my2; v += (__popc(m) - 2 * __popc(m & sxy)) << 2;
          m = mx1 & my1; v += (__popc(m) - 2 * __popc(m & sxy)) << 2;
          m = mx2 & my0; v += (__popc(m) - 2 * __popc(m & sxy)) << 2;
          m = mx1 & my2; v += (__popc(m) - 2 * __popc(m & sxy)) << 3;
          m = mx2 & my1; v += (__popc(m) - 2 * __popc(m & sxy)) << 3;
          m = mx2 & my2; v += (__popc(m) - 2 * __popc(m & sxy)) << 4;
          acc[i] += v;
        }
      }
    }
  }
  const int jb = warp * kAW;
#pragma unroll
  for (int i = 0; i < kAW; ++i) {
    const int64_t tau = 32 * (a_lo + jb + i) + r;
    if (tau >= P.lag_min && tau <= P.lag_max) {
      const int v = PL == 2 ? acc[i] - 2 * acc2[i] : acc[i];
      if (P.c64)
        static_cast<int64_t*>(P.c)[tau - P.lag_min] = v;
      else
        static_cast<int32_t*>(P.c)[tau - P.lag_min] = v;
    }
  }
}

}  // namespace

cudaError_t launch_pack_planes(const PlaneSig* d_sigs, int nsig, int64_t max_words, int bits,
                               uint32_t* d_status, cudaStream_t st) {
  dim3 grid((unsigned)ceil_div64(max_words, 8), nsig);
  k_pack<<<grid, 256, 0, st>>>(d_sigs, bits, d_status);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_xcorr_popc(const XcPair* d_pairs, const PopcItem* d_items, int nitems, int bits,
                              cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  if (bits == 4)
    k_xcorr_popc<4><<<nitems, 256, 0, st>>>(d_pairs, d_items);
  else
    k_xcorr_popc<2><<<nitems, 256, 0, st>>>(d_pairs, d_items);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}
