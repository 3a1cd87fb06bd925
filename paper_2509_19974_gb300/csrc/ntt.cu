// ntt.cu -- exact integer cross-correlation (Algorithm 1's correlation step; Eq. (1) of
// arXiv 2509.19974) by number-theoretic transforms, one of the paper's
// "multimodular method based on the Chinese remainder theorem" routes
// (Sec. 3.2), built for the GPU.
//
// For a pair, the shorter signal is the template t (length Nt) and the other
// signal a is cut into overlap-save blocks of length N = 2^logn:
//   R[k] = sum_j t[j] a[k + j],   tau = k (t = x)  or  tau = -k (t = y).
// Per block starting at a-index S, the circular correlation
//   R_blk[j'] = sum_j t[j] A[(j' + j) mod N],  A[m] = a[S + m]  (0 outside a)
// equals R[S + j'] for the block's "valid" outputs, and in the transform
// domain  R_blk^ = T_rev^ * A^  with  t_rev[m] = t[(-m) mod N].  Everything is
// done modulo primes below 2^31 with 2^25 | p - 1, so the result is exact:
//   one prime  (p0) when |R| <= Nt K^2 <= (p0 - 1) / 2, K the largest level
//              magnitude: the centred residue is R itself;
//   two primes (p0, p1) otherwise, recombined by CRT into the signed integer
//              (|R| < p0 p1 / 2 always holds here).
// Every kernel is a template on the number of primes NQ; the residues of the
// primes sit one after the other in each buffer (NQ * N uint32).
//
// Transform of length N = N1 * N2 (N1 = 2^ceil(logn/2)), four-step form, with
// element n = n1 + N1 n2 stored at n1 + N1 p2:
//   pass 1 (columns): DIF over n2 (natural -> bit-reversed slot p2), then
//     multiply by w^(n1 k2), k2 = bitrev(p2);
//   pass 2 (rows): DIF over n1, [templates: store the spectrum times 2^32 (its
//     Montgomery form) and stop], multiply by the pair's template spectrum
//     (Montgomery product), inverse DIT over the row (bit-reversed ->
//     natural n1);
//   pass 3 (columns): multiply by w^-(n1 k2) N^-1, inverse DIT over the column
//     (bit-reversed -> natural n2), CRT, write the valid outputs.
// Sub-transforms run in shared memory (columns 32 at a time, rows several at a
// time), twiddles for the sub-transform in shared memory; the block buffers
// live in global memory between passes.  Modular products: Shoup with
// precomputed companions for twiddles, Montgomery for data x data.
#include "common.cuh"
#include "ntt.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kCols = 32;            // columns per CTA in passes 1 and 3 (2^5)
constexpr int kRowElems = 2048;      // row elements per CTA in pass 2
// Montgomery constants: -p^-1 mod 2^32; 2^32 mod p with Shoup companion;
// p0^-1 mod p1 = 21 with Shoup companion; P = p0 p1.
__device__ __forceinline__ uint32_t pinv(int q) { return q ? 2113929215u : 2013265919u; }
__device__ __forceinline__ uint32_t rmod(int q) { return q ? 67108862u : 268435454u; }
__device__ __forceinline__ uint32_t rmod_s(int q) { return q ? 136348163u : 572662301u; }
constexpr uint32_t kInvP0 = 21u, kInvP0S = 42u;
constexpr uint64_t kP01 = 4255901651992313857ull;

// Rows per CTA in pass 2: kRowElems elements, at most all N2 rows.
__host__ __device__ __forceinline__ int rows_per_cta(int logn1, int logn2) {
  const int r = kRowElems >> logn1;
  return r < 1 ? 1 : (r > (1 << logn2) ? (1 << logn2) : r);
}

__device__ __forceinline__ uint32_t prime(int q) { return q ? kNttP1 : kNttP0; }
__device__ __forceinline__ uint32_t add_mod(uint32_t a, uint32_t b, uint32_t p) {
  const uint32_t r = a + b;
  return r >= p ? r - p : r;
}
__device__ __forceinline__ uint32_t sub_mod(uint32_t a, uint32_t b, uint32_t p) {
  const uint32_t r = a - b + p;
  return r >= p ? r - p : r;
}
// a * w mod p (a < 2^32, w < p, ws = floor(w 2^32 / p)): Shoup's method.
__device__ __forceinline__ uint32_t mul_shoup(uint32_t a, uint32_t w, uint32_t ws, uint32_t p) {
  const uint32_t q = __umulhi(a, ws);
  const uint32_t r = a * w - q * p;
  return r >= p ? r - p : r;
}
// a * b * 2^-32 mod p (a, b < p): Montgomery reduction.
__device__ __forceinline__ uint32_t mul_mont(uint32_t a, uint32_t b, int q) {
  const uint32_t p = prime(q);
  const uint64_t t = (uint64_t)a * b;
  const uint32_t m = (uint32_t)t * pinv(q);
  const uint32_t r = (uint32_t)((t + (uint64_t)m * p) >> 32);
  return r >= p ? r - p : r;
}

__device__ __forceinline__ uint32_t brev(uint32_t v, int bits) { return __brev(v) >> (32 - bits); }

__device__ __forceinline__ const uint32_t* tw_of(const NttTables& T, int q) { return q ? T.tw[1] : T.tw[0]; }
__device__ __forceinline__ const uint32_t* tws_of(const NttTables& T, int q) { return q ? T.tws[1] : T.tws[0]; }
__device__ __forceinline__ const uint32_t* itw_of(const NttTables& T, int q) { return q ? T.itw[1] : T.itw[0]; }
__device__ __forceinline__ const uint32_t* itws_of(const NttTables& T, int q) { return q ? T.itws[1] : T.itws[0]; }

// Loads the sub-transform twiddles w_M^j, j < M/2 (w_M = w_N^(N/M)), for the
// NQ primes into shared memory: tw_s[q][j], tws_s[q][j].
template <int NQ>
__device__ void load_sub_twiddles(const NttTables& T, int logn, int logm, uint32_t* tw_s,
                                  uint32_t* tws_s, bool inverse) {
  const int half = 1 << (logm - 1);
  const int n = 1 << logn;
  for (int i = threadIdx.x; i < NQ * half; i += kThreads) {
    const int q = NQ == 2 && i >= half, j = i - q * half;
    int e = j << (logn - logm);
    if (inverse) e = (n - e) & (n - 1);
    tw_s[i] = tw_of(T, q)[e];
    tws_s[i] = tws_of(T, q)[e];
  }
}

// In-place radix-2 transforms over shared memory.  Element (q, line, i) of a
// batch of `lines` sequences of length M = 2^logm per prime q < NQ is at
// s[q * qs + line * ls + i * is].
// DIF: natural -> bit-reversed; DIT: bit-reversed -> natural (inverse twiddles
// expected in tw_s).
template <int NQ>
__device__ void dif(uint32_t* s, int qs, int loglines, int ls, int is, int logm, const uint32_t* tw_s,
                    const uint32_t* tws_s, bool line_fastest) {
  const int half = 1 << (logm - 1);
  const int lines = 1 << loglines;
  const int per_q = lines * half;
  for (int loglen = logm - 1; loglen >= 0; --loglen) {
    const int len = 1 << loglen;
    for (int i = threadIdx.x; i < NQ * per_q; i += kThreads) {
      const int q = NQ == 2 && i >= per_q, r = i - q * per_q;
      const int line = line_fastest ? (r & (lines - 1)) : (r >> (logm - 1));
      const int bj = line_fastest ? (r >> loglines) : (r & (half - 1));
      const int j = bj & (len - 1), b = bj >> loglen;
      const int i0 = (b << (loglen + 1)) + j;
      uint32_t* base = s + q * qs + line * ls;
      const uint32_t p = prime(q);
      const uint32_t u = base[i0 * is], v = base[(i0 + len) * is];
      const int t = q * half + (j << (logm - 1 - loglen));
      base[i0 * is] = add_mod(u, v, p);
      base[(i0 + len) * is] = mul_shoup(sub_mod(u, v, p), tw_s[t], tws_s[t], p);
    }
    __syncthreads();
  }
}

template <int NQ>
__device__ void dit(uint32_t* s, int qs, int loglines, int ls, int is, int logm, const uint32_t* tw_s,
                    const uint32_t* tws_s, bool line_fastest) {
  const int half = 1 << (logm - 1);
  const int lines = 1 << loglines;
  const int per_q = lines * half;
  for (int loglen = 0; loglen < logm; ++loglen) {
    const int len = 1 << loglen;
    for (int i = threadIdx.x; i < NQ * per_q; i += kThreads) {
      const int q = NQ == 2 && i >= per_q, r = i - q * per_q;
      const int line = line_fastest ? (r & (lines - 1)) : (r >> (logm - 1));
      const int bj = line_fastest ? (r >> loglines) : (r & (half - 1));
      const int j = bj & (len - 1), b = bj >> loglen;
      const int i0 = (b << (loglen + 1)) + j;
      uint32_t* base = s + q * qs + line * ls;
      const uint32_t p = prime(q);
      const int t = q * half + (j << (logm - 1 - loglen));
      const uint32_t u = base[i0 * is];
      const uint32_t v = mul_shoup(base[(i0 + len) * is], tw_s[t], tws_s[t], p);
      base[i0 * is] = add_mod(u, v, p);
      base[(i0 + len) * is] = sub_mod(u, v, p);
    }
    __syncthreads();
  }
}

__device__ __forceinline__ int source_value(const NttJob& jb, int64_t n, int64_t N) {
  int64_t i;
  if (jb.is_template)
    i = n == 0 ? 0 : N - n;  // t_rev[n] = t[(-n) mod N]
  else
    i = jb.start + n;
  return (i >= 0 && i < jb.nsrc) ? (int)jb.src[i] : 0;
}

// Pass 1: columns n1 in [c0, c0 + 32), DIF over n2, times w^(n1 k2).
template <int NQ>
__global__ void __launch_bounds__(kThreads) k_ntt_col_fwd(const NttJob* __restrict__ jobs,
                                                          NttTables T, int logn, int logn1) {
  extern __shared__ uint32_t sm[];
  const int logn2 = logn - logn1, N2 = 1 << logn2, N1 = 1 << logn1;
  const int64_t N = (int64_t)1 << logn;
  uint32_t* s = sm;                         // [NQ][N2][kCols]
  uint32_t* tw_s = sm + NQ * N2 * kCols;    // [NQ][N2/2]
  uint32_t* tws_s = tw_s + NQ * N2 / 2;
  const NttJob jb = jobs[blockIdx.y];
  const int c0 = blockIdx.x * kCols;
  load_sub_twiddles<NQ>(T, logn, logn2, tw_s, tws_s, false);
  for (int idx = threadIdx.x; idx < N2 * kCols; idx += kThreads) {
    const int n2 = idx / kCols, c = idx % kCols;
    const int v = source_value(jb, (int64_t)(c0 + c) + (int64_t)N1 * n2, N);
    s[idx] = v >= 0 ? (uint32_t)v : (uint32_t)(v + (int)kNttP0);
    if (NQ == 2) s[N2 * kCols + idx] = v >= 0 ? (uint32_t)v : (uint32_t)(v + (int)kNttP1);
  }
  __syncthreads();
  dif<NQ>(s, N2 * kCols, 5, 1, kCols, logn2, tw_s, tws_s, true);
  for (int idx = threadIdx.x; idx < NQ * N2 * kCols; idx += kThreads) {
    const int q = NQ == 2 && idx >= N2 * kCols, r = idx - q * N2 * kCols;
    const int p2 = r / kCols, c = r % kCols;
    const int64_t e = ((int64_t)(c0 + c) * brev(p2, logn2)) & (N - 1);
    jb.buf[q * N + (c0 + c) + (int64_t)N1 * p2] = mul_shoup(s[idx], tw_of(T, q)[e], tws_of(T, q)[e], prime(q));
  }
}

// Pass 2: rows p2 in [r0, r0 + rows): DIF; templates store the Montgomery-form
// spectrum, blocks multiply by it and run the inverse DIT.
template <int NQ>
__global__ void __launch_bounds__(kThreads) k_ntt_row(const NttJob* __restrict__ jobs,
                                                      const NttPairOut* __restrict__ pairs,
                                                      NttTables T, int logn, int logn1) {
  extern __shared__ uint32_t sm[];
  const int N1 = 1 << logn1;
  const int rows = rows_per_cta(logn1, logn - logn1);
  const int64_t N = (int64_t)1 << logn;
  uint32_t* s = sm;                         // [NQ][rows][N1]
  uint32_t* tw_s = sm + NQ * rows * N1;     // [NQ][N1/2] forward
  uint32_t* tws_s = tw_s + NQ * N1 / 2;
  uint32_t* itw_s = tws_s + NQ * N1 / 2;    // [NQ][N1/2] inverse
  uint32_t* itws_s = itw_s + NQ * N1 / 2;
  const NttJob jb = jobs[blockIdx.y];
  const int r0 = blockIdx.x * rows;
  load_sub_twiddles<NQ>(T, logn, logn1, tw_s, tws_s, false);
  if (!jb.is_template) load_sub_twiddles<NQ>(T, logn, logn1, itw_s, itws_s, true);
  for (int idx = threadIdx.x; idx < NQ * rows * N1; idx += kThreads) {
    const int q = NQ == 2 && idx >= rows * N1, r = idx - q * rows * N1;
    s[idx] = jb.buf[q * N + (int64_t)r0 * N1 + r];
  }
  __syncthreads();
  dif<NQ>(s, rows * N1, __ffs(rows) - 1, N1, 1, logn1, tw_s, tws_s, false);
  if (jb.is_template) {
    for (int idx = threadIdx.x; idx < NQ * rows * N1; idx += kThreads) {
      const int q = NQ == 2 && idx >= rows * N1, r = idx - q * rows * N1;
      jb.buf[q * N + (int64_t)r0 * N1 + r] = mul_shoup(s[idx], rmod(q), rmod_s(q), prime(q));
    }
    return;
  }
  const uint32_t* spec = pairs[jb.pair].spec;
  for (int idx = threadIdx.x; idx < NQ * rows * N1; idx += kThreads) {
    const int q = NQ == 2 && idx >= rows * N1, r = idx - q * rows * N1;
    s[idx] = mul_mont(s[idx], spec[q * N + (int64_t)r0 * N1 + r], q);
  }
  __syncthreads();
  dit<NQ>(s, rows * N1, __ffs(rows) - 1, N1, 1, logn1, itw_s, itws_s, false);
  for (int idx = threadIdx.x; idx < NQ * rows * N1; idx += kThreads) {
    const int q = NQ == 2 && idx >= rows * N1, r = idx - q * rows * N1;
    jb.buf[q * N + (int64_t)r0 * N1 + r] = s[idx];
  }
}

// Pass 3: columns, times w^-(n1 k2) N^-1, inverse DIT, the signed value (the
// centred residue, or CRT of two), valid outputs.
template <int NQ>
__global__ void __launch_bounds__(kThreads) k_ntt_col_inv(const NttJob* __restrict__ jobs,
                                                          const NttPairOut* __restrict__ pairs,
                                                          NttTables T, int logn, int logn1) {
  extern __shared__ uint32_t sm[];
  const int logn2 = logn - logn1, N2 = 1 << logn2, N1 = 1 << logn1;
  const int64_t N = (int64_t)1 << logn;
  uint32_t* s = sm;
  uint32_t* tw_s = sm + NQ * N2 * kCols;
  uint32_t* tws_s = tw_s + NQ * N2 / 2;
  const NttJob jb = jobs[blockIdx.y];
  const NttPairOut P = pairs[jb.pair];
  const int c0 = blockIdx.x * kCols;
  load_sub_twiddles<NQ>(T, logn, logn2, tw_s, tws_s, true);
  for (int idx = threadIdx.x; idx < NQ * N2 * kCols; idx += kThreads) {
    const int q = NQ == 2 && idx >= N2 * kCols, r = idx - q * N2 * kCols;
    const int p2 = r / kCols, c = r % kCols;
    const int64_t e = ((int64_t)(c0 + c) * brev(p2, logn2)) & (N - 1);
    s[idx] = mul_shoup(jb.buf[q * N + (c0 + c) + (int64_t)N1 * p2], itw_of(T, q)[e], itws_of(T, q)[e],
                       prime(q));
  }
  __syncthreads();
  dit<NQ>(s, N2 * kCols, 5, 1, kCols, logn2, tw_s, tws_s, true);
  for (int idx = threadIdx.x; idx < N2 * kCols; idx += kThreads) {
    const int n2 = idx / kCols, c = idx % kCols;
    const int64_t jp = (int64_t)(c0 + c) + (int64_t)N1 * n2;  // block position j'
    if (jp >= jb.valid) continue;
    const int64_t tau = P.sign * (jb.start + jp);
    if (tau < P.lag_min || tau > P.lag_max) continue;
    const uint32_t a0 = s[idx];
    int64_t val;
    if (NQ == 1) {
      // |R| <= (p0 - 1) / 2: the centred residue
      val = a0 > kNttP0 / 2 ? (int64_t)a0 - (int64_t)kNttP0 : (int64_t)a0;
    } else {
      // CRT: v = r0 + p0 * ((r1 - r0) p0^-1 mod p1) in [0, p0 p1); signed.
      const uint32_t a1 = s[N2 * kCols + idx];
      const uint32_t h = mul_shoup(sub_mod(a1, a0, kNttP1), kInvP0, kInvP0S, kNttP1);
      const uint64_t v = (uint64_t)a0 + (uint64_t)kNttP0 * h;
      val = v > kP01 / 2 ? (int64_t)(v - kP01) : (int64_t)v;
    }
    if (P.c64)
      static_cast<int64_t*>(P.c)[tau - P.lag_min] = val;
    else
      static_cast<int32_t*>(P.c)[tau - P.lag_min] = (int32_t)val;
  }
}

int col_smem(int nq, int logn2) { return nq * ((1 << logn2) * kCols + (1 << logn2)) * 4; }
int row_smem(int nq, int logn1, int logn2) {
  const int n1 = 1 << logn1;
  return nq * (rows_per_cta(logn1, logn2) * n1 + 2 * n1) * 4;
}

template <int NQ>
cudaError_t templates_nq(const NttJob* d_jobs, int njobs, int logn, const NttTables& T,
                         cudaStream_t st) {
  const int logn1 = (logn + 1) / 2, logn2 = logn - logn1;
  cudaFuncSetAttribute(k_ntt_col_fwd<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       col_smem(NQ, logn2));
  cudaFuncSetAttribute(k_ntt_row<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       row_smem(NQ, logn1, logn2));
  const int rows = rows_per_cta(logn1, logn2);
  k_ntt_col_fwd<NQ><<<dim3((1 << logn1) / kCols, njobs), kThreads, col_smem(NQ, logn2), st>>>(
      d_jobs, T, logn, logn1);
  k_ntt_row<NQ><<<dim3((1 << logn2) / rows, njobs), kThreads, row_smem(NQ, logn1, logn2), st>>>(
      d_jobs, nullptr, T, logn, logn1);
  TDE_COUNT_LAUNCH(2);
  return cudaGetLastError();
}

template <int NQ>
cudaError_t blocks_nq(const NttJob* d_jobs, int njobs, const NttPairOut* d_pairs, int logn,
                      const NttTables& T, cudaStream_t st) {
  const int logn1 = (logn + 1) / 2, logn2 = logn - logn1;
  cudaFuncSetAttribute(k_ntt_col_fwd<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       col_smem(NQ, logn2));
  cudaFuncSetAttribute(k_ntt_row<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       row_smem(NQ, logn1, logn2));
  cudaFuncSetAttribute(k_ntt_col_inv<NQ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       col_smem(NQ, logn2));
  const int rows = rows_per_cta(logn1, logn2);
  k_ntt_col_fwd<NQ><<<dim3((1 << logn1) / kCols, njobs), kThreads, col_smem(NQ, logn2), st>>>(
      d_jobs, T, logn, logn1);
  k_ntt_row<NQ><<<dim3((1 << logn2) / rows, njobs), kThreads, row_smem(NQ, logn1, logn2), st>>>(
      d_jobs, d_pairs, T, logn, logn1);
  k_ntt_col_inv<NQ><<<dim3((1 << logn1) / kCols, njobs), kThreads, col_smem(NQ, logn2), st>>>(
      d_jobs, d_pairs, T, logn, logn1);
  TDE_COUNT_LAUNCH(3);
  return cudaGetLastError();
}

// ---- host-side table construction (exact, 128-bit intermediates)
uint64_t mulmod(uint64_t a, uint64_t b, uint64_t p) {
  return (uint64_t)((unsigned __int128)a * b % p);
}
uint64_t powmod(uint64_t a, uint64_t e, uint64_t p) {
  uint64_t r = 1;
  a %= p;
  while (e) {
    if (e & 1) r = mulmod(r, a, p);
    a = mulmod(a, a, p);
    e >>= 1;
  }
  return r;
}
uint32_t shoup(uint32_t w, uint32_t p) {
  return (uint32_t)(((unsigned __int128)w << 32) / p);
}

}  // namespace

void ntt_host_tables(int logn, uint32_t* out) {
  const uint64_t N = 1ull << logn;
  const uint32_t P[2] = {kNttP0, kNttP1};
  const uint32_t G[2] = {31u, 5u};
  for (int q = 0; q < 2; ++q) {
    const uint64_t p = P[q];
    const uint64_t w = powmod(G[q], (p - 1) / N, p);
    const uint64_t winv = powmod(w, p - 2, p);
    const uint64_t ninv = powmod(N, p - 2, p);
    uint32_t* tw = out + (0 + q) * N;
    uint32_t* tws = out + (2 + q) * N;
    uint32_t* itw = out + (4 + q) * N;
    uint32_t* itws = out + (6 + q) * N;
    uint64_t a = 1, b = ninv;
    for (uint64_t i = 0; i < N; ++i) {
      tw[i] = (uint32_t)a;
      tws[i] = shoup((uint32_t)a, (uint32_t)p);
      itw[i] = (uint32_t)b;
      itws[i] = shoup((uint32_t)b, (uint32_t)p);
      a = mulmod(a, w, p);
      b = mulmod(b, winv, p);
    }
  }
}

cudaError_t launch_ntt_templates(const NttJob* d_jobs, int njobs, int logn, int nprimes,
                                 const NttTables& T, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  return nprimes == 1 ? templates_nq<1>(d_jobs, njobs, logn, T, st)
                      : templates_nq<2>(d_jobs, njobs, logn, T, st);
}

cudaError_t launch_ntt_blocks(const NttJob* d_jobs, int njobs, const NttPairOut* d_pairs,
                              int logn, int nprimes, const NttTables& T, cudaStream_t st) {
  if (njobs <= 0) return cudaSuccess;
  return nprimes == 1 ? blocks_nq<1>(d_jobs, njobs, d_pairs, logn, T, st)
                      : blocks_nq<2>(d_jobs, njobs, d_pairs, logn, T, st);
}
