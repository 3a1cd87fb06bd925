// synth_gpu.cu -- tde_synth_pairs: a seeded, counter-based generator of
// shifted signal pairs on the GPU, for training the lag proposal on as many
// pairs as it needs.  It holds none of the estimator's arithmetic.
//
// Pair i of seed s: shift d ~ U[-dmax, dmax], AR(1) coefficient a ~ U[a_lo,
// a_hi], SNR ~ U[snr_lo, snr_hi] dB, all drawn from counters (s, i, k); the
// source s[n] = a s[n-1] + e[n] (e ~ N(0,1), s[0] stationary) of length
// N + 2 dmax; x = s[dmax : dmax+N] + noise, y = s[dmax-d : dmax-d+N] + noise, so
// x[n] = y[n + d] before noise (the correlation peak at lag d).  The noise
// scale uses the stationary variance 1 / (1 - a^2) of the source as the
// signal power.
//
// Random numbers: splitmix64 (Steele, Lea, Flood 2014; the finalizer of
// Vigna's SplitMix64) of a 64-bit counter, two uniforms per Box-Muller normal.
// The AR(1) recursion is split into chunks of 512 samples; each chunk restarts
// the recursion 1024 samples before its start from a stationary draw, so its
// state differs from the exact recursion by a factor a^1024 <= 0.98^1024
// (< 1e-8, below FP32 resolution); chunks within 1024 samples of the source's
// start follow the exact recursion from s[0].
#include "common.cuh"

namespace {

constexpr int kChunk = 512;
constexpr int kWarm = 1024;

__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Uniform in (0, 1) from a counter (24 random bits).
__device__ __forceinline__ float uniform01(uint64_t key) {
  return ((float)(uint32_t)(splitmix64(key) >> 40) + 0.5f) * (1.0f / 16777216.0f);
}

__device__ __forceinline__ uint64_t key(uint64_t seed, uint64_t pair, uint64_t stream, uint64_t n) {
  return splitmix64(seed * 0x632BE59BD9B4E019ull + pair) ^ (stream << 56) ^ n;
}

__device__ __forceinline__ float normal(uint64_t k) {
  const float u1 = uniform01(k * 2 + 0), u2 = uniform01(k * 2 + 1);
  return sqrtf(-2.0f * logf(u1)) * cospif(2.0f * u2);
}

struct PairParams {
  int64_t d;
  float a, sigma;
};

__device__ PairParams params(uint64_t seed, uint64_t pair, int64_t dmax, float a_lo, float a_hi,
                             float snr_lo, float snr_hi) {
  PairParams p;
  const uint64_t kp = key(seed, pair, 1, 0);
  p.d = (int64_t)(splitmix64(kp) % (uint64_t)(2 * dmax + 1)) - dmax;
  p.a = a_lo + (a_hi - a_lo) * uniform01(kp + 1);
  const float snr = snr_lo + (snr_hi - snr_lo) * uniform01(kp + 2);
  const float ps = 1.0f / (1.0f - p.a * p.a);
  p.sigma = sqrtf(ps / powf(10.0f, snr / 10.0f));
  return p;
}

// One thread per 512-sample chunk of one pair's x or y.
__global__ void k_synth(uint64_t seed, int64_t first, int npairs, int64_t n, int64_t dmax, float a_lo,
                        float a_hi, float snr_lo, float snr_hi, float* __restrict__ x,
                        float* __restrict__ y, int64_t* __restrict__ shift) {
  const int64_t chunks = (n + kChunk - 1) / kChunk;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per_pair = 2 * chunks;
  if (gid >= (int64_t)npairs * per_pair) return;
  const int64_t p = gid / per_pair, r = gid % per_pair;
  const int which = (int)(r / chunks);  // 0: x, 1: y
  const int64_t c0 = (r % chunks) * kChunk;
  const uint64_t pair = (uint64_t)(first + p);
  const PairParams pp = params(seed, pair, dmax, a_lo, a_hi, snr_lo, snr_hi);
  if (which == 0 && c0 == 0) shift[p] = pp.d;
  // source index of output sample c0: x -> dmax + c0, y -> dmax - d + c0
  const int64_t s0 = (which == 0 ? dmax : dmax - pp.d) + c0;
  int64_t t = s0 - kWarm;
  if (t < 0) t = 0;
  const float a = pp.a;
  const float stat = rsqrtf(fmaxf(1.0f - a * a, 1e-12f));
  float s = normal(key(seed, pair, 2, (uint64_t)t)) * stat;  // stationary start
  for (int64_t k = t + 1; k < s0; ++k) s = a * s + normal(key(seed, pair, 2, (uint64_t)k));
  float* out = (which == 0 ? x : y) + p * n;
  const uint64_t nstream = 3 + which;
  for (int64_t k = 0; k < kChunk && c0 + k < n; ++k) {
    if (s0 + k > t) s = a * s + normal(key(seed, pair, 2, (uint64_t)(s0 + k)));
    out[c0 + k] = s + pp.sigma * normal(key(seed, pair, nstream, (uint64_t)(c0 + k)));
  }
}

}  // namespace

cudaError_t launch_synth_pairs(uint64_t seed, int64_t first, int npairs, int64_t n, int64_t dmax,
                               float a_lo, float a_hi, float snr_lo, float snr_hi, float* x,
                               float* y, int64_t* shift, cudaStream_t st) {
  const int64_t threads = (int64_t)npairs * 2 * ((n + kChunk - 1) / kChunk);
  k_synth<<<(unsigned)((threads + 127) / 128), 128, 0, st>>>(seed, first, npairs, n, dmax, a_lo,
                                                             a_hi, snr_lo, snr_hi, x, y, shift);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}
