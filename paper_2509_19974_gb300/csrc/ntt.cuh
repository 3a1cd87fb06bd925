// ntt.cuh -- host/device interface of the number-theoretic-transform
// correlation engine (ntt.cu): exact integer correlation modulo one prime
// below 2^31 when the result's bound allows, else modulo two, recombined by
// the Chinese remainder theorem.
#pragma once

#include "common.cuh"

// p0 = 15 * 2^27 + 1 (generator 31), p1 = 63 * 2^25 + 1 (generator 5); both
// below 2^31 so values kept in [0, 2p) fit 32 bits; p0 p1 / 2 > 2^61.
constexpr uint32_t kNttP0 = 2013265921u;
constexpr uint32_t kNttP1 = 2113929217u;
constexpr int kNttMinLog = 10, kNttMaxLog = 19;  // column pass: N2 <= 512 in shared memory

// One prime suffices when every correlation value fits the centred residues
// of p0: |R[k]| <= nt * kmax^2 <= (p0 - 1) / 2, nt the template's length and
// kmax the largest level magnitude.
inline bool ntt_one_prime_ok(int64_t nt, int64_t kmax) {
  return nt * kmax * kmax <= (int64_t)(kNttP0 - 1) / 2;
}

// Per-prime tables for transform length N = 2^logn (device pointers):
// tw[i] = w^i and its Shoup companion floor(tw * 2^32 / p); itw[i] =
// w^-i * N^-1 and companion (w a primitive N-th root of unity).
struct NttTables {
  const uint32_t* tw[2];
  const uint32_t* tws[2];
  const uint32_t* itw[2];
  const uint32_t* itws[2];
};

// One transform: the (reversed, zero-padded) template of a pair, or one
// overlap-save block of the other signal.  buf holds nprimes * N uint32
// (prime 0, then prime 1 if used).
struct NttJob {
  const int8_t* src;
  int64_t nsrc;
  int64_t start;   // block: signal index of block element 0
  int64_t valid;   // block: leading block outputs that are correct
  uint32_t* buf;
  int32_t pair;
  int32_t is_template;
};

// Per pair: R[k] = sum_j t[j] a[k + j] is computed for the template t (the
// shorter signal) against a (the other); lag tau = sign * k.
struct NttPairOut {
  const uint32_t* spec;  // template spectrum, Montgomery form, nprimes * N uint32
  void* c;
  int64_t lag_min, lag_max;
  int32_t c64;
  int32_t sign;
};

// Host: fills 8 tables (tw, tws, itw, itws for p0 then p1), N entries each,
// into host memory `out` (8 * N uint32).
void ntt_host_tables(int logn, uint32_t* out);

// Launches the passes over `njobs` transforms of length 2^logn modulo
// `nprimes` (1: p0, the caller has checked ntt_one_prime_ok for every pair;
// 2: p0 and p1): templates (jobs with is_template) become spectra in their
// buf; blocks are multiplied by their pair's spectrum, transformed back and
// written to c.  d_jobs: device job array; the template jobs must finish
// first (same stream order guarantees it).
cudaError_t launch_ntt_templates(const NttJob* d_jobs, int njobs, int logn, int nprimes,
                                 const NttTables& T, cudaStream_t st);
cudaError_t launch_ntt_blocks(const NttJob* d_jobs, int njobs, const NttPairOut* d_pairs,
                              int logn, int nprimes, const NttTables& T, cudaStream_t st);
