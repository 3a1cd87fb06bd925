/*
 * oracle.c -- plain, slow, obviously correct CPU reference of the
 * time-difference estimator's hot path.  TEST INFRASTRUCTURE ONLY: it is
 * called by tests/, by __graft_entry__.smoke() and by the cpu_baseline /
 * reference legs of bench.py, never by the library.  It shares no source
 * with the CUDA path.
 *
 * What it computes (paper: "On the Invariance of Cross-Correlation Peak
 * Positions Under Monotonic Signal Transformations", arXiv 2509.19974):
 *   oracle_quantize   Algorithm 1's quantization step: u = phi(x), a monotone
 *                     non-decreasing integer map with phi(0) = 0.
 *                     bits = 1 is sign() with sign(0) = 0 (Sec. 4.2);
 *                     bits = 2, 4 is the sign-magnitude rank quantizer
 *                     (equal-population thresholds on |x|, 2^b - 1 levels),
 *                     a reading of the paper's "any quantization scheme,
 *                     including nonuniform" (Sec. 3.2).
 *   oracle_xcorr      Algorithm 1's correlation step / Eq. (1): the cross-correlation
 *                     (u * v)[tau] = sum_m u[m] v[m + tau], exact in int64,
 *                     written as the direct double loop over the overlap.
 *   oracle_argmax     Algorithm 1's argmax step: the maximiser; the paper returns
 *                     the whole set of maximisers, this collapses it to one
 *                     lag: smallest |tau|, then smallest tau.
 * Parity: pinned by tests/test_oracle_pins.py (brute force, library
 * correlation, Kronecker substitution, identities, Theorem 1, golden files).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORACLE_OK 0
#define ORACLE_ERR_INVALID 1

static int cmp_float(const void* a, const void* b) {
  float fa = *(const float*)a, fb = *(const float*)b;
  return (fa > fb) - (fa < fb);
}

static int finite_all(const float* x, int64_t n) {
  for (int64_t i = 0; i < n; ++i)
    if (!isfinite(x[i])) return 0;
  return 1;
}

/* Thresholds t_m, m = 1..M, of the b-bit rank quantizer, M = 2^(b-1) - 1:
 * a = |x| sorted ascending, t_m = a[min(n-1, floor((2m-1) n / L))],
 * L = 2^b - 1 levels.  Writes M floats. */
int oracle_rank_thresholds(const float* x, int64_t n, int bits, float* t) {
  if (n <= 0 || (bits != 2 && bits != 4)) return ORACLE_ERR_INVALID;
  if (!finite_all(x, n)) return ORACLE_ERR_INVALID;
  const int64_t L = ((int64_t)1 << bits) - 1;
  const int M = (1 << (bits - 1)) - 1;
  float* a = (float*)malloc(sizeof(float) * (size_t)n);
  if (!a) return ORACLE_ERR_INVALID;
  for (int64_t i = 0; i < n; ++i) a[i] = fabsf(x[i]);
  qsort(a, (size_t)n, sizeof(float), cmp_float);
  for (int m = 1; m <= M; ++m) {
    int64_t idx = ((2 * (int64_t)m - 1) * n) / L;
    if (idx > n - 1) idx = n - 1;
    t[m - 1] = a[idx];
  }
  free(a);
  return ORACLE_OK;
}

/* Algorithm 1's quantization step. */
int oracle_quantize(const float* x, int64_t n, int bits, int8_t* q) {
  if (n <= 0) return ORACLE_ERR_INVALID;
  if (bits == 1) {
    if (!finite_all(x, n)) return ORACLE_ERR_INVALID;
    for (int64_t i = 0; i < n; ++i) q[i] = (int8_t)((x[i] > 0.0f) - (x[i] < 0.0f));
    return ORACLE_OK;
  }
  if (bits != 2 && bits != 4) return ORACLE_ERR_INVALID;
  float t[8];
  int rc = oracle_rank_thresholds(x, n, bits, t);
  if (rc != ORACLE_OK) return rc;
  const int M = (1 << (bits - 1)) - 1;
  for (int64_t i = 0; i < n; ++i) {
    float ax = fabsf(x[i]);
    int level = 0;
    for (int m = 0; m < M; ++m)
      if (ax >= t[m]) level += 1;
    int s = (x[i] > 0.0f) - (x[i] < 0.0f);
    q[i] = (int8_t)(s * level);
  }
  return ORACLE_OK;
}

/* Eq. (1) on the quantized sequences, for tau = lag_min .. lag_max:
 * c[tau - lag_min] = sum over n with 0 <= n < nx, 0 <= n + tau < ny of
 * qx[n] * qy[n + tau], accumulated in int64. */
void oracle_xcorr(const int8_t* qx, int64_t nx, const int8_t* qy, int64_t ny,
                  int64_t lag_min, int64_t lag_max, int64_t* c) {
  int64_t count = lag_max - lag_min + 1;
#pragma omp parallel for schedule(dynamic, 64)
  for (int64_t i = 0; i < count; ++i) {
    int64_t tau = lag_min + i;
    int64_t lo = tau < 0 ? -tau : 0;
    int64_t hi = nx < ny - tau ? nx : ny - tau;
    int64_t s = 0;
    for (int64_t n = lo; n < hi; ++n) s += (int64_t)qx[n] * (int64_t)qy[n + tau];
    c[i] = s;
  }
}

/* Eq. (1) at an arbitrary list of lags (for sampled checks at full size). */
void oracle_xcorr_at(const int8_t* qx, int64_t nx, const int8_t* qy, int64_t ny,
                     const int64_t* lags, int64_t nlags, int64_t* c) {
#pragma omp parallel for schedule(dynamic, 16)
  for (int64_t i = 0; i < nlags; ++i) {
    int64_t tau = lags[i];
    int64_t lo = tau < 0 ? -tau : 0;
    int64_t hi = nx < ny - tau ? nx : ny - tau;
    int64_t s = 0;
    for (int64_t n = lo; n < hi; ++n) s += (int64_t)qx[n] * (int64_t)qy[n + tau];
    c[i] = s;
  }
}

/* Algorithm 1's argmax step, with the maximiser set collapsed to one lag:
 * largest value; among equal values the smallest |tau|; then smallest tau. */
void oracle_argmax(const int64_t* c, int64_t lag_min, int64_t count,
                   int64_t* lag_out, int64_t* val_out) {
  int64_t best_i = 0;
  for (int64_t i = 1; i < count; ++i) {
    int64_t v = c[i], bv = c[best_i];
    int64_t t = lag_min + i, bt = lag_min + best_i;
    int64_t at = t < 0 ? -t : t, abt = bt < 0 ? -bt : bt;
    if (v > bv || (v == bv && (at < abt || (at == abt && t < bt)))) best_i = i;
  }
  *lag_out = lag_min + best_i;
  *val_out = c[best_i];
}

#ifdef _OPENMP
#include <omp.h>
int oracle_num_threads(void) { return omp_get_max_threads(); }
#else
int oracle_num_threads(void) { return 1; }
#endif
