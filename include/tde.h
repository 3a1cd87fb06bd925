/*
 * tde.h -- C ABI of the GB300 time-difference estimator (libtde.so).
 *
 * The estimator is Algorithm 1 of "On the Invariance of
 * Cross-Correlation Peak Positions Under Monotonic Signal Transformations,
 * with Application to Fast Time Difference Estimation" (arXiv 2509.19974):
 *   1-2. quantize both signals with a monotone non-decreasing integer map phi
 *        with phi(0) = 0 (Theorem 1's hypotheses, Sec. 3.1),
 *   3.   compute their integer cross-correlation, Eq. (1),
 *   4.   take the maximiser.  The paper returns the set of maximisers; this
 *        library returns one lag: the largest value, ties to the smallest
 *        |tau|, then to the smallest tau.
 *
 * Conventions shared by every call below.
 *  - Lag convention, Eq. (1): c[tau] = sum_n qx[n] * qy[n + tau] over the
 *    overlap 0 <= n < nx, 0 <= n + tau < ny.  If x[n] = a * y[n + nu] (Eq. (2))
 *    the peak is at tau = nu.  Output element i holds lag lag_min + i.
 *  - Every array argument is DEVICE memory owned by the caller, unless the
 *    argument says "host".  The library never frees or retains caller memory.
 *  - Every call is asynchronous on `stream` (a cudaStream_t; NULL is the
 *    legacy default stream) and returns after enqueueing.  Host-side argument
 *    errors are returned immediately and nothing is enqueued.  Errors that only
 *    the device can see (NaN or Inf in the input, a bounded wait that ran out)
 *    are latched in the context's device status word and returned by
 *    tde_ctx_sync().
 *  - A context is bound to one device and is not thread-safe: use one context
 *    per host thread.  Calls on one context must not overlap in time on
 *    different streams, because they share the context's workspace.
 *  - Quantization levels (Algorithm 1's level map, phi : R -> Z):
 *      bits = 1: q = sign(x), with sign(0) = sign(-0.0) = 0 (Sec. 4.2).
 *      bits = 2, 4: sign-magnitude rank quantizer with L = 2^bits - 1 levels:
 *        a = |x| sorted ascending, t_m = a[min(n-1, floor((2m-1) n / L))]
 *        for m = 1 .. 2^(bits-1) - 1, q = sign(x) * #{m : |x| >= t_m}.
 *        Levels are {-1,0,1} for bits = 2 and -7..7 for bits = 4.
 *  - int32 correlation output requires min(nx, ny) * (2^(bits-1))^2 < 2^31;
 *    otherwise TDE_ERR_OVERFLOW is returned and the caller must ask for int64.
 */
#ifndef TDE_H_
#define TDE_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same object type as cudaStream_t. */
typedef struct CUstream_st* tde_stream_t;

typedef enum {
  TDE_OK = 0,
  TDE_ERR_INVALID = 1,     /* bad argument; or NaN/Inf input seen on the device */
  TDE_ERR_OVERFLOW = 2,    /* int32 output could overflow for these sizes */
  TDE_ERR_UNSUPPORTED = 3, /* valid request the library cannot serve */
  TDE_ERR_CUDA = 4,        /* a CUDA runtime call failed; see tde_last_error */
  TDE_ERR_TIMEOUT = 5      /* a bounded device-side wait gave up */
} tde_status;

/* Correlation engines (the "engine" argument). */
enum {
  TDE_ENGINE_AUTO = 0, /* pick by length and bits */
  TDE_ENGINE_POPC = 1, /* bit-plane AND/XOR + popcount direct sums */
  TDE_ENGINE_MMA = 2,  /* Toeplitz-as-GEMM on the tcgen05 tensor cores */
  TDE_ENGINE_NTT = 3   /* number-theoretic transform: one prime, or two + CRT */
};

/* Element types of the "dtype" arguments. */
enum { TDE_I32 = 0, TDE_I64 = 1, TDE_F32 = 2, TDE_I8 = 3 };

typedef struct tde_ctx tde_ctx;

/* Create a context on CUDA device `device` (0-based).  *out receives the
 * handle (host memory).  The context owns a device workspace that grows on
 * demand and a device status word.  Returns TDE_ERR_CUDA if the device cannot
 * be used. */
tde_status tde_ctx_create(int device, tde_ctx** out);

/* Synchronize the device, then free everything the context owns.  NULL is
 * accepted and ignored. */
tde_status tde_ctx_destroy(tde_ctx* ctx);

/* Wait for `stream`, then read and clear the device status word.  Returns
 * TDE_ERR_INVALID if a kernel saw NaN/Inf input, TDE_ERR_TIMEOUT if a bounded
 * wait gave up, TDE_ERR_CUDA on an asynchronous CUDA error, else TDE_OK. */
tde_status tde_ctx_sync(tde_ctx* ctx, tde_stream_t stream);

/* Text of the last error on this context (host string owned by the context,
 * valid until the next call on it).  Never NULL. */
const char* tde_last_error(const tde_ctx* ctx);

/* Instrumentation.  With profiling enabled, every launch of a correlation
 * engine's main kernel is bracketed by two CUDA events on its stream (the
 * events are the context's; no caller memory is touched). */
tde_status tde_ctx_set_profiling(tde_ctx* ctx, int enable);

/* Template search over an unbounded stream (the paper's closing remark on
 * long signals; Eq. (1) and Algorithm 1's argmax over the positions seen so
 * far).  A short template y is searched for in a signal x that arrives in
 * chunks; after every chunk the running answer equals Algorithm 1 on the
 * prefix of x seen so far, over the lags where y lies wholly inside it.
 * Positions are global: the template at position k of x is lag tau = -k of
 * c[tau] = sum_n x[n] y[n + tau]; ties go to the larger value, then the
 * smaller |tau| (the earlier position), as in tde_argmax.
 *
 * tde_stream_create: y is ny floats (device), quantized at creation; bits must
 * be 1 (the sign quantizer is pointwise, so a chunk quantizes the same alone
 * as inside the whole signal; the rank quantizer's thresholds are order
 * statistics of the whole signal: TDE_ERR_UNSUPPORTED).  Every chunk holds at
 * most max_chunk samples.  The stream owns device memory of about
 * 2 (ny + max_chunk) bytes + 8 max_chunk bytes.
 * tde_stream_push: the next chunk, n floats (device); asynchronous on
 * `stream`, no host synchronisation: the chunk is quantized behind the last
 * ny - 1 levels carried from before, correlated with the template (engine as
 * given, int64), and its tie-ruled maximum folded on the device into the
 * running best.  Pushes of one stream object must be ordered (one CUDA
 * stream); pushes of n = 0 do nothing.
 * tde_stream_best: *found (host, nullable) = 1 once ny samples have arrived;
 * then the running best lag and value go to lag_out, val_out (device int64,
 * each nullable), asynchronously on `stream`.
 * tde_stream_destroy waits for the device and frees the stream's memory. */
typedef struct tde_stream tde_stream;
tde_status tde_stream_create(tde_ctx* ctx, const float* y, int64_t ny, int bits, int engine,
                             int64_t max_chunk, tde_stream_t stream, tde_stream** out);
tde_status tde_stream_push(tde_stream* s, const float* x, int64_t n, tde_stream_t stream);
tde_status tde_stream_best(tde_stream* s, int64_t* lag_out, int64_t* val_out, int* found,
                           tde_stream_t stream);
tde_status tde_stream_destroy(tde_stream* s);

/* Issue rates the engines' rooflines are measured against, per SM per SM
 * clock, on `device` (the paper has no counterpart: this is a measurement
 * utility).  Each is timed with the SM's own cycle counter inside one CTA per
 * SM, so the rate does not depend on the clock; multiply by sm_count and a
 * sampled SM clock for a per-second peak.
 *   popc_per_sm_clk:      32-bit __popc results (the popc engine's operation);
 *   imad_per_sm_clk:      32-bit integer multiply-adds (the NTT engine's);
 *   e4m3_mac_per_sm_clk:  MACs of back-to-back tcgen05.mma kind::f8f6f4,
 *                         M = 128, N = 256, K = 32, issued by one thread;
 *   e2m1_mac_per_sm_clk:  the same for kind::mxf4 (E2M1, unit block scales),
 *                         K = 64.
 * Synchronous; allocates and frees a few bytes of device memory and runs for
 * tens of milliseconds.  TDE_ERR_CUDA if a CUDA call fails, TDE_ERR_TIMEOUT if
 * the MMA probe's bounded wait gives up. */
typedef struct {
  int sm_count;
  double popc_per_sm_clk;
  double imad_per_sm_clk;
  double e4m3_mac_per_sm_clk;
  double e2m1_mac_per_sm_clk;
} tde_peaks;
tde_status tde_measure_peaks(int device, tde_peaks* out);

/* Failure-detection self-test: launches one CTA whose bounded device waits
 * (the ones every tensor-core kernel uses: a spinning and a suspending
 * mbarrier wait, each limited to 2 s of %globaltimer) run out on a barrier
 * that nothing arrives on.  The CTA then flags a time-out in the context's
 * status word and returns, as a kernel whose wait gave up does, so the next
 * tde_ctx_sync on `stream` returns TDE_ERR_TIMEOUT (after about 4 s) and the
 * context stays usable.  No fault, trap or unbounded wait is involved. */
tde_status tde_selftest_wait_timeout(tde_ctx* ctx, tde_stream_t stream);

/* Prime count of the NTT engine (Sec. 3.2's multimodular route), for the
 * plans made after this call.  nprimes = 0 (the default): modulo one prime
 * p0 = 15 * 2^27 + 1 wherever every value fits its centred residues
 * (shorter length * largest level magnitude^2 <= (p0 - 1) / 2), else two
 * primes recombined by the Chinese remainder theorem; nprimes = 2: always
 * two.  Both are exact.  TDE_ERR_INVALID for any other value. */
tde_status tde_ctx_set_ntt_primes(tde_ctx* ctx, int nprimes);

/* Counters since the previous read, then reset: kernel launches this context
 * enqueued (host pointer *kernel_launches), engine-kernel launches
 * (*engine_launches) and their summed device time in milliseconds
 * (*engine_ms, waits for the recorded events).  Any pointer may be NULL. */
tde_status tde_ctx_read_profile(tde_ctx* ctx, int64_t* kernel_launches, int64_t* engine_launches,
                                double* engine_ms);

/* One autotuner measurement: for `bits` and a pair of min(nx, ny) = 2^log2_n
 * samples asking 2^log2_lags lags, the engine TDE_ENGINE_AUTO uses and the
 * measured device time per pair of each engine in ns (index by TDE_ENGINE_*;
 * entry 0 unused; < 0: not measured or not supported). */
typedef struct {
  int32_t bits;
  int32_t log2_n;
  int32_t log2_lags;
  int32_t engine;
  float ns_per_pair[4];
} tde_tune_entry;

/* Autotune the engine choice: for each of the npoints (n[i], lag_count[i])
 * (host arrays; equal-length pairs of n[i] samples, lag_count[i] lags
 * centred on 0) time every exact engine on a batch of random levels sized to
 * fill the GPU (best of `reps` runs) and record the fastest in the context.
 * From then on TDE_ENGINE_AUTO (in every call on this context) takes the
 * engine of the recorded point nearest in (log2 n, log2 lags) for the same
 * bits, falling back to the built-in rule when no point has those bits.
 * Synchronizes the device; allocates and frees its own device buffers. */
tde_status tde_autotune(tde_ctx* ctx, int bits, const int64_t* n, const int64_t* lag_count,
                        int npoints, int reps);
/* Copy the context's table (host array of capacity `cap`); *count receives
 * the number of entries. */
tde_status tde_autotune_table(const tde_ctx* ctx, tde_tune_entry* out, int cap, int* count);
/* Replace the context's table by `count` entries (e.g. a cached table). */
tde_status tde_autotune_load(tde_ctx* ctx, const tde_tune_entry* entries, int count);
/* The engine TDE_ENGINE_AUTO runs on this context (its autotuner table, else
 * the built-in rule of tde_pick_engine); -1 if the arguments are invalid. */
int tde_ctx_pick_engine(const tde_ctx* ctx, int bits, int64_t nx, int64_t ny, int64_t lag_count);

/* The engine TDE_ENGINE_AUTO picks for one pair of lengths nx, ny, `bits`
 * and lag_count lags (host-only, enqueues nothing).  Returns a
 * TDE_ENGINE_* value, or -1 if the arguments are invalid. */
int tde_pick_engine(int bits, int64_t nx, int64_t ny, int64_t lag_count);

/* Algorithm 1's quantization step.  x: n floats (device).  q_out: n int8 (device).
 * bits in {1, 2, 4}.  NaN/Inf inputs are latched as TDE_ERR_INVALID (see
 * tde_ctx_sync) and the output is then unspecified. */
tde_status tde_quantize(tde_ctx* ctx, const float* x, int64_t n, int bits, int8_t* q_out,
                        tde_stream_t stream);

/* tde_quantize for nsig signals of n samples each, stored one after another:
 * x: nsig * n floats, q_out: nsig * n int8 (device).  Same levels and error
 * reporting as tde_quantize on each signal; one launch per pass for all. */
tde_status tde_quantize_batch(tde_ctx* ctx, const float* x, int64_t n, int nsig, int bits,
                              int8_t* q_out, tde_stream_t stream);

/* Allocation-free quantizer: the paper has no counterpart to this entry
 * point; it exists for callers that cannot allocate device memory, such as a
 * real-time audio callback that must not block in the allocator, a host that
 * runs this library under its own device-memory manager, or code enqueueing
 * work while a stream is captured.  Every other call needs a tde_ctx, which
 * allocates its workspace and pinned staging on demand; this one needs no
 * context and allocates nothing (no cudaMalloc, cudaFree or allocating
 * library routine).
 *
 * It quantizes nsig signals of n samples each, exactly like tde_quantize on
 * each of them: x holds nsig * n floats (device, signal after signal), q_out
 * receives nsig * n int8 (device).  status_out is one uint32 of caller-owned
 * device memory: the call zeroes it, and bit 0 is set if any input was NaN or
 * Inf (the output is then unspecified).  The calling thread's current device
 * is used.
 *
 * Scratch: the rank quantizer's histograms and radix-select state live in a
 * fixed file-scope device array (about 0.9 MiB) that every GPU loading the
 * library keeps until the process exits.  Limits: 1 <= nsig <= 16 and
 * n <= 2^31 - 1; larger requests return TDE_ERR_UNSUPPORTED and enqueue
 * nothing.  Other argument errors return TDE_ERR_INVALID.  The first call on
 * a device looks up the array's device address (cudaGetSymbolAddress, once per
 * device); make that first call before any stream capture.  The address is
 * kept for the life of the process, so do not use this entry point across a
 * cudaDeviceReset of that device.  All calls share the array and it keeps the
 * last call's contents (each call clears what it needs): calls whose work may
 * overlap on the GPU, e.g. on two unordered streams, race and give wrong
 * results. */
tde_status tde_quantize_noalloc(const float* x, int64_t n, int nsig, int bits, int8_t* q_out,
                                uint32_t* status_out, tde_stream_t stream);

/* Algorithm 1's correlation step / Eq. (1) on quantized input.  qx: nx int8, qy: ny int8
 * (device), with |q| <= 2^(bits-1) - 1 (1 for bits <= 2, 7 for bits = 4).
 * Computes c[tau] for lag_min <= tau <= lag_max, which must lie inside
 * [-(nx-1), ny-1].  c_out: (lag_max - lag_min + 1) elements of `out_dtype`
 * (TDE_I32 or TDE_I64), device.  `engine` is a TDE_ENGINE_* value.  The
 * result is exact for every engine. */
tde_status tde_xcorr_int(tde_ctx* ctx, const int8_t* qx, int64_t nx, const int8_t* qy,
                         int64_t ny, int bits, int64_t lag_min, int64_t lag_max, int engine,
                         void* c_out, int out_dtype, tde_stream_t stream);

/* Algorithm 1's argmax step.  c: `count` elements of `dtype` (device), element i
 * holding lag lag_min + i.  Writes the maximising lag and its value to
 * lag_out[0] and val_out[0] (device int64).  Ties go to the smallest |tau|,
 * then to the smallest tau.  count >= 1 and |lag| < 2^31 are required. */
tde_status tde_argmax(tde_ctx* ctx, const void* c, int dtype, int64_t lag_min, int64_t count,
                      int64_t* lag_out, int64_t* val_out, tde_stream_t stream);

/* Algorithm 1's last steps (Sec. 3.3, after the argmax): the set of lags
 * where the integer correlation c is maximal and, when it holds several, its
 * subset where the real cross-correlation (x * y)[tau] = sum_n x[n] y[n+tau]
 * of the original signals (Eq. (1) without quantization) is maximal; plus the
 * sub-sample offset of the real cross-correlation's peak at the set's
 * representative (the vertex of the parabola through tau - 1, tau, tau + 1).
 *   x: nx floats, y: ny floats (device, the signals c was computed from);
 *   c: `count` elements of `dtype` (device), element i holding lag lag_min + i;
 *   out: one tde_refined (device), written asynchronously:
 *     lag         the set's representative (smallest |tau|, then tau);
 *     value       the maximum of c;
 *     lag_lo/hi   the smallest and largest lag of the set (the paper counts an
 *                 estimate correct only if every lag of the set is);
 *     n_int_ties  lags where c is maximal; n_ties: size of the re-ranked set;
 *     r           (x * y)[lag] in FP64 (exact FP32 products, FP64 sums in a
 *                 fixed order; real ties are exact FP64 equality);
 *     frac        parabola vertex offset in [-0.5, 0.5]; 0 when a neighbour
 *                 has no overlap or the three values are not a strict peak.
 * The work is one FP64 dot per tied lag.  Uses a context workspace of
 * 16 * count bytes.  Errors: TDE_ERR_INVALID for null pointers, bad dtype,
 * sizes <= 0 or lags outside [-(nx-1), ny-1]. */
typedef struct tde_refined {
  int64_t lag, value, lag_lo, lag_hi, n_int_ties, n_ties;
  double r, frac;
} tde_refined;
tde_status tde_refine(tde_ctx* ctx, const float* x, int64_t nx, const float* y, int64_t ny,
                      const void* c, int dtype, int64_t lag_min, int64_t count, tde_refined* out,
                      tde_stream_t stream);

/* Algorithm 1 for one pair.  x: nx floats, y: ny floats (device).
 * Lags lag_min..lag_max as in tde_xcorr_int.  lag_out[0], val_out[0]: device
 * int64.  Intermediate quantized signals and correlations live in the
 * context's workspace. */
tde_status tde_estimate(tde_ctx* ctx, const float* x, int64_t nx, const float* y, int64_t ny,
                        int bits, int64_t lag_min, int64_t lag_max, int engine,
                        int64_t* lag_out, int64_t* val_out, tde_stream_t stream);

/* FP32 FFT correlation comparator (the real-valued FFT baseline of Sec. 2.3;
 * not exact, not on the estimator's path): for npairs equal-shape pairs,
 * c_out[p * count + i] = sum_n x_p[n] * y_p[n + lag_min + i] computed as
 * IDFT(conj(DFT x) DFT y) over a zero-padded power-of-two length
 * >= nx + ny - 1 in FP32 (cuFFT).  x: npairs * nx and y: npairs * ny elements
 * of in_dtype (TDE_F32 or TDE_I8, e.g. quantized levels), device, pair after
 * pair.  count = lag_max - lag_min + 1; lags as in tde_xcorr_int.  c_out:
 * npairs * count floats, device.  Transform buffers live in the context's
 * workspace; the cuFFT plan is cached in the context. */
tde_status tde_xcorr_fft32(tde_ctx* ctx, const void* x, const void* y, int in_dtype, int64_t nx,
                           int64_t ny, int npairs, int64_t lag_min, int64_t lag_max, float* c_out,
                           tde_stream_t stream);

/* One pair of a batch: device pointers and sizes, lag range inclusive. */
typedef struct {
  const float* x; /* device, nx floats */
  const float* y; /* device, ny floats */
  int64_t nx;
  int64_t ny;
  int64_t lag_min;
  int64_t lag_max;
} tde_pair_desc;

/* Algorithm 1 for `npairs` independent pairs of possibly uneven
 * lengths and lag ranges.  descs: host array of npairs descriptors.
 * lag_out, val_out: npairs int64 each (device).  If c_out is not NULL it
 * receives every pair's correlation as int32, pair after pair (pair p starts
 * at the sum of the earlier pairs' lag counts).  Same bits and engine for all
 * pairs.  Pairs are independent: the result of each equals tde_estimate on
 * it. */
tde_status tde_estimate_batch(tde_ctx* ctx, const tde_pair_desc* descs, int npairs, int bits,
                              int engine, int32_t* c_out, int64_t* lag_out, int64_t* val_out,
                              tde_stream_t stream);

/* A planned batch: the whole step of tde_estimate_batch (quantize every
 * signal, correlate every pair -- each engine one persistent launch over all
 * of its pairs' work, longest work first --, argmax every pair) captured once
 * into a CUDA graph over memory the batch owns, then replayed.  Descriptors,
 * bits, engine and the output pointers (c_out may be NULL, as in
 * tde_estimate_batch) are fixed at creation; the caller refills the input
 * buffers the descriptors point to between runs.  *out (host) receives the
 * handle.  Creation allocates device memory and synchronizes; runs do not
 * allocate. */
typedef struct tde_batch tde_batch;
tde_status tde_batch_create(tde_ctx* ctx, const tde_pair_desc* descs, int npairs, int bits,
                            int engine, int32_t* c_out, int64_t* lag_out, int64_t* val_out,
                            tde_batch** out);
/* Replays the batch's graph on `stream` (asynchronous).  Device-side errors
 * are reported by tde_ctx_sync on the batch's context. */
tde_status tde_batch_run(tde_batch* batch, tde_stream_t stream);
/* Synchronizes the device, frees the batch.  NULL is accepted. */
tde_status tde_batch_destroy(tde_batch* batch);

/* ------------------------------------------------------------------------
 * Learned lag proposal.  Not part of the paper's method: a small 1-D CNN
 * reads the quantized pair decimated 16x (block sums) and proposes the 8 most
 * likely 257-lag windows; the exact integer correlation (Eq. 1) is then
 * evaluated only inside them, and over the full range when the proposal's
 * confidence is low.  The returned lag is always the tie-ruled maximiser of
 * exact integer values (Algorithm 1's argmax step) over the lags evaluated.
 *
 * Architecture (weights shared by x and y): d[i] = (sum of 16 levels) / 4;
 * 4 x [conv1d kernel 9, padding 4, 32 channels, bias, ReLU, max-pool 2] ->
 * features f[32][n/256]; score[l] = alpha * sum_c sum_i fx[c][i] fy[c][i + l]
 * for bins l in [-(n/256 - 1), n/256 - 1]; bin l stands for the lags
 * [256 l - 128, 256 l + 128].  Weights are BF16 in the forward pass, all
 * accumulation FP32 (inference also rounds the activations of layers 2-4 to
 * BF16, where the tensor cores read them); training keeps FP32 master
 * weights and AdamW moments and is deterministic.  Pair p's quantized signals are q[(2p) n ..] (x) and
 * q[(2p+1) n ..] (y), int8, device. */
typedef struct tde_model tde_model;

/* Number of FP32 parameters of a model (host-only). */
int64_t tde_model_param_count(void);

/* A model for signals of n samples (n a multiple of 2048 in [16384, 2^24]),
 * weights drawn from `seed` (He-uniform), Adam state zero.  Allocates device
 * memory on ctx's device. */
tde_status tde_model_create(tde_ctx* ctx, int64_t n, uint64_t seed, tde_model** out);
tde_status tde_model_destroy(tde_model* model);

/* Checkpointing: copy (after a device synchronize) the parameters, the two
 * AdamW moments, the last gradient and the step count to host arrays of
 * tde_model_param_count() floats each; any pointer may be NULL. */
tde_status tde_model_get(const tde_model* model, float* params, float* adam_m, float* adam_v,
                         float* grad, int64_t* step);
/* Restore parameters (required), moments (NULL: zero) and step. */
tde_status tde_model_set(tde_model* model, const float* params, const float* adam_m,
                         const float* adam_v, int64_t step);

/* One AdamW step (beta 0.9 / 0.999, eps 1e-8, decoupled weight decay on conv
 * weights) of softmax cross-entropy against the bin holding each pair's label
 * lag.  labels: npairs int64 (device); loss_out: npairs floats (device), the
 * per-pair loss before the update. */
tde_status tde_train_step(tde_ctx* ctx, tde_model* model, const int8_t* q, int npairs,
                          const int64_t* labels, float lr, float weight_decay, float* loss_out,
                          tde_stream_t stream);

/* Proposal only: centres[8 p + r] (device int32, samples, = 256 l) of pair
 * p's r-th best bin and margin[p] (device float) = softmax mass of its top 8
 * bins. */
tde_status tde_propose(tde_ctx* ctx, const tde_model* model, const int8_t* q, int npairs,
                       int32_t* centres, float* margin, tde_stream_t stream);

/* tde_estimate_learned planned once for fixed buffers, with its own device
 * memory, and captured in a CUDA graph: tde_learned_run replays it on the
 * current contents of x and y (refill them between runs).  The model must
 * outlive the plan; its current parameters are read on every run. */
typedef struct tde_learned tde_learned;
tde_status tde_learned_create(tde_ctx* ctx, const tde_model* model, const float* x, const float* y,
                              int npairs, int bits, float theta, int64_t* lag_out,
                              int64_t* val_out, int32_t* fallback_out, tde_learned** out);
tde_status tde_learned_run(tde_learned* plan, tde_stream_t stream);
tde_status tde_learned_destroy(tde_learned* plan);

/* Eq. (1) inside the proposal's windows, exactly: for pair p (x = q + 2 p n,
 * y = q + (2 p + 1) n; q: 2 npairs n int8 levels, device, as tde_propose
 * reads them) and window w with centre centres[8 p + w] (device int32),
 * c_out[(8 p + w) * 257 + i] (device int32) = c[centre - 128 + i] for
 * i in [0, 257); lags outside [-(n-1), n-1] read 0.  Computed on the tensor
 * cores in polyphase form: with samples split as k = 128 a + b, the blocks
 * D_u[b][j] = sum_a x[128 a + b] y[128 (a + u) + j] that the windows need are
 * GEMMs over the rows a (E4M3 operands, FP32 accumulation over at most 512
 * rows, so every value is an exact integer), and each lag tau is the sum of
 * the diagonals j - b = tau - 128 u of its blocks, added in int32; longer
 * signals' segments of 512 rows are added as integers, so the result is
 * exact for every n.  bits 1, 2 or 4; levels must lie in the bits' range
 * (|q| <= 1, or <= 7 for bits 4): one outside it sets the status word, and
 * tde_ctx_sync then returns TDE_ERR_INVALID.  TDE_ERR_OVERFLOW if
 * n * (2^(bits-1))^2 >= 2^31 (the int32 bound).  Uses a context workspace of
 * 2 npairs * round_up(n, 128) bytes for the levels in E4M3, 24 bytes per
 * window and 4 per pair for the window descriptors. */
tde_status tde_xcorr_windows(tde_ctx* ctx, const int8_t* q, int64_t n, int npairs, int bits,
                             const int32_t* centres, int32_t* c_out, tde_stream_t stream);

/* Algorithm 1 with the proposal, for npairs pairs of n samples
 * (x, y: npairs * n floats each, device, pair after pair; all lags).  Pairs
 * whose margin is below theta (theta > 1: all pairs) get the full exact
 * correlation instead, decided and run on the device (tensor-core engine),
 * and are flagged in fallback_out (device int32 per pair, may be NULL).
 * bits 1 or 2.  Asynchronous on `stream` (no host synchronization). */
tde_status tde_estimate_learned(tde_ctx* ctx, const tde_model* model, const float* x,
                                const float* y, int npairs, int bits, float theta,
                                int64_t* lag_out, int64_t* val_out, int32_t* fallback_out,
                                tde_stream_t stream);

/* Seeded synthetic pairs on the device (a workload generator, not part of
 * the estimator): pair first + i gets shift d ~ U[-dmax, dmax], AR(1)
 * coefficient ~ U[ar_lo, ar_hi], SNR ~ U[snr_lo, snr_hi] dB; x = s[dmax ..],
 * y = s[dmax - d ..] plus independent Gaussian noise, so x[n] = y[n + d]
 * before noise.  x_out, y_out: npairs * n floats, shift_out: npairs int64
 * (device). */
tde_status tde_synth_pairs(tde_ctx* ctx, uint64_t seed, int64_t first, int npairs, int64_t n,
                           int64_t dmax, float ar_lo, float ar_hi, float snr_lo, float snr_hi,
                           float* x_out, float* y_out, int64_t* shift_out, tde_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* TDE_H_ */
