// common.cuh -- types shared by the kernels and the C-ABI layer of libtde.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include "tde.h"

// An NVTX range named after one C-ABI call, for profiler timelines (a no-op
// unless a tool is attached).
struct ApiRange {
  explicit ApiRange(const char* name) { nvtxRangePushA(name); }
  ~ApiRange() { nvtxRangePop(); }
  ApiRange(const ApiRange&) = delete;
  ApiRange& operator=(const ApiRange&) = delete;
};

// Bits of the per-context device status word (see tde_ctx_sync).
#define TDE_ST_NONFINITE 1u  // NaN or Inf in a quantizer input
#define TDE_ST_TIMEOUT 2u    // a bounded wait gave up
#define TDE_ST_INTERNAL 4u   // a kernel's own bounds check refused an access

// ------------------------------------------------------------ E4M3 levels
#ifdef __CUDACC__
// Four int8 levels in [-7, 7] -> four E4M3 bytes (exact): magnitudes through
// a byte-permute table, sign bits copied.
__device__ __forceinline__ uint32_t e4m3x4(uint32_t w) {
  const uint32_t mag = __vabs4(w);
  const uint32_t sel = (mag & 0xFu) | ((mag >> 4) & 0xF0u) | ((mag >> 8) & 0xF00u) |
                       ((mag >> 12) & 0xF000u);
  // bytes of {hi:lo}: 0 -> 0x00, 1 -> 0x38, 2 -> 0x40, 3 -> 0x44, 4 -> 0x48,
  // 5 -> 0x4A, 6 -> 0x4C, 7 -> 0x4E
  return __byte_perm(0x44403800u, 0x4E4C4A48u, sel) | (w & 0x80808080u);
}
__device__ __forceinline__ uint4 e4m3x16(uint4 v) {
  return make_uint4(e4m3x4(v.x), e4m3x4(v.y), e4m3x4(v.z), e4m3x4(v.w));
}

// Four int8 levels in {-1, 0, 1} -> four packed E2M1 nibbles (exact: 0 ->
// 0x0, 1 -> 0x2 = 1.0, -1 -> 0xA = -1.0), level i in bits 4i .. 4i + 3, so
// sample 2j of a packed signal sits in the low nibble of byte j.  Nibble of
// byte b: bit 1 if b != 0, bit 3 = b's sign.
__device__ __forceinline__ uint32_t e2m1x4(uint32_t w) {
  const uint32_t t = (__vcmpne4(w, 0u) & 0x02020202u) | ((w >> 4) & 0x08080808u);
  const uint32_t u = t | (t >> 4);
  return (u & 0xFFu) | ((u >> 8) & 0xFF00u);
}
// 16 levels -> 8 bytes of packed E2M1
__device__ __forceinline__ uint2 e2m1x16(uint4 v) {
  return make_uint2(e2m1x4(v.x) | (e2m1x4(v.y) << 16), e2m1x4(v.z) | (e2m1x4(v.w) << 16));
}
#endif

// ---------------------------------------------------------------- quantize
// One signal to quantize: n floats at x -> n int8 at q.
struct QSig {
  const float* x;
  int8_t* q;
  int64_t n;
};

// Radix-select state of the rank quantizer for one signal: for each threshold
// m (0-based, at most 7) the bits of |x| fixed so far and the rank still to
// find among the elements that share them.
struct RankState {
  uint32_t prefix[7];
  uint32_t rank[7];
};

// Optional bit-plane output of the rank quantizer for one signal (layout of
// PlaneSig below: plane p word w at planes[p * words + w]).
struct QPlanes {
  uint32_t* planes;
  int64_t words;
};

// ------------------------------------------------------------- popc engine
// Bit-plane image of one quantized signal: plane 0 = sign (q < 0); for
// bits <= 2 plane 1 = (q != 0); for bits = 4 planes 1..3 = bits 0..2 of |q|.
// Word w of plane p is planes[p * words + w], bit i = sample 32 w + i.
struct PlaneSig {
  const int8_t* q;
  uint32_t* planes;
  int64_t n;
  int64_t words;
};

// One correlation problem for the direct engines.
struct XcPair {
  const uint32_t* px;  // planes of x
  const uint32_t* py;  // planes of y
  int64_t wx, wy;      // words per plane
  int64_t lag_min, lag_max;
  void* c;             // output, lag_max - lag_min + 1 elements
  int c64;             // 1: int64 output, 0: int32 output
};

// One CTA of the popc engine: pair index and the first 32-lag block index a0
// (lags 32*a0 .. 32*(a0 + 64) - 1, floor division).
struct PopcItem {
  int32_t pair;
  int32_t pad;
  int64_t a0;
};

// ------------------------------------------------------------------ argmax
struct ArgPair {
  const void* c;
  int64_t lag_min;
  int64_t count;
  int64_t* lag_out;
  int64_t* val_out;
};

// ----------------------------------------------------------- host launchers
// Each returns the first CUDA error it met (cudaSuccess otherwise).  All
// descriptor pointers below are device pointers.
cudaError_t launch_quantize_sign(const QSig* d_sigs, int nsig, int64_t max_n, uint32_t* d_status,
                                 cudaStream_t st);
// Rank quantizer for bits in {2,4}.  d_state: nsig RankState; d_hist:
// nsig * 7 * 2048 uint32 of scratch.
// Work memory of the streaming rank quantizer: a 4096-bin histogram, a
// 7 x 1024-bin candidate histogram and a QState per signal, and per signal a
// candidate list with room for n keys.
struct QState {
  uint32_t pre[7];   // threshold digits found so far
  uint32_t rank[7];  // rank within them
  uint32_t thr[7];   // final thresholds (FP32 bit patterns of |x|)
  int32_t owner[7];  // first threshold with the same prefix (shares its histogram)
  uint32_t ncand;    // keys in the candidate list
};
// Slack words of a candidate list beyond the signal's length: the one-launch
// quantizer keeps one column per thread (up to n + 2048 entries).
constexpr size_t kQCandSlack = 2048;
struct QWork {
  uint32_t* hist;               // [nsig][4096]
  QState* state;                // [nsig]
  uint32_t* const* cand;        // [nsig] device pointers to lists of 2 (n + kQCandSlack) words (keys, index | sign)
  uint32_t* chist;              // [nsig][7][1024] candidate histograms
};
// The rank quantizer (bits 2, 4) as five streaming launches; d_planes
// (nullable) receives each signal's bit planes as well.
cudaError_t launch_quantize_stream(const QSig* d_sigs, const QPlanes* d_planes, int nsig,
                                   int64_t max_n, int bits, QWork w, uint32_t* d_status,
                                   cudaStream_t st);
cudaError_t launch_quantize_rank(const QSig* d_sigs, int nsig, int64_t max_n, int bits,
                                 RankState* d_state, uint32_t* d_hist, uint32_t* d_status,
                                 cudaStream_t st);

// Flags TDE_ST_INTERNAL if a level exceeds the bits' range (|q| > 1 or > 7).
cudaError_t launch_pack_planes(const PlaneSig* d_sigs, int nsig, int64_t max_words, int bits,
                               uint32_t* d_status, cudaStream_t st);
// Number of lags one popc CTA covers.
constexpr int kPopcLagsPerCta = 2048;
cudaError_t launch_xcorr_popc(const XcPair* d_pairs, const PopcItem* d_items, int nitems, int bits,
                              cudaStream_t st);

// d_keys: npairs * 2 uint64 of scratch.  d_count (device, nullable): only
// pairs [0, *d_count) are reduced.
cudaError_t launch_argmax(const ArgPair* d_pairs, int npairs, int64_t max_count, int c64,
                          unsigned long long* d_keys, cudaStream_t st,
                          const int* d_count = nullptr);

// Kernel launches enqueued by this host thread (read by the context).
extern thread_local int64_t tde_launch_counter;
#define TDE_COUNT_LAUNCH(n) (tde_launch_counter += (n))

static inline int64_t ceil_div64(int64_t a, int64_t b) { return (a + b - 1) / b; }
static inline int64_t floor_div64(int64_t a, int64_t b) {
  return a >= 0 ? a / b : -((-a + b - 1) / b);
}
