// mma.cu -- exact integer cross-correlation (Algorithm 1, line 3; Eq. (1) of
// arXiv 2509.19974) as a Toeplitz-structured GEMM on the 5th-generation
// tensor cores (tcgen05.mma, accumulators in tensor memory).
//
// The levels q in [-7, 7] are exact in BF16 and every product and partial sum
// is an integer below 2^24 in magnitude (a CTA covers at most kKs = 12288
// samples of the sum, 12288 * 49 < 2^20), so FP32 accumulation is exact;
// partial sums of several CTAs are combined with integer atomics.
// (tcgen05 has no 8-bit integer kind on sm_103a, so BF16 operands with FP32
// accumulation carry the integer arithmetic.)
//
// Tile: a CTA computes 32768 lags  tau = T0 + (127 - m) + 128 n  for
// m in [0,128) (TMEM lane) and n in [0,256) (TMEM column):
//   D[m][n] = sum_k A[m][k] B[n][k],
//   A[m][k] = qx[k - 127 + m]       (Hankel in m + k)
//   B[n][k] = qy[k + T0 + 128 n]    (rows = windows of y at stride 128)
// so D[m][n] = sum_i qx[i] qy[i + tau] = c[tau].  Both operands are K-major.
//
// B costs nothing to build: y is stored once in shared memory as two arrays
// of 128-byte rows (64 BF16), E[r] = y[128 r .. 128 r + 63] and
// O[r] = y[128 r + 64 .. 128 r + 127], in the 128-byte swizzled layout; the
// 256 x 64 B tile of a K chunk starting at k is rows floor(u/2) .. +255 of E
// (u even) or O (u odd), u = (k + T0) / 64 -- a descriptor whose start moves
// by one row every two chunks.  The 128-byte swizzle is a function of the
// absolute shared-memory address (16-byte chunk bits 4..6 XOR row bits 7..9),
// so rows are written swizzled by their own address and a descriptor may start
// at any 128-byte row with base offset 0 (checked on the device: a start off
// the 1024-byte pattern with base offset = address bits 7..9 reads wrong data).
//
// A costs 1 KB per chunk instead of 16 KB: in the no-swizzle K-major layout a
// core matrix is 8 rows x 16 bytes and core matrix (g, h) (rows 8g.., k 8h..)
// of the Hankel A depends only on d = g + h:
//   S[d][r][c] = qx[8 d + r + c - 127].
// With leading- and stride-byte offsets both 128, consecutive 128-byte slots
// S[d] serve every (g, h).  One 64-wide K chunk reads 23 consecutive slots
// and adds 8 new ones; the slots live in a ring of 48 with the first 24
// mirrored past its end so every window is contiguous.
//
// Roles: warp 0 writes the slots and lane 0 issues the MMAs (M=128, N=256,
// K=16) and tcgen05.commit per chunk; all 8 warps load y first and read the
// accumulator out at the end (warp w reads lanes 32 (w % 4) .., columns
// 128 (w / 4) ..).  Every wait is bounded by %globaltimer; on time-out the
// CTA flags TDE_ST_TIMEOUT, waits (bounded) for its MMAs and frees TMEM.
#include "common.cuh"
#include "mma.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kM = 128, kN = 256, kKc = 64, kKStep = 16;
constexpr int kRing = 48, kMirror = 24, kSlots = kRing + kMirror;
constexpr int kNB = 8;                                  // chunk commit barriers
constexpr int kRowsMax = kMmaKs / 128 + 256 + 8;        // y rows per half
constexpr int kYBytes = kRowsMax * 128;
constexpr int kSlotBytes = kSlots * 128;
constexpr int kSmemUsed = 2 * kYBytes + kSlotBytes + (kNB + 1) * 8 + 16;
constexpr int kSmemBytes = kSmemUsed + 1024;            // room to align the base
constexpr uint64_t kTimeoutNs = 2000000000ull;         // 2 s per wait
static_assert(kMmaTileLags == kM * kN, "tile");
static_assert(kMmaKs % kKc == 0, "segment");
static_assert(kYBytes % 1024 == 0, "y arrays stay 1024-aligned");
static_assert(kRing % 8 == 0 && kMirror >= 23 && kRing >= kMirror, "slot ring");

// Instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kN >> 3) << 17) |
                            ((uint32_t)(kM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: start >> 4 (bits 0-13), leading byte
// offset >> 4 (16-29), stride byte offset >> 4 (32-45), version 1 (46-47),
// base offset (49-51), layout (61-63: 0 none, 2 = 128-byte swizzle).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo,
                                          uint32_t layout, uint32_t base_off) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) |
         ((uint64_t)(base_off & 7u) << 49) | ((uint64_t)(layout & 7u) << 61);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ uint64_t now_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Waits for the phase of parity `parity` to complete; false after the limit.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  if (mbar_try(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  for (;;) {
    for (int i = 0; i < 32; ++i)
      if (mbar_try(bar, parity)) return true;
    if (now_ns() - t0 > kTimeoutNs) return false;
  }
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(kIdesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   bar)
               : "memory");
}

__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c,
                                             uint32_t d) {
  asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c),
               "r"(d)
               : "memory");
}

// 32 lanes x 32 consecutive columns of FP32 accumulator -> registers.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Exact BF16 encoding of a small integer: the top half of its FP32 pattern.
__device__ __forceinline__ uint32_t bf16_bits(int v) {
  return __float_as_uint((float)v) >> 16;
}
__device__ __forceinline__ uint32_t pack2(int lo, int hi) {
  return bf16_bits(lo) | (bf16_bits(hi) << 16);
}

__device__ __forceinline__ int64_t fdiv(int64_t a, int64_t b) {  // floor division, b > 0
  return a >= 0 ? a / b : -((-a + b - 1) / b);
}

__global__ void __launch_bounds__(kThreads, 2)
    k_xcorr_mma(const MmaPair* __restrict__ pairs, const MmaItem* __restrict__ items,
                uint32_t* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t yE = base, yO = base + kYBytes, slots = base + 2 * kYBytes;
  const uint32_t bars = slots + kSlotBytes;           // kNB chunk barriers + 1 "done"
  const uint32_t done_bar = bars + kNB * 8;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem_raw + (done_bar + 8 - raw));

  const MmaItem it = items[blockIdx.x];
  const MmaPair P = pairs[it.pair];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t T0 = it.T0, ks = it.ks, ke = it.ke;
  const int nchunks = (int)((ke - ks) / kKc);
  const int64_t u_s = (ks + T0) / kKc, u_l = (ke - kKc + T0) / kKc;  // exact
  const int64_t r_lo = fdiv(fdiv(u_s, 2), 8) * 8;
  const int64_t nrows = fdiv(u_l, 2) + 255 - r_lo + 1;
  // The CTA's own bounds check: the y window must fit its arrays.
  if (nrows > kRowsMax || nchunks <= 0) {
    if (threadIdx.x == 0) atomicOr(status, TDE_ST_INTERNAL);
    return;
  }

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(256)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    for (int i = 0; i <= kNB; ++i) mbar_init(bars + 8 * i, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }

  // y window: rows r_lo .. r_lo + nrows - 1 of E and O, zero outside [0, ny).
  const int8_t* qy = P.qy;
  const bool y_al8 = (reinterpret_cast<uintptr_t>(qy) & 7) == 0;
  for (int idx = threadIdx.x; idx < nrows * 16; idx += kThreads) {
    const int row = idx >> 4, half = (idx >> 3) & 1, ch = idx & 7;
    const int64_t q0 = 128 * (r_lo + row) + 64 * half + 8 * ch;
    int v[8];
    if (y_al8 && q0 >= 0 && q0 + 8 <= P.ny) {
      const uint2 w = *reinterpret_cast<const uint2*>(qy + q0);
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        v[t] = (int)(int8_t)(w.x >> (8 * t));
        v[4 + t] = (int)(int8_t)(w.y >> (8 * t));
      }
    } else {
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        const int64_t q = q0 + t;
        v[t] = (q >= 0 && q < P.ny) ? (int)qy[q] : 0;
      }
    }
    const uint32_t row_addr = (half ? yO : yE) + 128u * (uint32_t)row;
    const uint32_t phys = (uint32_t)ch ^ ((row_addr >> 7) & 7u);
    st_shared_v4(row_addr + 16u * phys, pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]),
                 pack2(v[6], v[7]));
  }
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  bool ok = true;
  if (warp == 0) {
    const int8_t* qx = P.qx;
    const int64_t d_begin = ks / 8;
    for (int c = 0; c < nchunks && ok; ++c) {
      // Slots written now overwrite those last read by chunk c - (kRing/8 - 2).
      const int prev = c - (kRing / 8 - 2);
      if (prev >= 0) ok = mbar_wait(bars + 8 * (prev % kNB), (uint32_t)((prev / kNB) & 1));
      ok = __all_sync(0xffffffffu, ok);
      if (!ok) break;
      const int e0 = c == 0 ? 0 : 8 * c + 15, e1 = 8 * c + 22;
      for (int idx = lane; idx < (e1 - e0 + 1) * 8; idx += 32) {
        const int e = e0 + (idx >> 3), r = idx & 7;
        const int64_t x0 = 8 * (d_begin + e) + r - 127;
        int v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) {
          const int64_t i = x0 + t;
          v[t] = (i >= 0 && i < P.nx) ? (int)qx[i] : 0;
        }
        const int p = e % kRing;
        const uint32_t a = slots + 128u * p + 16u * r;
        st_shared_v4(a, pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]),
                     pack2(v[6], v[7]));
        if (p < kMirror)
          st_shared_v4(a + 128u * kRing, pack2(v[0], v[1]), pack2(v[2], v[3]), pack2(v[4], v[5]),
                       pack2(v[6], v[7]));
      }
      fence_proxy_async();
      __syncwarp();
      if (lane == 0) {
        tc_fence_after();
        const int64_t u = u_s + c;
        const int64_t half = u & 1;  // two's complement: u mod 2
        const int64_t row0 = fdiv(u, 2) - r_lo;
        const uint32_t a_start = slots + 128u * (uint32_t)((8 * c) % kRing);
        const uint32_t b_row = (half ? yO : yE) + 128u * (uint32_t)row0;
#pragma unroll
        for (int s = 0; s < kKc / kKStep; ++s) {
          const uint64_t ad = sdesc(a_start + 256u * s, 128, 128, 0, 0);
          const uint32_t bs = b_row + 32u * s;
          const uint64_t bd = sdesc(bs, 16, 1024, 2, 0);
          mma_bf16(tmem, ad, bd, (c > 0 || s > 0) ? 1u : 0u);
        }
        mma_commit(bars + 8 * (c % kNB));
      }
      __syncwarp();
    }
    if (lane == 0) mma_commit(done_bar);
    __syncwarp();
  }

  // Epilogue: every thread waits for the accumulator.
  const bool done = mbar_wait(done_bar, 0);
  ok = __syncthreads_and(ok && done);
  if (!ok) {
    if (threadIdx.x == 0) atomicOr(status, TDE_ST_TIMEOUT);
  } else {
    tc_fence_after();
    const int q = warp & 3, colh = warp >> 2;
    const int m = 32 * q + lane;
    for (int cb = 0; cb < 4; ++cb) {
      const int col0 = 128 * colh + 32 * cb;
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)col0, v);
#pragma unroll
      for (int j = 0; j < 32; ++j) {
        const int64_t tau = T0 + 127 - m + 128 * (int64_t)(col0 + j);
        if (tau < P.lag_min || tau > P.lag_max) continue;
        const int val = __float2int_rn(__uint_as_float(v[j]));
        const int64_t o = tau - P.lag_min;
        if (P.c64) {
          if (it.single)
            static_cast<long long*>(P.c)[o] = val;
          else
            atomicAdd(reinterpret_cast<unsigned long long*>(P.c) + o, (unsigned long long)(long long)val);
        } else {
          if (it.single)
            static_cast<int*>(P.c)[o] = val;
          else
            atomicAdd(static_cast<int*>(P.c) + o, val);
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(256)
                 : "memory");
  }
}

// Zeroes the outputs of pairs whose tiles are split over several CTAs.
__global__ void k_zero_outputs(const MmaPair* __restrict__ pairs) {
  const MmaPair P = pairs[blockIdx.y];
  if (!P.zero_first) return;
  const int64_t count = P.lag_max - P.lag_min + 1;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
    if (P.c64)
      static_cast<long long*>(P.c)[i] = 0;
    else
      static_cast<int*>(P.c)[i] = 0;
  }
}

}  // namespace

int mma_smem_bytes() { return kSmemBytes; }

cudaError_t launch_mma_zero(const MmaPair* d_pairs, int npairs, int64_t max_count, cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  int64_t gx = ceil_div64(max_count, 256 * 8);
  if (gx > 1024) gx = 1024;
  if (gx < 1) gx = 1;
  k_zero_outputs<<<dim3((unsigned)gx, npairs), 256, 0, st>>>(d_pairs);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_xcorr_mma(const MmaPair* d_pairs, const MmaItem* d_items, int nitems,
                             uint32_t* d_status, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_xcorr_mma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSmemBytes);
  if (e != cudaSuccess) return e;
  k_xcorr_mma<<<nitems, kThreads, kSmemBytes, st>>>(d_pairs, d_items, d_status);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}
