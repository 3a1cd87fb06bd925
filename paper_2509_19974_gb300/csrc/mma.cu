// mma.cu -- exact integer cross-correlation (Algorithm 1's correlation step; Eq. (1) of
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
// Only column groups (32 columns = 4096 lags) whose overlap meets a chunk are
// multiplied: the MMA's N shrinks at the ends of a tile's K range, so the
// MACs issued stay within a few percent of the overlap MACs for long pairs.
//
// Roles: all 8 warps stage y (BF16, swizzled) and the segment of x (int8) in
// shared memory; warps 1-2 (64 threads) write one 16-byte slot row each per
// chunk and arrive on the chunk's "full" barrier; warp 0 lane 0 waits on it,
// issues the chunk's MMAs (M=128, K=16, N = 32..256) and tcgen05.commit's the
// chunk's barrier, which the producers wait on before overwriting ring slots;
// at the end all warps read the accumulator (warp w: lanes 32 (w % 4) ..,
// columns 128 (w / 4) ..).  Every wait is bounded by %globaltimer; on time-out
// the CTA flags TDE_ST_TIMEOUT, waits (bounded) for its MMAs and frees TMEM.
#include "cnn.cuh"
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
constexpr int kXBytes = kMmaKs + 272;                   // x samples a segment's slots read
constexpr int kProducers = 64;                          // slot-writing threads (warps 1, 2)
constexpr int kGroups = 8, kGroupCols = kN / kGroups;   // column groups of 32 (4096 lags)
constexpr int kSmemUsed = 2 * kYBytes + kSlotBytes + kXBytes + (2 * kNB + 1) * 8 + 16;  // + tmem/item words
constexpr int kSmemBytes = kSmemUsed + 1024;            // room to align the base
constexpr uint64_t kTimeoutNs = 2000000000ull;         // 2 s per wait
static_assert(kMmaTileLags == kM * kN, "tile");
static_assert(kMmaKs % kKc == 0, "segment");
static_assert(kYBytes % 1024 == 0, "y arrays stay 1024-aligned");
static_assert(kRing % 8 == 0 && kMirror >= 23 && kRing >= kMirror, "slot ring");
static_assert(kXBytes % 16 == 0, "x stage");
static_assert(2 * (kSmemBytes + 1024) <= 228 * 1024, "two CTAs per SM");

// Instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28.
__host__ __device__ constexpr uint32_t idesc_for(int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(kM >> 4) << 24);
}

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

// As mbar_wait, but each try may suspend the thread in hardware for up to
// ~20 us awaiting the phase (no issue slots spent spinning).
__device__ __forceinline__ bool mbar_try_sleep(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(20000u)
      : "memory");
  return ok != 0;
}
__device__ __noinline__ bool mbar_wait_sleep(uint32_t bar, uint32_t parity) {
  if (mbar_try_sleep(bar, parity)) return true;
  const uint64_t t0 = now_ns();
  for (;;) {
    if (mbar_try_sleep(bar, parity)) return true;
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

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

// Zeroes 32 lanes x 32 columns of tensor memory.
__device__ __forceinline__ void tmem_zero32(uint32_t taddr) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
      "{%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
      "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(taddr),
      "r"(0u)
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

// Unpacks 8 int8 levels (little-endian in w) to 8 BF16 and stores them as one
// 16-byte core-matrix row at `addr` (and at `addr2` if non-zero).
__device__ __forceinline__ void store_row8(uint32_t addr, uint32_t addr2, uint64_t w) {
  int v[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) v[t] = (int)(int8_t)(w >> (8 * t));
  const uint32_t w0 = pack2(v[0], v[1]), w1 = pack2(v[2], v[3]);
  const uint32_t w2 = pack2(v[4], v[5]), w3 = pack2(v[6], v[7]);
  st_shared_v4(addr, w0, w1, w2, w3);
  if (addr2) st_shared_v4(addr2, w0, w1, w2, w3);
}

__device__ __forceinline__ uint64_t ld_shared_u64(uint32_t addr) {
  uint64_t v;
  asm volatile("ld.shared.b64 %0, [%1];" : "=l"(v) : "r"(addr) : "memory");
  return v;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
  asm volatile("{\n\t.reg .b64 st;\n\tmbarrier.arrive.shared::cta.b64 st, [%0];\n\t}" ::"r"(bar)
               : "memory");
}

// 16 int8 from global memory (zero outside [0, n)); vector load when aligned.
__device__ __forceinline__ uint4 load16(const int8_t* q, int64_t i0, int64_t n, bool al16) {
  if (al16 && i0 >= 0 && i0 + 16 <= n) return __ldg(reinterpret_cast<const uint4*>(q + i0));
  uint32_t w[4] = {0u, 0u, 0u, 0u};
#pragma unroll
  for (int t = 0; t < 16; ++t) {
    const int64_t i = i0 + t;
    const uint32_t b = (i >= 0 && i < n) ? (uint32_t)(uint8_t)q[i] : 0u;
    w[t >> 2] |= b << (8 * (t & 3));
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}

__global__ void __launch_bounds__(kThreads, 2)
    k_xcorr_mma(const MmaPair* __restrict__ pairs, const MmaItem* __restrict__ items, int nitems,
                int* __restrict__ counter, uint32_t* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t yE = base, yO = base + kYBytes, slots = base + 2 * kYBytes;
  const uint32_t xs = slots + kSlotBytes;   // int8 x segment
  const uint32_t full_bar = xs + kXBytes;   // kNB "slots written" barriers
  const uint32_t cmt_bar = full_bar + 8 * kNB;  // kNB "chunk MMAs done" barriers
  const uint32_t done_bar = cmt_bar + 8 * kNB;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem_raw + (done_bar + 8 - raw));
  volatile int* item_slot = reinterpret_cast<volatile int*>(tmem_slot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(256)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    for (int i = 0; i < kNB; ++i) {
      mbar_init(full_bar + 8 * i, kProducers);
      mbar_init(cmt_bar + 8 * i, 1);
    }
    mbar_init(done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // Persistent loop: items (pair, 32768-lag tile, K segment) are taken in
  // the host's order (longest first) from a global counter.  Barrier phases
  // continue across items: chunk cc0 + c of this CTA uses barrier
  // (cc0 + c) % kNB with parity ((cc0 + c) / kNB) & 1; "done" completes once per
  // item.
  int64_t cc0 = 0;
  uint32_t iter = 0;
  bool ok = true;
  for (;; ++iter) {
    if (threadIdx.x == 0) *item_slot = atomicAdd(counter, 1);
    __syncthreads();
    tc_fence_after();
    const int w_item = *item_slot;
    if (w_item >= nitems) break;
    const MmaItem it = items[w_item];
    const MmaPair P = pairs[it.pair];
    const int64_t T0 = it.T0, ks = it.ks, ke = it.ke;
    const int nchunks = (int)((ke - ks) / kKc);
    const int64_t u_s = (ks + T0) / kKc, u_l = (ke - kKc + T0) / kKc;  // exact
    const int64_t r_lo = fdiv(fdiv(u_s, 2), 8) * 8;
    const int64_t nrows = fdiv(u_l, 2) + 255 - r_lo + 1;
    // x is staged from a 16-byte aligned index; window o (x index ks - 127 + o)
    // sits at xs + xoff + o.
    const int64_t xs_base = fdiv(ks - 127, 16) * 16;
    const uint32_t xoff = (uint32_t)(ks - 127 - xs_base);
    // The CTA's own bounds checks: the y window and the x segment must fit.
    if (nrows > kRowsMax || nchunks <= 0 || (ke - ks) + 272 > kXBytes) {
      if (threadIdx.x == 0) atomicOr(status, TDE_ST_INTERNAL);
      --iter;  // "done" was not used
      __syncthreads();
      continue;
    }

    // y window: rows r_lo .. r_lo + nrows - 1 of E and O (zero outside [0, ny)),
    // 16 samples per load, four loads in flight per thread.
    {
      const int8_t* qy = P.qy;
      const bool al16 = (reinterpret_cast<uintptr_t>(qy) & 15) == 0;
      const int total = (int)nrows * 8;  // (row, half, quarter)
      for (int b0 = threadIdx.x; b0 < total; b0 += 4 * kThreads) {
        uint4 w[4];
  #pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int idx = b0 + k * kThreads;
          if (idx < total) {
            const int row = idx >> 3, half = (idx >> 2) & 1, j = idx & 3;
            w[k] = load16(qy, 128 * (r_lo + row) + 64 * half + 16 * j, P.ny, al16);
          }
        }
  #pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int idx = b0 + k * kThreads;
          if (idx < total) {
            const int row = idx >> 3, half = (idx >> 2) & 1, j = idx & 3;
            const uint32_t row_addr = (half ? yO : yE) + 128u * (uint32_t)row;
            const uint32_t sw = (row_addr >> 7) & 7u;
            store_row8(row_addr + 16u * ((uint32_t)(2 * j) ^ sw), 0u,
                       (uint64_t)w[k].x | ((uint64_t)w[k].y << 32));
            store_row8(row_addr + 16u * ((uint32_t)(2 * j + 1) ^ sw), 0u,
                       (uint64_t)w[k].z | ((uint64_t)w[k].w << 32));
          }
        }
      }
    }
    // x segment x[xs_base .. xs_base + kXBytes), zero outside [0, nx).
    {
      const int8_t* qx = P.qx;
      const bool al16 = (reinterpret_cast<uintptr_t>(qx) & 15) == 0;
      for (int i = threadIdx.x; i < kXBytes / 16; i += kThreads) {
        const uint4 w = load16(qx, xs_base + 16 * i, P.nx, al16);
        st_shared_v4(xs + 16u * i, w.x, w.y, w.z, w.w);
      }
    }
    // The accumulator starts at zero: column groups join the sum at different
    // chunks, so every MMA accumulates.
    if (warp < 4) {
      const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
      for (int cb = 0; cb < kN; cb += 32) tmem_zero32(tmem + lane_base + (uint32_t)cb);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    if (warp == 1 || warp == 2) {
      // Slot producers: thread t writes window o = 64 c + 120 + t of chunk c
      // (chunk 0 writes windows 0..183): slot e = o / 8, row r = o % 8, i.e.
      // x[ks - 127 + o .. + 7] as BF16.
      const int t = threadIdx.x - 32;
      for (int c = 0; c < nchunks; ++c) {
        // The slots written now were last read by chunk c - (kRing/8 - 2).
        const int64_t prev = cc0 + c - (kRing / 8 - 2);
        if (prev >= 0 && !mbar_wait(cmt_bar + 8 * (uint32_t)(prev % kNB), (uint32_t)((prev / kNB) & 1))) {
          ok = false;
          break;
        }
        const int o_first = c == 0 ? t : 64 * c + 120 + t;
        const int o_end = c == 0 ? 184 : 64 * c + 184;
        for (int o = o_first; o < o_end; o += kProducers) {
          const uint32_t pa = xs + xoff + (uint32_t)o;
          const uint32_t al = pa & ~7u, sh = 8u * (pa & 7u);
          const uint64_t lo = ld_shared_u64(al), hi = ld_shared_u64(al + 8u);
          const uint64_t w = sh ? (lo >> sh) | (hi << (64u - sh)) : lo;
          const int e = o >> 3, r = o & 7;
          const int ps = e % kRing;
          const uint32_t a = slots + 128u * ps + 16u * r;
          store_row8(a, ps < kMirror ? a + 128u * kRing : 0u, w);
        }
        fence_proxy_async();
        mbar_arrive(full_bar + 8 * (uint32_t)((cc0 + c) % kNB));
      }
    } else if (warp == 0) {
      // MMA issuer: the whole warp waits (a divergent warp whose other lanes sit
      // in a barrier wait would stall the issuing lane); lane 0 issues.  k range of column group g (columns 32 g .. 32 g + 31, lags
      // T0 + 4096 g ..): [lo_g, hi_g), relative to ks.
      int64_t glo[kGroups], ghi[kGroups];
  #pragma unroll
      for (int g = 0; g < kGroups; ++g) {
        const int64_t lo = -T0 - 128 * (int64_t)(kGroupCols * g + kGroupCols - 1);
        const int64_t hi = P.ny - T0 - 128 * (int64_t)(kGroupCols * g);
        glo[g] = (lo > 0 ? lo : 0) - ks;
        ghi[g] = (hi < P.nx + 127 ? hi : P.nx + 127) - ks;
      }
      for (int c = 0; c < nchunks; ++c) {
        const int64_t cc = cc0 + c;
        ok = __all_sync(0xffffffffu, mbar_wait(full_bar + 8 * (uint32_t)(cc % kNB), (uint32_t)((cc / kNB) & 1)));
        if (!ok) break;
        tc_fence_after();
        const int64_t kc = (int64_t)kKc * c;
        int ga = kGroups, gb = -1;
  #pragma unroll
        for (int g = 0; g < kGroups; ++g)
          if (glo[g] < kc + kKc && ghi[g] > kc) {
            ga = g < ga ? g : ga;
            gb = g;
          }
        if (gb >= ga && lane == 0) {
          const uint32_t idesc = idesc_for(kGroupCols * (gb - ga + 1));
          const int64_t u = u_s + c;
          const int64_t half = u & 1;  // two's complement: u mod 2
          const int64_t row0 = fdiv(u, 2) - r_lo + kGroupCols * ga;
          const uint32_t a_start = slots + 128u * (uint32_t)((8 * c) % kRing);
          const uint32_t b_row = (half ? yO : yE) + 128u * (uint32_t)row0;
          const uint32_t d_col = tmem + (uint32_t)(kGroupCols * ga);
  #pragma unroll
          for (int s2 = 0; s2 < kKc / kKStep; ++s2) {
            const uint64_t ad = sdesc(a_start + 256u * s2, 128, 128, 0, 0);
            const uint64_t bd = sdesc(b_row + 32u * s2, 16, 1024, 2, 0);
            mma_bf16(d_col, ad, bd, idesc, 1u);
          }
        }
        if (lane == 0) mma_commit(cmt_bar + 8 * (uint32_t)(cc % kNB));
        __syncwarp();
      }
      if (lane == 0) mma_commit(done_bar);
      __syncwarp();
    }

    // Epilogue: every thread waits for the accumulator.
    const bool done = mbar_wait(done_bar, iter & 1u);
    ok = __syncthreads_and(ok && done);
    if (!ok) {
      if (threadIdx.x == 0) atomicOr(status, TDE_ST_TIMEOUT);
      break;
    }
    {
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
    cc0 += nchunks;
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


// ---------------------------------------------------------------------------
// Windowed form (the learned proposal's exact check): for one pair and its 8
// windows, window w's lags are covered by tau = T_w + 128 j + 127 - m
// (j = 0..7, T_w = its first lag rounded down to a multiple of 128), 1024
// lags of which the window's <= 257 are kept.  A is the same Hankel slot ring
// as above.  B needs no per-chunk copies: each window's y segment is staged
// once per item as E/O arrays of 128-byte swizzled rows,
//   E_w[r] = y[ks + T_w + 128 r .. + 63],  O_w[r] = y[ks + T_w + 128 r + 64 .. + 127],
// and because ks and T_w are multiples of 128, the 8 B rows of window w for
// K chunk c are rows floor(c/2) .. + 7 of E_w (c even) or O_w (c odd) -- the
// same rows for every window.  Windows' arrays sit at a fixed stride, so one
// descriptor (stride byte offset = that stride) gives an N = 64 tile: 8
// windows x 8 columns.  A CTA takes items (pair, K segment) round-robin;
// partial sums are added into the zeroed window outputs with integer atomics.

constexpr int kWinW = kCnnTopK;                  // windows per pair (8)
constexpr int kWinJ = 8;                         // columns per window (one core-matrix group)
constexpr int kWinN = kWinW * kWinJ;             // MMA N = 64
constexpr int kWinKs = 4096;                     // max samples of the sum per item
constexpr int kWinRows = (kWinKs / kKc + 1) / 2 + kWinJ;  // E/O rows per window (40)
constexpr int kWinArr = kWinRows * 128;          // bytes per E (or O) array, = the SBO
constexpr int kWinXBytes = kWinKs + 272;
// Producers and the issuer synchronize once per super-chunk of kWinSC chunks
// (16 MMAs), on a slot ring of 128 (+ 24 mirrored): a super-chunk writes
// logical slots [32 s + 15, 32 s + 47) and its chunks read [32 s, 32 s + 47),
// so the slots it writes were last read by super-chunk s - 3.
constexpr int kWinSC = 4;
constexpr int kWinRing = 128, kWinMirror = 24;
constexpr int kWinSlotBytes = (kWinRing + kWinMirror) * 128;
constexpr int kWinSmemUsed = 2 * kWinW * kWinArr + kWinSlotBytes + kWinXBytes + (2 * kNB + 1) * 8 + 16;
constexpr int kWinSmemBytes = kWinSmemUsed + 1024;
static_assert(kWinArr % 1024 == 0, "windows' arrays keep the 1024-byte swizzle pattern");
static_assert(kWinXBytes % 16 == 0, "staging");
static_assert(kWinSmemBytes + 1024 <= 114 * 1024, "two CTAs per SM");
static_assert(kWinRing % 32 == 0 && kWinMirror >= 23, "slot ring");

__global__ void __launch_bounds__(kThreads, 2)
    k_xcorr_mma_win(const int8_t* __restrict__ q, int64_t n, int npairs, const WinJob* __restrict__ jobs,
                    int nseg, int seg, uint32_t* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t yE = base;                                 // window w at yE + w * kWinArr
  const uint32_t yO = yE + kWinW * kWinArr;
  const uint32_t slots = yO + kWinW * kWinArr;
  const uint32_t xs = slots + kWinSlotBytes;
  const uint32_t full_bar = xs + kWinXBytes;
  const uint32_t cmt_bar = full_bar + 8 * kNB;
  const uint32_t done_bar = cmt_bar + 8 * kNB;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem_raw + (done_bar + 8 - raw));
  __shared__ int64_t sT[kWinW], sLo[kWinW], sHi[kWinW];  // per window: T_w, lag range
  __shared__ int32_t* sC[kWinW];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kWinN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    for (int i = 0; i < kNB; ++i) {
      mbar_init(full_bar + 8 * i, kProducers);
      mbar_init(cmt_bar + 8 * i, 1);
    }
    mbar_init(done_bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  int64_t sc0 = 0;  // super-chunks issued by this CTA so far (barrier phases)
  uint32_t iter = 0;
  bool ok = true;
  const int nitems = npairs * nseg;
  const int64_t kmax = (n + 127 + 127) / 128 * 128;
  for (int item = blockIdx.x; item < nitems; item += gridDim.x, ++iter) {
    const int p = item / nseg, sgi = item - p * nseg;
    const int64_t ks = (int64_t)sgi * seg;
    const int64_t ke = ks + seg < kmax ? ks + seg : kmax;
    const int nchunks = (int)((ke - ks) / kKc);
    const int8_t* qx = q + (int64_t)(2 * p) * n;
    const int8_t* qy = q + (int64_t)(2 * p + 1) * n;
    const WinJob* J = jobs + (int64_t)p * kWinW;
    if (nchunks <= 0 || ke - ks > kWinKs || (ks & 127) != 0) {  // not for the host's segmentation
      if (threadIdx.x == 0 && nchunks > 0) atomicOr(status, TDE_ST_INTERNAL);
      --iter;
      continue;
    }
    const int64_t xs_base = fdiv(ks - 127, 16) * 16;
    const uint32_t xoff = (uint32_t)(ks - 127 - xs_base);
    const int nrows = (nchunks + 1) / 2 + kWinJ;  // rows of each E/O array this item reads
    if (threadIdx.x < kWinW) {
      const WinJob jw = J[threadIdx.x];
      sT[threadIdx.x] = fdiv(jw.lag_lo, 128) * 128;
      sLo[threadIdx.x] = jw.lag_lo;
      sHi[threadIdx.x] = jw.lag_hi;
      sC[threadIdx.x] = jw.c;
    }
    __syncthreads();
    // staging: x segment, then every window's E/O rows (int8 -> BF16, swizzled)
    {
      const bool alx = (reinterpret_cast<uintptr_t>(qx) & 15) == 0;
      const bool aly = (reinterpret_cast<uintptr_t>(qy) & 15) == 0;
      constexpr int kXV = kWinXBytes / 16;
      const int per_w = nrows * 8;  // (row, half, quarter) per window
      const int total = kXV + kWinW * per_w;
      for (int b0 = threadIdx.x; b0 < total; b0 += 8 * kThreads) {
        uint4 v[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int idx = b0 + k * kThreads;
          if (idx < kXV) {
            v[k] = load16(qx, xs_base + 16 * idx, n, alx);
          } else if (idx < total) {
            const int w = (idx - kXV) / per_w, r8 = (idx - kXV) - w * per_w;
            const int row = r8 >> 3, half = (r8 >> 2) & 1, jq = r8 & 3;
            v[k] = load16(qy, ks + sT[w] + 128 * row + 64 * half + 16 * jq, n, aly);
          }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int idx = b0 + k * kThreads;
          if (idx < kXV) {
            st_shared_v4(xs + 16u * (uint32_t)idx, v[k].x, v[k].y, v[k].z, v[k].w);
          } else if (idx < total) {
            const int w = (idx - kXV) / per_w, r8 = (idx - kXV) - w * per_w;
            const int row = r8 >> 3, half = (r8 >> 2) & 1, jq = r8 & 3;
            const uint32_t row_addr = (half ? yO : yE) + (uint32_t)(w * kWinArr + 128 * row);
            const uint32_t sw = (row_addr >> 7) & 7u;
            store_row8(row_addr + 16u * ((uint32_t)(2 * jq) ^ sw), 0u,
                       (uint64_t)v[k].x | ((uint64_t)v[k].y << 32));
            store_row8(row_addr + 16u * ((uint32_t)(2 * jq + 1) ^ sw), 0u,
                       (uint64_t)v[k].z | ((uint64_t)v[k].w << 32));
          }
        }
      }
    }
    if (warp < 4) {
      const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
      tmem_zero32(tmem + lane_base);
      tmem_zero32(tmem + lane_base + 32u);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    const int nsc = (nchunks + kWinSC - 1) / kWinSC;
    if (warp == 1 || warp == 2) {
      // Hankel slots of x (as in k_xcorr_mma), one super-chunk at a time
      const int t = threadIdx.x - 32;
      for (int sc = 0; sc < nsc; ++sc) {
        const int64_t g = sc0 + sc;
        const int64_t prev = g - 3;
        if (prev >= 0 && !mbar_wait_sleep(cmt_bar + 8 * (uint32_t)(prev % kNB), (uint32_t)((prev / kNB) & 1))) {
          ok = false;
          break;
        }
        const int c_last = (sc + 1) * kWinSC < nchunks ? (sc + 1) * kWinSC - 1 : nchunks - 1;
        const int o_first = sc == 0 ? 0 : 64 * (sc * kWinSC) + 120;
        const int o_end = 64 * c_last + 184;
        for (int o = o_first + t; o < o_end; o += kProducers) {
          const uint32_t pa = xs + xoff + (uint32_t)o;
          const uint32_t al = pa & ~7u, sh = 8u * (pa & 7u);
          const uint64_t lo = ld_shared_u64(al), hi = ld_shared_u64(al + 8u);
          const uint64_t w = sh ? (lo >> sh) | (hi << (64u - sh)) : lo;
          const int e = o >> 3, r = o & 7;
          const int ps = e % kWinRing;
          const uint32_t a = slots + 128u * ps + 16u * r;
          store_row8(a, ps < kWinMirror ? a + 128u * kWinRing : 0u, w);
        }
        fence_proxy_async();
        mbar_arrive(full_bar + 8 * (uint32_t)(g % kNB));
      }
    } else if (warp == 0) {
      const uint32_t idesc = idesc_for(kWinN);
      for (int sc = 0; sc < nsc; ++sc) {
        const int64_t g = sc0 + sc;
        ok = __all_sync(0xffffffffu, mbar_wait_sleep(full_bar + 8 * (uint32_t)(g % kNB), (uint32_t)((g / kNB) & 1)));
        if (!ok) break;
        tc_fence_after();
        if (lane == 0) {
          const int c_end = (sc + 1) * kWinSC < nchunks ? (sc + 1) * kWinSC : nchunks;
          for (int c = sc * kWinSC; c < c_end; ++c) {
            const uint32_t a_start = slots + 128u * (uint32_t)((8 * c) % kWinRing);
            const uint32_t b_start = ((c & 1) ? yO : yE) + 128u * (uint32_t)(c >> 1);
#pragma unroll
            for (int s2 = 0; s2 < kKc / kKStep; ++s2)
              mma_bf16(tmem, sdesc(a_start + 256u * s2, 128, 128, 0, 0),
                       sdesc(b_start + 32u * s2, 16, kWinArr, 2, 0), idesc, 1u);
          }
          mma_commit(cmt_bar + 8 * (uint32_t)(g % kNB));
        }
        __syncwarp();
      }
      if (lane == 0) mma_commit(done_bar);
      __syncwarp();
    }

    // one warp waits for the accumulator; the others block in the barrier
    bool done = true;
    if (warp == 3) done = mbar_wait_sleep(done_bar, iter & 1u);
    ok = __syncthreads_and(ok && done);
    if (!ok) {
      if (threadIdx.x == 0) atomicOr(status, TDE_ST_TIMEOUT);
      break;
    }
    {
      // warp w: TMEM lanes 32 (w % 4) .., windows 4 (w / 4) .. + 3 (columns 32 (w / 4) ..)
      tc_fence_after();
      const int qd = warp & 3, colh = warp >> 2;
      const int m = 32 * qd + lane;
      uint32_t v[32];
      tmem_ld32(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(32 * colh), v);
#pragma unroll
      for (int jj = 0; jj < 32; ++jj) {
        const int w = 4 * colh + (jj >> 3), j = jj & 7;
        const int64_t lo = sLo[w], hi = sHi[w];
        const int64_t tau = sT[w] + 128 * j + 127 - m;
        if (tau < lo || tau > hi) continue;
        const int val = __float2int_rn(__uint_as_float(v[jj]));
        if (val != 0) atomicAdd(sC[w] + (tau - lo), val);
      }
    }
    tc_fence_before();
    __syncthreads();
    sc0 += nsc;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kWinN)
                 : "memory");
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
                             int* d_counter, int grid, uint32_t* d_status, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_xcorr_mma, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSmemBytes);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(d_counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (grid > nitems) grid = nitems;
  k_xcorr_mma<<<grid, kThreads, kSmemBytes, st>>>(d_pairs, d_items, nitems, d_counter, d_status);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_xcorr_mma_windows(const int8_t* d_q, int64_t n, int npairs, const WinJob* d_jobs,
                                     uint32_t* d_status, cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  // K range [0, n + 127) rounded up to 128; segments are multiples of 128
  // (so that each segment's windows start on a 128-sample row)
  const int64_t kmax = ceil_div64(n + 127, 128) * 128;
  const int nseg = (int)ceil_div64(kmax, kWinKs);
  const int seg = (int)(ceil_div64(ceil_div64(kmax, nseg), 128) * 128);
  cudaError_t e = cudaFuncSetAttribute(k_xcorr_mma_win, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kWinSmemBytes);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t nitems = (int64_t)npairs * nseg;
  const int grid = (int)(nitems < 2 * sms ? nitems : 2 * sms);
  k_xcorr_mma_win<<<grid, kThreads, kWinSmemBytes, st>>>(d_q, n, npairs, d_jobs, nseg, seg, d_status);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}
