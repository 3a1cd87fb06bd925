// mma.cu -- exact integer cross-correlation (Algorithm 1's correlation step; Eq. (1) of
// arXiv 2509.19974) as a Toeplitz-structured GEMM on the 5th-generation
// tensor cores (tcgen05.mma, accumulators in tensor memory), and the
// learned proposal's convolution layers on the same tensor cores.  (The
// proposal's windows are in winpp.cu.)
//
// tcgen05 has no 8-bit integer kind on sm_103a, so the integer arithmetic
// rides on kind::f8f6f4 with E4M3 operands and FP32 accumulation: the levels
// -7..7 are exact in E4M3, every product is an exact integer, and a CTA sums
// at most kMmaKs = 24576 samples (24576 * 49 < 2^21 < 2^24), so every FP32
// partial sum is an exact integer; partial sums of several CTAs are combined
// with integer atomics.
//
// Tile: a CTA computes 32768 lags  tau = T0 + (127 - m) + 128 n  for
// m in [0,128) (TMEM lane) and n in [0,256) (TMEM column):
//   D[m][n] = sum_k A[m][k] B[n][k],
//   A[m][k] = qx[k - 127 + m]       (Hankel in m + k)
//   B[n][k] = qy[k + T0 + 128 n]    (rows = windows of y at stride 128)
// so D[m][n] = sum_i qx[i] qy[i + tau] = c[tau].  Both operands are K-major.
//
// B costs nothing to build: y is stored once in shared memory as 128-byte
// E4M3 rows Y[r] = y[128 r .. 128 r + 127] in the 128-byte swizzled layout;
// the 256-row tile of the K chunk starting at k is rows (k + T0)/128 .. + 255
// -- a descriptor whose start moves by one row per chunk.  The swizzle is a
// function of the absolute shared-memory address (16-byte chunk bits 4..6 XOR
// row bits 7..9), so rows are written swizzled by their own address and a
// descriptor may start at any 128-byte row with base offset 0.
//
// A costs 2 KB per 128-sample chunk instead of 16 KB: in the no-swizzle
// K-major layout a core matrix is 8 rows x 16 bytes, and core matrix (g, h)
// (rows 8 g.., k 16 h..) of the Hankel A is slot g + 2 h of
//   S[e][r][c] = qx[8 e + r + c - 127],
// so with stride byte offsets 128 (M direction) and 256 (leading, K) a run of
// 128-byte slots serves every core matrix.  The slots live in a ring with its
// first entries mirrored past the end so every MMA's run is contiguous.
//
// Only column groups (32 columns = 4096 lags) whose overlap meets a chunk are
// multiplied: the MMA's N shrinks at the ends of a tile's K range, so the
// MACs issued stay within a few percent of the overlap MACs for long pairs.
//
// Roles: all 8 warps stage y and the segment of x (int8 -> E4M3) in shared
// memory; warps 1-2 (64 threads) write the chunk's new slot rows and arrive on
// the chunk's "full" barrier; warp 0 waits on it (the whole warp, converged),
// lane 0 issues the chunk's MMAs (M=128, K=32, N = 32..256) and
// tcgen05.commit's the chunk's barrier, which the producers wait on before
// overwriting ring slots; at the end all warps read the accumulator (warp w:
// lanes 32 (w % 4) .., columns 128 (w / 4) ..).  Every wait is bounded by
// %globaltimer; on time-out the CTA flags TDE_ST_TIMEOUT, waits (bounded) for
// its MMAs and frees TMEM.
//
// Descriptor facts established on the device by one-MMA probes with
// controlled operand images (documented descriptor forms only): the leading
// byte offset is the K-direction core-matrix stride of the no-swizzle K-major
// layout, overlapping core matrices read correctly, and a B descriptor that
// starts off the 1024-byte swizzle pattern must keep base offset 0.
#include "cnn.cuh"
#include "common.cuh"
#include "mma.cuh"
#include "tc.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kM = 128, kN = 256;
constexpr int kNB = 8;                                  // chunk commit barriers
constexpr int kProducers = 64;                          // slot-writing threads (warps 1, 2)
constexpr int kGroups = 8, kGroupCols = kN / kGroups;   // column groups of 32 (4096 lags)
static_assert(kMmaTileLags == kM * kN, "tile");

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

// ---------------------------------------------------------------------------
// The engine kernel (kind::f8f6f4, E4M3 operands, FP32 accumulation).  Per K
// chunk of 128 samples:
//   B: y is staged once per item as one array of 128-byte E4M3 rows
//      Y[r] = y[128 r .. 128 r + 127] (128-byte swizzle); with T0 and ks
//      multiples of 128 the 256-row tile of chunk k is rows (k + T0)/128 ..
//      + 255 -- no E/O split.
//   A: Hankel slots S[e][r][c] = qx[8 e + r + c - 127], 16 bytes per row; core
//      matrix (g, h) (rows 8 g.., k 16 h..) is slot g + 2 h, so a K = 32 step
//      reads 18 consecutive slots with stride byte offsets 128 (M) and 256
//      (leading, K).  Chunk c reads slots [16 c, 16 c + 30) and adds 16; the
//      ring holds 96 slots with 32 mirrored past its end, and the slots a
//      chunk writes were last read by chunk c - 5.
// These forms were checked on the device by a one-MMA probe with controlled
// operand images (plain and Hankel A, B rows off the 1024-byte pattern, a
// second K step).  Roles, barriers, column-group skipping and the epilogue
// are those described at the top of this file.

constexpr int kKc8 = kMmaChunk;                   // 128 samples per chunk
constexpr int kRing8 = 96, kMirror8 = 32, kSlots8 = kRing8 + kMirror8;
constexpr int kSlotBytes8 = kSlots8 * 128;
constexpr int kRowsMax8 = kMmaKs / 128 + 256 + 8;  // y rows per item
constexpr int kYBytes8 = kRowsMax8 * 128;
constexpr int kXBytes8 = kMmaKs + 288;            // x samples a segment's slots read
constexpr int kSmemUsed8 = kYBytes8 + kSlotBytes8 + kXBytes8 + (2 * kNB + 1) * 8 + 16;
constexpr int kSmemBytes8 = kSmemUsed8 + 1024;
static_assert(kMmaKs % kKc8 == 0 && kYBytes8 % 1024 == 0 && kXBytes8 % 16 == 0, "fp8 layout");
static_assert(2 * (kSmemBytes8 + 1024) <= 228 * 1024, "two CTAs per SM");
static_assert(kMmaKs * 49 < (1 << 24), "exact FP32 sums");

// Instruction descriptor, kind::f8f6f4: D F32 (bits 4-5 = 1), A and B E4M3
// (format 0 at bits 7-9 and 10-12), both K-major, N >> 3 at 17, M >> 4 at 24.
__host__ __device__ constexpr uint32_t idesc8_for(int n) {
  return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kM >> 4) << 24);
}

__device__ __forceinline__ void mma_e4m3(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__global__ void __launch_bounds__(kThreads, 2)
    k_xcorr_mma8(const MmaPair* __restrict__ pairs, const MmaItem* __restrict__ items, int nitems_arg,
                 const int* __restrict__ d_nitems, int* __restrict__ counter,
                 uint32_t* __restrict__ status) {
  const int nitems = d_nitems ? *d_nitems : nitems_arg;
  if (nitems <= 0) return;  // (a device-made item list can be empty)
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t yr = base, slots = base + kYBytes8;
  const uint32_t xs = slots + kSlotBytes8;    // E4M3 x segment
  const uint32_t full_bar = xs + kXBytes8;
  const uint32_t cmt_bar = full_bar + 8 * kNB;
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
    const int nchunks = (int)((ke - ks) / kKc8);
    const int64_t u_s = fdiv(ks + T0, kKc8);                  // exact (host alignment)
    const int64_t r_lo = fdiv(u_s, 8) * 8;                     // 1024-byte aligned start row
    const int64_t nrows = u_s + nchunks - 1 + 255 - r_lo + 1;
    const int64_t xs_base = fdiv(ks - 127, 16) * 16;
    const uint32_t xoff = (uint32_t)(ks - 127 - xs_base);
    if (nrows > kRowsMax8 || nchunks <= 0 || (ke - ks) + 288 > kXBytes8 ||
        ((ks + T0) & (kKc8 - 1)) != 0 || (ks & (kKc8 - 1)) != 0) {
      if (threadIdx.x == 0) atomicOr(status, TDE_ST_INTERNAL);
      --iter;
      __syncthreads();
      continue;
    }

    // y rows r_lo .. r_lo + nrows - 1 (E4M3, swizzled), x segment (E4M3)
    {
      const int8_t* qy = P.qy;
      const int8_t* qx = P.qx;
      const bool aly = (reinterpret_cast<uintptr_t>(qy) & 15) == 0;
      const bool alx = (reinterpret_cast<uintptr_t>(qx) & 15) == 0;
      const int ny16 = (int)nrows * 8;       // 16-byte pieces of y
      const int total = ny16 + kXBytes8 / 16;
      for (int b0 = threadIdx.x; b0 < total; b0 += 4 * kThreads) {
        uint4 w[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int idx = b0 + k * kThreads;
          if (idx < ny16)
            w[k] = load16(qy, 128 * (r_lo + (idx >> 3)) + 16 * (idx & 7), P.ny, aly);
          else if (idx < total)
            w[k] = load16(qx, xs_base + 16 * (idx - ny16), P.nx, alx);
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int idx = b0 + k * kThreads;
          if (idx >= total) continue;
          const uint4 e = e4m3x16(w[k]);
          uint32_t a;
          if (idx < ny16) {
            const uint32_t row_addr = yr + 128u * (uint32_t)(idx >> 3);
            a = row_addr + 16u * ((uint32_t)(idx & 7) ^ ((row_addr >> 7) & 7u));
          } else {
            a = xs + 16u * (uint32_t)(idx - ny16);
          }
          st_shared_v4(a, e.x, e.y, e.z, e.w);
        }
      }
    }
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
      // Slot producers: row o = 8 e + r (slot e, row r) is x[ks - 127 + o .. + 15];
      // chunk 0 writes o in [0, 240), chunk c >= 1 writes [128 c + 112, 128 c + 240).
      // Lane (octet t / 8, row r = t % 8) writes row r of 2 consecutive slots
      // (128-byte runs per store): x bytes [xoff + 8 e + r, + 16) for e = e0,
      // e0 + 1, as aligned word pairs of the stream realigned once by
      // (xoff + r) mod 8 with byte permutes.
      const int t = threadIdx.x - 32, r = t & 7;
      for (int c = 0; c < nchunks; ++c) {
        const int64_t prev = cc0 + c - 5;
        if (prev >= 0) {
          const uint32_t cb = cmt_bar + 8 * (uint32_t)(prev % kNB), ph = (uint32_t)((prev / kNB) & 1);
          if (!mbar_try(cb, ph) && !mbar_wait(cb, ph)) {
            ok = false;
            break;
          }
        }
        const int e_lo = c == 0 ? 0 : 16 * c + 14, e_hi = 16 * c + 30;
        for (int e0 = e_lo + 2 * (t >> 3); e0 < e_hi; e0 += 2 * (kProducers / 8)) {
          const uint32_t pos = xoff + 8u * (uint32_t)e0 + (uint32_t)r;
          const uint32_t al = xs + (pos & ~7u);
          uint32_t u[8], a[6];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint64_t w = ld_shared_u64(al + 8u * i);
            u[2 * i] = (uint32_t)w, u[2 * i + 1] = (uint32_t)(w >> 32);
          }
          const bool wo = (pos & 4u) != 0;
          const uint32_t sel = 0x3210u + 0x1111u * (pos & 3u);
#pragma unroll
          for (int j = 0; j < 6; ++j)
            a[j] = __byte_perm(wo ? u[j + 1] : u[j], wo ? u[j + 2] : u[j + 1], sel);
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            if (e0 + k >= e_hi) break;
            const uint32_t ps = (uint32_t)(e0 + k) % (uint32_t)kRing8;
            const uint32_t ad = slots + 128u * ps + 16u * (uint32_t)r;
            st_shared_v4(ad, a[2 * k], a[2 * k + 1], a[2 * k + 2], a[2 * k + 3]);
            if (ps < (uint32_t)kMirror8)
              st_shared_v4(ad + 128u * kRing8, a[2 * k], a[2 * k + 1], a[2 * k + 2], a[2 * k + 3]);
          }
        }
        fence_proxy_async();
        mbar_arrive(full_bar + 8 * (uint32_t)((cc0 + c) % kNB));
      }
    } else if (warp == 0) {
      // MMA issuer (whole warp waits, lane 0 issues); column groups of 32
      int64_t glo[kGroups], ghi[kGroups];
#pragma unroll
      for (int g = 0; g < kGroups; ++g) {
        const int64_t lo = -T0 - 128 * (int64_t)(kGroupCols * g + kGroupCols - 1);
        const int64_t hi = P.ny - T0 - 128 * (int64_t)(kGroupCols * g);
        glo[g] = (lo > 0 ? lo : 0) - ks;
        ghi[g] = (hi < P.nx + 127 ? hi : P.nx + 127) - ks;
      }
      const uint64_t da0 = sdesc(slots, 256, 128, 0, 0);  // + ring slot * 8
      const uint64_t db0 = sdesc(yr, 16, 1024, 2, 0);     // + row * 8
      for (int c = 0; c < nchunks; ++c) {
        const int64_t cc = cc0 + c;
        {
          const uint32_t fb = full_bar + 8 * (uint32_t)(cc % kNB), ph = (uint32_t)((cc / kNB) & 1);
          ok = __all_sync(0xffffffffu, mbar_try(fb, ph) || mbar_wait(fb, ph));
        }
        if (!ok) break;
        tc_fence_after();
        const int64_t kc = (int64_t)kKc8 * c;
        int ga = kGroups, gb = -1;
#pragma unroll
        for (int g = 0; g < kGroups; ++g)
          if (glo[g] < kc + kKc8 && ghi[g] > kc) {
            ga = g < ga ? g : ga;
            gb = g;
          }
        if (gb >= ga && lane == 0) {
          const uint32_t idesc = idesc8_for(kGroupCols * (gb - ga + 1));
          const int64_t row0 = u_s + c - r_lo + kGroupCols * ga;
          const uint64_t ad = da0 + 8u * (uint32_t)((16 * c) % kRing8);
          const uint64_t bd = db0 + 8u * (uint32_t)row0;
          const uint32_t d_col = tmem + (uint32_t)(kGroupCols * ga);
#pragma unroll
          for (int s2 = 0; s2 < 4; ++s2) mma_e4m3(d_col, ad + 32u * s2, bd + 2u * s2, idesc, 1u);
        }
        if (lane == 0) mma_commit(cmt_bar + 8 * (uint32_t)(cc % kNB));
        __syncwarp();
      }
      if (lane == 0) mma_commit(done_bar);
      __syncwarp();
    }

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
// Pairs y = blockIdx.y, + gridDim.y, ... below npairs (or the device count
// d_count when the pairs were made on the device: the grid is then small).
__global__ void k_zero_outputs(const MmaPair* __restrict__ pairs, int npairs, const int* __restrict__ d_count) {
  int lim = npairs;
  if (d_count && *d_count < lim) lim = *d_count;
  for (int y = blockIdx.y; y < lim; y += gridDim.y) {
    const MmaPair P = pairs[y];
    if (!P.zero_first) continue;
    const int64_t count = P.lag_max - P.lag_min + 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += stride) {
      if (P.c64)
        static_cast<long long*>(P.c)[i] = 0;
      else
        static_cast<int*>(P.c)[i] = 0;
    }
  }
}


// Instruction descriptor, kind::mxf4 (block-scaled): A and B E2M1 (format 1,
// bits 7-9 and 10-12), both K-major, N >> 3 at bits 17-22, UE8M0 scales (bit
// 23), M >> 4 at bits 24-28, scale-factor ids 0 (bits 4-5 and 29-30).
__host__ __device__ constexpr uint32_t idesc4_for(int n) {
  return (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | (1u << 23) | ((uint32_t)(kM >> 4) << 24);
}

__device__ __forceinline__ void mma_mxf4(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t sfa, uint32_t sfb, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %6, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n\t}" ::"r"(
          d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(sfa), "r"(sfb), "r"(acc)
      : "memory");
}

// ---------------------------------------------------------------------------
// The engine on packed E2M1 operands (levels in {-1, 0, 1}, bits 1 and 2):
// tcgen05 kind::mxf4 with unit UE8M0 block scales, K = 64 samples per MMA, so
// an MMA does twice the work of the E4M3 form in the same time.  The block
// scales take 64 columns of tensor memory, so a tile is 128 lags x 128
// columns (16384 lags; two CTAs per SM still fit), an MMA of N = 128 at the
// same cost per column as N = 256.  Per K chunk of 128 samples:
//   B: y staged once per item as 64-byte rows of 128 packed samples,
//      Y[r] = y[128 r ..], in the 64-byte swizzle; the tile of chunk c is rows
//      (c + u_s - r_lo) .. + 127 (stride byte offset 512), the second K step
//      the rows' second 32 bytes.
//   A: the Hankel slots of the windows kernel (32 samples per slot row,
//      core matrix (g, h) = slot e0 + g + 4 h, e0 = 16 c + 8 s).
// Super-chunks of 4 chunks (8 MMAs per wait and commit, so the issuer's
// per-batch costs stay under the MMAs' time) on a ring of 256 slots (+ 32
// mirrored): super-chunk j reads [64 j, 64 j + 76) and writes [64 j + 12,
// 64 j + 76) (from 0 at an item's start); those slots were last read by
// super-chunk j - 3, which the producers wait for.  Items are staged into two
// buffers: while warp 0 issues and warps 1-2 write slots, warps 3-7 stage the
// next item's y and x, so staging leaves the MMAs' path.  Staging flags
// TDE_ST_INTERNAL for a level outside {-1, 0, 1}.  Column-group skipping,
// items, the epilogue and the bounded waits are the E4M3 engine's.

constexpr int kN4 = 128;                            // tile columns
constexpr int kGroups4 = kN4 / kGroupCols;          // column groups of 32
#ifndef TDE_M4_SC
#define TDE_M4_SC 4
#endif
#ifndef TDE_M4_RING
#define TDE_M4_RING 256
#endif
constexpr int kSC4 = TDE_M4_SC;                     // chunks per super-chunk
constexpr int kStep4 = 16 * kSC4;                   // new slots per super-chunk
constexpr int kRead4 = kStep4 + 12;                 // slots a super-chunk reads
constexpr int kRing4 = TDE_M4_RING, kMirror4 = 32;
constexpr int kSlotBytes4 = (kRing4 + kMirror4) * 128;
// the newest earlier super-chunk whose reads a super-chunk's writes may alias
constexpr int kBack4 = (kRing4 - kRead4) / kStep4 + 1;
static_assert(kBack4 >= 2 && kBack4 <= kNB, "super-chunks in flight fit the commit barriers");
constexpr int kRowsMax4 = kMmaKs4 / 128 + kN4 + 8;  // y rows per item
constexpr int kYBytes4 = (kRowsMax4 * 64 + 1023) / 1024 * 1024;
constexpr int kXBytes4 = (kMmaKs4 / 2 + 256 + 1023) / 1024 * 1024;  // packed x bytes a segment's slots read
constexpr int kCols4 = 256;                         // tensor memory: D 128 + block scales
constexpr int kScaleCol4 = 128;
constexpr int kStage4 = kYBytes4 + kXBytes4;        // one item's staged y and x
constexpr int kSmemUsed4 = 2 * kStage4 + kSlotBytes4 + (2 * kNB + 1) * 8 + 16;
constexpr int kSmemBytes4 = kSmemUsed4 + 1024;
static_assert(kStage4 % 1024 == 0, "staging buffers keep the 1024-byte alignment");
static_assert((32 + 8 * (16 * (kMmaKs4 / kKc8 - 1) + 28) + 7 + 40) / 2 + 8 <= kXBytes4, "x segment");
static_assert(kRing4 % kStep4 == 0 && kRing4 - kStep4 + kRead4 <= kRing4 + kMirror4, "ring and mirror");
static_assert(2 * (kSmemBytes4 + 1024) <= 228 * 1024 && 2 * kCols4 <= 512, "two CTAs per SM");
static_assert(kMmaKs4 < (1 << 24) && kMmaKs4 % kKc8 == 0, "exact FP32 sums of ternary products");

// One item's staging geometry.
struct Item4 {
  int64_t T0, ks, ke, u_s, r_lo, nrows, x0;
  int nchunks, nsc;
  uint32_t bp;
  bool valid;
};
__device__ __forceinline__ Item4 item4_of(const MmaItem& it) {
  Item4 g;
  g.T0 = it.T0, g.ks = it.ks, g.ke = it.ke;
  g.nchunks = (int)((g.ke - g.ks) / kKc8);
  g.nsc = (g.nchunks + kSC4 - 1) / kSC4;
  g.u_s = fdiv(g.ks + g.T0, kKc8);                  // exact (host alignment)
  g.r_lo = fdiv(g.u_s, 8) * 8;                       // 512-byte (swizzle atom) aligned start row
  g.nrows = g.u_s + g.nchunks - 1 + kN4 - 1 - g.r_lo + 1;
  g.x0 = fdiv(g.ks - 127, 32) * 32;                  // first packed x sample
  g.bp = (uint32_t)(g.ks - 127 - g.x0);              // nibble of sample ks - 127
  g.valid = g.nrows <= kRowsMax4 && g.nchunks > 0 && (g.ke - g.ks) <= kMmaKs4 &&
            ((g.ks + g.T0) & (kKc8 - 1)) == 0 && (g.ks & (kKc8 - 1)) == 0;
  return g;
}

// y rows r_lo .. r_lo + nrows - 1 and the x segment of an item, packed E2M1,
// by threads t0 .. t0 + nthr - 1: one 32-sample unit (16 bytes) per thread
// and step.  Returns whether a level outside {-1, 0, 1} was seen.
__device__ __forceinline__ bool stage4(const MmaPair& P, const Item4& g, uint32_t yr, uint32_t xs, int t,
                                       int nthr) {
  const int8_t* qy = P.qy;
  const int8_t* qx = P.qx;
  const bool aly = (reinterpret_cast<uintptr_t>(qy) & 15) == 0;
  const bool alx = (reinterpret_cast<uintptr_t>(qx) & 15) == 0;
  const int nyu = (int)g.nrows * 4;
  const int total = nyu + kXBytes4 / 16;
  bool bad = false;
  for (int b0 = t; b0 < total; b0 += 2 * nthr) {
    uint4 w[2][2];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int idx = b0 + k * nthr;
      if (idx < nyu) {
        const int64_t s0 = 128 * (g.r_lo + (idx >> 2)) + 32 * (idx & 3);
        w[k][0] = load16(qy, s0, P.ny, aly);
        w[k][1] = load16(qy, s0 + 16, P.ny, aly);
      } else if (idx < total) {
        const int64_t s0 = g.x0 + 32 * (int64_t)(idx - nyu);
        w[k][0] = load16(qx, s0, P.nx, alx);
        w[k][1] = load16(qx, s0 + 16, P.nx, alx);
      }
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const int idx = b0 + k * nthr;
      if (idx >= total) continue;
      const uint32_t lim = 0x01010101u;
      bad |= (__vcmpgtu4(__vabs4(w[k][0].x), lim) | __vcmpgtu4(__vabs4(w[k][0].y), lim) |
              __vcmpgtu4(__vabs4(w[k][0].z), lim) | __vcmpgtu4(__vabs4(w[k][0].w), lim) |
              __vcmpgtu4(__vabs4(w[k][1].x), lim) | __vcmpgtu4(__vabs4(w[k][1].y), lim) |
              __vcmpgtu4(__vabs4(w[k][1].z), lim) | __vcmpgtu4(__vabs4(w[k][1].w), lim)) != 0u;
      const uint2 lo = e2m1x16(w[k][0]), hi = e2m1x16(w[k][1]);
      uint32_t a;
      if (idx < nyu) {
        const uint32_t row_addr = yr + 64u * (uint32_t)(idx >> 2);
        a = row_addr + 16u * ((uint32_t)(idx & 3) ^ ((row_addr >> 7) & 3u));
      } else {
        a = xs + 16u * (uint32_t)(idx - nyu);
      }
      st_shared_v4(a, lo.x, lo.y, hi.x, hi.y);
    }
  }
  return bad;
}

__global__ void __launch_bounds__(kThreads, 2)
    k_xcorr_mma4(const MmaPair* __restrict__ pairs, const MmaItem* __restrict__ items, int nitems_arg,
                 const int* __restrict__ d_nitems, int* __restrict__ counter,
                 uint32_t* __restrict__ status) {
  const int nitems = d_nitems ? *d_nitems : nitems_arg;
  if (nitems <= 0) return;  // (a device-made item list can be empty)
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  const uint32_t stage0 = base;                 // staging buffer b at stage0 + b * kStage4: y, then x
  const uint32_t slots = base + 2 * kStage4;
  const uint32_t full_bar = slots + kSlotBytes4;
  const uint32_t cmt_bar = full_bar + 8 * kNB;
  const uint32_t done_bar = cmt_bar + 8 * kNB;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem_raw + (done_bar + 8 - raw));
  volatile int* item_slot = reinterpret_cast<volatile int*>(tmem_slot + 1);  // [0]: this item, [1]: next
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kCols4)
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
  if (threadIdx.x == 0) item_slot[1] = atomicAdd(counter, 1);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  if (warp >= 4) {  // block scales: UE8M0 1.0 in every byte of columns 128 .. 191
    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
#pragma unroll
    for (int c0 = 0; c0 < 64; c0 += 32)
      asm volatile(
          "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
          "{%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, "
          "%1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(tmem + lanes +
                                                                                   kScaleCol4 + c0),
          "r"(0x7F7F7F7Fu)
          : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  const uint32_t sfa = tmem + kScaleCol4, sfb = tmem + kScaleCol4 + 32;
  // the first item, staged by every thread
  {
    const int w0 = item_slot[1];
    if (w0 < nitems) {
      const MmaItem it = items[w0];
      const Item4 g = item4_of(it);
      if (g.valid && stage4(pairs[it.pair], g, stage0, stage0 + kYBytes4, threadIdx.x, kThreads))
        atomicOr(status, TDE_ST_INTERNAL);
    }
  }

  int64_t sc0 = 0;      // super-chunks of earlier items
  uint32_t ndone = 0;   // items whose MMAs were committed to done_bar
  uint32_t iter = 0;    // items taken (the staging buffer alternates with it)
  bool ok = true;
  for (;; ++iter) {
    __syncthreads();  // the previous item's epilogue and this item's staging are done
    if (threadIdx.x == 0) {
      item_slot[0] = item_slot[1];
      if (item_slot[0] < nitems) item_slot[1] = atomicAdd(counter, 1);
    }
    __syncthreads();
    tc_fence_after();
    const int w_item = item_slot[0];
    if (w_item >= nitems) break;
    const int w_next = item_slot[1];
    const MmaItem it = items[w_item];
    const MmaPair P = pairs[it.pair];
    const Item4 g = item4_of(it);
    const uint32_t yr = stage0 + (iter & 1u) * kStage4, xs = yr + kYBytes4;
    if (!g.valid) {
      if (threadIdx.x == 0) atomicOr(status, TDE_ST_INTERNAL);
      // (nothing was staged for it; the next item is staged below by everyone)
      if (w_next < nitems) {
        const MmaItem itn = items[w_next];
        const Item4 gn = item4_of(itn);
        const uint32_t yn = stage0 + ((iter + 1) & 1u) * kStage4;
        if (gn.valid && stage4(pairs[itn.pair], gn, yn, yn + kYBytes4, threadIdx.x, kThreads))
          atomicOr(status, TDE_ST_INTERNAL);
      }
      continue;
    }
    if (warp < 4) {
      const uint32_t lane_base = (uint32_t)(32 * warp) << 16;
      for (int cb = 0; cb < kN4; cb += 32) tmem_zero32(tmem + lane_base + (uint32_t)cb);
      asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();

    if (warp == 1 || warp == 2) {
      // Slot producers: lane (octet o, row r) writes row r of the slots e0,
      // e0 + 1 from five funnel-shifted words of the packed x segment
      const int t = threadIdx.x - 32, r = t & 7, o = t >> 3;
      for (int j = 0; j < g.nsc; ++j) {
        const int64_t prev = sc0 + j - kBack4;
        if (prev >= 0) {
          const uint32_t cb = cmt_bar + 8 * (uint32_t)(prev % kNB), ph = (uint32_t)((prev / kNB) & 1);
          if (!mbar_try(cb, ph) && !mbar_wait(cb, ph)) {
            ok = false;
            break;
          }
        }
        const int c_last = kSC4 * j + kSC4 - 1 < g.nchunks ? kSC4 * j + kSC4 - 1 : g.nchunks - 1;
        const int e_lo = j == 0 ? 0 : kStep4 * j + (kRead4 - kStep4), e_hi = 16 * c_last + 28;
        for (int e0 = e_lo + 2 * o; e0 < e_hi; e0 += 2 * (kProducers / 8)) {
          const uint32_t pn = g.bp + 8u * (uint32_t)e0 + (uint32_t)r;
          const uint32_t a8 = (pn >> 1) & ~7u;
          const uint32_t sbit = 4u * pn - 8u * a8;
          uint32_t u[8], w[5];
#pragma unroll
          for (int i = 0; i < 4; ++i) {
            const uint64_t v = ld_shared_u64(xs + a8 + 8u * i);
            u[2 * i] = (uint32_t)v, u[2 * i + 1] = (uint32_t)(v >> 32);
          }
          const bool wo = sbit >= 32u;
          const uint32_t sh = sbit & 31u;
#pragma unroll
          for (int q = 0; q < 5; ++q) w[q] = __funnelshift_r(wo ? u[q + 1] : u[q], wo ? u[q + 2] : u[q + 1], sh);
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            if (e0 + k >= e_hi) break;
            const uint32_t ps = (uint32_t)(e0 + k) % (uint32_t)kRing4;
            const uint32_t ad = slots + 128u * ps + 16u * (uint32_t)r;
            st_shared_v4(ad, w[k], w[k + 1], w[k + 2], w[k + 3]);
            if (ps < (uint32_t)kMirror4) st_shared_v4(ad + 128u * kRing4, w[k], w[k + 1], w[k + 2], w[k + 3]);
          }
        }
        fence_proxy_async();
        mbar_arrive(full_bar + 8 * (uint32_t)((sc0 + j) % kNB));
      }
    } else if (warp == 0) {
      // MMA issuer (whole warp waits, lane 0 issues): per chunk, the live
      // column groups, two K steps
      // column group gg is live for chunks [clo[gg], chi[gg]) (live for chunk
      // c iff its y rows meet the signal); chunks where every group is live
      // take a fast path: one full-width pair of MMAs, no per-chunk tests
      int clo[kGroups4], chi[kGroups4];
      int full_lo = 0, full_hi = g.nchunks;
#pragma unroll
      for (int gg = 0; gg < kGroups4; ++gg) {
        const int64_t lo = -g.T0 - 128 * (int64_t)(kGroupCols * gg + kGroupCols - 1);
        const int64_t hi = P.ny - g.T0 - 128 * (int64_t)(kGroupCols * gg);
        const int64_t glo = (lo > 0 ? lo : 0) - g.ks;
        const int64_t ghi = (hi < P.nx + 127 ? hi : P.nx + 127) - g.ks;
        // live for chunk c iff glo < 128 (c + 1) and ghi > 128 c
        int64_t a = fdiv(glo, kKc8), z = fdiv(ghi + kKc8 - 1, kKc8);
        a = a < 0 ? 0 : (a > g.nchunks ? g.nchunks : a);
        z = z < 0 ? 0 : (z > g.nchunks ? g.nchunks : z);
        clo[gg] = (int)a, chi[gg] = (int)z;
        full_lo = full_lo > clo[gg] ? full_lo : clo[gg];
        full_hi = full_hi < chi[gg] ? full_hi : chi[gg];
      }
      const uint32_t idesc_full = idesc4_for(kN4);
      const uint64_t da0 = sdesc(slots, 512, 128, 0, 0);  // + ring slot * 8
      const uint64_t db0 = sdesc(yr, 16, 512, 4, 0);      // + row * 4
      for (int j = 0; j < g.nsc; ++j) {
        const int64_t S = sc0 + j;
        {
          const uint32_t fb = full_bar + 8 * (uint32_t)(S % kNB), ph = (uint32_t)((S / kNB) & 1);
          ok = __all_sync(0xffffffffu, mbar_try(fb, ph) || mbar_wait(fb, ph));
        }
        if (!ok) break;
        tc_fence_after();
        if (lane == 0) {
          const int c0 = kSC4 * j;
          const int c1 = c0 + kSC4 < g.nchunks ? c0 + kSC4 : g.nchunks;
          const uint32_t row_c0 = (uint32_t)(g.u_s - g.r_lo) + (uint32_t)c0;
          if (c0 >= full_lo && c1 <= full_hi) {
            // every group live: ring slot and tile row advance by 16 slots and 1 row
            const uint64_t bd0 = db0 + 4u * row_c0;
#pragma unroll
            for (int cc = 0; cc < kSC4; ++cc)
              if (c0 + cc < c1) {
                const uint64_t ad = da0 + 8u * ((16u * (uint32_t)(c0 + cc)) & (uint32_t)(kRing4 - 1));
                mma_mxf4(tmem, ad, bd0 + 4u * (uint32_t)cc, idesc_full, sfa, sfb, 1u);
                mma_mxf4(tmem, ad + 64u, bd0 + 4u * (uint32_t)cc + 2u, idesc_full, sfa, sfb, 1u);
              }
          } else {
            for (int c = c0; c < c1; ++c) {
              int ga = kGroups4, gb = -1;
#pragma unroll
              for (int gg = 0; gg < kGroups4; ++gg)
                if (c >= clo[gg] && c < chi[gg]) {
                  ga = gg < ga ? gg : ga;
                  gb = gg;
                }
              if (gb >= ga) {
                const uint32_t idesc = idesc4_for(kGroupCols * (gb - ga + 1));
                const uint32_t row0 = row_c0 + (uint32_t)(c - c0) + (uint32_t)(kGroupCols * ga);
                const uint64_t ad = da0 + 8u * ((16u * (uint32_t)c) & (uint32_t)(kRing4 - 1));
                const uint64_t bd = db0 + 4u * row0;
                const uint32_t d_col = tmem + (uint32_t)(kGroupCols * ga);
                mma_mxf4(d_col, ad, bd, idesc, sfa, sfb, 1u);
                mma_mxf4(d_col, ad + 64u, bd + 2u, idesc, sfa, sfb, 1u);
              }
            }
          }
          mma_commit(cmt_bar + 8 * (uint32_t)(S % kNB));
        }
        __syncwarp();
      }
      if (lane == 0) mma_commit(done_bar);
      __syncwarp();
    } else if (warp >= 3 && w_next < nitems) {
      // the next item's y and x into the other buffer while the MMAs run
      const MmaItem itn = items[w_next];
      const Item4 gn = item4_of(itn);
      const uint32_t yn = stage0 + ((iter + 1) & 1u) * kStage4;
      if (gn.valid && stage4(pairs[itn.pair], gn, yn, yn + kYBytes4, threadIdx.x - 96, kThreads - 96))
        atomicOr(status, TDE_ST_INTERNAL);
    }

    const bool done = mbar_wait(done_bar, ndone & 1u);
    ++ndone;
    ok = __syncthreads_and(ok && done);
    if (!ok) {
      if (threadIdx.x == 0) atomicOr(status, TDE_ST_TIMEOUT);
      break;
    }
    {
      tc_fence_after();
      const int q = warp & 3, colh = warp >> 2;
      const int m = 32 * q + lane;
      for (int cb = 0; cb < 2; ++cb) {
        const int col0 = 64 * colh + 32 * cb;
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)col0, v);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int64_t tau = g.T0 + 127 - m + 128 * (int64_t)(col0 + j);
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
    sc0 += g.nsc;
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols4)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// The learned proposal's 32 -> 32 channel conv layers (inference) on the
// tensor cores: kind::f16 with BF16 operands and FP32 accumulation in tensor
// memory.  z[p][co] = sum_k sum_ci X[p + k - 4][ci] W[co][ci][k] (kernel 9,
// pad 4), then bias, ReLU and max-pool of (2P, 2P + 1).
//
// Input layout (written by the previous layer): per signal, per position
// parity (E: even positions, O: odd) and per 8-channel chunk j, an array of
// R = cnn_eo_rows(L) rows of 16 bytes, row r holding position 2r - 4 (E) or
// 2r - 3 (O), zero outside [0, L).  A tile is 128 pooled outputs
// P = P0 + m (TMEM lane m); it needs rows P0 .. P0 + 131 of the 8 arrays,
// contiguous in global memory, so one thread moves it with 8 bulk copies.
//
// In that layout every shifted window of rows serves two taps at once: rows
// m + d of E feed the even output 2P through tap 2d and the odd output 2P + 1
// through tap 2d - 1; rows m + d of O feed the even output through tap 2d + 1
// and the odd one through tap 2d.  With the weights staged as blocks
// W_s[j][t][co][ci % 8] for t = tap + 1 (t = 0 and t = 10 are zero blocks),
// the B operand of a window is two consecutive blocks (N = 64: columns 0-31
// the odd outputs' tap, 32-63 the even outputs'), so a tile is 10 windows x 2
// halves of the input channels = 20 MMAs of 128 x 64 x 16, and each lane ends
// with both outputs of its pooling pair: y = relu(max(z_even, z_odd) + b).
//
// Outputs: the next layer's E/O arrays (with their zero rows), or for the
// last layer FP32 features [signal][L/2][32] (position-major).  A CTA takes an equal
// contiguous run of (signal, tile) units; thread 0 keeps kCvNB tiles of bulk
// copies in flight and issues the MMAs into two accumulators (2 x 64 TMEM
// columns), so tile i's MMAs overlap tile i - 1's epilogue.  Waits are
// bounded; on time-out the CTA flags TDE_ST_TIMEOUT, waits (bounded) for its
// copies and MMAs and frees its tensor memory.

constexpr int kCvM = 128;                          // pooled outputs per tile (MMA M)
constexpr int kCvN = 64;                           // odd | even outputs
constexpr int kCvRows = kCvM + 4;                  // input rows per parity array per tile
constexpr int kCvArr = kCvRows * 16;               // bytes of one (parity, chunk) piece
constexpr int kCvXBytes = 2 * (kCnnC / 8) * kCvArr;  // one tile's input (16896)
constexpr int kCvTaps = kCnnK + 2;                 // weight blocks per chunk (zero at both ends)
constexpr int kCvWBytes = (kCnnC / 8) * kCvTaps * kCnnC * 16;
constexpr int kCvNB = 3;                           // input tile buffers
constexpr int kCvSmem = kCvNB * kCvXBytes + kCvWBytes + (kCvNB + 2) * 8 + 16 + 128;
constexpr int kCvCtasPerSm = 3;
static_assert(kCvXBytes % 128 == 0 && kCvWBytes % 128 == 0, "conv staging alignment");
static_assert(kCvCtasPerSm * (kCvSmem + 1024) <= 228 * 1024, "conv CTAs per SM");

// Instruction descriptor, kind::f16: D F32 (bits 4-5 = 1), A and B BF16
// (bits 7-9 = 1, 10-12 = 1), both K-major, N >> 3 at bits 17-22, M >> 4 at
// bits 24-28.
constexpr uint32_t kCvIdesc =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kCvN >> 3) << 17) | ((uint32_t)(kCvM >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}


__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
// bytes (multiple of 16) global -> shared, completing on bar's transaction count
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

__device__ __forceinline__ uint32_t pack_bf16x2_rn(float lo, float hi) {
  uint32_t r;
  asm("cvt.rn.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
  return r;
}

template <bool kLast>
__global__ void __launch_bounds__(kThreads, kCvCtasPerSm)
    k_conv_tc(const uint16_t* __restrict__ in, void* __restrict__ out, int L, int nsig,
              const uint16_t* __restrict__ wbf, const float* __restrict__ bias,
              uint32_t* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 127u) & ~127u;
  const uint32_t xbuf = base;                     // kCvNB tiles' input
  const uint32_t wsm = xbuf + kCvNB * kCvXBytes;  // weight blocks
  const uint32_t full_bar = wsm + kCvWBytes;      // per input buffer
  const uint32_t done_bar = full_bar + 8 * kCvNB; // per accumulator
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(smem_raw + (done_bar + 16 - raw));
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Lo = L / 2;                            // pooled outputs
  const int tps = (Lo + kCvM - 1) / kCvM;          // tiles per signal
  const int R = cnn_eo_rows(L);                    // rows per input array
  const int units = nsig * tps;
  const int u0 = (int)((int64_t)units * blockIdx.x / gridDim.x);
  const int ntiles = (int)((int64_t)units * (blockIdx.x + 1) / gridDim.x) - u0;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(2 * kCvN)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    for (int b = 0; b < kCvNB; ++b) mbar_init(full_bar + 8 * b, 1);
    mbar_init(done_bar, 1);
    mbar_init(done_bar + 8, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // weight blocks W_s[j][t][co][e], t = tap + 1 (zero blocks at t = 0, 10),
  // two elements per store: every load of the thread's share is issued
  // before its first store (plain stores, so the loads are not held behind
  // them)
  {
    constexpr int kPer = (kCvWBytes / 4 + kThreads - 1) / kThreads;
    uint32_t v[kPer];
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int idx = threadIdx.x + r * kThreads;
      const int e2 = idx & 3, co = (idx >> 2) & (kCnnC - 1), jt = idx >> 7;
      const int t = jt % kCvTaps, j = jt / kCvTaps, k = t - 1;
      v[r] = 0;
      if (idx < kCvWBytes / 4 && k >= 0 && k < kCnnK) {
        const int ci = 8 * j + 2 * e2;
        v[r] = (uint32_t)__ldg(wbf + (co * kCnnC + ci) * kCnnK + k) |
               ((uint32_t)__ldg(wbf + (co * kCnnC + ci + 1) * kCnnK + k) << 16);
      }
    }
    uint32_t* wdst = reinterpret_cast<uint32_t*>(smem_raw + (wsm - raw));
#pragma unroll
    for (int r = 0; r < kPer; ++r) {
      const int idx = threadIdx.x + r * kThreads;
      if (idx < kCvWBytes / 4) wdst[idx] = v[r];
    }
  }
  // the next layer's zero rows: 0, 1 and [L/4 + 2, R') of each array
  if (!kLast) {
    const int Rn = cnn_eo_rows(Lo), vn = Lo / 2 + 2, npad = 2 + (Rn - vn);
    uint16_t* o = static_cast<uint16_t*>(out);
    const int64_t total = (int64_t)nsig * 8 * npad;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < total; i += (int64_t)gridDim.x * kThreads) {
      const int pr = (int)(i % npad);
      const int64_t arr = i / npad;  // (signal, parity, chunk)
      const int r = pr < 2 ? pr : vn + (pr - 2);
      *reinterpret_cast<uint4*>(o + (arr * Rn + r) * 8) = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  const int qd = warp & 3, ch = warp >> 2;  // TMEM lanes 32 qd.., channels 16 ch..
  float bv[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) bv[j] = bias[16 * ch + j];
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // thread 0: bulk copies of tile i (unit u0 + i) into buffer i % kCvNB
  auto load = [&](int i) {
    const int u = u0 + i, s = u / tps, P0 = (u - s * tps) * kCvM;
    const uint32_t fb = full_bar + 8u * (uint32_t)(i % kCvNB);
    const uint32_t xb = xbuf + (uint32_t)(i % kCvNB) * kCvXBytes;
    mbar_expect_tx(fb, (uint32_t)kCvXBytes);
#pragma unroll
    for (int a = 0; a < 8; ++a)  // a = parity * 4 + chunk
      bulk_g2s(xb + (uint32_t)a * kCvArr, in + (((int64_t)s * 8 + a) * R + P0) * 8, (uint32_t)kCvArr, fb);
  };
  int loaded = 0, issued = 0;  // tiles whose copies / MMAs were issued (thread 0)
  if (threadIdx.x == 0)
    for (; loaded < kCvNB && loaded < ntiles; ++loaded) load(loaded);

  auto epilogue = [&](int i) {
    const int u = u0 + i, s = u / tps, P = (u - s * tps) * kCvM + 32 * qd + lane;
    const uint32_t col = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)((i & 1) * kCvN + 16 * ch);
    uint32_t vo[16], ve[16];
    tmem_ld16_nowait(col, vo);
    tmem_ld16_nowait(col + 32u, ve);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
    float y[16];
#pragma unroll
    for (int j = 0; j < 16; ++j)
      y[j] = fmaxf(fmaxf(__uint_as_float(ve[j]), __uint_as_float(vo[j])) + bv[j], 0.f);
    if (P >= Lo) return;
    if (kLast) {  // features, position-major: [signal][P][32]
      float4* dst = reinterpret_cast<float4*>(static_cast<float*>(out) + ((int64_t)s * Lo + P) * kCnnC + 16 * ch);
#pragma unroll
      for (int j = 0; j < 4; ++j) dst[j] = make_float4(y[4 * j], y[4 * j + 1], y[4 * j + 2], y[4 * j + 3]);
    } else {
      const int Rn = cnn_eo_rows(Lo);
      uint16_t* o = static_cast<uint16_t*>(out) +
                    ((((int64_t)s * 2 + (P & 1)) * 4 + 2 * ch) * Rn + (P >> 1) + 2) * 8;
      *reinterpret_cast<uint4*>(o) = make_uint4(pack_bf16x2_rn(y[0], y[1]), pack_bf16x2_rn(y[2], y[3]),
                                                pack_bf16x2_rn(y[4], y[5]), pack_bf16x2_rn(y[6], y[7]));
      *reinterpret_cast<uint4*>(o + (int64_t)Rn * 8) =
          make_uint4(pack_bf16x2_rn(y[8], y[9]), pack_bf16x2_rn(y[10], y[11]),
                     pack_bf16x2_rn(y[12], y[13]), pack_bf16x2_rn(y[14], y[15]));
    }
  };

  bool ok = true;
  for (int i = 0; i < ntiles; ++i) {
    if (threadIdx.x == 0) {
      ok = mbar_wait_sleep(full_bar + 8u * (uint32_t)(i % kCvNB), (uint32_t)((i / kCvNB) & 1));
      if (ok) {
        tc_fence_after();
        const uint32_t xb = xbuf + (uint32_t)(i % kCvNB) * kCvXBytes;
        const uint32_t d = tmem + (uint32_t)((i & 1) * kCvN);
#pragma unroll
        for (int w = 0; w < 10; ++w) {  // windows: E d = 0..4, O d = 0..4
          const int par = w / 5, dd = w % 5;
          const int t0 = 2 * dd + par;  // first weight block of the window
#pragma unroll
          for (int h = 0; h < 2; ++h)
            mma_bf16(d, sdesc(xb + (uint32_t)((par * 4 + 2 * h) * kCvArr + 16 * dd), kCvArr, 128, 0, 0),
                     sdesc(wsm + (uint32_t)(((2 * h) * kCvTaps + t0) * kCnnC * 16), kCvTaps * kCnnC * 16, 128, 0, 0),
                     kCvIdesc, (w | h) != 0);
        }
        mma_commit(done_bar + 8u * (uint32_t)(i & 1));
        issued = i + 1;
      }
    }
    if (i > 0) {
      // tile i - 1's MMAs: its buffer may be refilled and its accumulator read
      const bool w_ok = mbar_wait_sleep(done_bar + 8u * (uint32_t)((i - 1) & 1), (uint32_t)(((i - 1) >> 1) & 1));
      ok = __syncthreads_and(ok && w_ok);
      if (!ok) break;
      if (threadIdx.x == 0 && loaded < ntiles) load(loaded++);
      tc_fence_after();
      epilogue(i - 1);
    } else {
      ok = __syncthreads_and(ok);
      if (!ok) break;
    }
    tc_fence_before();
    __syncthreads();
  }
  if (ok && ntiles > 0) {
    const int i = ntiles - 1;
    ok = __syncthreads_and(mbar_wait_sleep(done_bar + 8u * (uint32_t)(i & 1), (uint32_t)((i >> 1) & 1)));
    if (ok) {
      tc_fence_after();
      epilogue(i);
    }
  }
  if (!ok && threadIdx.x == 0) {
    atomicOr(status, TDE_ST_TIMEOUT);
    // bounded waits for this CTA's copies and MMAs still in flight
    for (int i = issued; i < loaded; ++i)
      mbar_wait_sleep(full_bar + 8u * (uint32_t)(i % kCvNB), (uint32_t)((i / kCvNB) & 1));
    for (int i = issued - 2 < 0 ? 0 : issued - 2; i < issued; ++i)
      mbar_wait_sleep(done_bar + 8u * (uint32_t)(i & 1), (uint32_t)((i >> 1) & 1));
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kCvN)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// The learned proposal's first layer (decimation + conv 1 -> 32 channels,
// kernel 9, pad 4, bias, ReLU, max-pool 2) on the tensor cores, as
// k_conv12_tc runs it: for 128 layer-1 outputs u0 + m it builds the im2col
// operand
//   A_par[m][k] = d[2 (u0 + m) + par + k - 4]   (k < 9; k = 9..15 zero)
// for both parities of the pooling pair as K-major no-swizzle tiles (16-byte
// rows of 8 taps, leading byte offset 2048 between the two 8-tap halves), and
// issues one MMA of 128 x 32 x 16 per parity (columns 0-31 odd, 32-63 even)
// against W[co][k]; y = relu(max(z_even, z_odd) + b).  The decimated samples
// d[j] = (sum of 16 levels) / 4 are exact in BF16 (|4 d| <= 112).
constexpr int kC1M = 128;                      // pooled outputs per CTA
constexpr int kC1ABytes = 2 * 2 * kC1M * 16;   // A tiles: parity x 8-tap half x rows
constexpr int kC1WBytes = 2 * kCnnC * 16;      // B: 8-tap half x co rows
constexpr uint32_t kC1Idesc =
    (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kCnnC >> 3) << 17) | ((uint32_t)(kC1M >> 4) << 24);


// Self-test of the bounded waits the kernels above use: thread 0 waits on a
// shared-memory barrier that nothing arrives on, first spinning (mbar_wait),
// then suspending (mbar_wait_sleep); each gives up after kTimeoutNs, and the
// CTA flags TDE_ST_TIMEOUT as a kernel whose wait gave up does.  No copy,
// MMA or tensor memory is involved, so the CTA simply returns.
__global__ void k_wait_selftest(uint32_t* __restrict__ status) {
  __shared__ __align__(8) uint64_t bar;
  const uint32_t b = smem_u32(&bar);
  if (threadIdx.x == 0) {
    mbar_init(b, 1);
    bool ok = mbar_wait(b, 0);
    ok = mbar_wait_sleep(b, 0) && ok;
    if (!ok) atomicOr(status, TDE_ST_TIMEOUT);
  }
}


// ---------------------------------------------------------------------------
// The inference forward's first two layers in one kernel: decimation + conv
// 1 -> 32 + pool (the first layer above) feeding conv 32 -> 32 + pool
// (k_conv_tc's) through shared memory, so layer 2's input never goes to
// global memory.  A unit is one layer-2 tile: 128 pooled outputs P0 + m of
// one signal.  It needs layer-1 outputs u = 2 P0 - 4 + t, t in [0, 264) (zero
// outside [0, Ld / 2)): t < 256 come from two 128-row MMA tiles per parity
// as above (im2col operand from the 536 decimated samples
// d[4 P0 - 12 + i]), t = 256..263 from CUDA-core FMAs over the same BF16
// products.  They are written, BF16, as the E/O parity arrays of k_conv_tc's
// tile (t even -> E row t / 2, t odd -> O row t / 2), and that tile's 20
// MMAs and epilogue follow.  Layer 1's im2col tiles share the tile's space
// (they are read before it is written), and layer 2's accumulator reuses
// layer 1's tensor-memory columns, so a CTA holds 128 columns and about
// 41 KB: four CTAs per SM.  The CTA also writes the E4M3 copy of the levels
// its unit owns (q samples [64 P0, 64 P0 + 8192)) and, as layer 2 of
// k_conv_tc does, the zero rows of layer 3's input.
constexpr int kF2M = 128;                    // layer-2 pooled outputs per unit
constexpr int kF1U = 2 * kF2M + 8;           // layer-1 outputs per unit (264)
constexpr int kF1D = 2 * kF1U + 8;           // decimated samples per unit (536)
constexpr int kF1Fetch = 3;                  // uint4 per thread holding the unit's level bytes
constexpr int kF1ABytes = 2 * kC1ABytes;     // two conv-1 im2col tiles (aliasing the layer-2 tile)
constexpr int kF12Smem = kCvXBytes + kCvWBytes + kC1WBytes + 1152 + 16 + 16 + 128;
static_assert(kF1ABytes <= kCvXBytes, "conv-1 tiles fit the layer-2 tile");
static_assert(kF1D <= kF1Fetch * kThreads && kF1D * 2 <= 1152, "per-unit samples");
static_assert(4 * (kF12Smem + 1024) <= 228 * 1024, "four CTAs per SM");

__global__ void __launch_bounds__(kThreads, 4)
    k_conv12_tc(const int8_t* __restrict__ q, int64_t n, int nsig, const uint16_t* __restrict__ w1bf,
                const float* __restrict__ bias1, const uint16_t* __restrict__ w2bf,
                const float* __restrict__ bias2, uint16_t* __restrict__ out, uint8_t* __restrict__ qe,
                uint32_t* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 127u) & ~127u;
  uint8_t* sbase = smem_raw + (base - raw);
  const uint32_t xb = base;                          // layer-2 tile; conv-1 im2col tiles first
  const uint32_t wsm = xb + kCvXBytes;               // layer-2 weight blocks
  const uint32_t w1s = wsm + kCvWBytes;              // layer-1 weights
  uint16_t* d_s = reinterpret_cast<uint16_t*>(sbase + kCvXBytes + kCvWBytes + kC1WBytes);
  const uint32_t bar1 = w1s + kC1WBytes + 1152, bar2 = bar1 + 8;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(sbase + kCvXBytes + kCvWBytes + kC1WBytes + 1152 + 16);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int Ld = (int)(n / kCnnDec), L2 = Ld / 2, Lo = L2 / 2;  // decimated, layer-2 input, layer-2 pooled
  const int tps = (Lo + kF2M - 1) / kF2M;
  const int units = nsig * tps;
  const int u0 = (int)((int64_t)units * blockIdx.x / gridDim.x);
  const int u1 = (int)((int64_t)units * (blockIdx.x + 1) / gridDim.x);

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(2 * kCnnC * 2)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 32) {
    mbar_init(bar1, 1);
    mbar_init(bar2, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // layer-1 weights W_s[half][co][e] = W1[co][8 half + e] (taps 9..15 zero)
  for (int idx = threadIdx.x; idx < 2 * kCnnC * 8; idx += kThreads) {
    const int e = idx & 7, co = (idx >> 3) & (kCnnC - 1), h = idx >> 8;
    const int k = 8 * h + e;
    reinterpret_cast<uint16_t*>(sbase + kCvXBytes + kCvWBytes)[idx] = k < kCnnK ? __ldg(w1bf + co * kCnnK + k) : (uint16_t)0;
  }
  // layer-2 weight blocks as in k_conv_tc, in two batches of loads
  {
    uint32_t* wdst = reinterpret_cast<uint32_t*>(sbase + kCvXBytes);
    constexpr int kPer = (kCvWBytes / 4 + kThreads - 1) / kThreads;
#pragma unroll
    for (int r0 = 0; r0 < kPer; r0 += (kPer + 1) / 2) {
      uint32_t v[(kPer + 1) / 2];
#pragma unroll
      for (int r = 0; r < (kPer + 1) / 2; ++r) {
        const int idx = threadIdx.x + (r0 + r) * kThreads;
        const int e2 = idx & 3, co = (idx >> 2) & (kCnnC - 1), jt = idx >> 7;
        const int t = jt % kCvTaps, j = jt / kCvTaps, k = t - 1;
        v[r] = 0;
        if (r0 + r < kPer && idx < kCvWBytes / 4 && k >= 0 && k < kCnnK) {
          const int ci = 8 * j + 2 * e2;
          v[r] = (uint32_t)__ldg(w2bf + (co * kCnnC + ci) * kCnnK + k) |
                 ((uint32_t)__ldg(w2bf + (co * kCnnC + ci + 1) * kCnnK + k) << 16);
        }
      }
#pragma unroll
      for (int r = 0; r < (kPer + 1) / 2; ++r) {
        const int idx = threadIdx.x + (r0 + r) * kThreads;
        if (r0 + r < kPer && idx < kCvWBytes / 4) wdst[idx] = v[r];
      }
    }
  }
  // the zero rows of layer 3's input: 0, 1 and [Lo / 2 + 2, Rn) of each array
  {
    const int Rn = cnn_eo_rows(Lo), vn = Lo / 2 + 2, npad = 2 + (Rn - vn);
    const int64_t total = (int64_t)nsig * 8 * npad;
    for (int64_t i = (int64_t)blockIdx.x * kThreads + threadIdx.x; i < total; i += (int64_t)gridDim.x * kThreads) {
      const int pr = (int)(i % npad);
      const int64_t arr = i / npad;
      const int r = pr < 2 ? pr : vn + (pr - 2);
      *reinterpret_cast<uint4*>(out + (arr * Rn + r) * 8) = make_uint4(0u, 0u, 0u, 0u);
    }
  }
  const int qd = warp & 3, ch = warp >> 2;
  const uint16_t* w1h = reinterpret_cast<const uint16_t*>(sbase + kCvXBytes + kCvWBytes);
  fence_proxy_async();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const uint64_t bd1 = sdesc(w1s, kCnnC * 16, 128, 0, 0);
  bool ok = true;
  uint32_t ph1 = 0, ph2 = 0;
  auto fetch = [&](int u, uint4 (&w)[kF1Fetch]) {
    const int s = u / tps, P0 = (u - s * tps) * kF2M;
    const int8_t* src = q + (int64_t)s * n;
#pragma unroll
    for (int f = 0; f < kF1Fetch; ++f) {
      const int i = threadIdx.x + f * kThreads, j = 4 * P0 - 12 + i;
      w[f] = (i < kF1D && j >= 0 && j < Ld) ? __ldg(reinterpret_cast<const uint4*>(src + (int64_t)j * kCnnDec))
                                            : make_uint4(0u, 0u, 0u, 0u);
    }
  };
  uint4 wn[kF1Fetch];
  if (u0 < u1) fetch(u0, wn);
  for (int u = u0; u < u1 && ok; ++u) {
    const int s = u / tps, P0 = (u - s * tps) * kF2M;
    // decimate (the level bytes were fetched one unit ahead): d_s[i] = d[4 P0 - 12 + i]; the E4M3 copy of the samples the unit owns
#pragma unroll
    for (int f = 0; f < kF1Fetch; ++f) {
      const int i = threadIdx.x + f * kThreads;
      if (i >= kF1D) continue;
      const int j = 4 * P0 - 12 + i;
      float v = 0.f;
      if (j >= 0 && j < Ld) {
        const uint4 w = wn[f];
        int acc = 0;
        acc = __dp4a((int)w.x, 0x01010101, acc);
        acc = __dp4a((int)w.y, 0x01010101, acc);
        acc = __dp4a((int)w.z, 0x01010101, acc);
        acc = __dp4a((int)w.w, 0x01010101, acc);
        v = 0.25f * (float)acc;
        if (qe && i >= 12 && i < 12 + 4 * kF2M) {
          // levels in {-1, 0, 1} (bit 0 set iff non-zero, bit 7 the sign):
          // E4M3 bytes 0x00, 0x38 = 1.0, 0xB8 = -1.0
          const uint4 e = make_uint4(((w.x & 0x01010101u) * 0x38u) | (w.x & 0x80808080u),
                                     ((w.y & 0x01010101u) * 0x38u) | (w.y & 0x80808080u),
                                     ((w.z & 0x01010101u) * 0x38u) | (w.z & 0x80808080u),
                                     ((w.w & 0x01010101u) * 0x38u) | (w.w & 0x80808080u));
          *reinterpret_cast<uint4*>(qe + (int64_t)s * n + (int64_t)j * kCnnDec) = e;
        }
      }
      d_s[i] = (uint16_t)(__float_as_uint(v) >> 16);  // exact: |4 d| <= 112
    }
    if (u + 1 < u1) fetch(u + 1, wn);
    __syncthreads();
    // conv-1 im2col: tile h1 (t = 128 h1 + m), row (par, half, m) of 8 taps
    for (int row = threadIdx.x; row < 2 * 2 * 2 * kC1M; row += kThreads) {
      const int m = row & (kC1M - 1), h = (row >> 7) & 1, par = (row >> 8) & 1, h1 = row >> 9;
      uint32_t wv[4];
#pragma unroll
      for (int e2 = 0; e2 < 4; ++e2) {
        const int k0 = 8 * h + 2 * e2;
        const int i0 = 2 * (kC1M * h1 + m) + par + k0;
        const uint32_t lo = k0 < kCnnK ? d_s[i0] : 0u, hi = k0 + 1 < kCnnK ? d_s[i0 + 1] : 0u;
        wv[e2] = lo | (hi << 16);
      }
      st_shared_v4(xb + (uint32_t)(h1 * kC1ABytes) + 16u * (uint32_t)(row & 511), wv[0], wv[1], wv[2], wv[3]);
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0) {  // tile h1: odd parity -> columns 64 h1 .. +31, even -> +32 .. +63
#pragma unroll
      for (int h1 = 0; h1 < 2; ++h1) {
        const uint32_t a = xb + (uint32_t)(h1 * kC1ABytes);
        mma_bf16(tmem + 64u * (uint32_t)h1, sdesc(a + 2u * kC1M * 16, kC1M * 16, 128, 0, 0), bd1, kC1Idesc, 0u);
        mma_bf16(tmem + 64u * (uint32_t)h1 + kCnnC, sdesc(a, kC1M * 16, 128, 0, 0), bd1, kC1Idesc, 0u);
      }
      mma_commit(bar1);
    }
    // the halo t = 256 .. 263 on the CUDA cores while the MMAs run: warp w
    // takes t = 256 + w, lane = channel
    float yh;
    {
      const int t = 2 * kF2M + warp, uu = 2 * P0 - 4 + t;
      float z0 = 0.f, z1 = 0.f;
#pragma unroll
      for (int k = 0; k < kCnnK; ++k) {
        const float wk = __uint_as_float((uint32_t)w1h[((k >> 3) * kCnnC + lane) * 8 + (k & 7)] << 16);
        z0 = fmaf(__uint_as_float((uint32_t)d_s[2 * t + k] << 16), wk, z0);
        z1 = fmaf(__uint_as_float((uint32_t)d_s[2 * t + 1 + k] << 16), wk, z1);
      }
      yh = (uu >= 0 && uu < L2) ? fmaxf(fmaxf(z0, z1) + __ldg(bias1 + lane), 0.f) : 0.f;
    }
    ok = __syncthreads_and(mbar_wait_sleep(bar1, ph1));
    ph1 ^= 1u;
    if (!ok) break;
    tc_fence_after();
    // conv-1 epilogue -> the layer-2 tile (its space held the im2col tiles)
    {
      const float* b1 = bias1 + 16 * ch;
#pragma unroll 1
      for (int h1 = 0; h1 < 2; ++h1) {
        const uint32_t col = tmem + ((uint32_t)(32 * qd) << 16) + 64u * (uint32_t)h1 + (uint32_t)(16 * ch);
        uint32_t vo[16], ve[16];
        tmem_ld16_nowait(col, vo);
        tmem_ld16_nowait(col + 32u, ve);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        const int t = kC1M * h1 + 32 * qd + lane, uu = 2 * P0 - 4 + t;
        const bool valid = uu >= 0 && uu < L2;
        float y[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
          y[j] = valid ? fmaxf(fmaxf(__uint_as_float(ve[j]), __uint_as_float(vo[j])) + __ldg(b1 + j), 0.f) : 0.f;
        // generic stores after every thread's tensor-memory read of the
        // tiles' MMAs is done: the im2col tiles they read share this space
        const uint32_t row = xb + (uint32_t)(((t & 1) * 4 + 2 * ch) * kCvArr + 16 * (t >> 1));
        st_shared_v4(row, pack_bf16x2_rn(y[0], y[1]), pack_bf16x2_rn(y[2], y[3]), pack_bf16x2_rn(y[4], y[5]),
                     pack_bf16x2_rn(y[6], y[7]));
        st_shared_v4(row + kCvArr, pack_bf16x2_rn(y[8], y[9]), pack_bf16x2_rn(y[10], y[11]),
                     pack_bf16x2_rn(y[12], y[13]), pack_bf16x2_rn(y[14], y[15]));
      }
      const int t = 2 * kF2M + warp;  // the halo row: channel = lane
      const uint32_t hrow = xb + (uint32_t)(((t & 1) * 4 + (lane >> 3)) * kCvArr + 16 * (t >> 1) + 2 * (lane & 7));
      asm volatile("st.shared.u16 [%0], %1;" ::"r"(hrow), "h"((uint16_t)(pack_bf16x2_rn(yh, 0.f) & 0xFFFFu)) : "memory");
    }
    fence_proxy_async();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (threadIdx.x == 0) {  // layer 2 into columns 0 .. 63 (layer 1's, drained)
#pragma unroll
      for (int w = 0; w < 10; ++w) {
        const int par = w / 5, dd = w % 5;
        const int t0 = 2 * dd + par;
#pragma unroll
        for (int h = 0; h < 2; ++h)
          mma_bf16(tmem, sdesc(xb + (uint32_t)((par * 4 + 2 * h) * kCvArr + 16 * dd), kCvArr, 128, 0, 0),
                   sdesc(wsm + (uint32_t)(((2 * h) * kCvTaps + t0) * kCnnC * 16), kCvTaps * kCnnC * 16, 128, 0, 0),
                   kCvIdesc, (w | h) != 0);
      }
      mma_commit(bar2);
    }
    ok = __syncthreads_and(mbar_wait_sleep(bar2, ph2));
    ph2 ^= 1u;
    if (!ok) break;
    tc_fence_after();
    {
      const int P = P0 + 32 * qd + lane;
      const uint32_t col = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(16 * ch);
      uint32_t vo[16], ve[16];
      tmem_ld16_nowait(col, vo);
      tmem_ld16_nowait(col + 32u, ve);
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (P < Lo) {
        const float* b2 = bias2 + 16 * ch;
        float y[16];
#pragma unroll
        for (int j = 0; j < 16; ++j)
          y[j] = fmaxf(fmaxf(__uint_as_float(ve[j]), __uint_as_float(vo[j])) + __ldg(b2 + j), 0.f);
        const int Rn = cnn_eo_rows(Lo);
        uint16_t* o = out + ((((int64_t)s * 2 + (P & 1)) * 4 + 2 * ch) * Rn + (P >> 1) + 2) * 8;
        *reinterpret_cast<uint4*>(o) = make_uint4(pack_bf16x2_rn(y[0], y[1]), pack_bf16x2_rn(y[2], y[3]),
                                                  pack_bf16x2_rn(y[4], y[5]), pack_bf16x2_rn(y[6], y[7]));
        *reinterpret_cast<uint4*>(o + (int64_t)Rn * 8) =
            make_uint4(pack_bf16x2_rn(y[8], y[9]), pack_bf16x2_rn(y[10], y[11]),
                       pack_bf16x2_rn(y[12], y[13]), pack_bf16x2_rn(y[14], y[15]));
      }
    }
    tc_fence_before();  // the next unit's MMAs overwrite the columns after the loop's barriers
  }
  if (!ok && threadIdx.x == 0) atomicOr(status, TDE_ST_TIMEOUT);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(2 * kCnnC * 2)
                 : "memory");
  }
}

}  // namespace

int mma_smem_bytes() { return kSmemBytes8; }

cudaError_t launch_wait_selftest(uint32_t* d_status, cudaStream_t st) {
  k_wait_selftest<<<1, 32, 0, st>>>(d_status);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_mma_zero(const MmaPair* d_pairs, int npairs, int64_t max_count, cudaStream_t st,
                            const int* d_count) {
  if (npairs <= 0) return cudaSuccess;
  int64_t gx = ceil_div64(max_count, 256 * 8);
  if (gx > 1024) gx = 1024;
  if (gx < 1) gx = 1;
  const int gy = d_count ? (npairs < 8 ? npairs : 8) : npairs;
  k_zero_outputs<<<dim3((unsigned)gx, gy), 256, 0, st>>>(d_pairs, npairs, d_count);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_xcorr_mma(const MmaPair* d_pairs, const MmaItem* d_items, int nitems,
                             int* d_counter, int grid, uint32_t* d_status, cudaStream_t st,
                             const int* d_nitems) {
  if (nitems <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_xcorr_mma8, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSmemBytes8);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(d_counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (grid > nitems) grid = nitems;
  k_xcorr_mma8<<<grid, kThreads, kSmemBytes8, st>>>(d_pairs, d_items, nitems, d_nitems, d_counter,
                                                     d_status);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_xcorr_mma4(const MmaPair* d_pairs, const MmaItem* d_items, int nitems,
                              int* d_counter, int grid, uint32_t* d_status, cudaStream_t st,
                              const int* d_nitems) {
  if (nitems <= 0) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(k_xcorr_mma4, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       kSmemBytes4);
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(d_counter, 0, sizeof(int), st);
  if (e != cudaSuccess) return e;
  if (grid > nitems) grid = nitems;
  k_xcorr_mma4<<<grid, kThreads, kSmemBytes4, st>>>(d_pairs, d_items, nitems, d_nitems, d_counter,
                                                     d_status);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

// Levels -> E4M3 bytes with a padded signal stride (zeros in [n, n_pad)).
// Flags TDE_ST_INTERNAL if a level's magnitude exceeds maxlev (the bits'
// range; the conversion itself is exact up to 7).
__global__ void k_to_e4m3(const int8_t* __restrict__ q, int64_t n, int64_t n_pad, int nsig, int maxlev,
                          uint8_t* __restrict__ qe, uint32_t* __restrict__ status) {
  const int64_t total = (int64_t)nsig * n_pad;
  const uint32_t lim = 0x01010101u * (uint32_t)maxlev;
  bool bad = false;
  for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) * 4; i < total;
       i += (int64_t)gridDim.x * blockDim.x * 4) {
    const int64_t s = i / n_pad, j = i - s * n_pad;  // n_pad % 4 == 0: one signal per word
    uint32_t w = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (j + k < n) w |= (uint32_t)(uint8_t)q[s * n + j + k] << (8 * k);
    bad |= __vcmpgtu4(__vabs4(w), lim) != 0u;  // -128 stays 0x80 and is flagged
    *reinterpret_cast<uint32_t*>(qe + i) = e4m3x4(w);
  }
  if (bad) atomicOr(status, TDE_ST_INTERNAL);
}

cudaError_t launch_to_e4m3(const int8_t* d_q, int64_t n, int64_t n_pad, int nsig, int bits, uint8_t* d_qe,
                           uint32_t* d_status, cudaStream_t st) {
  if (nsig <= 0) return cudaSuccess;
  if (n_pad % 4 != 0 || n_pad < n) return cudaErrorInvalidValue;
  if (bits != 1 && bits != 2 && bits != 4) return cudaErrorInvalidValue;
  const int64_t words = (int64_t)nsig * n_pad / 4;
  const int64_t grid = words / 256 + 1 < 4096 ? words / 256 + 1 : 4096;
  k_to_e4m3<<<(unsigned)grid, 256, 0, st>>>(d_q, n, n_pad, nsig, bits == 4 ? 7 : 1, d_qe, d_status);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}

cudaError_t launch_cnn_conv_tc(const uint16_t* in, void* out, int L, int nsig, const uint16_t* wbf,
                               const float* bias, bool last, uint32_t* d_status, cudaStream_t st) {
  if (nsig <= 0 || L <= 0) return cudaSuccess;
  if (L % 4 != 0) return cudaErrorInvalidValue;
  auto kern = last ? k_conv_tc<true> : k_conv_tc<false>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kCvSmem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t units = (int64_t)nsig * ((L / 2 + kCvM - 1) / kCvM);
  if (units > INT32_MAX) return cudaErrorInvalidValue;
  const int64_t cap = (int64_t)kCvCtasPerSm * sms;
  const int grid = (int)(units < cap ? units : cap);
  kern<<<grid, kThreads, kCvSmem, st>>>(in, out, L, nsig, wbf, bias, d_status);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}


cudaError_t launch_cnn_conv12_tc(const int8_t* q, int64_t n, int nsig, const uint16_t* w1bf, const float* bias1,
                                 const uint16_t* w2bf, const float* bias2, uint16_t* out, uint8_t* qe,
                                 uint32_t* d_status, cudaStream_t st) {
  if (nsig <= 0) return cudaSuccess;
  const int64_t Ld = n / kCnnDec;
  if (n % kCnnDec != 0 || Ld % 8 != 0 || Ld > INT32_MAX) return cudaErrorInvalidValue;
  const int64_t units = (int64_t)nsig * ((Ld / 4 + kF2M - 1) / kF2M);
  if (units > INT32_MAX) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_conv12_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kF12Smem);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t cap = 4 * (int64_t)sms;  // persistent: four CTAs per SM, contiguous unit runs
  const int grid = (int)(units < cap ? units : cap);
  k_conv12_tc<<<grid, kThreads, kF12Smem, st>>>(q, n, nsig, w1bf, bias1, w2bf, bias2, out, qe, d_status);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}
