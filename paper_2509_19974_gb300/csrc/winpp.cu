// winpp.cu -- the learned proposal's windows of the exact integer
// cross-correlation (Eq. (1) of arXiv 2509.19974, evaluated only at the
// proposed lags) in polyphase form on the 5th-generation tensor cores.
//
// Write a sample index as k = 128 a + b: a is a 128-sample row, b the phase in
// the row.  For a block offset u the 128 x 128 matrix
//   D_u[b][j] = sum_a x[128 a + b] * y[128 (a + u) + j]          (b, j < 128)
// is a plain GEMM over the rows a, and each of its terms is a term of one
// lag: x[128 a + b] y[128 (a + u) + j] belongs to c[tau] with
// tau = 128 u + j - b.  Conversely a term x[k] y[k + tau] of c[tau] lies in
// exactly one block, u = floor((b + tau) / 128), so
//   c[tau] = sum over u of the diagonal (j - b = tau - 128 u) of D_u.
// A window of lags [lo, hi] needs the blocks floor(lo / 128) ..
// floor((hi + 127) / 128): three for a window of 257 lags starting on a
// multiple of 128, and windows of neighbouring proposal bins share a block,
// so the 8 windows of a pair need between 17 blocks (adjacent bins: ~94 % of
// the MACs issued fall in the windows) and 24 (isolated bins: 67 %).
//
// The GEMM reads the levels' own rows, unchanged.  With E4M3 bytes a row is
// 128 bytes; A[b][a] = byte b of x row a and B[j][a] = byte j of y row
// a + u are MN-major operands in the 128-byte swizzle (K rows 128 bytes
// apart, 8-row groups 1024 bytes apart), so both arrive by plain tiled TMA
// loads of 32 rows.  Blocks u and u + 1 form one N = 256 MMA: block u + 1's
// operand is block u's shifted by one row, a leading byte offset (the MN
// atom stride) of 128 bytes.  An MMA is M = 128 x N = 256 x K = 32 rows
// (128 cycles on the tensor pipe, 12 KB of operand reads); a job (one or two
// blocks) is one MMA per 32-row K tile into an FP32 accumulator in tensor
// memory.  These operand forms were checked on the device with a one-MMA
// probe of controlled operands (MN-major A and B, overlapping B atoms, a B
// start off the 1024-byte pattern with base offset 0).
//
// Exactness: a job sums at most kPpSegRows = 512 rows (65536 samples) per
// accumulator, so |D| <= 512 * 49 < 2^24 and every FP32 value is an exact
// integer; diagonals are summed in int32 and longer signals' segments are
// added as integers (|c| <= n K_b^2 < 2^31 is checked by the caller).
//
// Work: the jobs of the batch, in (pair, segment, block) order, are dealt to
// the CTAs (one per SM) as contiguous runs of equal length; every CTA first
// scans all pairs' job counts (written with the windows) to find its run.  Within a run, a visit is the run's
// jobs of one (pair, segment): its x rows are loaded once, as one or two
// halves of 256 rows, and its y rows once per group of jobs whose rows fit
// the y ring, as units of 64 rows.  Roles (11 warps):
//   warp 1:          lane 0 plans each visit (jobs, groups, block slots) into
//                    a ring of 4 plans the other roles read; lanes 0-3 issue
//                    the TMA loads, slot s of a ring by lane s % 4 (one
//                    thread issues a tiled load in about 600 cycles).  x
//                    halves go to a ring of 3, y units to a ring of 11 (the
//                    first 32 rows of unit slot 0 mirrored past the end, so an
//                    MMA's 33 rows are always contiguous).  A slot is refilled
//                    once the last MMA that reads it has completed (an
//                    "empty" barrier committed by the issuer), so the next
//                    visit's loads overlap this visit's MMAs.
//   warps 0, 10:     MMAs (lane 0 of each), one per K tile of a job, the two
//                    issuers taking alternate jobs, each into its own
//                    256-column accumulator; a slot's release takes both.
//   warps 2-9:       epilogue: a warp reads 32 lanes x 128 (or 64) columns of
//                    the finished accumulator, converts to int32 and adds each
//                    value to its block's diagonal with a shared-memory
//                    atomic; at the end of a visit the diagonals go to the
//                    pair's windows with integer atomics (the outputs must be
//                    zero first).
// Every wait is bounded by %globaltimer; a role whose wait gives up raises
// the CTA's abort flag, and the CTA flags TDE_ST_TIMEOUT, waits (bounded) for
// its loads and MMAs in flight and frees its tensor memory.
#include "cnn.cuh"
#include "common.cuh"
#include "mma.cuh"
#include "tc.cuh"

namespace {

constexpr int kPpThreads = 352;                   // 11 warps
constexpr int kPpIssuerB = 10;                    // the second MMA warp
constexpr int kPpSegRows = 512;                   // rows summed per accumulator
constexpr int kPpTileRows = 32;                   // K rows per MMA (E4M3: K = 32)
constexpr int kPpHalfRows = 256;                  // x rows per load (and per release)
constexpr int kPpHalfBytes = kPpHalfRows * 128;
constexpr int kPpXHalves = 3;                     // x ring: the visit's halves + one ahead
constexpr int kPpUnitRows = 64;                   // y rows per load (and per release)
constexpr int kPpUnitBytes = kPpUnitRows * 128;
constexpr int kPpYUnits = 11;                     // y ring
constexpr int kPpYRows = kPpYUnits * kPpUnitRows;
constexpr int kPpMirrorRows = 32;                 // rows of unit slot 0 mirrored past the ring's end
constexpr int kPpGroupUnits = kPpYUnits - 2;      // a group leaves 2 units to load ahead
constexpr int kPpWin = kCnnTopK;                  // windows per pair (8)
constexpr int kPpWinLen = kCnnWin;                // lags per window (257)
constexpr int kPpMaxJobs = 2 * kPpWin;            // a window of <= 257 lags spans <= 4 blocks
constexpr int kPpMaxBlocks = 4 * kPpWin;
constexpr int kPpCols = 512;                      // two 256-column accumulators
constexpr int kPpEpi = 256;                       // epilogue threads (warps 2-9)
constexpr int kPpPlans = 4;                       // visits planned ahead

constexpr int kPpOffX = 0;
constexpr int kPpOffY = kPpOffX + kPpXHalves * kPpHalfBytes;
constexpr int kPpOffDiag = kPpOffY + kPpYUnits * kPpUnitBytes + kPpMirrorRows * 128;
constexpr int kPpDiagBytes = kPpMaxBlocks * 256 * 4;                    // 255 diagonals per block
constexpr int kPpOffBar = kPpOffDiag + kPpDiagBytes;
constexpr int kPpNBar = 2 * kPpXHalves + 2 * kPpYUnits + 2 + 2 + 1 + 2 * kPpPlans;
constexpr int kPpOffPlans = kPpOffBar + kPpNBar * 8;
constexpr int kPpPlanBytes = kPpPlans * 512;  // (static_assert below)
constexpr int kPpOffMisc = kPpOffPlans + kPpPlanBytes;
// misc words: tensor-memory address, abort flag, the run's first pair, pad,
// its job offset (int64), loads issued per x and y slot, the warps' job
// counts (int64) and the visit's block slots per window
constexpr int kPpMiscFills = 6;
constexpr int kPpMiscWarp = ((kPpMiscFills + kPpXHalves + kPpYUnits) * 4 + 7) / 8 * 8;
constexpr int kPpMiscWslot = kPpMiscWarp + 8 * 2 * (kPpThreads / 32);
constexpr int kPpMiscWin = kPpMiscWslot + 4 * 4 * kPpWin;  // the visit's windows: lo, c, length
constexpr int kPpMisc = kPpMiscWin + (8 + 8 + 8) * kPpWin;
constexpr int kPpSmemBytes = kPpOffMisc + kPpMisc + 1024;
static_assert(kPpOffY % 1024 == 0 && kPpUnitBytes % 1024 == 0 && kPpHalfBytes % 1024 == 0 &&
                  (kPpYRows * 128) % 1024 == 0,
              "loads and the mirror keep the 1024-byte swizzle pattern");
static_assert(kPpSmemBytes <= 232448, "one CTA per SM");
static_assert(kPpSegRows * 49 < (1 << 24), "exact FP32 sums of E4M3 level products");
static_assert(kPpSegRows == 2 * kPpHalfRows && kPpHalfRows % kPpTileRows == 0, "a visit's x is one or two halves");
static_assert(kPpGroupUnits * kPpUnitRows >= kPpSegRows + 1, "a single job's rows fit a group");
static_assert(kPpMirrorRows >= kPpTileRows + 1 - 1, "an MMA reads at most 33 rows from its start");

// Instruction descriptor, kind::f8f6f4: D F32 (bits 4-5 = 1), A and B E4M3
// (format 0), A and B MN-major (bits 15, 16), N >> 3 at 17, M >> 4 at 24.
__device__ __forceinline__ uint32_t pp_idesc(int nb) {
  return (1u << 4) | (1u << 15) | (1u << 16) | ((uint32_t)(128 * nb >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void pp_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void red_shared_s32(uint32_t addr, int v) {
  asm volatile("red.shared.add.s32 [%0], %1;" ::"r"(addr), "r"(v) : "memory");
}

// 16 lanes x 32 consecutive columns of FP32 accumulator -> v[0 .. 15] (the
// caller waits with tcgen05.wait::ld).  Thread t receives lanes t / 4 and
// t / 4 + 8 of the 16: v[4 g + e] = (lane t / 4, column 8 g + 2 (t % 4) + e)
// and v[4 g + 2 + e] = (lane t / 4 + 8, the same column), g < 4, e < 2 (the
// 16x256b shape's layout, checked on the device with a one-warp probe).
__device__ __forceinline__ void tmem_ld16x256_x4(uint32_t taddr, uint32_t* v) {
  asm volatile(
      "tcgen05.ld.sync.aligned.16x256b.x4.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(taddr));
}

// The diagonal sums of one warp's share of a finished accumulator: TMEM lanes
// 32 qd .. 32 qd + 31 (rows b) and kCols columns from c0 (columns j = jcol0 +
// the column's offset within them, in its block).  Thread t holds rows
// b_k = 32 qd + t / 4 + 8 k (k < 4) and columns 8 g + 2 (t % 4) + e, so its
// values with the same g - k lie on one diagonal j - b: it sums each such
// chain of four in FP32 (exact: |D| <= 512 * 49 and 4 * 512 * 49 < 2^24) and
// adds the 2 (kCols / 8 + 3) chain sums to the block's diagonals with
// shared-memory atomics, a third of one atomic per value.
template <int kCols>
__device__ __forceinline__ void pp_drain(uint32_t tcol, int qd, int lane, uint32_t drow) {
  constexpr int G = kCols / 8;
  float acc[2][G + 3];
#pragma unroll
  for (int e = 0; e < 2; ++e)
#pragma unroll
    for (int i = 0; i < G + 3; ++i) acc[e][i] = 0.f;
#pragma unroll
  for (int cb = 0; cb < kCols; cb += 32) {
    uint32_t lo[16], hi[16];  // lanes 32 qd + 0..15 (k = 0, 1) and + 16..31 (k = 2, 3)
    tmem_ld16x256_x4(tcol + (uint32_t)cb, lo);
    tmem_ld16x256_x4(tcol + (16u << 16) + (uint32_t)cb, hi);
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int gg = 0; gg < 4; ++gg) {
      const int g = cb / 8 + gg;
#pragma unroll
      for (int e = 0; e < 2; ++e) {
        acc[e][g + 3] += __uint_as_float(lo[4 * gg + e]);      // k = 0: g - k = g
        acc[e][g + 2] += __uint_as_float(lo[4 * gg + 2 + e]);  // k = 1
        acc[e][g + 1] += __uint_as_float(hi[4 * gg + e]);      // k = 2
        acc[e][g] += __uint_as_float(hi[4 * gg + 2 + e]);      // k = 3
      }
    }
  }
  // chain s = g - k (acc index s + 3) of column parity e lies on diagonal
  // j - b + 127 = 8 s + e + 2 (t % 4) - t / 4 - 32 qd + 127 (+ the columns' offset)
  const uint32_t d0 = drow + 4u * (uint32_t)(2 * (lane & 3) - (lane >> 2) - 32 * qd + 127 - 24);
#pragma unroll
  for (int i = 0; i < G + 3; ++i)
#pragma unroll
    for (int e = 0; e < 2; ++e)  // |sum| < 2^22: adding 1.5 * 2^23 leaves it in the low mantissa bits
      red_shared_s32(d0 + 4u * (uint32_t)(8 * i + e), __float_as_int(acc[e][i] + 12582912.0f) - 0x4B400000);
}

// Named barrier of the epilogue's 256 threads.
__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, 256;" ::: "memory"); }

__device__ __forceinline__ int64_t fdiv128(int64_t a) { return win_fdiv128(a); }

// The sorted block ranges of pair p's windows (win_blocks); the 16 lag bounds
// are loaded before any is used.
__device__ __forceinline__ void pp_ranges(const WinJob* __restrict__ jobs, int p, int (&a)[kPpWin], int (&b)[kPpWin]) {
  int64_t L[kPpWin], H[kPpWin];
#pragma unroll
  for (int w = 0; w < kPpWin; ++w) {
    L[w] = jobs[(int64_t)p * kPpWin + w].lag_lo;
    H[w] = jobs[(int64_t)p * kPpWin + w].lag_hi;
  }
  win_blocks(L, H, a, b);
}

// A pair's jobs in block order: job k covers blocks u[k], u[k] + nb[k] - 1.
struct PpPlan {
  int njobs;
  int u[kPpMaxJobs];
  int nb[kPpMaxJobs];
};

__device__ __noinline__ void pp_plan(const WinJob* __restrict__ jobs, int p, PpPlan& P) {
  int a[kPpWin], b[kPpWin];
  pp_ranges(jobs, p, a, b);
  P.njobs = 0;
  if (a[0] == INT_MAX) return;
  int r0 = a[0], r1 = b[0];
  for (int i = 1; i <= kPpWin; ++i) {
    if (i < kPpWin && a[i] != INT_MAX && a[i] <= r1 + 1) {
      r1 = b[i] > r1 ? b[i] : r1;
      continue;
    }
    for (int u = r0; u <= r1; u += 2) {
      P.u[P.njobs] = u;
      P.nb[P.njobs] = r1 - u >= 1 ? 2 : 1;
      ++P.njobs;
    }
    if (i == kPpWin || a[i] == INT_MAX) break;
    r0 = a[i], r1 = b[i];
  }
}

// One visit -- the run's jobs of one (pair, segment) -- as the loader plans it
// for the other roles: its jobs in block order, their groups (jobs whose y
// rows share one load) and each job's first slot in the diagonal store.
struct PpVisit {
  int p, s, tiles, nj, ng, pad;
  long long xh;                     // x half counter at the visit's first half
  int u[kPpMaxJobs], nb[kPpMaxJobs], slot[kPpMaxJobs];
  int gbeg[kPpMaxJobs + 1];         // first job of each group; gbeg[ng] = nj
  int gun[kPpMaxJobs];              // y units of each group
  long long gyu[kPpMaxJobs];        // logical index of each group's first y unit
};
static_assert(kPpPlans * sizeof(PpVisit) <= kPpPlanBytes && sizeof(PpVisit) % 8 == 0, "plan ring");

// The loader's position in the CTA's run of jobs, in (pair, segment, job)
// order.
struct PpRun {
  const WinJob* jobs;
  int nseg;
  int64_t rows_total, left;  // rows per signal, jobs still to plan
  int p, s, k;               // the next job
  long long xh, yu;          // x half and y unit counters
  PpPlan P;

  __device__ void init(const WinJob* j, int ns, int64_t rt, int p0, int64_t off, int64_t count) {
    jobs = j, nseg = ns, rows_total = rt, left = count;
    p = p0;
    pp_plan(jobs, p, P);
    s = (int)(off / P.njobs);
    k = (int)(off - (int64_t)s * P.njobs);
    xh = yu = 0;
  }
  // y units holding the rows of jobs [g0, g1] of a group: rows u_g0 + a ..
  // u_g1 + nb_g1 - 1 + a for a < 32 tiles
  __device__ int units(int g0, int g1, int tiles) const {
    const int rows = P.u[g1] + P.nb[g1] - 1 - P.u[g0] + kPpTileRows * tiles;
    return (rows + kPpUnitRows - 1) / kPpUnitRows;
  }
  // Plans the next visit into V; false at the run's end.
  __device__ bool next(PpVisit& V) {
    if (left <= 0) return false;
    if (k >= P.njobs) {  // past the pair's jobs in this segment
      k = 0;
      if (++s >= nseg) {
        s = 0;
        do {
          ++p;
          pp_plan(jobs, p, P);
        } while (P.njobs == 0);
      }
    }
    const int kb = k, ke = P.njobs - k < left ? P.njobs : k + (int)left, nj = ke - kb;
    const int64_t r = rows_total - (int64_t)kPpSegRows * s;
    const int tiles = (int)(((r < kPpSegRows ? r : kPpSegRows) + kPpTileRows - 1) / kPpTileRows);
    V.p = p, V.s = s, V.tiles = tiles, V.nj = nj, V.xh = xh;
    int slot = 0;
    for (int j = 0; j < nj; ++j) {
      V.u[j] = P.u[kb + j], V.nb[j] = P.nb[kb + j], V.slot[j] = slot;
      slot += P.nb[kb + j];
    }
    int ng = 0;
    for (int g0 = kb; g0 < ke;) {
      int g1 = g0 + 1;
      while (g1 < ke && units(g0, g1, tiles) <= kPpGroupUnits) ++g1;
      V.gbeg[ng] = g0 - kb, V.gun[ng] = units(g0, g1 - 1, tiles), V.gyu[ng] = yu;
      yu += V.gun[ng];
      ++ng;
      g0 = g1;
    }
    V.gbeg[ng] = nj, V.ng = ng;
    left -= nj, k = ke;
    xh += (tiles * kPpTileRows + kPpHalfRows - 1) / kPpHalfRows;
    return true;
  }
};

__global__ void __launch_bounds__(kPpThreads, 1)
    k_xcorr_win_pp(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap ymap,
                   const __grid_constant__ CUtensorMap mmap, int64_t rows_total, int npairs, int nseg,
                   const WinJob* __restrict__ jobs, const int32_t* __restrict__ njobs,
                   uint32_t* __restrict__ status) {
  extern __shared__ uint8_t smem_raw[];
  const uint32_t raw = smem_u32(smem_raw);
  const uint32_t base = (raw + 1023u) & ~1023u;
  uint8_t* const sb = smem_raw + (base - raw);
  const uint32_t xbuf = base + kPpOffX, ybuf = base + kPpOffY;
  const uint32_t diag_s = base + kPpOffDiag;
  int* const diag = reinterpret_cast<int*>(sb + kPpOffDiag);  // [block slot][256]
  const uint32_t xfull = base + kPpOffBar, xempty = xfull + 8 * kPpXHalves;
  const uint32_t yfull = xempty + 8 * kPpXHalves, yempty = yfull + 8 * kPpYUnits;
  const uint32_t accf = yempty + 8 * kPpYUnits, acce = accf + 16, done_bar = acce + 16;
  const uint32_t plan_full = done_bar + 8, plan_empty = plan_full + 8 * kPpPlans;
  PpVisit* const plans = reinterpret_cast<PpVisit*>(sb + kPpOffPlans);
  uint32_t* const misc = reinterpret_cast<uint32_t*>(sb + kPpOffMisc);
  uint32_t* const tmem_slot = misc;
  volatile int* const abort_flag = reinterpret_cast<volatile int*>(misc + 1);
  int* const run_sh = reinterpret_cast<int*>(misc + 2);  // first pair of the run, -1: empty
  int64_t* const off_sh = reinterpret_cast<int64_t*>(misc + 4);
  int* const xfills = reinterpret_cast<int*>(misc + kPpMiscFills);  // loads issued per x half slot
  int* const yfills = xfills + kPpXHalves;                         // per y unit slot
  long long* const wsum = reinterpret_cast<long long*>(sb + kPpOffMisc + kPpMiscWarp);
  int* const wslot = reinterpret_cast<int*>(sb + kPpOffMisc + kPpMiscWslot);  // [window][4]
  long long* const wlo = reinterpret_cast<long long*>(sb + kPpOffMisc + kPpMiscWin);  // [window]
  int** const wc = reinterpret_cast<int**>(wlo + kPpWin);
  long long* const wlen = wlo + 2 * kPpWin;  // lags - 1, or -1 for an empty window
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tid = threadIdx.x;
  constexpr int kWarps = kPpThreads / 32;

  // ---- the run: every pair's jobs counted (each thread a contiguous range
  // of pairs, their bounds loaded together), an exclusive scan, and the
  // pair holding the run's first job
  int64_t mine = 0;
  const int pl = (int)((int64_t)npairs * tid / kPpThreads), ph = (int)((int64_t)npairs * (tid + 1) / kPpThreads);
  for (int p = pl; p < ph; ++p) mine += (int64_t)njobs[p] * nseg;
  int64_t incl = mine;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t v = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += v;
  }
  if (lane == 31) wsum[warp] = incl;
  if (tid == 0) {
    *abort_flag = 0;
    run_sh[0] = -1;
  }
  __syncthreads();
  int64_t before = 0, J = 0;
#pragma unroll
  for (int i = 0; i < kWarps; ++i) {
    const int64_t v = wsum[i];
    before += i < warp ? v : 0;
    J += v;
  }
  const int64_t excl = before + incl - mine;
  const int64_t J0 = J * blockIdx.x / gridDim.x, J1 = J * (blockIdx.x + 1) / gridDim.x;
  if (J1 > J0 && mine > 0 && excl <= J0 && J0 < excl + mine) {
    int64_t a = excl;
    for (int p = pl; p < ph; ++p) {
      const int64_t c = (int64_t)njobs[p] * nseg;
      if (J0 < a + c) {
        run_sh[0] = p;
        *off_sh = J0 - a;
        break;
      }
      a += c;
    }
  }
  __syncthreads();
  const int p0 = run_sh[0];
  if (p0 < 0) return;  // no jobs for this CTA (no tensor memory held yet)
  const int64_t off0 = *off_sh;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kPpCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 32) {
    // a slot is released by both issuers (each after its last MMA reading it)
    for (int i = 0; i < kPpXHalves; ++i) mbar_init(xfull + 8 * i, 1), mbar_init(xempty + 8 * i, 2);
    for (int i = 0; i < kPpYUnits; ++i) mbar_init(yfull + 8 * i, 1), mbar_init(yempty + 8 * i, 2);
    for (int i = 0; i < 2; ++i) mbar_init(accf + 8 * i, 1), mbar_init(acce + 8 * i, kPpEpi / 32);
    mbar_init(done_bar, 2);
    for (int i = 0; i < kPpPlans; ++i) mbar_init(plan_full + 8 * i, 1), mbar_init(plan_empty + 8 * i, 3);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = tid; i < kPpMaxBlocks * 256; i += kPpThreads) diag[i] = 0;
  for (int i = tid; i < kPpXHalves + kPpYUnits; i += kPpThreads) xfills[i] = 0;
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 1) {
    // ---- the plans (lane 0) and the TMA loads (lanes 0-3: slot s of each
    // ring by lane s % 4, so a slot's fills are issued in order and a lap's
    // empty-barrier wait can never see a phase two behind)
    PpRun R;
    if (lane == 0) {
      R.init(jobs, nseg, rows_total, p0, off0, J1 - J0);
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&xmap)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&ymap)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&mmap)) : "memory");
    }
    bool ok = true;
    // x half i goes to slot xs (lap xl), y unit i to slot ys (lap yl); a
    // slot's lap l >= 1 waits for the release of lap l - 1
    int xs = 0, ys = 0;
    uint32_t xl = 0, yl = 0;
    auto load_x = [&](int row, int sig) -> bool {
      if ((xs & 3) == lane) {
        if (xl > 0 && !mbar_wait_sleep(xempty + 8 * xs, (xl - 1) & 1u)) return false;
        const uint32_t fb = xfull + 8 * xs;
        mbar_expect_tx_win(fb, kPpHalfBytes);
        tma_load3(xbuf + (uint32_t)(xs * kPpHalfBytes), &xmap, 0, row, sig, fb);
      }
      if (++xs == kPpXHalves) xs = 0, ++xl;
      return true;
    };
    auto load_y = [&](int row, int sig) -> bool {
      if ((ys & 3) == lane) {
        if (yl > 0 && !mbar_wait_sleep(yempty + 8 * ys, (yl - 1) & 1u)) return false;
        const uint32_t fb = yfull + 8 * ys;
        mbar_expect_tx_win(fb, ys == 0 ? kPpUnitBytes + kPpMirrorRows * 128 : kPpUnitBytes);
        tma_load3(ybuf + (uint32_t)(ys * kPpUnitBytes), &ymap, 0, row, sig, fb);
        if (ys == 0) tma_load3(ybuf + (uint32_t)(kPpYRows * 128), &mmap, 0, row, sig, fb);
      }
      if (++ys == kPpYUnits) ys = 0, ++yl;
      return true;
    };
    for (long long v = 0; !*abort_flag; ++v) {
      const int ps = (int)(v % kPpPlans);
      PpVisit& V = plans[ps];
      int more = 1;
      if (lane == 0) {
        if (v >= kPpPlans && !mbar_wait_sleep(plan_empty + 8 * ps, (uint32_t)(((v / kPpPlans) - 1) & 1))) {
          ok = false;
        } else {
          more = R.next(V) ? 1 : 0;
          if (!more) V.nj = 0;  // the end of the run
          mbar_arrive(plan_full + 8 * ps);
        }
      }
      more = __shfl_sync(0xffffffffu, ok && more ? 1 : 0, 0);
      __syncwarp();
      if (!more) break;
      if (lane < 4) {
        const int sig = 2 * V.p, rowbase = V.s * kPpSegRows, ng = V.ng;
        const int nh = (V.tiles * kPpTileRows + kPpHalfRows - 1) / kPpHalfRows;
        for (int g = 0; g < ng && ok; ++g) {
          const int ubase = rowbase + V.u[V.gbeg[g]], gun = V.gun[g];
          int c = 0;
          if (g == 0) {  // x half h, then the y units the group's first job reads with it
            for (int h = 0; h < nh && ok; ++h) {
              ok = load_x(rowbase + kPpHalfRows * h, sig);
              const int need = (kPpHalfRows * (h + 1) + kPpTileRows) / kPpUnitRows;
              for (; ok && c < gun && c <= need; ++c) ok = load_y(ubase + kPpUnitRows * c, sig + 1);
            }
          }
          for (; ok && c < gun; ++c) ok = load_y(ubase + kPpUnitRows * c, sig + 1);
          if (*abort_flag) ok = false;
        }
      }
      if (!__all_sync(0xffffffffu, ok)) {
        ok = false;
        break;
      }
    }
    if (!ok) *abort_flag = 1;
    // loads issued per slot, for the final wait on loads in flight
    if (lane == 0) {
      for (int i = 0; i < kPpXHalves; ++i) xfills[i] = (int)xl + (i < xs ? 1 : 0);
      for (int i = 0; i < kPpYUnits; ++i) yfills[i] = (int)yl + (i < ys ? 1 : 0);
    }
  } else if (warp == 0 || warp == kPpIssuerB) {
    // ---- MMAs: two issuers (lane 0 of warps 0 and kPpIssuerB) take
    // alternate jobs, each into its own accumulator, so that one thread's
    // issue cost (about 65 cycles per MMA plus its loop) has twice the
    // tensor pipe's time per MMA.  A slot's release takes both: the issuer of
    // the last job that reads it commits after that job's batch, the other
    // after its own last job of the group (y) or visit (x).  Ring slots and
    // phases advance incrementally: no division in the loops.
    if (lane == 0) {
      const int me = warp == 0 ? 0 : 1;
      bool ok = true;
      int64_t jc = 0;  // jobs walked (both issuers'); this issuer's are those with jc % 2 == me
      const uint64_t da0 = sdesc(xbuf, 128u, 1024u, 2u, 0u), db0 = sdesc(ybuf, 128u, 1024u, 2u, 0u);
      constexpr int kTilesPerHalf = kPpHalfRows / kPpTileRows;
      auto wait = [&](uint32_t bar, uint32_t parity) { return mbar_try(bar, parity) || mbar_wait_sleep(bar, parity); };
      const uint32_t d = tmem + 256u * (uint32_t)me;  // this issuer's accumulator
      for (long long v = 0; ok && !*abort_flag; ++v) {
        const int ps = (int)(v % kPpPlans);
        if (!wait(plan_full + 8 * ps, (uint32_t)((v / kPpPlans) & 1))) {
          ok = false;
          break;
        }
        const PpVisit& V = plans[ps];
        const int nj = V.nj, tiles = V.tiles, ng = V.ng;
        if (nj == 0) break;
        // the visit's x halves: slots and fill phases
        const int nh = (tiles + kTilesPerHalf - 1) / kTilesPerHalf;
        const int xs0 = (int)(V.xh % kPpXHalves), xs1 = xs0 + 1 == kPpXHalves ? 0 : xs0 + 1;
        const uint32_t xp0 = (uint32_t)((V.xh / kPpXHalves) & 1), xp1 = xs1 == 0 ? xp0 ^ 1u : xp0;
        const uint32_t xa0 = (uint32_t)(xs0 * kPpHalfBytes), xa1 = (uint32_t)(xs1 * kPpHalfBytes);
        const int vlast = (int)((jc + nj - 1) & 1);  // the issuer of the visit's last job
        bool xwaited = false;
        for (int g = 0; g < ng && ok; ++g) {
          const int gb = V.gbeg[g], ge = V.gbeg[g + 1], ufirst = V.u[gb], gun = V.gun[g];
          const int gys = (int)(V.gyu[g] % kPpYUnits);                  // slot of the group's unit 0
          const uint32_t gyp = (uint32_t)((V.gyu[g] / kPpYUnits) & 1);  // and its fill phase
          int ywaited = -1;               // group units known loaded
          int wys = gys;                  // slot and phase of unit ywaited + 1
          uint32_t wyp = gyp;
          int freed = 0, fys = gys;       // group units released; slot of unit freed
          const int yrow0 = gys * kPpUnitRows;  // ring row of the group's row 0
          const int64_t jg = jc + (ge - gb);    // jc after the group
          const int glast = (int)((jg - 1) & 1);  // the issuer of the group's last job
          for (int kk = gb; kk < ge && ok; ++kk, ++jc) {
            if ((int)(jc & 1) != me) continue;
            const int nb = V.nb[kk], urel = V.u[kk] - ufirst;
            const bool last_visit = kk == nj - 1, last_group = kk == ge - 1;
            const int64_t mine = jc >> 1;  // this issuer's job count
            if (mine >= 1 && !wait(acce + 8 * me, (uint32_t)((mine - 1) & 1))) {
              ok = false;
              break;
            }
            tc_fence_after();
            const uint32_t idesc = pp_idesc(nb);
            int row = yrow0 + urel;  // ring row of this job's tile 0
            if (row >= kPpYRows) row -= kPpYRows;
            uint64_t db = db0 + (uint64_t)(row * 8);
            if (xwaited && !last_visit && !last_group &&
                (urel + kPpTileRows * tiles + nb - 2) / kPpUnitRows <= ywaited) {
              // every operand is loaded and no slot is released: one run of MMAs
              uint64_t da = da0 + (xa0 >> 4);
              for (int t = 0; t < tiles; ++t) {
                pp_mma(d, da, db, idesc, t > 0 ? 1u : 0u);
                da = t == kTilesPerHalf - 1 ? da0 + (xa1 >> 4) : da + (kPpTileRows * 128 >> 4);
                db += kPpTileRows * 128 >> 4;
                row += kPpTileRows;
                if (row >= kPpYRows) row -= kPpYRows, db -= kPpYRows * 128 >> 4;
              }
              mma_commit(accf + 8 * me);
              continue;
            }
            // the K tiles in batches of one x half: waits before a batch,
            // releases after it, the batch's MMAs back to back
            for (int h = 0, t0 = 0; t0 < tiles; ++h, t0 += kTilesPerHalf) {
              const int t1 = t0 + kTilesPerHalf < tiles ? t0 + kTilesPerHalf : tiles;
              bool waited = false;
              if (!xwaited) {
                if (!wait(xfull + 8 * (h ? xs1 : xs0), h ? xp1 : xp0)) {
                  ok = false;
                  break;
                }
                if (t1 == tiles) xwaited = true;
                waited = true;
              }
              // tile t reads group rows urel + 32 t .. urel + 32 t + 32 + nb - 2
              const int need = (urel + kPpTileRows * t1 + nb - 2) / kPpUnitRows;
              while (ywaited < need) {
                if (!wait(yfull + 8 * wys, wyp)) {
                  ok = false;
                  break;
                }
                ++ywaited;
                if (++wys == kPpYUnits) wys = 0, wyp ^= 1u;
                waited = true;
              }
              if (!ok) break;
              if (waited) tc_fence_after();
              uint64_t da = da0 + ((h ? xa1 : xa0) >> 4);
              for (int t = t0; t < t1; ++t) {
                pp_mma(d, da, db, idesc, t > 0 ? 1u : 0u);
                da += kPpTileRows * 128 >> 4;
                db += kPpTileRows * 128 >> 4;
                row += kPpTileRows;
                if (row >= kPpYRows) row -= kPpYRows, db -= kPpYRows * 128 >> 4;
              }
              if (last_visit) mma_commit(xempty + 8 * (h ? xs1 : xs0));  // the visit's last reads of this half
              if (last_group) {
                // units below the next batch's first row are read by no later MMA
                const int upto = t1 == tiles ? gun : (urel + kPpTileRows * t1) / kPpUnitRows;
                for (; freed < upto; ++freed) {
                  mma_commit(yempty + 8 * fys);
                  if (++fys == kPpYUnits) fys = 0;
                }
              }
            }
            if (!ok) break;
            mma_commit(accf + 8 * me);
          }
          // the other issuer's share of the group's releases: after its own
          // last MMAs of the group (all of them precede the commit), and only
          // once the group's units are loaded, so that no release runs ahead
          // of the fill it answers
          if (ok && glast != me) {
            while (ok && ywaited < gun - 1) {
              ok = wait(yfull + 8 * wys, wyp);
              ++ywaited;
              if (++wys == kPpYUnits) wys = 0, wyp ^= 1u;
            }
            for (int i = 0, sl = gys; ok && i < gun; ++i) {
              mma_commit(yempty + 8 * sl);
              if (++sl == kPpYUnits) sl = 0;
            }
          }
        }
        if (ok && vlast != me) {  // and of the visit's x halves
          for (int h = 0; ok && !xwaited && h < nh; ++h) ok = wait(xfull + 8 * (h ? xs1 : xs0), h ? xp1 : xp0);
          for (int h = 0; ok && h < nh; ++h) mma_commit(xempty + 8 * (h ? xs1 : xs0));
        }
        mbar_arrive(plan_empty + 8 * ps);  // this issuer is done with the plan
      }
      if (!ok) *abort_flag = 1;
      mma_commit(done_bar);
    }
    __syncwarp();
  } else if (warp >= 2 && warp < 10) {
    // ---- epilogue (warps 2-9): TMEM lanes 32 (warp & 3) .., column half h
    const int qd = warp & 3, h = (warp - 2) >> 2;
    const int e = tid - 64;  // 0 .. 255
    int64_t jc = 0;
    bool ok = true;
    for (long long v = 0; ok && !*abort_flag; ++v) {
      const int ps = (int)(v % kPpPlans);
      if (!warp_wait(plan_full + 8 * ps, (uint32_t)((v / kPpPlans) & 1))) {
        ok = false;
        break;
      }
      const PpVisit& V = plans[ps];
      const int nj = V.nj;
      if (nj == 0) break;
      if (e < 4 * kPpWin) {  // the windows and their blocks' slots (or -1), read at the visit's end
        const int w = e >> 2, i = e & 3;
        const WinJob J = jobs[(int64_t)V.p * kPpWin + w];
        int sl = -1;
        if (J.lag_hi >= J.lag_lo) {
          const int64_t ub = fdiv128(J.lag_lo) + i;
          for (int kk = 0; kk < nj; ++kk) {
            const int u = V.u[kk], nbk = V.nb[kk];
            if (ub >= u && ub < u + nbk) sl = V.slot[kk] + (int)(ub - u);
          }
        }
        wslot[e] = sl;
        if (i == 0) wlo[w] = J.lag_lo, wc[w] = J.c, wlen[w] = J.lag_hi >= J.lag_lo ? J.lag_hi - J.lag_lo : -1;
      }
      for (int kk = 0; kk < nj; ++kk, ++jc) {
        const int nb = V.nb[kk], slot = V.slot[kk];
        const int jb = (int)(jc & 1);
        if (!warp_wait(accf + 8 * jb, (uint32_t)((jc >> 1) & 1))) {
          ok = false;
          break;
        }
        tc_fence_after();
        // block h (two blocks) or columns 64 h .. (one block) of this warp's
        // lanes: value D[b][j] to diagonal j - b + 127 of its block's slot
        const uint32_t tcol = tmem + ((uint32_t)(32 * qd) << 16) + 256u * (uint32_t)jb;
        if (nb == 2)  // block h: its 128 columns
          pp_drain<128>(tcol + 128u * (uint32_t)h, qd, lane, diag_s + 4u * (uint32_t)(256 * (slot + h)));
        else  // columns 64 h .. 64 h + 63 of the one block
          pp_drain<64>(tcol + 64u * (uint32_t)h, qd, lane, diag_s + 4u * (uint32_t)(256 * slot + 64 * h));
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(acce + 8 * jb);
      }
      if (!ok) break;
      const int nslots = V.slot[nj - 1] + V.nb[nj - 1];
      // ---- the visit's blocks to its pair's windows: c[tau] = diagonal
      // tau - 128 q + 127 of block q plus diagonal tau - 128 (q + 1) + 127 of
      // block q + 1 (q = floor(tau / 128)), for the blocks this visit holds
      epi_sync();
      for (int idx = e; idx < kPpWin * kPpWinLen; idx += kPpEpi) {
        const int w = idx / kPpWinLen, t = idx - w * kPpWinLen;
        if (t > wlen[w]) continue;
        const long long lo = wlo[w];
        const int64_t tau = lo + t, q = fdiv128(tau);
        const int r = (int)(tau - 128 * q), i0 = (int)(q - fdiv128(lo));
        int val = 0;
        const int s0 = wslot[4 * w + i0];
        if (s0 >= 0) val += diag[256 * s0 + r + 127];
        if (r >= 1) {
          const int s1 = wslot[4 * w + i0 + 1];
          if (s1 >= 0) val += diag[256 * s1 + r - 1];
        }
        if (val != 0) atomicAdd(wc[w] + t, val);
      }
      epi_sync();
      for (int i = e; i < 256 * nslots; i += kPpEpi) diag[i] = 0;
      epi_sync();
      if (e == 0) mbar_arrive(plan_empty + 8 * ps);  // the epilogue is done with the plan
    }
    if (!ok) *abort_flag = 1;
  }

  tc_fence_before();
  __syncthreads();
  // the MMAs and every load issued have completed before the buffers and
  // tensor memory are released (bounded waits, one barrier per thread)
  if (tid == 0) {
    if (*abort_flag) atomicOr(status, TDE_ST_TIMEOUT);
    mbar_wait(done_bar, 0u);
  } else if (tid <= kPpXHalves) {
    const int i = tid - 1;
    if (xfills[i] > 0) mbar_wait(xfull + 8 * i, (uint32_t)((xfills[i] - 1) & 1));
  } else if (tid <= kPpXHalves + kPpYUnits) {
    const int i = tid - 1 - kPpXHalves;
    if (yfills[i] > 0) mbar_wait(yfull + 8 * i, (uint32_t)((yfills[i] - 1) & 1));
  }
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kPpCols) : "memory");
  }
}

}  // namespace

cudaError_t launch_xcorr_win_pp(const uint8_t* d_qe, int64_t n, int64_t n_pad, int npairs, const WinJob* d_jobs,
                                const int32_t* d_njobs, uint32_t* d_status, cudaStream_t st) {
  if (npairs <= 0) return cudaSuccess;
  if (n <= 0 || n_pad % 128 != 0 || n_pad < n || (reinterpret_cast<uintptr_t>(d_qe) & 15) != 0)
    return cudaErrorInvalidValue;
  const int64_t rows = n_pad / 128;
  // TMA row coordinates (int32) reach a segment start plus a block offset of
  // at most (n + 127) / 128 plus a group's rows
  if (rows > (int64_t)1 << 28 || 2 * (int64_t)npairs > INT32_MAX) return cudaErrorInvalidValue;
  const int nseg = (int)((rows + kPpSegRows - 1) / kPpSegRows);
  CUtensorMap xmap, ymap, mmap;
  if (!tmap_bytes3(&xmap, d_qe, n_pad, 2 * npairs, 128, kPpHalfRows, 128) ||
      !tmap_bytes3(&ymap, d_qe, n_pad, 2 * npairs, 128, kPpUnitRows, 128) ||
      !tmap_bytes3(&mmap, d_qe, n_pad, 2 * npairs, 128, kPpMirrorRows, 128))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(k_xcorr_win_pp, cudaFuncAttributeMaxDynamicSharedMemorySize, kPpSmemBytes);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  k_xcorr_win_pp<<<sms, kPpThreads, kPpSmemBytes, st>>>(xmap, ymap, mmap, rows, npairs, nseg, d_jobs, d_njobs, d_status);
  TDE_COUNT_LAUNCH(1);
  return cudaGetLastError();
}
