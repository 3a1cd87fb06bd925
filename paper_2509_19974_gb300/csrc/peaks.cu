// peaks.cu -- tde_measure_peaks: the issue rates, per SM per clock, that the
// engines' rooflines are measured against on the GPU at hand.  Each rate is
// timed with clock64 inside one CTA per SM (a large dynamic shared-memory
// request keeps a second CTA off the SM), so it does not depend on the SM
// clock; a caller multiplies by the SM count and the clock it sampled.
//   POPC: __popc on 32-bit words (the popc engine's inner operation);
//   IMAD: 32-bit integer multiply-add (the NTT engine's modular arithmetic);
//   E4M3 / E2M1 MMA: back-to-back tcgen05.mma of M = 128, N = 256 from one
//   thread, kind::f8f6f4 (K = 32) and kind::mxf4 with unit block scales
//   (K = 64), operands fixed in shared memory, MACs per clock.
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace {

constexpr int kPkThreads = 1024;
constexpr int kPkSmem = 120 * 1024;  // one CTA per SM
constexpr int kPkIters = 4096;

__global__ void __launch_bounds__(kPkThreads, 1) k_peak_popc(uint32_t seed, uint32_t* sink, long long* cyc) {
  uint32_t v[8], a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = seed * (threadIdx.x + 7 * i + 1), a[i] = 0;
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < kPkIters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      a[i] += __popc(v[i]);
      v[i] ^= a[i];
    }
  }
  __syncthreads();
  const long long t1 = clock64();
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  if (s == 0x9E3779B9u) sink[0] = s;  // keeps the loop
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

__global__ void __launch_bounds__(kPkThreads, 1) k_peak_imad(uint32_t seed, uint32_t* sink, long long* cyc) {
  uint32_t v[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = seed + threadIdx.x + 3 * i;
  const uint32_t m = seed | 1u;
  __syncthreads();
  const long long t0 = clock64();
  for (int it = 0; it < kPkIters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = v[i] * m + (uint32_t)i;
  }
  __syncthreads();
  const long long t1 = clock64();
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s ^= v[i];
  if (s == 0x9E3779B9u) sink[0] = s;
  if (threadIdx.x == 0) cyc[blockIdx.x] = t1 - t0;
}

__device__ __forceinline__ uint32_t pk_smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// K-major no-swizzle descriptor (start, leading 128 B, stride 256 B, version 1)
__device__ __forceinline__ uint64_t pk_desc(uint32_t addr) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(128 >> 4) << 16) | ((uint64_t)(256 >> 4) << 32) |
         (1ull << 46);
}

// kind: 0 = E4M3 (kind::f8f6f4), 1 = E2M1 (kind::mxf4, unit UE8M0 scales)
template <int KIND>
__global__ void __launch_bounds__(128, 1) k_peak_mma(int iters, long long* cyc, uint32_t* status) {
  extern __shared__ __align__(1024) uint8_t pk_smem[];
  uint8_t* sa = pk_smem;              // A: 128 rows x 32 bytes
  uint8_t* sb = pk_smem + 128 * 32;   // B: 256 rows x 32 bytes
  uint64_t* bar = reinterpret_cast<uint64_t*>(pk_smem + 128 * 32 + 256 * 32);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 1);
  for (int i = threadIdx.x; i < 384 * 32; i += blockDim.x) sa[i] = 0;
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  const int warp = threadIdx.x >> 5;
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(pk_smem_u32(tslot)),
                 "r"(512)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(pk_smem_u32(bar)), "r"(1u) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  {  // block scales (E2M1): UE8M0 1.0 in columns 256 .. 511 of this warp's lanes
    const uint32_t lanes = (uint32_t)(32 * warp) << 16;
    for (int c0 = 256; c0 < 512; c0 += 8)
      asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1, %1, %1, %1, %1, %1, %1, %1};" ::"r"(
                       tmem + lanes + (uint32_t)c0),
                   "r"(0x7F7F7F7Fu)
                   : "memory");
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  if (threadIdx.x == 0) {
    const uint64_t da = pk_desc(pk_smem_u32(sa)), db = pk_desc(pk_smem_u32(sb));
    const uint32_t idesc = KIND == 0 ? ((1u << 4) | (32u << 17) | (8u << 24))
                                     : ((1u << 7) | (1u << 10) | (32u << 17) | (1u << 23) | (8u << 24));
    const long long t0 = clock64();
    for (int i = 0; i < iters; ++i) {
      if (KIND == 0)
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(i)
            : "memory");
      else
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %6, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::mxf4.block_scale.scale_vec::2X [%0], %1, %2, %3, [%4], [%5], p;\n\t}" ::"r"(
                tmem),
            "l"(da), "l"(db), "r"(idesc), "r"(tmem + 256u), "r"(tmem + 384u), "r"(i)
            : "memory");
    }
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     pk_smem_u32(bar))
                 : "memory");
    // bounded wait for the MMAs (about 2 s at 2 GHz)
    uint32_t done = 0;
    for (long long tw = clock64(); !done && clock64() - tw < 4000000000ll;)
      asm volatile(
          "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
          : "=r"(done)
          : "r"(pk_smem_u32(bar)), "r"(0u)
          : "memory");
    cyc[blockIdx.x] = done ? clock64() - t0 : -1;
    if (!done) atomicOr(status, TDE_ST_TIMEOUT);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512) : "memory");
  }
}

// max over CTAs of their cycle counts (the slowest SM sets the rate); -1 if any failed
double max_cycles(const long long* h, int n) {
  long long m = 0;
  for (int i = 0; i < n; ++i) {
    if (h[i] < 0) return -1.0;
    m = h[i] > m ? h[i] : m;
  }
  return (double)m;
}

}  // namespace

extern "C" tde_status tde_measure_peaks(int device, tde_peaks* out) {
  if (!out) return TDE_ERR_INVALID;
  int prev = 0;
  if (cudaGetDevice(&prev) != cudaSuccess || cudaSetDevice(device) != cudaSuccess) return TDE_ERR_CUDA;
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  long long* d_cyc = nullptr;
  uint32_t* d_aux = nullptr;
  long long* h = nullptr;
  tde_status st = TDE_OK;
  const int mma_iters = 20000;
  auto fail = [&](cudaError_t e) { return e != cudaSuccess ? (st = TDE_ERR_CUDA, true) : false; };
  do {
    if (fail(cudaMalloc(&d_cyc, sizeof(long long) * sms)) || fail(cudaMalloc(&d_aux, 8)) ||
        fail(cudaMemset(d_aux, 0, 8)) || fail(cudaMallocHost(&h, sizeof(long long) * sms)))
      break;
    if (fail(cudaFuncSetAttribute(k_peak_popc, cudaFuncAttributeMaxDynamicSharedMemorySize, kPkSmem)) ||
        fail(cudaFuncSetAttribute(k_peak_imad, cudaFuncAttributeMaxDynamicSharedMemorySize, kPkSmem)) ||
        fail(cudaFuncSetAttribute(k_peak_mma<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPkSmem)) ||
        fail(cudaFuncSetAttribute(k_peak_mma<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, kPkSmem)))
      break;
    double rate[4] = {0, 0, 0, 0};
    for (int k = 0; k < 4 && st == TDE_OK; ++k) {
      for (int rep = 0; rep < 2; ++rep) {  // the first run warms up
        if (k == 0) k_peak_popc<<<sms, kPkThreads, kPkSmem>>>(12345u, d_aux + 1, d_cyc);
        if (k == 1) k_peak_imad<<<sms, kPkThreads, kPkSmem>>>(12345u, d_aux + 1, d_cyc);
        if (k == 2) k_peak_mma<0><<<sms, 128, kPkSmem>>>(mma_iters, d_cyc, d_aux);
        if (k == 3) k_peak_mma<1><<<sms, 128, kPkSmem>>>(mma_iters, d_cyc, d_aux);
        if (fail(cudaGetLastError()) || fail(cudaDeviceSynchronize())) break;
      }
      if (st != TDE_OK || fail(cudaMemcpy(h, d_cyc, sizeof(long long) * sms, cudaMemcpyDeviceToHost))) break;
      const double c = max_cycles(h, sms);
      if (c <= 0) {
        st = TDE_ERR_TIMEOUT;
        break;
      }
      const double ops = k < 2 ? (double)kPkThreads * kPkIters * 8 : (double)mma_iters * 128.0 * 256.0 * (k == 2 ? 32 : 64);
      rate[k] = ops / c;
    }
    if (st != TDE_OK) break;
    out->sm_count = sms;
    out->popc_per_sm_clk = rate[0];
    out->imad_per_sm_clk = rate[1];
    out->e4m3_mac_per_sm_clk = rate[2];
    out->e2m1_mac_per_sm_clk = rate[3];
  } while (false);
  if (h) cudaFreeHost(h);
  if (d_aux) cudaFree(d_aux);
  if (d_cyc) cudaFree(d_cyc);
  cudaSetDevice(prev);
  return st;
}
