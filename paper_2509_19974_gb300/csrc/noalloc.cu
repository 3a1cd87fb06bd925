// noalloc.cu -- tde_quantize_noalloc: the quantizer (Algorithm 1's quantization step)
// for callers that cannot allocate device memory.
//
// Every other entry point works through a tde_ctx, and a context allocates:
// its device workspace and its pinned staging buffer grow with cudaMalloc /
// cudaMallocHost on demand.  Some callers cannot do that -- a real-time audio
// callback that must not block inside the allocator, a host that runs this
// library under its own device-memory manager and forbids foreign
// allocations, code that enqueues work while a stream is being captured.
// This entry point needs no context: the rank quantizer's scratch (the
// per-signal signal descriptor, radix-select state and 7 x 2048-bin
// histograms) lives in one file-scope __device__ array, sized for at most
// kMaxSignals signals per call, which every GPU that loads the library keeps
// until the process exits.  The caller passes inputs, outputs and a one-word
// device status output; nothing is allocated or freed.
//
// Host code must not hand the array's name to a kernel (on the host it is a
// stand-in symbol, not a device address): the first call on each device asks
// the runtime for the device address with cudaGetSymbolAddress (with that
// device current) and caches it for the life of the process (a
// cudaDeviceReset of that device would make the cached address stale, so the
// entry point must not be used across one).  All calls share the array, and it keeps the
// previous call's contents, so each call clears the histograms it uses and
// rewrites the descriptors and state; calls whose kernels overlap on the GPU
// (different streams, no ordering between them) race on it.
#include <cstddef>
#include <mutex>

#include "common.cuh"

namespace {

constexpr int kMaxSignals = 16;
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
  QSig sigs[kMaxSignals];
  RankState state[kMaxSignals];
  uint32_t hist[kMaxSignals * 7 * 2048];
};

// 16 x (24 + 56 + 57344) bytes, about 0.9 MiB per device.
__device__ __align__(256) unsigned char tde_noalloc_scratch[sizeof(NoAllocScratch)];

std::mutex g_mu;
char* g_scratch[kMaxDevices] = {};

__global__ void k_noalloc_sigs(QSig* __restrict__ dst, const float* x, int8_t* q, int64_t n,
                               int nsig) {
  const int i = threadIdx.x;
  if (i < nsig) dst[i] = QSig{x + (int64_t)i * n, q + (int64_t)i * n, n};
}

// Device address of the scratch array on the current device (set-up once).
cudaError_t scratch_on_current_device(char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_scratch[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, tde_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_scratch[dev] = static_cast<char*>(p);
  }
  *out = g_scratch[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" tde_status tde_quantize_noalloc(const float* x, int64_t n, int nsig, int bits,
                                           int8_t* q_out, uint32_t* status_out,
                                           tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  if (!x || !q_out || !status_out) return TDE_ERR_INVALID;
  if (bits != 1 && bits != 2 && bits != 4) return TDE_ERR_INVALID;
  if (n <= 0 || nsig <= 0) return TDE_ERR_INVALID;
  if (n > INT32_MAX) return TDE_ERR_UNSUPPORTED;
  if (nsig > kMaxSignals) return TDE_ERR_UNSUPPORTED;
  char* base = nullptr;
  if (scratch_on_current_device(&base) != cudaSuccess) return TDE_ERR_CUDA;
  QSig* d_sigs = reinterpret_cast<QSig*>(base + offsetof(NoAllocScratch, sigs));
  RankState* d_state = reinterpret_cast<RankState*>(base + offsetof(NoAllocScratch, state));
  uint32_t* d_hist = reinterpret_cast<uint32_t*>(base + offsetof(NoAllocScratch, hist));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (cudaMemsetAsync(status_out, 0, sizeof(uint32_t), st) != cudaSuccess) return TDE_ERR_CUDA;
  k_noalloc_sigs<<<1, kMaxSignals, 0, st>>>(d_sigs, x, q_out, n, nsig);
  TDE_COUNT_LAUNCH(1);
  if (cudaGetLastError() != cudaSuccess) return TDE_ERR_CUDA;
  // launch_quantize_rank clears the histograms of these nsig signals and
  // re-initialises their radix-select state before using them.
  const cudaError_t e =
      bits == 1 ? launch_quantize_sign(d_sigs, nsig, n, status_out, st)
                : launch_quantize_rank(d_sigs, nsig, n, bits, d_state, d_hist, status_out, st);
  return e == cudaSuccess ? TDE_OK : TDE_ERR_CUDA;
}
