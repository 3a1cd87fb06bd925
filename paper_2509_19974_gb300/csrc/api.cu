// api.cu -- the C ABI of libtde (declared in include/tde.h): argument checks,
// the context (device workspace, pinned descriptor staging, device status
// word), and the dispatch of Algorithm 1's steps (arXiv 2509.19974, Sec. 3.2)
// to the kernels.  No step of the path runs on the host.
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "mma.cuh"
#include "fftcmp.cuh"
#include "ntt.cuh"
#include "refine.cuh"
#include "cnn.cuh"

struct tde_ctx {
  int device = 0;
  int sm_count = 0;
  uint32_t* d_status = nullptr;
  char* ws = nullptr;          // device workspace
  size_t ws_cap = 0;
  char* stage = nullptr;       // pinned host staging for descriptor uploads
  size_t stage_cap = 0;
  cudaEvent_t stage_ev = nullptr;
  bool stage_busy = false;
  std::string err;
  // instrumentation
  bool profile = false;
  std::vector<cudaEvent_t> ev;  // start/end pairs around engine kernels
  size_t ev_used = 0;
  int64_t launches = 0, engine_launches = 0;
  FftPlan fft;
  uint32_t* ntt_tables[kNttMaxLog + 1] = {};  // per log2 length, 8 * N uint32
  bool ntt_two_primes = false;                 // NTT engine: CRT even where one prime suffices
  std::vector<tde_tune_entry> tune;           // autotuner table (empty: built-in rule)
};

thread_local int64_t tde_launch_counter = 0;

namespace {

tde_status set_err(tde_ctx* ctx, tde_status s, const char* fmt, ...) {
  if (ctx) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    ctx->err = buf;
  }
  return s;
}

tde_status cuda_err(tde_ctx* ctx, cudaError_t e, const char* what) {
  return set_err(ctx, TDE_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define TDE_CK(call)                                          \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_err(ctx, e_, #call);   \
  } while (0)

// Makes ctx->device current for the lifetime of the guard.
struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (prev != dev) cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Bump allocator over a region whose size is computed first (dry run) and
// then carved for real.
struct Carve {
  char* base;
  size_t off = 0;
  explicit Carve(char* b) : base(b) {}
  template <typename T>
  T* take(size_t count) {
    off = align_up(off, 256);
    T* p = reinterpret_cast<T*>(base ? base + off : nullptr);
    off += count * sizeof(T);
    return p;
  }
};

tde_status ensure_ws(tde_ctx* ctx, size_t bytes) {
  if (bytes <= ctx->ws_cap) return TDE_OK;
  // Earlier calls may still use the old workspace on any stream.
  TDE_CK(cudaDeviceSynchronize());
  if (ctx->ws) TDE_CK(cudaFree(ctx->ws));
  ctx->ws = nullptr;
  ctx->ws_cap = 0;
  size_t cap = align_up(bytes + bytes / 4, 1 << 20);
  TDE_CK(cudaMalloc(&ctx->ws, cap));
  ctx->ws_cap = cap;
  return TDE_OK;
}

// Host staging of descriptors: waits until the previous upload has left the
// pinned buffer before it is rewritten.
tde_status stage_begin(tde_ctx* ctx, size_t bytes, char** host) {
  if (ctx->stage_busy) {
    TDE_CK(cudaEventSynchronize(ctx->stage_ev));
    ctx->stage_busy = false;
  }
  if (bytes > ctx->stage_cap) {
    if (ctx->stage) TDE_CK(cudaFreeHost(ctx->stage));
    ctx->stage = nullptr;
    ctx->stage_cap = 0;
    size_t cap = align_up(bytes + bytes / 4, 1 << 16);
    TDE_CK(cudaMallocHost(&ctx->stage, cap));
    ctx->stage_cap = cap;
  }
  *host = ctx->stage;
  return TDE_OK;
}

tde_status stage_upload(tde_ctx* ctx, void* dev, size_t bytes, cudaStream_t st) {
  if (bytes) TDE_CK(cudaMemcpyAsync(dev, ctx->stage, bytes, cudaMemcpyHostToDevice, st));
  TDE_CK(cudaEventRecord(ctx->stage_ev, st));
  ctx->stage_busy = true;
  return TDE_OK;
}

// Adds the kernel launches enqueued during its lifetime to the context.
struct LaunchCount {
  tde_ctx* ctx;
  int64_t before;
  explicit LaunchCount(tde_ctx* c) : ctx(c), before(tde_launch_counter) {}
  ~LaunchCount() { ctx->launches += tde_launch_counter - before; }
};

// Brackets one engine-kernel launch with the context's events when profiling.
struct EngineTimer {
  tde_ctx* ctx;
  cudaStream_t st;
  cudaEvent_t end = nullptr;
  EngineTimer(tde_ctx* c, cudaStream_t s) : ctx(c), st(s) {
    if (!ctx->profile) return;
    while (ctx->ev.size() < ctx->ev_used + 2) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;
      ctx->ev.push_back(e);
    }
    cudaEventRecord(ctx->ev[ctx->ev_used], st);
    end = ctx->ev[ctx->ev_used + 1];
    ctx->ev_used += 2;
  }
  ~EngineTimer() {
    if (!end) return;
    cudaEventRecord(end, st);
    ctx->engine_launches += 1;
  }
};

bool valid_bits(int bits) { return bits == 1 || bits == 2 || bits == 4; }
int planes_for(int bits) { return bits == 4 ? 4 : 2; }

tde_status check_xcorr_args(tde_ctx* ctx, int64_t nx, int64_t ny, int bits, int64_t lag_min,
                            int64_t lag_max, int engine, int out_dtype) {
  if (!valid_bits(bits)) return set_err(ctx, TDE_ERR_INVALID, "bits must be 1, 2 or 4 (got %d)", bits);
  if (nx <= 0 || ny <= 0) return set_err(ctx, TDE_ERR_INVALID, "signal lengths must be positive");
  if (nx > INT32_MAX || ny > INT32_MAX)
    return set_err(ctx, TDE_ERR_UNSUPPORTED, "signal lengths above 2^31-1 are not supported");
  if (lag_min > lag_max) return set_err(ctx, TDE_ERR_INVALID, "lag_min > lag_max");
  if (lag_min < -(nx - 1) || lag_max > ny - 1)
    return set_err(ctx, TDE_ERR_INVALID,
                   "lag range [%lld, %lld] outside the overlap range [%lld, %lld]",
                   (long long)lag_min, (long long)lag_max, (long long)-(nx - 1),
                   (long long)(ny - 1));
  if (engine < TDE_ENGINE_AUTO || engine > TDE_ENGINE_NTT)
    return set_err(ctx, TDE_ERR_INVALID, "unknown engine %d", engine);
  if (out_dtype != TDE_I32 && out_dtype != TDE_I64)
    return set_err(ctx, TDE_ERR_INVALID, "unknown output dtype %d", out_dtype);
  if (out_dtype == TDE_I32) {
    // The bound N * (2^(bits-1))^2 < 2^31, asserted as stated.
    const int64_t k = (int64_t)1 << (bits - 1);
    const int64_t n = nx < ny ? nx : ny;
    if (n * k * k >= ((int64_t)1 << 31))
      return set_err(ctx, TDE_ERR_OVERFLOW,
                     "int32 output may overflow: min(nx,ny)*(2^(bits-1))^2 = %lld >= 2^31; "
                     "request TDE_I64", (long long)(n * k * k));
  }
  return TDE_OK;
}

}  // namespace

// ===================================================================== ABI

extern "C" tde_status tde_ctx_create(int device, tde_ctx** out) {
  if (!out) return TDE_ERR_INVALID;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev)
    return TDE_ERR_CUDA;
  tde_ctx* ctx = new tde_ctx();
  ctx->device = device;
  DeviceGuard g(device);
  if (cudaDeviceGetAttribute(&ctx->sm_count, cudaDevAttrMultiProcessorCount, device) != cudaSuccess ||
      cudaMalloc(&ctx->d_status, sizeof(uint32_t)) != cudaSuccess ||
      cudaMemset(ctx->d_status, 0, sizeof(uint32_t)) != cudaSuccess ||
      cudaEventCreateWithFlags(&ctx->stage_ev, cudaEventDisableTiming) != cudaSuccess) {
    tde_ctx_destroy(ctx);
    return TDE_ERR_CUDA;
  }
  *out = ctx;
  return TDE_OK;
}

extern "C" tde_status tde_ctx_destroy(tde_ctx* ctx) {
  if (!ctx) return TDE_OK;
  {
    DeviceGuard g(ctx->device);
    cudaDeviceSynchronize();
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->stage) cudaFreeHost(ctx->stage);
    if (ctx->stage_ev) cudaEventDestroy(ctx->stage_ev);
    for (cudaEvent_t e : ctx->ev) cudaEventDestroy(e);
    fft_plan_destroy(&ctx->fft);
    for (uint32_t* t : ctx->ntt_tables)
      if (t) cudaFree(t);
  }
  delete ctx;
  return TDE_OK;
}

extern "C" const char* tde_last_error(const tde_ctx* ctx) {
  return ctx ? ctx->err.c_str() : "null context";
}

extern "C" tde_status tde_ctx_sync(tde_ctx* ctx, tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  if (!ctx) return TDE_ERR_INVALID;
  DeviceGuard g(ctx->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  TDE_CK(cudaStreamSynchronize(st));
  uint32_t s = 0;
  TDE_CK(cudaMemcpy(&s, ctx->d_status, sizeof s, cudaMemcpyDeviceToHost));
  TDE_CK(cudaMemset(ctx->d_status, 0, sizeof s));
  if (s & TDE_ST_NONFINITE) return set_err(ctx, TDE_ERR_INVALID, "NaN or Inf in a quantizer input");
  if (s & TDE_ST_INTERNAL)
    return set_err(ctx, TDE_ERR_INVALID, "a quantized level is outside the range of `bits`");
  if (s & TDE_ST_TIMEOUT) return set_err(ctx, TDE_ERR_TIMEOUT, "a bounded device wait gave up");
  return TDE_OK;
}


extern "C" tde_status tde_ctx_set_profiling(tde_ctx* ctx, int enable) {
  if (!ctx) return TDE_ERR_INVALID;
  ctx->profile = enable != 0;
  return TDE_OK;
}

extern "C" tde_status tde_selftest_wait_timeout(tde_ctx* ctx, tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  if (!ctx) return TDE_ERR_INVALID;
  DeviceGuard g(ctx->device);
  LaunchCount lc(ctx);
  const cudaError_t e = launch_wait_selftest(ctx->d_status, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? TDE_OK : cuda_err(ctx, e, "wait self-test");
}

extern "C" tde_status tde_ctx_set_ntt_primes(tde_ctx* ctx, int nprimes) {
  if (!ctx) return TDE_ERR_INVALID;
  if (nprimes != 0 && nprimes != 2)
    return set_err(ctx, TDE_ERR_INVALID, "nprimes must be 0 (automatic) or 2, got %d", nprimes);
  ctx->ntt_two_primes = nprimes == 2;
  return TDE_OK;
}

extern "C" tde_status tde_ctx_read_profile(tde_ctx* ctx, int64_t* kernel_launches,
                                           int64_t* engine_launches, double* engine_ms) {
  if (!ctx) return TDE_ERR_INVALID;
  DeviceGuard g(ctx->device);
  double ms = 0.0;
  for (size_t i = 0; i + 1 < ctx->ev_used; i += 2) {
    TDE_CK(cudaEventSynchronize(ctx->ev[i + 1]));
    float t = 0.f;
    TDE_CK(cudaEventElapsedTime(&t, ctx->ev[i], ctx->ev[i + 1]));
    ms += t;
  }
  if (kernel_launches) *kernel_launches = ctx->launches;
  if (engine_launches) *engine_launches = ctx->engine_launches;
  if (engine_ms) *engine_ms = ms;
  ctx->launches = ctx->engine_launches = 0;
  ctx->ev_used = 0;
  return TDE_OK;
}

namespace {

// Offsets of one API call's regions: a descriptor block (uploaded in one copy
// from the pinned staging buffer) followed by a data block, both inside the
// context workspace.
struct Layout {
  size_t desc = 0, data = 0;
  template <typename T>
  size_t d(size_t n) {
    desc = align_up(desc, 16);
    size_t o = desc;
    desc += n * sizeof(T);
    return o;
  }
  template <typename T>
  size_t w(size_t n) {
    data = align_up(data, 256);
    size_t o = data;
    data += n * sizeof(T);
    return o;
  }
  size_t data_base() const { return align_up(desc, 256); }
  size_t total() const { return data_base() + data; }
};

// Resolved base pointers once the workspace and the staging exist.
struct Bases {
  char* hdesc;  // pinned host copy of the descriptor block
  char* ddesc;  // device descriptor block
  char* ddata;  // device data block
  template <typename T>
  T* hd(size_t o) const { return reinterpret_cast<T*>(hdesc + o); }
  template <typename T>
  T* dd(size_t o) const { return reinterpret_cast<T*>(ddesc + o); }
  template <typename T>
  T* dw(size_t o) const { return reinterpret_cast<T*>(ddata + o); }
};

// ---- step A: quantize a list of signals
struct QuantStage {
  int nsig = 0, bits = 1;
  int64_t max_n = 0;
  bool with_planes = false;
  size_t o_sigs = 0, o_hist = 0, o_chist = 0, o_state = 0, o_candp = 0, o_planes = 0;
  std::vector<size_t> o_cand;  // per signal: room for all its keys, then their indices (+ slack)
  // ns: the signals' lengths (host), or nullptr when all are max_n.  With
  // want_planes the rank quantizer also writes bit planes (set_planes);
  // callers check planes_written() and pack themselves otherwise.
  void plan(Layout& L, int n, int b, const int64_t* ns, int64_t mx, bool want_planes = false) {
    nsig = n, bits = b, max_n = mx;
    with_planes = bits != 1 && want_planes;
    o_sigs = L.d<QSig>(nsig);
    if (bits == 1) return;
    if (with_planes) o_planes = L.d<QPlanes>(nsig);
    o_candp = L.d<uint32_t*>(nsig);
    o_hist = L.w<uint32_t>((size_t)nsig * 4096);
    o_chist = L.w<uint32_t>((size_t)nsig * 7 * 1024);
    o_state = L.w<QState>(nsig);
    o_cand.resize(nsig);
    for (int i = 0; i < nsig; ++i) o_cand[i] = L.w<uint32_t>(2 * ((size_t)(ns ? ns[i] : mx) + kQCandSlack));
  }
  bool planes_written() const { return with_planes; }
  void fill(const Bases& B, const float* const* xs, int8_t* const* qs, const int64_t* ns) const {
    QSig* h = B.hd<QSig>(o_sigs);
    for (int i = 0; i < nsig; ++i) h[i] = QSig{xs[i], qs[i], ns[i]};
    if (bits == 1) return;
    uint32_t** cp = B.hd<uint32_t*>(o_candp);
    for (int i = 0; i < nsig; ++i) cp[i] = B.dw<uint32_t>(o_cand[i]);
  }
  void set_planes(const Bases& B, int i, uint32_t* planes, int64_t words) const {
    if (with_planes) B.hd<QPlanes>(o_planes)[i] = QPlanes{planes, words};
  }
  cudaError_t launch(const Bases& B, uint32_t* status, cudaStream_t st) const {
    if (nsig == 0) return cudaSuccess;
    if (bits == 1) return launch_quantize_sign(B.dd<QSig>(o_sigs), nsig, max_n, status, st);
    const QWork w{B.dw<uint32_t>(o_hist), B.dw<QState>(o_state), B.dd<uint32_t*>(o_candp),
                  B.dw<uint32_t>(o_chist)};
    return launch_quantize_stream(B.dd<QSig>(o_sigs), with_planes ? B.dd<QPlanes>(o_planes) : nullptr,
                                  nsig, max_n, bits, w, status, st);
  }
};

// One correlation job on quantized inputs already in device memory.
struct Job {
  const int8_t* qx;
  const int8_t* qy;
  int64_t nx, ny, lag_min, lag_max;
  void* c;
  int c64;
};

// ---- step B, popc engine
struct PopcStage {
  int njobs = 0, bits = 1, nitems = 0;
  int64_t max_words = 0;
  size_t o_psig = 0, o_pairs = 0, o_items = 0;
  std::vector<size_t> o_planes;  // per signal (2 per job)
  std::vector<int64_t> words;
  void plan(Layout& L, const std::vector<Job>& jobs, int b) {
    njobs = (int)jobs.size(), bits = b;
    const int pl = planes_for(bits);
    o_psig = L.d<PlaneSig>(2 * njobs);
    o_pairs = L.d<XcPair>(njobs);
    nitems = 0;
    for (const Job& j : jobs) {
      int64_t a_lo = floor_div64(j.lag_min, 32), a_hi = floor_div64(j.lag_max, 32);
      nitems += (int)ceil_div64(a_hi - a_lo + 1, kPopcLagsPerCta / 32);
    }
    o_items = L.d<PopcItem>(nitems);
    o_planes.resize(2 * njobs);
    words.resize(2 * njobs);
    max_words = 0;
    for (int i = 0; i < njobs; ++i)
      for (int s = 0; s < 2; ++s) {
        int64_t n = s ? jobs[i].ny : jobs[i].nx;
        words[2 * i + s] = ceil_div64(n, 32);
        max_words = words[2 * i + s] > max_words ? words[2 * i + s] : max_words;
        o_planes[2 * i + s] = L.w<uint32_t>((size_t)pl * words[2 * i + s]);
      }
  }
  void fill(const Bases& B, const std::vector<Job>& jobs) const {
    PlaneSig* ps = B.hd<PlaneSig>(o_psig);
    XcPair* xp = B.hd<XcPair>(o_pairs);
    PopcItem* it = B.hd<PopcItem>(o_items);
    int k = 0;
    for (int i = 0; i < njobs; ++i) {
      const Job& j = jobs[i];
      uint32_t* px = B.dw<uint32_t>(o_planes[2 * i]);
      uint32_t* py = B.dw<uint32_t>(o_planes[2 * i + 1]);
      ps[2 * i] = PlaneSig{j.qx, px, j.nx, words[2 * i]};
      ps[2 * i + 1] = PlaneSig{j.qy, py, j.ny, words[2 * i + 1]};
      xp[i] = XcPair{px, py, words[2 * i], words[2 * i + 1], j.lag_min, j.lag_max, j.c, j.c64};
      int64_t a_lo = floor_div64(j.lag_min, 32), a_hi = floor_div64(j.lag_max, 32);
      for (int64_t a = a_lo; a <= a_hi; a += kPopcLagsPerCta / 32) it[k++] = PopcItem{i, 0, a};
    }
  }
  // The planes of job i's signal `side` (0: x, 1: y).
  uint32_t* planes_of(const Bases& B, int i, int side) const {
    return B.dw<uint32_t>(o_planes[2 * i + side]);
  }
  bool prepacked = false;  // the quantizer already wrote every job's planes
  cudaError_t launch(tde_ctx* ctx, const Bases& B, cudaStream_t st) const {
    if (njobs == 0) return cudaSuccess;
    cudaError_t e = prepacked ? cudaSuccess
                              : launch_pack_planes(B.dd<PlaneSig>(o_psig), 2 * njobs, max_words,
                                                   bits, ctx->d_status, st);
    if (e != cudaSuccess) return e;
    EngineTimer t(ctx, st);
    return launch_xcorr_popc(B.dd<XcPair>(o_pairs), B.dd<PopcItem>(o_items), nitems, bits, st);
  }
};

// ---- step B, tensor-core engine
struct MmaStage {
  int njobs = 0, nitems = 0, any_zero = 0;
  int64_t max_count = 0;
  size_t o_pairs = 0, o_items = 0, o_counter = 0;
  std::vector<MmaItem> items;
  std::vector<int> zero_first;
  // split_small: a plan with few items (fewer than half the SMs) cuts its K
  // ranges into shorter segments (>= kMinSeg samples) so that its items spread
  // over the SMs; the partial sums are added with integer atomics as usual.
  static constexpr int64_t kMinSeg = 2 * kMmaChunk;
  // fp4: levels in {-1, 0, 1} run on the packed E2M1 kernel, whose tiles are
  // 128 columns (16384 lags) wide; otherwise E4M3 tiles of 256 columns.
  bool fp4 = false;
  void plan(Layout& L, const std::vector<Job>& jobs, bool split_small = true, bool use_fp4 = false) {
    njobs = (int)jobs.size();
    fp4 = use_fp4;
    const int64_t tile = fp4 ? kMmaTileLags4 : kMmaTileLags, cols = tile / 128;
    const int64_t ks_cap = fp4 ? kMmaKs4 : kMmaKs;
    items.clear();
    zero_first.assign(njobs, 0);
    struct Tile {
      int job;
      int64_t T0, klo, khi;
    };
    std::vector<Tile> tiles;
    int64_t n_default = 0;  // items at the default segment length
    for (int i = 0; i < njobs; ++i) {
      const Job& j = jobs[i];
      max_count = std::max<int64_t>(max_count, j.lag_max - j.lag_min + 1);
      const int64_t t0 = floor_div64(j.lag_min, kMmaChunk) * kMmaChunk;
      const int64_t ntiles = ceil_div64(j.lag_max - t0 + 1, tile);
      for (int64_t t = 0; t < ntiles; ++t) {
        const int64_t T0 = t0 + t * tile;
        // k = x index + (127 - m); nonzero terms need k in [0, nx + 127) and
        // y index k + T0 + 128 n in [0, ny) for some n in [0, cols).
        int64_t klo = std::max<int64_t>(0, -T0 - 128 * (cols - 1));
        int64_t khi = std::min<int64_t>(j.nx + 127, j.ny - T0);
        klo = floor_div64(klo, kMmaChunk) * kMmaChunk;
        khi = ceil_div64(khi, kMmaChunk) * kMmaChunk;
        if (khi <= klo) {  // no overlap anywhere in this tile: its lags are 0
          zero_first[i] = 1;
          continue;
        }
        tiles.push_back(Tile{i, T0, klo, khi});
        n_default += ceil_div64(khi - klo, ks_cap);
      }
    }
    int64_t seg_cap = ks_cap;
    if (split_small && !tiles.empty()) {
      int dev = 0, sms = 0;
      cudaGetDevice(&dev);
      if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess &&
          n_default < sms / 2) {
        int64_t total = 0;
        for (const Tile& t : tiles) total += t.khi - t.klo;
        const int64_t want = ceil_div64(ceil_div64(total, sms), kMmaChunk) * kMmaChunk;
        seg_cap = std::min<int64_t>(ks_cap, std::max<int64_t>(kMinSeg, want));
      }
    }
    for (const Tile& t : tiles) {
      const int64_t nseg = ceil_div64(t.khi - t.klo, seg_cap);
      const int64_t seg = ceil_div64(ceil_div64(t.khi - t.klo, nseg), kMmaChunk) * kMmaChunk;
      if (nseg > 1) zero_first[t.job] = 1;
      for (int64_t s = 0; s < nseg; ++s) {
        const int64_t ks = t.klo + s * seg, ke = std::min(t.khi, ks + seg);
        if (ke > ks) items.push_back(MmaItem{t.job, nseg == 1 ? 1 : 0, t.T0, ks, ke});
      }
    }
    for (int i = 0; i < njobs; ++i) any_zero |= zero_first[i];
    // Longest first: the persistent CTAs then finish close together.
    std::stable_sort(items.begin(), items.end(), [](const MmaItem& a, const MmaItem& b) {
      return a.ke - a.ks > b.ke - b.ks;
    });
    nitems = (int)items.size();
    o_pairs = L.d<MmaPair>(njobs);
    o_items = L.d<MmaItem>(nitems);
    o_counter = L.w<int>(1);
  }
  void fill(const Bases& B, const std::vector<Job>& jobs) const {
    MmaPair* p = B.hd<MmaPair>(o_pairs);
    for (int i = 0; i < njobs; ++i) {
      const Job& j = jobs[i];
      p[i] = MmaPair{j.qx, j.qy, j.nx, j.ny, j.lag_min, j.lag_max, j.c, j.c64, zero_first[i]};
    }
    if (nitems) memcpy(B.hd<MmaItem>(o_items), items.data(), sizeof(MmaItem) * nitems);
  }
  cudaError_t launch(tde_ctx* ctx, const Bases& B, cudaStream_t st) const {
    if (njobs == 0) return cudaSuccess;
    if (any_zero) {
      cudaError_t e = launch_mma_zero(B.dd<MmaPair>(o_pairs), njobs, max_count, st);
      if (e != cudaSuccess) return e;
    }
    EngineTimer t(ctx, st);
    return (fp4 ? launch_xcorr_mma4 : launch_xcorr_mma)(B.dd<MmaPair>(o_pairs), B.dd<MmaItem>(o_items), nitems,
                                                        B.dw<int>(o_counter), 2 * ctx->sm_count, ctx->d_status, st,
                                                        nullptr);
  }
};

// ---- step B, number-theoretic-transform engine
// Template = the shorter signal; the other is cut into overlap-save blocks.
struct NttPlanPair {
  int logn = 0;
  int sign = 1;
  const int8_t* t = nullptr;
  const int8_t* a = nullptr;
  int64_t nt = 0, na = 0;
  std::vector<std::pair<int64_t, int64_t>> blocks;  // (start, valid)
};

// Valid outputs of an overlap-save block of length N starting at S: R[S + j']
// for j' < V.  Outputs j' <= N - nt never wrap.  Beyond that the circular sum
// drops a[S + j' + j] and adds a[S + j' + j - N] for j >= N - j'; both are
// zero when the block reaches past the end of a (S + N >= na) and the wrapped
// indices stay below 0 (j' < N - nt + 1 - S).
int64_t ntt_valid(int64_t N, int64_t nt, int64_t na, int64_t S) {
  if (S < 0 && S + N >= na) return std::min<int64_t>(N, N - nt + 1 - S);
  return N - nt + 1;
}

// Overlap-save blocks of length N = 2^logn covering k in [k0, k1].
std::vector<std::pair<int64_t, int64_t>> ntt_blocks(int logn, int64_t nt, int64_t na, int64_t k0,
                                                    int64_t k1) {
  std::vector<std::pair<int64_t, int64_t>> out;
  const int64_t N = (int64_t)1 << logn;
  for (int64_t S = k0; S <= k1;) {
    const int64_t V = ntt_valid(N, nt, na, S);
    out.emplace_back(S, V);
    S += V;
  }
  return out;
}

// False if no length up to 2^kNttMaxLog holds the template with at least
// N/8 outputs per overlap-save block.
bool ntt_plan_pair(const Job& j, NttPlanPair* pp) {
  const bool tx = j.nx <= j.ny;  // template = x: R[k] = c[k]; else c[-k]
  pp->t = tx ? j.qx : j.qy;
  pp->a = tx ? j.qy : j.qx;
  pp->nt = tx ? j.nx : j.ny;
  pp->na = tx ? j.ny : j.nx;
  pp->sign = tx ? 1 : -1;
  const int64_t k0 = tx ? j.lag_min : -j.lag_max, k1 = tx ? j.lag_max : -j.lag_min;
  double best = -1.0;
  for (int logn = kNttMinLog; logn <= kNttMaxLog; ++logn) {
    const int64_t N = (int64_t)1 << logn;
    // a block must keep at least N/8 outputs (else the plan is mostly waste)
    if (N - pp->nt + 1 < N / 8) continue;
    // count blocks without building the list
    int64_t nb = 0;
    for (int64_t S = k0; S <= k1 && nb < (1 << 22);) {
      S += ntt_valid(N, pp->nt, pp->na, S);
      ++nb;
    }
    const double cost = (double)(nb + 1) * (double)N * logn;
    if (best < 0 || cost < best) {
      best = cost;
      pp->logn = logn;
    }
  }
  if (best < 0) return false;
  pp->blocks = ntt_blocks(pp->logn, pp->nt, pp->na, k0, k1);
  return true;
}

tde_status ntt_tables(tde_ctx* ctx, int logn, NttTables* T) {
  if (!ctx->ntt_tables[logn]) {
    const size_t N = (size_t)1 << logn;
    std::vector<uint32_t> h(8 * N);
    ntt_host_tables(logn, h.data());
    uint32_t* d = nullptr;
    TDE_CK(cudaMalloc(&d, 8 * N * sizeof(uint32_t)));
    TDE_CK(cudaMemcpy(d, h.data(), 8 * N * sizeof(uint32_t), cudaMemcpyHostToDevice));
    ctx->ntt_tables[logn] = d;
  }
  const size_t N = (size_t)1 << logn;
  const uint32_t* d = ctx->ntt_tables[logn];
  for (int q = 0; q < 2; ++q) {
    T->tw[q] = d + (0 + q) * N;
    T->tws[q] = d + (2 + q) * N;
    T->itw[q] = d + (4 + q) * N;
    T->itws[q] = d + (6 + q) * N;
  }
  return TDE_OK;
}

struct NttStage {
  int njobs = 0;
  bool ok = true;
  std::vector<NttPlanPair> pp;
  size_t o_pairs = 0;
  // per (log2 length, primes): template jobs, block jobs and their buffers
  struct Group {
    int logn, nprimes;
    std::vector<int> pairs;
    size_t o_tjobs = 0, o_bjobs = 0;
    int ntemplates = 0, nblocks = 0;
    std::vector<size_t> o_tbuf, o_bbuf;
  };
  std::vector<Group> groups;
  // bits: the levels' width (largest magnitude 1, 1, 7 for b = 1, 2, 4);
  // two_primes: CRT even where one prime suffices.
  void plan(Layout& L, const std::vector<Job>& jobs, int bits, bool two_primes) {
    njobs = (int)jobs.size();
    pp.assign(njobs, NttPlanPair{});
    groups.clear();
    const int64_t kmax = bits == 4 ? 7 : 1;
    for (int i = 0; i < njobs; ++i) {
      if (!ntt_plan_pair(jobs[i], &pp[i])) {
        ok = false;
        return;
      }
      const int nq = (!two_primes && ntt_one_prime_ok(pp[i].nt, kmax)) ? 1 : 2;
      Group* g = nullptr;
      for (Group& x : groups)
        if (x.logn == pp[i].logn && x.nprimes == nq) g = &x;
      if (!g) {
        groups.push_back(Group{});
        g = &groups.back();
        g->logn = pp[i].logn;
        g->nprimes = nq;
      }
      g->pairs.push_back(i);
    }
    o_pairs = L.d<NttPairOut>(njobs);
    for (Group& g : groups) {
      const size_t words = (size_t)g.nprimes << g.logn;
      g.ntemplates = (int)g.pairs.size();
      g.nblocks = 0;
      for (int i : g.pairs) g.nblocks += (int)pp[i].blocks.size();
      g.o_tjobs = L.d<NttJob>(g.ntemplates);
      g.o_bjobs = L.d<NttJob>(g.nblocks);
      g.o_tbuf.clear(), g.o_bbuf.clear();
      for (int t = 0; t < g.ntemplates; ++t) g.o_tbuf.push_back(L.w<uint32_t>(words));
      for (int b = 0; b < g.nblocks; ++b) g.o_bbuf.push_back(L.w<uint32_t>(words));
    }
  }
  void fill(const Bases& B, const std::vector<Job>& jobs) {
    NttPairOut* po = B.hd<NttPairOut>(o_pairs);
    for (Group& g : groups) {
      NttJob* tj = B.hd<NttJob>(g.o_tjobs);
      NttJob* bj = B.hd<NttJob>(g.o_bjobs);
      int b = 0;
      for (int t = 0; t < g.ntemplates; ++t) {
        const int i = g.pairs[t];
        NttPlanPair& P = pp[i];
        // the pointers of a Job are bound only now
        const bool tx = jobs[i].nx <= jobs[i].ny;
        P.t = tx ? jobs[i].qx : jobs[i].qy;
        P.a = tx ? jobs[i].qy : jobs[i].qx;
        uint32_t* spec = B.dw<uint32_t>(g.o_tbuf[t]);
        tj[t] = NttJob{P.t, P.nt, 0, 0, spec, i, 1};
        po[i] = NttPairOut{spec, jobs[i].c, jobs[i].lag_min, jobs[i].lag_max, jobs[i].c64, P.sign};
        for (auto& blk : P.blocks) {
          bj[b] = NttJob{P.a, P.na, blk.first, blk.second, B.dw<uint32_t>(g.o_bbuf[b]), i, 0};
          ++b;
        }
      }
    }
  }
  cudaError_t launch(tde_ctx* ctx, const Bases& B, cudaStream_t st) const {
    for (const Group& g : groups) {
      NttTables T;
      if (ntt_tables(ctx, g.logn, &T) != TDE_OK) return cudaErrorMemoryAllocation;
      cudaError_t e = launch_ntt_templates(B.dd<NttJob>(g.o_tjobs), g.ntemplates, g.logn,
                                           g.nprimes, T, st);
      if (e != cudaSuccess) return e;
      EngineTimer t(ctx, st);
      e = launch_ntt_blocks(B.dd<NttJob>(g.o_bjobs), g.nblocks, B.dd<NttPairOut>(o_pairs), g.logn,
                            g.nprimes, T, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
};

// Both engines over one job list: each job goes to the engine picked for it.
struct XcorrStage {
  std::vector<int> eng;                 // per job
  std::vector<Job> popc_jobs, mma_jobs, ntt_jobs;
  PopcStage popc;
  MmaStage mma;
  NttStage ntt;
  int bits = 1;
  std::vector<Job>& list(int e) {
    return e == TDE_ENGINE_MMA ? mma_jobs : (e == TDE_ENGINE_NTT ? ntt_jobs : popc_jobs);
  }
  // False if some job cannot be served by its engine.  ntt_two_primes: the
  // NTT engine recombines two primes even where one suffices.
  bool plan(Layout& L, const std::vector<Job>& jobs, const std::vector<int>& engines, int b,
            bool ntt_two_primes) {
    bits = b;
    eng = engines;
    popc_jobs.clear(), mma_jobs.clear(), ntt_jobs.clear();
    for (size_t i = 0; i < jobs.size(); ++i) list(eng[i]).push_back(jobs[i]);
    popc.plan(L, popc_jobs, bits);
    mma.plan(L, mma_jobs, true, bits <= 2);
    ntt.plan(L, ntt_jobs, bits, ntt_two_primes);
    return ntt.ok;
  }
  // Binds pointers (known after realize) and writes the descriptors.
  void fill(const Bases& B, const std::vector<Job>& jobs) {
    size_t a = 0, m = 0, t = 0;
    for (size_t i = 0; i < jobs.size(); ++i) {
      if (eng[i] == TDE_ENGINE_MMA)
        mma_jobs[m++] = jobs[i];
      else if (eng[i] == TDE_ENGINE_NTT)
        ntt_jobs[t++] = jobs[i];
      else
        popc_jobs[a++] = jobs[i];
    }
    popc.fill(B, popc_jobs);
    mma.fill(B, mma_jobs);
    ntt.fill(B, ntt_jobs);
  }
  cudaError_t launch(tde_ctx* ctx, const Bases& B, cudaStream_t st) const {
    cudaError_t e = cudaSuccess;
    if (!popc_jobs.empty()) e = popc.launch(ctx, B, st);
    if (e == cudaSuccess && !mma_jobs.empty()) e = mma.launch(ctx, B, st);
    if (e == cudaSuccess && !ntt_jobs.empty()) e = ntt.launch(ctx, B, st);
    return e;
  }
};

// ---- step C
struct ArgStage {
  int n = 0, c64 = 0;
  int64_t max_count = 0;
  size_t o_pairs = 0, o_keys = 0;
  void plan(Layout& L, int npairs, int64_t maxc, int is64) {
    n = npairs, max_count = maxc, c64 = is64;
    o_pairs = L.d<ArgPair>(n);
    o_keys = L.w<unsigned long long>(2 * (size_t)n);
  }
  void set(const Bases& B, int i, const void* c, int64_t lag_min, int64_t count, int64_t* lag_out,
           int64_t* val_out) const {
    B.hd<ArgPair>(o_pairs)[i] = ArgPair{c, lag_min, count, lag_out, val_out};
  }
  cudaError_t launch(const Bases& B, cudaStream_t st) const {
    return launch_argmax(B.dd<ArgPair>(o_pairs), n, max_count, c64,
                         B.dw<unsigned long long>(o_keys), st);
  }
};

// Allocates the workspace and the staging for a planned call.
tde_status realize(tde_ctx* ctx, const Layout& L, Bases* B) {
  tde_status s = ensure_ws(ctx, L.total());
  if (s != TDE_OK) return s;
  char* host = nullptr;
  s = stage_begin(ctx, L.desc ? L.desc : 16, &host);
  if (s != TDE_OK) return s;
  B->hdesc = host;
  B->ddesc = ctx->ws;
  B->ddata = ctx->ws + L.data_base();
  return TDE_OK;
}

// AUTO: the tensor-core engine pays for a whole 32768-lag tile; it runs about
// 16x (bits <= 2) or 150x (bits = 4) more MACs per clock than the POPC pipe,
// so it wins once a pair asks for more lags than ~1/16 (1/128) of a tile.
int pick_engine(int engine, int bits, int64_t nx, int64_t ny, int64_t lag_count) {
  if (engine != TDE_ENGINE_AUTO) return engine;
  const int64_t n = nx < ny ? nx : ny;
  const int64_t need = bits == 4 ? kMmaTileLags / 128 : kMmaTileLags / 16;
  return (n >= 1024 && lag_count >= need) ? TDE_ENGINE_MMA : TDE_ENGINE_POPC;
}

int ilog2_round(int64_t v) {
  int l = 0;
  while (((int64_t)1 << (l + 1)) <= v) ++l;
  // round to the nearer power of two
  if (l < 62 && v - ((int64_t)1 << l) > ((int64_t)1 << (l + 1)) - v) ++l;
  return l;
}

// AUTO with the context's autotuner table when it has entries for `bits`.
int pick_engine_ctx(const tde_ctx* ctx, int engine, int bits, int64_t nx, int64_t ny,
                    int64_t lag_count) {
  if (engine != TDE_ENGINE_AUTO || ctx->tune.empty()) return pick_engine(engine, bits, nx, ny, lag_count);
  const int ln = ilog2_round(nx < ny ? nx : ny), ll = ilog2_round(lag_count);
  int best = -1, bd = 1 << 30;
  for (const tde_tune_entry& t : ctx->tune) {
    if (t.bits != bits) continue;
    const int d = std::abs(t.log2_n - ln) + std::abs(t.log2_lags - ll);
    if (d < bd) bd = d, best = t.engine;
  }
  return best >= 0 ? best : pick_engine(engine, bits, nx, ny, lag_count);
}

tde_status engine_available(tde_ctx* ctx, int engine) {
  if (engine == TDE_ENGINE_POPC || engine == TDE_ENGINE_MMA || engine == TDE_ENGINE_NTT)
    return TDE_OK;
  return set_err(ctx, TDE_ERR_UNSUPPORTED, "engine %d is not available in this library", engine);
}

}  // namespace

extern "C" int tde_pick_engine(int bits, int64_t nx, int64_t ny, int64_t lag_count) {
  if (!valid_bits(bits) || nx <= 0 || ny <= 0 || lag_count <= 0) return -1;
  return pick_engine(TDE_ENGINE_AUTO, bits, nx, ny, lag_count);
}

extern "C" tde_status tde_quantize(tde_ctx* ctx, const float* x, int64_t n, int bits,
                                   int8_t* q_out, tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  if (!ctx) return TDE_ERR_INVALID;
  if (!x || !q_out) return set_err(ctx, TDE_ERR_INVALID, "null pointer");
  if (n <= 0) return set_err(ctx, TDE_ERR_INVALID, "n must be positive");
  if (n > INT32_MAX) return set_err(ctx, TDE_ERR_UNSUPPORTED, "n above 2^31-1 is not supported");
  if (!valid_bits(bits)) return set_err(ctx, TDE_ERR_INVALID, "bits must be 1, 2 or 4");
  DeviceGuard g(ctx->device);
  LaunchCount lc(ctx);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Layout L;
  QuantStage Q;
  Q.plan(L, 1, bits, nullptr, n);
  Bases B;
  tde_status s = realize(ctx, L, &B);
  if (s != TDE_OK) return s;
  Q.fill(B, &x, &q_out, &n);
  if ((s = stage_upload(ctx, B.ddesc, L.desc, st)) != TDE_OK) return s;
  cudaError_t e = Q.launch(B, ctx->d_status, st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "quantize launch");
  return TDE_OK;
}

extern "C" tde_status tde_quantize_batch(tde_ctx* ctx, const float* x, int64_t n, int nsig,
                                         int bits, int8_t* q_out, tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  if (!ctx) return TDE_ERR_INVALID;
  if (!x || !q_out) return set_err(ctx, TDE_ERR_INVALID, "null pointer");
  if (n <= 0 || nsig <= 0) return set_err(ctx, TDE_ERR_INVALID, "n and nsig must be positive");
  if (n > INT32_MAX) return set_err(ctx, TDE_ERR_UNSUPPORTED, "n above 2^31-1 is not supported");
  if (!valid_bits(bits)) return set_err(ctx, TDE_ERR_INVALID, "bits must be 1, 2 or 4");
  DeviceGuard g(ctx->device);
  LaunchCount lc(ctx);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Layout L;
  QuantStage Q;
  Q.plan(L, nsig, bits, nullptr, n);
  Bases B;
  tde_status s = realize(ctx, L, &B);
  if (s != TDE_OK) return s;
  std::vector<const float*> xs(nsig);
  std::vector<int8_t*> qs(nsig);
  std::vector<int64_t> ns(nsig, n);
  for (int i = 0; i < nsig; ++i) xs[i] = x + (int64_t)i * n, qs[i] = q_out + (int64_t)i * n;
  Q.fill(B, xs.data(), qs.data(), ns.data());
  if ((s = stage_upload(ctx, B.ddesc, L.desc, st)) != TDE_OK) return s;
  const cudaError_t e = Q.launch(B, ctx->d_status, st);
  return e == cudaSuccess ? TDE_OK : cuda_err(ctx, e, "quantize launch");
}

extern "C" tde_status tde_xcorr_int(tde_ctx* ctx, const int8_t* qx, int64_t nx, const int8_t* qy,
                                    int64_t ny, int bits, int64_t lag_min, int64_t lag_max,
                                    int engine, void* c_out, int out_dtype, tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  if (!ctx) return TDE_ERR_INVALID;
  if (!qx || !qy || !c_out) return set_err(ctx, TDE_ERR_INVALID, "null pointer");
  tde_status s = check_xcorr_args(ctx, nx, ny, bits, lag_min, lag_max, engine, out_dtype);
  if (s != TDE_OK) return s;
  const int eng = pick_engine_ctx(ctx, engine, bits, nx, ny, lag_max - lag_min + 1);
  if ((s = engine_available(ctx, eng)) != TDE_OK) return s;
  DeviceGuard g(ctx->device);
  LaunchCount lc(ctx);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  std::vector<Job> jobs{Job{qx, qy, nx, ny, lag_min, lag_max, c_out, out_dtype == TDE_I64}};
  Layout L;
  XcorrStage E;
  if (!E.plan(L, jobs, std::vector<int>{eng}, bits, ctx->ntt_two_primes))
    return set_err(ctx, TDE_ERR_UNSUPPORTED,
                   "NTT engine: the shorter signal needs a transform above 2^%d",
                   kNttMaxLog);
  Bases B;
  if ((s = realize(ctx, L, &B)) != TDE_OK) return s;
  E.fill(B, jobs);
  if ((s = stage_upload(ctx, B.ddesc, L.desc, st)) != TDE_OK) return s;
  cudaError_t e = E.launch(ctx, B, st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "xcorr launch");
  return TDE_OK;
}

extern "C" tde_status tde_argmax(tde_ctx* ctx, const void* c, int dtype, int64_t lag_min,
                                 int64_t count, int64_t* lag_out, int64_t* val_out,
                                 tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  if (!ctx) return TDE_ERR_INVALID;
  if (!c || !lag_out || !val_out) return set_err(ctx, TDE_ERR_INVALID, "null pointer");
  if (dtype != TDE_I32 && dtype != TDE_I64) return set_err(ctx, TDE_ERR_INVALID, "unknown dtype");
  if (count <= 0) return set_err(ctx, TDE_ERR_INVALID, "count must be positive");
  const int64_t lim = INT32_MAX;
  if (lag_min < -lim || lag_min + count - 1 > lim)
    return set_err(ctx, TDE_ERR_UNSUPPORTED, "lags beyond +-(2^31-1) are not supported");
  DeviceGuard g(ctx->device);
  LaunchCount lc(ctx);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Layout L;
  ArgStage A;
  A.plan(L, 1, count, dtype == TDE_I64);
  Bases B;
  tde_status s = realize(ctx, L, &B);
  if (s != TDE_OK) return s;
  A.set(B, 0, c, lag_min, count, lag_out, val_out);
  if ((s = stage_upload(ctx, B.ddesc, L.desc, st)) != TDE_OK) return s;
  cudaError_t e = A.launch(B, st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "argmax launch");
  return TDE_OK;
}

extern "C" tde_status tde_refine(tde_ctx* ctx, const float* x, int64_t nx, const float* y, int64_t ny,
                                 const void* c, int dtype, int64_t lag_min, int64_t count,
                                 tde_refined* out, tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  if (!ctx) return TDE_ERR_INVALID;
  if (!x || !y || !c || !out) return set_err(ctx, TDE_ERR_INVALID, "null pointer");
  if (dtype != TDE_I32 && dtype != TDE_I64) return set_err(ctx, TDE_ERR_INVALID, "unknown dtype");
  if (nx <= 0 || ny <= 0 || count <= 0) return set_err(ctx, TDE_ERR_INVALID, "sizes must be positive");
  if (lag_min < -(nx - 1) || lag_min + count - 1 > ny - 1)
    return set_err(ctx, TDE_ERR_INVALID, "lags outside [-(nx-1), ny-1]");
  const int64_t lim = INT32_MAX;
  if (lag_min < -lim || lag_min + count - 1 > lim)
    return set_err(ctx, TDE_ERR_UNSUPPORTED, "lags beyond +-(2^31-1) are not supported");
  DeviceGuard g(ctx->device);
  LaunchCount lc(ctx);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Layout L;
  ArgStage A;
  A.plan(L, 1, count, dtype == TDE_I64);
  const size_t o_lv = L.w<int64_t>(2);
  const size_t o_list = L.w<int64_t>((size_t)count);
  const size_t o_r = L.w<double>((size_t)count);
  const size_t o_n = L.w<unsigned long long>(1);
  Bases B;
  tde_status s = realize(ctx, L, &B);
  if (s != TDE_OK) return s;
  int64_t* lv = B.dw<int64_t>(o_lv);  // [lag, value] of the maximum
  A.set(B, 0, c, lag_min, count, lv, lv + 1);
  if ((s = stage_upload(ctx, B.ddesc, L.desc, st)) != TDE_OK) return s;
  cudaError_t e = A.launch(B, st);
  if (e == cudaSuccess)
    e = launch_refine(x, nx, y, ny, c, dtype == TDE_I64, lag_min, count, lv + 1, B.dw<int64_t>(o_list),
                      B.dw<double>(o_r), B.dw<unsigned long long>(o_n), out, ctx->sm_count, st);
  return e == cudaSuccess ? TDE_OK : cuda_err(ctx, e, "refine launch");
}

namespace {

// Everything one batch (Algorithm 1 over many pairs) needs, planned
// from the descriptors alone; pointers are bound by fill() once memory exists.
struct BatchWork {
  int npairs = 0, bits = 1;
  Layout L;
  QuantStage Q;
  XcorrStage E;
  ArgStage A;
  std::vector<int> engs;
  std::vector<size_t> o_q;
  std::vector<int64_t> c_start;
  size_t o_call = 0;
  bool own_c = true;
  std::vector<Job> jobs;
};

tde_status batch_plan(tde_ctx* ctx, const tde_pair_desc* descs, int npairs, int bits, int engine,
                      bool have_c_out, BatchWork* w) {
  if (npairs <= 0) return set_err(ctx, TDE_ERR_INVALID, "npairs must be positive");
  tde_status s;
  w->npairs = npairs;
  w->bits = bits;
  w->engs.assign(npairs, 0);
  int64_t max_n = 0, max_count = 0;
  for (int p = 0; p < npairs; ++p) {
    const tde_pair_desc& d = descs[p];
    if (!d.x || !d.y) return set_err(ctx, TDE_ERR_INVALID, "null signal pointer in pair %d", p);
    s = check_xcorr_args(ctx, d.nx, d.ny, bits, d.lag_min, d.lag_max, engine, TDE_I32);
    if (s != TDE_OK) return s;
    const int64_t cnt = d.lag_max - d.lag_min + 1;
    w->engs[p] = pick_engine_ctx(ctx, engine, bits, d.nx, d.ny, cnt);
    if ((s = engine_available(ctx, w->engs[p])) != TDE_OK) return s;
    max_n = std::max(max_n, std::max(d.nx, d.ny));
    max_count = std::max(max_count, cnt);
  }
  // Quantized signals and (unless the caller gives c_out) correlations live
  // in the work memory.
  bool any_popc = false;
  for (int p = 0; p < npairs; ++p) any_popc |= w->engs[p] == TDE_ENGINE_POPC;
  std::vector<int64_t> lens(2 * (size_t)npairs);
  for (int p = 0; p < npairs; ++p) lens[2 * p] = descs[p].nx, lens[2 * p + 1] = descs[p].ny;
  w->Q.plan(w->L, 2 * npairs, bits, lens.data(), max_n, any_popc);
  w->o_q.assign(2 * npairs, 0);
  w->c_start.assign(npairs, 0);
  int64_t c_total = 0;
  for (int p = 0; p < npairs; ++p) {
    w->o_q[2 * p] = w->L.w<int8_t>((size_t)descs[p].nx);
    w->o_q[2 * p + 1] = w->L.w<int8_t>((size_t)descs[p].ny);
    w->c_start[p] = c_total;
    c_total += descs[p].lag_max - descs[p].lag_min + 1;
  }
  w->own_c = !have_c_out;
  w->o_call = have_c_out ? 0 : w->L.w<int32_t>((size_t)c_total);
  w->jobs.assign(npairs, Job{});
  for (int p = 0; p < npairs; ++p)
    w->jobs[p] = Job{nullptr, nullptr, descs[p].nx, descs[p].ny, descs[p].lag_min,
                     descs[p].lag_max, nullptr, 0};
  if (!w->E.plan(w->L, w->jobs, w->engs, bits, ctx->ntt_two_primes))
    return set_err(ctx, TDE_ERR_UNSUPPORTED,
                   "NTT engine: a pair's shorter signal exceeds the largest transform (2^%d)",
                   kNttMaxLog);
  w->E.popc.prepacked = w->Q.planes_written();
  w->A.plan(w->L, npairs, max_count, 0);
  return TDE_OK;
}

void batch_fill(BatchWork* w, const Bases& B, const tde_pair_desc* descs, int32_t* c_out,
                int64_t* lag_out, int64_t* val_out) {
  const int np = w->npairs;
  std::vector<const float*> xs(2 * np);
  std::vector<int8_t*> qs(2 * np);
  std::vector<int64_t> ns(2 * np);
  int32_t* c_base = w->own_c ? B.dw<int32_t>(w->o_call) : c_out;
  for (int p = 0; p < np; ++p) {
    xs[2 * p] = descs[p].x, xs[2 * p + 1] = descs[p].y;
    qs[2 * p] = B.dw<int8_t>(w->o_q[2 * p]), qs[2 * p + 1] = B.dw<int8_t>(w->o_q[2 * p + 1]);
    ns[2 * p] = descs[p].nx, ns[2 * p + 1] = descs[p].ny;
    w->jobs[p].qx = qs[2 * p], w->jobs[p].qy = qs[2 * p + 1];
    w->jobs[p].c = c_base + w->c_start[p];
    w->A.set(B, p, w->jobs[p].c, descs[p].lag_min, descs[p].lag_max - descs[p].lag_min + 1,
             lag_out + p, val_out + p);
  }
  w->Q.fill(B, xs.data(), qs.data(), ns.data());
  w->E.fill(B, w->jobs);
  // popc pairs get their planes from the quantizer (the k-th popc job is the
  // k-th pair routed to popc)
  for (int p = 0, k = 0; p < np; ++p)
    for (int side = 0; side < 2; ++side) {
      const bool popc = w->engs[p] == TDE_ENGINE_POPC;
      const int64_t n = side ? descs[p].ny : descs[p].nx;
      w->Q.set_planes(B, 2 * p + side, popc ? w->E.popc.planes_of(B, k, side) : nullptr,
                      popc ? ceil_div64(n, 32) : 0);
      if (side == 1 && popc) ++k;
    }
}

cudaError_t batch_launch(tde_ctx* ctx, const BatchWork& w, const Bases& B, cudaStream_t st) {
  cudaError_t e = w.Q.launch(B, ctx->d_status, st);
  if (e == cudaSuccess) e = w.E.launch(ctx, B, st);
  if (e == cudaSuccess) e = w.A.launch(B, st);
  return e;
}

}  // namespace

extern "C" tde_status tde_estimate_batch(tde_ctx* ctx, const tde_pair_desc* descs, int npairs,
                                         int bits, int engine, int32_t* c_out, int64_t* lag_out,
                                         int64_t* val_out, tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  if (!ctx) return TDE_ERR_INVALID;
  if (!descs || !lag_out || !val_out) return set_err(ctx, TDE_ERR_INVALID, "null pointer");
  BatchWork w;
  tde_status s = batch_plan(ctx, descs, npairs, bits, engine, c_out != nullptr, &w);
  if (s != TDE_OK) return s;
  DeviceGuard g(ctx->device);
  LaunchCount lc(ctx);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Bases B;
  if ((s = realize(ctx, w.L, &B)) != TDE_OK) return s;
  batch_fill(&w, B, descs, c_out, lag_out, val_out);
  if ((s = stage_upload(ctx, B.ddesc, w.L.desc, st)) != TDE_OK) return s;
  const cudaError_t e = batch_launch(ctx, w, B, st);
  if (e != cudaSuccess) return cuda_err(ctx, e, "estimate launch");
  return TDE_OK;
}

// A batch planned once, with its own device memory and descriptors, whose
// whole step is captured in a CUDA graph.
struct tde_batch {
  tde_ctx* ctx = nullptr;
  BatchWork w;
  char* mem = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;  // kernels in the graph
};

extern "C" tde_status tde_batch_create(tde_ctx* ctx, const tde_pair_desc* descs, int npairs,
                                       int bits, int engine, int32_t* c_out, int64_t* lag_out,
                                       int64_t* val_out, tde_batch** out) {
  ApiRange nvtx_range(__func__);
  if (!ctx) return TDE_ERR_INVALID;
  if (!descs || !lag_out || !val_out || !out) return set_err(ctx, TDE_ERR_INVALID, "null pointer");
  *out = nullptr;
  tde_batch* b = new tde_batch();
  b->ctx = ctx;
  tde_status s = batch_plan(ctx, descs, npairs, bits, engine, c_out != nullptr, &b->w);
  if (s != TDE_OK) {
    delete b;
    return s;
  }
  DeviceGuard g(ctx->device);
  auto fail = [&](cudaError_t e, const char* what) {
    tde_batch_destroy(b);
    return cuda_err(ctx, e, what);
  };
  cudaError_t e = cudaMalloc(&b->mem, b->w.L.total());
  if (e != cudaSuccess) return fail(e, "cudaMalloc(batch memory)");
  std::vector<char> host(b->w.L.desc ? b->w.L.desc : 16);
  Bases B{host.data(), b->mem, b->mem + b->w.L.data_base()};
  batch_fill(&b->w, B, descs, c_out, lag_out, val_out);
  e = cudaMemcpy(b->mem, host.data(), b->w.L.desc, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(e, "descriptor upload");
  // Tables the engines need are built before capture (capture forbids cudaMalloc).
  for (const auto& grp : b->w.E.ntt.groups) {
    NttTables T;
    if (ntt_tables(ctx, grp.logn, &T) != TDE_OK) {
      tde_batch_destroy(b);
      return TDE_ERR_CUDA;
    }
  }
  cudaStream_t cs;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fail(e, "cudaStreamCreate");
  const bool prof = ctx->profile;
  ctx->profile = false;
  const int64_t before = tde_launch_counter;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    const cudaError_t le = batch_launch(ctx, b->w, B, cs);
    e = cudaStreamEndCapture(cs, &b->graph);
    if (le != cudaSuccess) e = le;
  }
  b->launches = tde_launch_counter - before;
  tde_launch_counter = before;
  ctx->profile = prof;
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return fail(e, "graph capture");
  e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) return fail(e, "cudaGraphInstantiate");
  *out = b;
  return TDE_OK;
}

extern "C" tde_status tde_batch_run(tde_batch* b, tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  if (!b || !b->exec) return TDE_ERR_INVALID;
  tde_ctx* ctx = b->ctx;
  DeviceGuard g(ctx->device);
  const cudaError_t e = cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaGraphLaunch");
  ctx->launches += b->launches;
  return TDE_OK;
}

extern "C" tde_status tde_batch_destroy(tde_batch* b) {
  if (!b) return TDE_OK;
  {
    DeviceGuard g(b->ctx->device);
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->mem) cudaFree(b->mem);
  }
  delete b;
  return TDE_OK;
}

extern "C" tde_status tde_estimate(tde_ctx* ctx, const float* x, int64_t nx, const float* y,
                                   int64_t ny, int bits, int64_t lag_min, int64_t lag_max,
                                   int engine, int64_t* lag_out, int64_t* val_out,
                                   tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  tde_pair_desc d{x, y, nx, ny, lag_min, lag_max};
  return tde_estimate_batch(ctx, &d, 1, bits, engine, nullptr, lag_out, val_out, stream);
}

extern "C" tde_status tde_xcorr_fft32(tde_ctx* ctx, const void* x, const void* y, int in_dtype,
                                      int64_t nx, int64_t ny, int npairs, int64_t lag_min,
                                      int64_t lag_max, float* c_out, tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  if (!ctx) return TDE_ERR_INVALID;
  if (!x || !y || !c_out) return set_err(ctx, TDE_ERR_INVALID, "null pointer");
  if (in_dtype != TDE_F32 && in_dtype != TDE_I8)
    return set_err(ctx, TDE_ERR_INVALID, "in_dtype must be TDE_F32 or TDE_I8");
  if (nx <= 0 || ny <= 0 || npairs <= 0)
    return set_err(ctx, TDE_ERR_INVALID, "sizes must be positive");
  if (lag_min > lag_max || lag_min < -(nx - 1) || lag_max > ny - 1)
    return set_err(ctx, TDE_ERR_INVALID, "lag range outside [-(nx-1), ny-1]");
  const int64_t L = fft_length(nx, ny);
  if (L > ((int64_t)1 << 30)) return set_err(ctx, TDE_ERR_UNSUPPORTED, "transform too long");
  DeviceGuard g(ctx->device);
  LaunchCount lc(ctx);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (fft_plan(&ctx->fft, L, npairs) != 0)
    return set_err(ctx, TDE_ERR_CUDA, "cuFFT plan creation failed (L=%lld, batch=%d)",
                   (long long)L, npairs);
  Layout Lay;
  const size_t o_rx = Lay.w<float>((size_t)npairs * L), o_ry = Lay.w<float>((size_t)npairs * L);
  const size_t o_sx = Lay.w<float2>((size_t)npairs * (L / 2 + 1));
  const size_t o_sy = Lay.w<float2>((size_t)npairs * (L / 2 + 1));
  Bases B;
  tde_status s = realize(ctx, Lay, &B);
  if (s != TDE_OK) return s;
  if (fft_xcorr(ctx->fft, x, y, in_dtype == TDE_I8, nx, ny, lag_min, lag_max - lag_min + 1, c_out,
                B.dw<float>(o_rx), B.dw<float>(o_ry), B.dw<float2>(o_sx), B.dw<float2>(o_sy),
                st) != 0)
    return set_err(ctx, TDE_ERR_CUDA, "FFT comparator failed");
  return TDE_OK;
}

// ====================================================== learned lag proposal

cudaError_t launch_synth_pairs(uint64_t seed, int64_t first, int npairs, int64_t n, int64_t dmax,
                               float a_lo, float a_hi, float snr_lo, float snr_hi, float* x,
                               float* y, int64_t* shift, cudaStream_t st);

extern "C" tde_status tde_synth_pairs(tde_ctx* ctx, uint64_t seed, int64_t first, int npairs,
                                      int64_t n, int64_t dmax, float ar_lo, float ar_hi,
                                      float snr_lo, float snr_hi, float* x_out, float* y_out,
                                      int64_t* shift_out, tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  if (!ctx) return TDE_ERR_INVALID;
  if (!x_out || !y_out || !shift_out) return set_err(ctx, TDE_ERR_INVALID, "null pointer");
  if (npairs <= 0 || n <= 0 || dmax < 0 || first < 0)
    return set_err(ctx, TDE_ERR_INVALID, "sizes must be positive (dmax, first >= 0)");
  if (!(ar_lo >= 0.f && ar_hi < 1.f && ar_lo <= ar_hi) || !(snr_lo <= snr_hi))
    return set_err(ctx, TDE_ERR_INVALID, "need 0 <= ar_lo <= ar_hi < 1 and snr_lo <= snr_hi");
  DeviceGuard g(ctx->device);
  LaunchCount lc(ctx);
  const cudaError_t e =
      launch_synth_pairs(seed, first, npairs, n, dmax, ar_lo, ar_hi, snr_lo, snr_hi, x_out, y_out,
                         shift_out, reinterpret_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? TDE_OK : cuda_err(ctx, e, "synth launch");
}

struct tde_model {
  tde_ctx* ctx = nullptr;
  int64_t n = 0;
  float* params = nullptr;  // FP32 master
  uint16_t* wbf = nullptr;  // BF16 copy used by the forward pass
  float* m = nullptr;
  float* v = nullptr;
  float* grad = nullptr;
  int64_t step = 0;
};

namespace {

uint64_t host_splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

bool model_len_ok(int64_t n) { return n >= 16384 && n % 2048 == 0 && n <= ((int64_t)1 << 24); }

// Work memory of the CNN for npairs pairs (2 npairs signals): decimated input,
// per-layer outputs (and, for training, pre-pool activations and gradients).
struct CnnPlan {
  int P = 0, Ld = 0, Lf = 0;
  size_t o_d = 0, o_out[kCnnLayers] = {}, o_pre[kCnnLayers] = {}, o_scores = 0;
  size_t o_act[kCnnLayers - 1] = {};  // inference: BF16 activation rows
  bool train_ = false;
  size_t o_dscores = 0, o_dalpha = 0, o_dz = 0, o_dA = 0, o_dB = 0, o_partial = 0, o_loss = 0;
  void plan(Layout& L, int npairs, int64_t n, bool train) {
    P = npairs;
    train_ = train;
    Ld = (int)(n / kCnnDec);
    Lf = Ld / 16;
    const size_t S = 2 * (size_t)P;
    if (!train) {
      for (int l = 0; l + 1 < kCnnLayers; ++l)
        o_act[l] = L.w<uint16_t>(S * (size_t)cnn_eo_elems(Ld >> (l + 1)));
      o_out[kCnnLayers - 1] = L.w<float>(S * kCnnC * (size_t)Lf);
    } else {
      o_d = L.w<float>(S * Ld);
      for (int l = 0; l < kCnnLayers; ++l) {
        const size_t len = (size_t)Ld >> l;  // input length of layer l
        o_out[l] = L.w<float>(S * kCnnC * (len / 2));
        o_pre[l] = L.w<float>(S * kCnnC * len);
      }
    }
    o_scores = L.w<float>((size_t)P * (2 * Lf - 1));
    if (train) {
      o_dscores = L.w<float>((size_t)P * (2 * Lf - 1));
      o_dalpha = L.w<float>((size_t)P);
      o_loss = L.w<float>((size_t)P);
      o_dz = L.w<float>(S * kCnnC * Ld);
      o_dA = L.w<float>(S * kCnnC * (Ld / 2));
      o_dB = L.w<float>(S * kCnnC * (Ld / 2));
      o_partial = L.w<float>(S * (kCnnC * kCnnC * kCnnK + kCnnC));
    }
  }
  float* layer_in(const Bases& B, int l) const {
    return l == 0 ? B.dw<float>(o_d) : B.dw<float>(o_out[l - 1]);
  }
  // scores = false (inference only): stop at the features, for a caller
  // that scores them itself.
  cudaError_t forward(const Bases& B, const tde_model* m, const int8_t* q, int64_t n, bool train,
                      uint32_t* status, cudaStream_t st, uint8_t* qe = nullptr,
                      bool scores = true) const {
    if (!train) {
      uint16_t* act[kCnnLayers - 1];
      for (int l = 0; l + 1 < kCnnLayers; ++l) act[l] = B.dw<uint16_t>(o_act[l]);
      cudaError_t e = launch_cnn_infer(q, n, 2 * P, m->wbf, m->params, act,
                                       B.dw<float>(o_out[kCnnLayers - 1]), qe, status, st);
      if (e == cudaSuccess && scores)
        e = launch_cnn_scores(B.dw<float>(o_out[kCnnLayers - 1]), P, Lf, m->params,
                              B.dw<float>(o_scores), st, true, status);
      return e;
    }
    cudaError_t e = launch_cnn_decimate(q, n, 2 * P, B.dw<float>(o_d), st);
    for (int l = 0; l < kCnnLayers && e == cudaSuccess; ++l) {
      CnnLayerIO io{layer_in(B, l), train ? B.dw<float>(o_pre[l]) : nullptr, B.dw<float>(o_out[l]),
                    Ld >> l};
      e = launch_cnn_layer(io, l, 2 * P, m->wbf, m->params, st);
    }
    if (e == cudaSuccess)
      e = launch_cnn_scores(B.dw<float>(o_out[kCnnLayers - 1]), P, Lf, m->params,
                            B.dw<float>(o_scores), st);
    return e;
  }
};

tde_status check_model(tde_ctx* ctx, const tde_model* m) {
  if (!m || !m->params) return set_err(ctx, TDE_ERR_INVALID, "null model");
  if (m->ctx && m->ctx->device != ctx->device)
    return set_err(ctx, TDE_ERR_INVALID, "model lives on another device");
  return TDE_OK;
}

// Window w of pair p: lags [c - 128, c + 128] clipped to the overlap range;
// lag tau lands at cbuf[i * stride + tau - (c - 128)].
__global__ void k_make_windows(const int32_t* __restrict__ centres, int npairs, int64_t n,
                               int32_t* __restrict__ cbuf, int stride, WinJob* __restrict__ jobs,
                               int32_t* __restrict__ njobs) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= npairs * kCnnTopK) return;
  jobs[i] = win_job_of(centres[i], n, cbuf + (int64_t)i * stride);
  if (i % kCnnTopK == 0) {  // the pair's job count in the polyphase windows kernel
    int64_t lo[kCnnTopK], hi[kCnnTopK];
#pragma unroll
    for (int w = 0; w < kCnnTopK; ++w) {
      const WinJob J = win_job_of(centres[i + w], n, cbuf);
      lo[w] = J.lag_lo, hi[w] = J.lag_hi;
    }
    int a[kCnnTopK], b[kCnnTopK];
    win_blocks(lo, hi, a, b);
    njobs[i / kCnnTopK] = win_jobs(a, b);
  }
}


}  // namespace

extern "C" tde_status tde_model_create(tde_ctx* ctx, int64_t n, uint64_t seed, tde_model** out) {
  if (!ctx || !out) return TDE_ERR_INVALID;
  *out = nullptr;
  if (!model_len_ok(n))
    return set_err(ctx, TDE_ERR_UNSUPPORTED,
                   "proposal model needs n a multiple of 2048 in [16384, 2^24] (got %lld)",
                   (long long)n);
  DeviceGuard g(ctx->device);
  tde_model* m = new tde_model();
  m->ctx = ctx;
  m->n = n;
  // He-uniform conv weights from a seeded splitmix64 stream; zero biases;
  // alpha scaled to the feature length.
  std::vector<float> h(kCnnParams, 0.f);
  uint64_t st = seed * 0x9E3779B97F4A7C15ull + 12345;
  for (int l = 0; l < kCnnLayers; ++l) {
    const int fan_in = cnn_cin(l) * kCnnK;
    const float bound = sqrtf(6.0f / (float)fan_in);
    for (int i = cnn_woff(l); i < cnn_boff(l); ++i) {
      const double u = (double)(host_splitmix(st) >> 11) / 9007199254740992.0;
      h[i] = (float)((2.0 * u - 1.0) * bound);
    }
  }
  h[kCnnAlpha] = 1.0f / (float)(kCnnC * (n / kCnnDec / 16));
  const size_t bytes = sizeof(float) * kCnnParams;
  if (cudaMalloc(&m->params, bytes) != cudaSuccess || cudaMalloc(&m->m, bytes) != cudaSuccess ||
      cudaMalloc(&m->v, bytes) != cudaSuccess || cudaMalloc(&m->grad, bytes) != cudaSuccess ||
      cudaMalloc(&m->wbf, sizeof(uint16_t) * kCnnParams) != cudaSuccess ||
      cudaMemcpy(m->params, h.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(m->m, 0, bytes) != cudaSuccess || cudaMemset(m->v, 0, bytes) != cudaSuccess ||
      cudaMemset(m->grad, 0, bytes) != cudaSuccess ||
      launch_cnn_to_bf16(m->params, m->wbf, nullptr) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess) {
    tde_model_destroy(m);
    return set_err(ctx, TDE_ERR_CUDA, "model allocation failed");
  }
  *out = m;
  return TDE_OK;
}

extern "C" tde_status tde_model_destroy(tde_model* m) {
  if (!m) return TDE_OK;
  {
    DeviceGuard g(m->ctx ? m->ctx->device : 0);
    cudaDeviceSynchronize();
    cudaFree(m->params), cudaFree(m->wbf), cudaFree(m->m), cudaFree(m->v), cudaFree(m->grad);
  }
  delete m;
  return TDE_OK;
}

extern "C" int64_t tde_model_param_count(void) { return kCnnParams; }

extern "C" tde_status tde_model_get(const tde_model* m, float* params, float* adam_m, float* adam_v,
                                    float* grad, int64_t* step) {
  if (!m) return TDE_ERR_INVALID;
  DeviceGuard g(m->ctx->device);
  const size_t bytes = sizeof(float) * kCnnParams;
  if (cudaDeviceSynchronize() != cudaSuccess) return TDE_ERR_CUDA;
  if ((params && cudaMemcpy(params, m->params, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (adam_m && cudaMemcpy(adam_m, m->m, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (adam_v && cudaMemcpy(adam_v, m->v, bytes, cudaMemcpyDeviceToHost) != cudaSuccess) ||
      (grad && cudaMemcpy(grad, m->grad, bytes, cudaMemcpyDeviceToHost) != cudaSuccess))
    return TDE_ERR_CUDA;
  if (step) *step = m->step;
  return TDE_OK;
}

extern "C" tde_status tde_model_set(tde_model* m, const float* params, const float* adam_m,
                                    const float* adam_v, int64_t step) {
  if (!m || !params) return TDE_ERR_INVALID;
  DeviceGuard g(m->ctx->device);
  const size_t bytes = sizeof(float) * kCnnParams;
  if (cudaDeviceSynchronize() != cudaSuccess ||
      cudaMemcpy(m->params, params, bytes, cudaMemcpyHostToDevice) != cudaSuccess ||
      (adam_m && cudaMemcpy(m->m, adam_m, bytes, cudaMemcpyHostToDevice) != cudaSuccess) ||
      (adam_v && cudaMemcpy(m->v, adam_v, bytes, cudaMemcpyHostToDevice) != cudaSuccess) ||
      launch_cnn_to_bf16(m->params, m->wbf, nullptr) != cudaSuccess ||
      cudaDeviceSynchronize() != cudaSuccess)
    return TDE_ERR_CUDA;
  if (!adam_m) cudaMemset(m->m, 0, bytes);
  if (!adam_v) cudaMemset(m->v, 0, bytes);
  m->step = step;
  return TDE_OK;
}

extern "C" tde_status tde_train_step(tde_ctx* ctx, tde_model* m, const int8_t* q, int npairs,
                                     const int64_t* labels, float lr, float weight_decay,
                                     float* loss_out, tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  if (!ctx) return TDE_ERR_INVALID;
  tde_status s = check_model(ctx, m);
  if (s != TDE_OK) return s;
  if (!q || !labels || !loss_out) return set_err(ctx, TDE_ERR_INVALID, "null pointer");
  if (npairs <= 0) return set_err(ctx, TDE_ERR_INVALID, "npairs must be positive");
  DeviceGuard g(ctx->device);
  LaunchCount lc(ctx);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Layout L;
  CnnPlan C;
  C.plan(L, npairs, m->n, true);
  Bases B;
  if ((s = realize(ctx, L, &B)) != TDE_OK) return s;
  const int S = 2 * npairs, Ld = C.Ld, Lf = C.Lf;
  cudaError_t e = C.forward(B, m, q, m->n, true, ctx->d_status, st);
  if (e == cudaSuccess)
    e = launch_cnn_softmax_ce(B.dw<float>(C.o_scores), labels, npairs, Lf, loss_out,
                              B.dw<float>(C.o_dscores), st);
  // d features -> dA (gradient w.r.t. the last layer's pooled output)
  if (e == cudaSuccess)
    e = launch_cnn_scores_bwd(B.dw<float>(C.o_out[kCnnLayers - 1]), B.dw<float>(C.o_dscores),
                              npairs, Lf, m->params, B.dw<float>(C.o_dA), B.dw<float>(C.o_dalpha),
                              st);
  float* dout = B.dw<float>(C.o_dA);
  float* dnext = B.dw<float>(C.o_dB);
  for (int l = kCnnLayers - 1; l >= 0 && e == cudaSuccess; --l) {
    const int len = Ld >> l;
    float* dz = B.dw<float>(C.o_dz);
    e = launch_cnn_pool_relu_bwd(B.dw<float>(C.o_pre[l]), dout, S, len, dz, st);
    if (e == cudaSuccess)
      e = launch_cnn_wgrad(dz, C.layer_in(B, l), S, len, l, B.dw<float>(C.o_partial), st);
    if (e == cudaSuccess)
      e = launch_cnn_reduce(B.dw<float>(C.o_partial), S,
                            kCnnC * cnn_cin(l) * kCnnK + kCnnC, m->grad + cnn_woff(l), st);
    if (e == cudaSuccess && l > 0) {
      e = launch_cnn_dgrad(dz, S, len, l, m->wbf, dnext, st);
      std::swap(dout, dnext);
    }
  }
  if (e == cudaSuccess)
    e = launch_cnn_reduce(B.dw<float>(C.o_dalpha), npairs, 1, m->grad + kCnnAlpha, st);
  if (e == cudaSuccess) {
    m->step += 1;
    e = launch_cnn_adamw(m->params, m->grad, m->m, m->v, m->wbf, m->step, lr, 0.9f, 0.999f, 1e-8f,
                         weight_decay, st);
  }
  return e == cudaSuccess ? TDE_OK : cuda_err(ctx, e, "train step");
}

extern "C" tde_status tde_propose(tde_ctx* ctx, const tde_model* m, const int8_t* q, int npairs,
                                  int32_t* centres, float* margin, tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  if (!ctx) return TDE_ERR_INVALID;
  tde_status s = check_model(ctx, m);
  if (s != TDE_OK) return s;
  if (!q || !centres || !margin) return set_err(ctx, TDE_ERR_INVALID, "null pointer");
  if (npairs <= 0) return set_err(ctx, TDE_ERR_INVALID, "npairs must be positive");
  DeviceGuard g(ctx->device);
  LaunchCount lc(ctx);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Layout L;
  CnnPlan C;
  C.plan(L, npairs, m->n, false);
  Bases B;
  if ((s = realize(ctx, L, &B)) != TDE_OK) return s;
  cudaError_t e = C.forward(B, m, q, m->n, false, ctx->d_status, st);
  if (e == cudaSuccess) e = launch_cnn_topk(B.dw<float>(C.o_scores), npairs, C.Lf, centres, margin, st);
  return e == cudaSuccess ? TDE_OK : cuda_err(ctx, e, "propose");
}

extern "C" tde_status tde_xcorr_windows(tde_ctx* ctx, const int8_t* q, int64_t n, int npairs,
                                        int bits, const int32_t* centres, int32_t* c_out,
                                        tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  if (!ctx) return TDE_ERR_INVALID;
  if (!q || !centres || !c_out) return set_err(ctx, TDE_ERR_INVALID, "null pointer");
  if (!valid_bits(bits)) return set_err(ctx, TDE_ERR_INVALID, "bits must be 1, 2 or 4");
  if (n <= 0 || npairs <= 0) return set_err(ctx, TDE_ERR_INVALID, "n and npairs must be positive");
  if (n > INT32_MAX) return set_err(ctx, TDE_ERR_UNSUPPORTED, "n beyond 2^31 - 1");
  {
    // the int32 windows hold values up to n * (2^(bits-1))^2 in magnitude
    const int64_t k = (int64_t)1 << (bits - 1);
    if (n * k * k >= ((int64_t)1 << 31))
      return set_err(ctx, TDE_ERR_OVERFLOW,
                     "int32 windows may overflow: n*(2^(bits-1))^2 = %lld >= 2^31", (long long)(n * k * k));
  }
  DeviceGuard g(ctx->device);
  LaunchCount lc(ctx);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Layout L;
  const size_t o_jobs = L.w<WinJob>((size_t)npairs * kCnnTopK);
  const size_t o_njobs = L.w<int32_t>((size_t)npairs);
  const int64_t n_pad = (n + 127) / 128 * 128;
  const size_t o_qe = L.w<uint8_t>((size_t)2 * npairs * n_pad);
  Bases B;
  tde_status s = realize(ctx, L, &B);
  if (s != TDE_OK) return s;
  WinJob* jobs = B.dw<WinJob>(o_jobs);
  uint8_t* qe = B.dw<uint8_t>(o_qe);
  cudaError_t e = cudaMemsetAsync(c_out, 0, sizeof(int32_t) * (size_t)npairs * kCnnTopK * kCnnWin, st);
  if (e == cudaSuccess) {
    k_make_windows<<<(npairs * kCnnTopK + 255) / 256, 256, 0, st>>>(centres, npairs, n, c_out,
                                                                     kCnnWin, jobs, B.dw<int32_t>(o_njobs));
    TDE_COUNT_LAUNCH(1);
    e = cudaGetLastError();
  }
  // the levels as E4M3 bytes (a level outside the bits' range sets the status
  // word), then the windows in polyphase form
  if (e == cudaSuccess) e = launch_to_e4m3(q, n, n_pad, 2 * npairs, bits, qe, ctx->d_status, st);
  if (e == cudaSuccess) {
    EngineTimer t(ctx, st);
    e = launch_xcorr_win_pp(qe, n, n_pad, npairs, jobs, B.dw<int32_t>(o_njobs), ctx->d_status, st);
  }
  return e == cudaSuccess ? TDE_OK : cuda_err(ctx, e, "windows");
}

namespace {

// Fallback on the device: the pairs whose margin is below theta (in any
// order) -> fb_idx[0 .. *nfb).  One CTA.
__global__ void k_fb_select(const float* __restrict__ marg, int P, float theta,
                            int32_t* __restrict__ fb_idx, int* __restrict__ nfb,
                            int32_t* __restrict__ fb_out) {
  __shared__ int cnt;
  if (threadIdx.x == 0) cnt = 0;
  __syncthreads();
  for (int p = threadIdx.x; p < P; p += blockDim.x) {
    const bool f = !(marg[p] >= theta);
    if (fb_out) fb_out[p] = f ? 1 : 0;
    if (f) fb_idx[atomicAdd(&cnt, 1)] = p;
  }
  __syncthreads();
  if (threadIdx.x == 0) *nfb = cnt;
}

// Descriptors of the fallback's full correlations: slot k < *nfb is pair
// fb_idx[k] (all lags, output row k of cfb), its engine items are the
// one-pair template with pair = k, and its argmax writes tlag/tval[k].
__global__ void k_fb_build(const int32_t* __restrict__ fb_idx, const int* __restrict__ nfb, int P,
                           const int8_t* __restrict__ qbuf, int64_t n,
                           const MmaItem* __restrict__ tmpl, int nt, int zero_first,
                           int32_t* __restrict__ cfb, MmaPair* __restrict__ pairs,
                           MmaItem* __restrict__ items, ArgPair* __restrict__ args,
                           int64_t* __restrict__ tlag, int64_t* __restrict__ tval,
                           int* __restrict__ nitems) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int cnt = *nfb;
  const int64_t lags = 2 * n - 1;
  if (i == 0) *nitems = cnt * nt;
  if (i < (int64_t)cnt * nt) {
    MmaItem it = tmpl[i % nt];
    it.pair = (int32_t)(i / nt);
    items[i] = it;
  }
  if (i < cnt) {
    const int64_t p = fb_idx[i];
    int32_t* c = cfb + i * lags;
    pairs[i] = MmaPair{qbuf + 2 * p * n, qbuf + (2 * p + 1) * n, n, n, -(n - 1), n - 1, c, 0,
                       zero_first};
    args[i] = ArgPair{c, -(n - 1), lags, tlag + i, tval + i};
  } else if (i < P) {
    pairs[i] = MmaPair{qbuf, qbuf, n, n, -(n - 1), n - 1, cfb, 0, 0};  // idle slot
  }
}

__global__ void k_fb_scatter(const int32_t* __restrict__ fb_idx, const int* __restrict__ nfb,
                             const int64_t* __restrict__ tlag, const int64_t* __restrict__ tval,
                             int64_t* __restrict__ lag, int64_t* __restrict__ val) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= *nfb) return;
  lag[fb_idx[i]] = tlag[i];
  val[fb_idx[i]] = tval[i];
}

// Everything one learned estimate needs: quantize, proposal, windows, window
// argmax, and the device-side fallback (full correlations of the pairs whose
// margin is below theta), planned from the sizes alone.
struct LearnedWork {
  int P = 0, bits = 2;
  int64_t n = 0;
  float theta = 0.f;
  Layout L;
  QuantStage Q;
  CnnPlan C;
  MmaStage T;  // one full-range pair: the fallback's item template
  size_t o_q = 0, o_qe = 0, o_cent = 0, o_marg = 0, o_jobs = 0, o_njobs = 0, o_cwin = 0;
  size_t o_fbidx = 0, o_nfb = 0, o_fbpairs = 0, o_fbitems = 0, o_nitems = 0, o_counter = 0;
  size_t o_fbargs = 0, o_keys = 0, o_tlag = 0, o_tval = 0, o_cfb = 0;
};

void learned_plan(LearnedWork* w, int npairs, int64_t n, int bits, float theta) {
  w->P = npairs, w->n = n, w->bits = bits, w->theta = theta;
  Layout& L = w->L;
  const int S = 2 * npairs;
  w->Q.plan(L, S, bits, nullptr, n);
  w->o_q = L.w<int8_t>((size_t)S * n);
  w->o_qe = L.w<uint8_t>((size_t)S * n);  // the levels as E4M3 bytes (n % 2048 == 0)
  w->C.plan(L, npairs, n, false);
  w->o_cent = L.w<int32_t>((size_t)npairs * kCnnTopK);
  w->o_marg = L.w<float>((size_t)npairs);
  w->o_jobs = L.w<WinJob>((size_t)npairs * kCnnTopK);
  w->o_njobs = L.w<int32_t>((size_t)npairs);
  w->o_cwin = L.w<int32_t>((size_t)npairs * kCnnTopK * kCnnWin);
  std::vector<Job> one{Job{nullptr, nullptr, n, n, -(n - 1), n - 1, nullptr, 0}};
  w->T.plan(L, one, false, bits <= 2);  // replicated per fallback pair: keep the default segments
  const int nt = w->T.nitems;
  w->o_fbidx = L.w<int32_t>((size_t)npairs);
  w->o_nfb = L.w<int>(1);
  w->o_fbpairs = L.w<MmaPair>((size_t)npairs);
  w->o_fbitems = L.w<MmaItem>((size_t)npairs * nt);
  w->o_nitems = L.w<int>(1);
  w->o_counter = L.w<int>(1);
  w->o_fbargs = L.w<ArgPair>((size_t)npairs);
  w->o_keys = L.w<unsigned long long>(2 * (size_t)npairs);
  w->o_tlag = L.w<int64_t>((size_t)npairs);
  w->o_tval = L.w<int64_t>((size_t)npairs);
  w->o_cfb = L.w<int32_t>((size_t)npairs * (size_t)(2 * n - 1));
}

void learned_fill(LearnedWork* w, const Bases& B, const float* x, const float* y) {
  const int S = 2 * w->P;
  const int64_t n = w->n;
  std::vector<const float*> xs(S);
  std::vector<int8_t*> qs(S);
  std::vector<int64_t> ns(S, n);
  int8_t* qbuf = B.dw<int8_t>(w->o_q);
  for (int p = 0; p < w->P; ++p)
    for (int k = 0; k < 2; ++k) {
      const int i = 2 * p + k;
      xs[i] = (k ? y : x) + (int64_t)p * n;
      qs[i] = qbuf + (int64_t)i * n;
    }
  w->Q.fill(B, xs.data(), qs.data(), ns.data());
  std::vector<Job> one{Job{qbuf, qbuf + n, n, n, -(n - 1), n - 1, B.dw<int32_t>(w->o_cfb), 0}};
  w->T.fill(B, one);  // only its items (the template) are used
}

cudaError_t learned_launch(tde_ctx* ctx, const tde_model* m, const LearnedWork& w, const Bases& B,
                           int64_t* lag_out, int64_t* val_out, int32_t* fb_out, cudaStream_t st) {
  const int P = w.P;
  const int64_t n = w.n;
  int8_t* qbuf = B.dw<int8_t>(w.o_q);
  int32_t* cent = B.dw<int32_t>(w.o_cent);
  float* marg = B.dw<float>(w.o_marg);
  WinJob* jobs = B.dw<WinJob>(w.o_jobs);
  cudaError_t e = w.Q.launch(B, ctx->d_status, st);
  uint8_t* qe = B.dw<uint8_t>(w.o_qe);
  // features up to kCnnFusedMaxLf: scores, top 8, window jobs and their
  // zeroed outputs in one launch; longer ones in separate steps
  const bool fused = w.C.Lf <= kCnnFusedMaxLf;
  if (e == cudaSuccess) e = w.C.forward(B, m, qbuf, n, false, ctx->d_status, st, qe, !fused);
  if (e == cudaSuccess && fused)
    e = launch_cnn_scores_propose(B.dw<float>(w.C.o_out[kCnnLayers - 1]), P, w.C.Lf, m->params,
                                  B.dw<float>(w.C.o_scores), cent, marg, jobs,
                                  B.dw<int32_t>(w.o_cwin), n, B.dw<int32_t>(w.o_njobs), st,
                                  ctx->d_status);
  if (e == cudaSuccess && !fused) {
    e = launch_cnn_topk(B.dw<float>(w.C.o_scores), P, w.C.Lf, cent, marg, st);
    if (e == cudaSuccess) {
      k_make_windows<<<(P * kCnnTopK + 255) / 256, 256, 0, st>>>(
          cent, P, n, B.dw<int32_t>(w.o_cwin), kCnnWin, jobs, B.dw<int32_t>(w.o_njobs));
      TDE_COUNT_LAUNCH(1);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess)
      e = cudaMemsetAsync(B.dw<int32_t>(w.o_cwin), 0,
                          sizeof(int32_t) * (size_t)P * kCnnTopK * kCnnWin, st);
  }
  if (e == cudaSuccess) {
    EngineTimer t(ctx, st);
    e = launch_xcorr_win_pp(qe, n, n, P, jobs, B.dw<int32_t>(w.o_njobs), ctx->d_status, st);
  }
  if (e == cudaSuccess) e = launch_window_argmax(jobs, P, lag_out, val_out, st);
  // fallback, decided and run on the device
  int32_t* fb_idx = B.dw<int32_t>(w.o_fbidx);
  int* nfb = B.dw<int>(w.o_nfb);
  if (e == cudaSuccess) {
    k_fb_select<<<1, 1024, 0, st>>>(marg, P, w.theta, fb_idx, nfb, fb_out);
    TDE_COUNT_LAUNCH(1);
    e = cudaGetLastError();
  }
  const int nt = w.T.nitems;
  if (e == cudaSuccess) {
    const int64_t total = (int64_t)P * (nt > 1 ? nt : 1);
    k_fb_build<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(
        fb_idx, nfb, P, qbuf, n, B.dd<MmaItem>(w.T.o_items), nt, w.T.zero_first[0],
        B.dw<int32_t>(w.o_cfb), B.dw<MmaPair>(w.o_fbpairs), B.dw<MmaItem>(w.o_fbitems),
        B.dw<ArgPair>(w.o_fbargs), B.dw<int64_t>(w.o_tlag), B.dw<int64_t>(w.o_tval),
        B.dw<int>(w.o_nitems));
    TDE_COUNT_LAUNCH(1);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && w.T.any_zero) e = launch_mma_zero(B.dw<MmaPair>(w.o_fbpairs), P, 2 * n - 1, st, nfb);
  if (e == cudaSuccess)
    e = (w.T.fp4 ? launch_xcorr_mma4 : launch_xcorr_mma)(B.dw<MmaPair>(w.o_fbpairs), B.dw<MmaItem>(w.o_fbitems),
                                                          P * nt, B.dw<int>(w.o_counter), 2 * ctx->sm_count,
                                                          ctx->d_status, st, B.dw<int>(w.o_nitems));
  if (e == cudaSuccess)
    e = launch_argmax(B.dw<ArgPair>(w.o_fbargs), P, 2 * n - 1, 0,
                      B.dw<unsigned long long>(w.o_keys), st, nfb);
  if (e == cudaSuccess) {
    k_fb_scatter<<<(P + 255) / 256, 256, 0, st>>>(fb_idx, nfb, B.dw<int64_t>(w.o_tlag),
                                                  B.dw<int64_t>(w.o_tval), lag_out, val_out);
    TDE_COUNT_LAUNCH(1);
    e = cudaGetLastError();
  }
  return e;
}

tde_status check_learned_args(tde_ctx* ctx, const tde_model* m, const float* x, const float* y,
                              int npairs, int bits, const int64_t* lag_out, const int64_t* val_out) {
  tde_status s = check_model(ctx, m);
  if (s != TDE_OK) return s;
  if (!x || !y || !lag_out || !val_out) return set_err(ctx, TDE_ERR_INVALID, "null pointer");
  if (npairs <= 0) return set_err(ctx, TDE_ERR_INVALID, "npairs must be positive");
  if (bits != 1 && bits != 2)
    return set_err(ctx, TDE_ERR_UNSUPPORTED, "the learned path supports bits 1 and 2");
  return TDE_OK;
}

}  // namespace

extern "C" tde_status tde_estimate_learned(tde_ctx* ctx, const tde_model* m, const float* x,
                                           const float* y, int npairs, int bits, float theta,
                                           int64_t* lag_out, int64_t* val_out,
                                           int32_t* fallback_out, tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  if (!ctx) return TDE_ERR_INVALID;
  tde_status s = check_learned_args(ctx, m, x, y, npairs, bits, lag_out, val_out);
  if (s != TDE_OK) return s;
  DeviceGuard g(ctx->device);
  LaunchCount lc(ctx);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  LearnedWork w;
  learned_plan(&w, npairs, m->n, bits, theta);
  Bases B;
  if ((s = realize(ctx, w.L, &B)) != TDE_OK) return s;
  learned_fill(&w, B, x, y);
  if ((s = stage_upload(ctx, B.ddesc, w.L.desc, st)) != TDE_OK) return s;
  const cudaError_t e = learned_launch(ctx, m, w, B, lag_out, val_out, fallback_out, st);
  return e == cudaSuccess ? TDE_OK : cuda_err(ctx, e, "learned estimate");
}

// A learned estimate planned once, with its own device memory, captured in a
// CUDA graph; every run replays it on the current contents of x and y.
struct tde_learned {
  tde_ctx* ctx = nullptr;
  LearnedWork w;
  char* mem = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;
};

extern "C" tde_status tde_learned_create(tde_ctx* ctx, const tde_model* m, const float* x,
                                         const float* y, int npairs, int bits, float theta,
                                         int64_t* lag_out, int64_t* val_out,
                                         int32_t* fallback_out, tde_learned** out) {
  ApiRange nvtx_range(__func__);
  if (!ctx) return TDE_ERR_INVALID;
  if (!out) return set_err(ctx, TDE_ERR_INVALID, "null pointer");
  *out = nullptr;
  tde_status s = check_learned_args(ctx, m, x, y, npairs, bits, lag_out, val_out);
  if (s != TDE_OK) return s;
  DeviceGuard g(ctx->device);
  tde_learned* b = new tde_learned();
  b->ctx = ctx;
  learned_plan(&b->w, npairs, m->n, bits, theta);
  auto fail = [&](cudaError_t e, const char* what) {
    tde_learned_destroy(b);
    return cuda_err(ctx, e, what);
  };
  cudaError_t e = cudaMalloc(&b->mem, b->w.L.total());
  if (e != cudaSuccess) return fail(e, "cudaMalloc(learned plan memory)");
  std::vector<char> host(b->w.L.desc ? b->w.L.desc : 16);
  Bases B{host.data(), b->mem, b->mem + b->w.L.data_base()};
  learned_fill(&b->w, B, x, y);
  e = cudaMemcpy(b->mem, host.data(), b->w.L.desc, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) return fail(e, "descriptor upload");
  cudaStream_t cs;
  e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fail(e, "cudaStreamCreate");
  const bool prof = ctx->profile;
  ctx->profile = false;
  const int64_t before = tde_launch_counter;
  e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed);
  if (e == cudaSuccess) {
    const cudaError_t le = learned_launch(ctx, m, b->w, B, lag_out, val_out, fallback_out, cs);
    e = cudaStreamEndCapture(cs, &b->graph);
    if (le != cudaSuccess) e = le;
  }
  b->launches = tde_launch_counter - before;
  tde_launch_counter = before;
  ctx->profile = prof;
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return fail(e, "graph capture");
  e = cudaGraphInstantiate(&b->exec, b->graph, 0);
  if (e != cudaSuccess) return fail(e, "cudaGraphInstantiate");
  *out = b;
  return TDE_OK;
}

extern "C" tde_status tde_learned_run(tde_learned* b, tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  if (!b || !b->exec) return TDE_ERR_INVALID;
  tde_ctx* ctx = b->ctx;
  DeviceGuard g(ctx->device);
  const cudaError_t e = cudaGraphLaunch(b->exec, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_err(ctx, e, "cudaGraphLaunch");
  ctx->launches += b->launches;
  return TDE_OK;
}

extern "C" tde_status tde_learned_destroy(tde_learned* b) {
  if (!b) return TDE_OK;
  {
    DeviceGuard g(b->ctx->device);
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->mem) cudaFree(b->mem);
  }
  delete b;
  return TDE_OK;
}

// ================================================================ autotuner

namespace {

__global__ void k_random_levels(int8_t* q, int64_t n, int bits, uint64_t seed) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  const int k = bits == 4 ? 7 : 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
    uint64_t z = seed + (uint64_t)i * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    q[i] = (int8_t)((int)(z % (uint64_t)(2 * k + 1)) - k);
  }
}

}  // namespace

extern "C" tde_status tde_autotune(tde_ctx* ctx, int bits, const int64_t* n,
                                   const int64_t* lag_count, int npoints, int reps) {
  ApiRange nvtx_range(__func__);
  if (!ctx) return TDE_ERR_INVALID;
  if (!valid_bits(bits) || !n || !lag_count || npoints <= 0 || reps <= 0)
    return set_err(ctx, TDE_ERR_INVALID, "bad autotune arguments");
  DeviceGuard g(ctx->device);
  cudaStream_t st = nullptr;
  TDE_CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
  cudaEvent_t e0, e1;
  TDE_CK(cudaEventCreate(&e0));
  TDE_CK(cudaEventCreate(&e1));
  std::vector<tde_tune_entry> found;
  tde_status result = TDE_OK;
  for (int i = 0; i < npoints && result == TDE_OK; ++i) {
    const int64_t N = n[i];
    const int64_t lags = std::min<int64_t>(std::max<int64_t>(lag_count[i], 1), 2 * N - 1);
    if (N <= 0 || N > INT32_MAX) {
      result = set_err(ctx, TDE_ERR_INVALID, "autotune point %d: bad length", i);
      break;
    }
    const int64_t lo = -(lags / 2), hi = lo + lags - 1;
    const double work = (double)N * (double)lags;
    const int B = (int)std::max<double>(1.0, std::min<double>(512.0, 2e11 / work));
    int8_t* q = nullptr;
    int32_t* c = nullptr;
    if (cudaMalloc(&q, (size_t)2 * B * N) != cudaSuccess ||
        cudaMalloc(&c, sizeof(int32_t) * (size_t)B * lags) != cudaSuccess) {
      cudaFree(q);
      result = set_err(ctx, TDE_ERR_CUDA, "autotune allocation failed");
      break;
    }
    k_random_levels<<<1024, 256, 0, st>>>(q, 2 * B * N, bits, 12345 + i);
    tde_tune_entry te{bits, ilog2_round(N), ilog2_round(lags), TDE_ENGINE_POPC, {-1.f, -1.f, -1.f, -1.f}};
    float best = -1.f;
    for (int eng = TDE_ENGINE_POPC; eng <= TDE_ENGINE_NTT; ++eng) {
      cudaGetLastError();  // an earlier engine's failure must not be charged to this one
      std::vector<Job> jobs(B);
      for (int b = 0; b < B; ++b)
        jobs[b] = Job{q + (int64_t)(2 * b) * N, q + (int64_t)(2 * b + 1) * N, N, N, lo, hi,
                      c + (int64_t)b * lags, 0};
      Layout L;
      XcorrStage E;
      if (!E.plan(L, jobs, std::vector<int>(B, eng), bits, ctx->ntt_two_primes))
        continue;  // engine cannot serve it
      Bases Bs;
      if (realize(ctx, L, &Bs) != TDE_OK) {
        cudaGetLastError();
        continue;
      }
      E.fill(Bs, jobs);
      if (stage_upload(ctx, Bs.ddesc, L.desc, st) != TDE_OK) continue;
      float ms_best = -1.f;
      for (int r = 0; r <= reps; ++r) {  // the first run warms up
        cudaEventRecord(e0, st);
        const cudaError_t le = E.launch(ctx, Bs, st);
        cudaEventRecord(e1, st);
        if (le != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
          ms_best = -1.f;
          break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (r > 0 && (ms_best < 0.f || ms < ms_best)) ms_best = ms;
      }
      if (ms_best < 0.f) continue;
      te.ns_per_pair[eng] = ms_best * 1e6f / (float)B;
      if (best < 0.f || te.ns_per_pair[eng] < best) best = te.ns_per_pair[eng], te.engine = eng;
    }
    cudaStreamSynchronize(st);
    cudaFree(q);
    cudaFree(c);
    found.push_back(te);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(st);
  if (result != TDE_OK) return result;
  // replace the entries of these bits, keep the others
  std::vector<tde_tune_entry> keep;
  for (const tde_tune_entry& t : ctx->tune)
    if (t.bits != bits) keep.push_back(t);
  keep.insert(keep.end(), found.begin(), found.end());
  ctx->tune = keep;
  return TDE_OK;
}

extern "C" tde_status tde_autotune_table(const tde_ctx* ctx, tde_tune_entry* out, int cap,
                                         int* count) {
  if (!ctx || !count) return TDE_ERR_INVALID;
  *count = (int)ctx->tune.size();
  if (out)
    for (int i = 0; i < cap && i < (int)ctx->tune.size(); ++i) out[i] = ctx->tune[i];
  return TDE_OK;
}

extern "C" int tde_ctx_pick_engine(const tde_ctx* ctx, int bits, int64_t nx, int64_t ny,
                                   int64_t lag_count) {
  if (!ctx || !valid_bits(bits) || nx <= 0 || ny <= 0 || lag_count <= 0) return -1;
  return pick_engine_ctx(ctx, TDE_ENGINE_AUTO, bits, nx, ny, lag_count);
}

extern "C" tde_status tde_autotune_load(tde_ctx* ctx, const tde_tune_entry* entries, int count) {
  if (!ctx || count < 0 || (count > 0 && !entries)) return TDE_ERR_INVALID;
  for (int i = 0; i < count; ++i)
    if (!valid_bits(entries[i].bits) || entries[i].engine < TDE_ENGINE_POPC ||
        entries[i].engine > TDE_ENGINE_NTT)
      return set_err(ctx, TDE_ERR_INVALID, "bad autotune entry %d", i);
  ctx->tune.assign(entries, entries + count);
  return TDE_OK;
}

// ===================================================================== streaming
// Template search over a stream of chunks (overlap-save): each chunk is
// quantized into the stream's own buffer behind the last ny - 1 levels carried
// from before, the template is correlated there over the lags where it lies
// wholly inside, and the chunk's tie-ruled maximum is folded on the device
// into the running best in global positions.
struct tde_stream {
  tde_ctx* ctx = nullptr;
  int bits = 1, engine = TDE_ENGINE_AUTO;
  int64_t ny = 0, max_chunk = 0;
  int8_t* qy = nullptr;                  // the quantized template
  int8_t* buf[2] = {nullptr, nullptr};   // carry (<= ny - 1 levels) then a chunk, alternating
  int cur = 0;                           // the buffer holding the carry
  int64_t carry = 0, consumed = 0;       // levels carried; samples pushed so far
  int64_t* c = nullptr;                  // one push's correlations (<= max_chunk lags)
  int64_t* d = nullptr;                  // chunk lag, chunk value, found, best lag, best value
};

namespace {

// The chunk's maximum (relative lag d[0], value d[1]) at global lag
// -(base - d[0]) folded into the running best (d[2] = found, d[3], d[4]) in
// the argmax's order: the larger value, then the smaller |lag|, then the
// smaller lag.
__global__ void k_stream_fold(int64_t* __restrict__ d, int64_t base) {
  const int64_t lag = -(base - d[0]), val = d[1];
  if (d[2] == 0) {
    d[2] = 1, d[3] = lag, d[4] = val;
    return;
  }
  const int64_t bl = d[3], bv = d[4];
  const int64_t al = lag < 0 ? -lag : lag, abl = bl < 0 ? -bl : bl;
  if (val > bv || (val == bv && (al < abl || (al == abl && lag < bl)))) d[3] = lag, d[4] = val;
}

void stream_free(tde_stream* s) {
  if (!s) return;
  DeviceGuard g(s->ctx->device);
  cudaFree(s->qy);
  cudaFree(s->buf[0]);
  cudaFree(s->buf[1]);
  cudaFree(s->c);
  cudaFree(s->d);
  delete s;
}

}  // namespace

extern "C" tde_status tde_stream_create(tde_ctx* ctx, const float* y, int64_t ny, int bits, int engine,
                                        int64_t max_chunk, tde_stream_t stream, tde_stream** out) {
  ApiRange nvtx_range(__func__);
  if (!ctx) return TDE_ERR_INVALID;
  if (!y || !out) return set_err(ctx, TDE_ERR_INVALID, "null pointer");
  *out = nullptr;
  if (bits != 1)
    return set_err(ctx, TDE_ERR_UNSUPPORTED,
                   "streaming needs the pointwise sign quantizer (bits 1): the rank quantizer's "
                   "thresholds are order statistics of the whole signal");
  if (ny <= 0 || max_chunk <= 0) return set_err(ctx, TDE_ERR_INVALID, "ny and max_chunk must be positive");
  if (ny > INT32_MAX || max_chunk > INT32_MAX)
    return set_err(ctx, TDE_ERR_UNSUPPORTED, "ny and max_chunk must stay below 2^31");
  if (engine < TDE_ENGINE_AUTO || engine > TDE_ENGINE_NTT)
    return set_err(ctx, TDE_ERR_INVALID, "unknown engine %d", engine);
  DeviceGuard g(ctx->device);
  tde_stream* s = new tde_stream();
  s->ctx = ctx, s->bits = bits, s->engine = engine, s->ny = ny, s->max_chunk = max_chunk;
  const size_t nbuf = (size_t)(ny - 1 + max_chunk);
  cudaError_t e = cudaMalloc(&s->qy, (size_t)ny);
  if (e == cudaSuccess) e = cudaMalloc(&s->buf[0], nbuf);
  if (e == cudaSuccess) e = cudaMalloc(&s->buf[1], nbuf);
  if (e == cudaSuccess) e = cudaMalloc(&s->c, sizeof(int64_t) * (size_t)max_chunk);
  if (e == cudaSuccess) e = cudaMalloc(&s->d, 5 * sizeof(int64_t));
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d, 0, 5 * sizeof(int64_t), st);
  if (e != cudaSuccess) {
    stream_free(s);
    return cuda_err(ctx, e, "stream create");
  }
  const tde_status q = tde_quantize(ctx, y, ny, bits, s->qy, stream);
  if (q != TDE_OK) {
    stream_free(s);
    return q;
  }
  *out = s;
  return TDE_OK;
}

extern "C" tde_status tde_stream_push(tde_stream* s, const float* x, int64_t n, tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  if (!s) return TDE_ERR_INVALID;
  tde_ctx* ctx = s->ctx;
  if (n == 0) return TDE_OK;
  if (!x) return set_err(ctx, TDE_ERR_INVALID, "null pointer");
  if (n < 0 || n > s->max_chunk)
    return set_err(ctx, TDE_ERR_INVALID, "chunk of %lld samples: at most max_chunk = %lld", (long long)n,
                   (long long)s->max_chunk);
  DeviceGuard g(ctx->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int8_t* b = s->buf[s->cur];
  tde_status r = tde_quantize(ctx, x, n, s->bits, b + s->carry, stream);
  if (r != TDE_OK) return r;
  const int64_t nb = s->carry + n, base = s->consumed - s->carry;  // base: position of b[0] in x
  if (nb >= s->ny) {
    // the template wholly inside b: tau in [-(nb - ny), 0], position base - tau
    const int64_t lo = -(nb - s->ny);
    r = tde_xcorr_int(ctx, b, nb, s->qy, s->ny, s->bits, lo, 0, s->engine, s->c, TDE_I64, stream);
    if (r == TDE_OK) r = tde_argmax(ctx, s->c, TDE_I64, lo, nb - s->ny + 1, s->d, s->d + 1, stream);
    if (r != TDE_OK) return r;
    k_stream_fold<<<1, 1, 0, st>>>(s->d, base);
    TDE_COUNT_LAUNCH(1);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_err(ctx, e, "stream fold");
  }
  // the last ny - 1 levels become the other buffer's carry
  const int64_t keep = nb < s->ny - 1 ? nb : s->ny - 1;
  if (keep > 0) {
    const cudaError_t e = cudaMemcpyAsync(s->buf[s->cur ^ 1], b + nb - keep, (size_t)keep,
                                          cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_err(ctx, e, "stream carry");
  }
  s->cur ^= 1;
  s->carry = keep;
  s->consumed += n;
  return TDE_OK;
}

extern "C" tde_status tde_stream_best(tde_stream* s, int64_t* lag_out, int64_t* val_out, int* found,
                                      tde_stream_t stream) {
  ApiRange nvtx_range(__func__);
  if (!s) return TDE_ERR_INVALID;
  if (found) *found = s->consumed >= s->ny ? 1 : 0;
  if (s->consumed < s->ny || (!lag_out && !val_out)) return TDE_OK;
  DeviceGuard g(s->ctx->device);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaSuccess;
  if (lag_out) e = cudaMemcpyAsync(lag_out, s->d + 3, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
  if (e == cudaSuccess && val_out) e = cudaMemcpyAsync(val_out, s->d + 4, sizeof(int64_t), cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? TDE_OK : cuda_err(s->ctx, e, "stream best");
}

extern "C" tde_status tde_stream_destroy(tde_stream* s) {
  if (!s) return TDE_OK;
  {
    DeviceGuard g(s->ctx->device);
    cudaDeviceSynchronize();  // no push of this stream may still be running
  }
  stream_free(s);
  return TDE_OK;
}
