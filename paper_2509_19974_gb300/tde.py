"""Thin Python binding of libtde (include/tde.h) -- argument marshalling only.

Every step of the estimator runs in libtde's CUDA kernels; torch supplies
device memory (``Tensor.data_ptr()``) and the current CUDA stream.  There is
no CPU fallback: if libtde.so is missing or no GPU is present, the calls raise.

The functions keep the C names (``tde_quantize`` ...) and take a
:class:`Context`; :class:`Context` also offers them as methods without the
prefix.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libtde.so")

TDE_OK, TDE_ERR_INVALID, TDE_ERR_OVERFLOW, TDE_ERR_UNSUPPORTED, TDE_ERR_CUDA, TDE_ERR_TIMEOUT = range(6)
STATUS_NAMES = {0: "TDE_OK", 1: "TDE_ERR_INVALID", 2: "TDE_ERR_OVERFLOW", 3: "TDE_ERR_UNSUPPORTED",
                4: "TDE_ERR_CUDA", 5: "TDE_ERR_TIMEOUT"}
ENGINES = {"auto": 0, "popc": 1, "mma": 2, "ntt": 3}
TDE_I32, TDE_I64, TDE_F32, TDE_I8 = 0, 1, 2, 3

# Every symbol include/tde.h declares.
EXPORTS = ("tde_ctx_create", "tde_ctx_destroy", "tde_ctx_sync", "tde_last_error",
           "tde_ctx_set_profiling", "tde_ctx_set_ntt_primes", "tde_selftest_wait_timeout", "tde_measure_peaks", "tde_ctx_read_profile", "tde_pick_engine", "tde_quantize",
           "tde_quantize_noalloc", "tde_quantize_batch", "tde_xcorr_int", "tde_argmax", "tde_xcorr_fft32",
           "tde_estimate", "tde_estimate_batch", "tde_batch_create", "tde_batch_run",
           "tde_batch_destroy", "tde_model_param_count", "tde_model_create", "tde_model_destroy",
           "tde_model_get", "tde_model_set", "tde_train_step", "tde_propose",
           "tde_estimate_learned", "tde_synth_pairs", "tde_autotune", "tde_autotune_table",
           "tde_autotune_load", "tde_ctx_pick_engine", "tde_xcorr_windows",
           "tde_learned_create", "tde_learned_run", "tde_learned_destroy", "tde_refine",
           "tde_stream_create", "tde_stream_push", "tde_stream_best", "tde_stream_destroy")


class TdeError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class PairDesc(ctypes.Structure):
    _fields_ = [("x", ctypes.c_void_p), ("y", ctypes.c_void_p), ("nx", ctypes.c_int64),
                ("ny", ctypes.c_int64), ("lag_min", ctypes.c_int64), ("lag_max", ctypes.c_int64)]


class TuneEntry(ctypes.Structure):
    _fields_ = [("bits", ctypes.c_int32), ("log2_n", ctypes.c_int32), ("log2_lags", ctypes.c_int32),
                ("engine", ctypes.c_int32), ("ns_per_pair", ctypes.c_float * 4)]


_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libtde.so (built by ``paper_2509_19974_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libtde.so not found at {path}: run paper_2509_19974_gb300.build.build()")
    lib = ctypes.CDLL(path)
    i64, p, i32, f32 = ctypes.c_int64, ctypes.c_void_p, ctypes.c_int, ctypes.c_float
    st = ctypes.c_int
    sig = {
        "tde_ctx_create": ([i32, ctypes.POINTER(p)], st),
        "tde_ctx_destroy": ([p], st),
        "tde_ctx_sync": ([p, p], st),
        "tde_last_error": ([p], ctypes.c_char_p),
        "tde_ctx_set_profiling": ([p, i32], st),
        "tde_ctx_set_ntt_primes": ([p, i32], st),
        "tde_selftest_wait_timeout": ([p, p], st),
        "tde_measure_peaks": ([i32, p], st),
        "tde_ctx_read_profile": ([p, p, p, p], st),
        "tde_pick_engine": ([i32, i64, i64, i64], i32),
        "tde_quantize": ([p, p, i64, i32, p, p], st),
        "tde_quantize_noalloc": ([p, i64, i32, i32, p, p, p], st),
        "tde_quantize_batch": ([p, p, i64, i32, i32, p, p], st),
        "tde_xcorr_int": ([p, p, i64, p, i64, i32, i64, i64, i32, p, i32, p], st),
        "tde_argmax": ([p, p, i32, i64, i64, p, p, p], st),
        "tde_xcorr_fft32": ([p, p, p, i32, i64, i64, i32, i64, i64, p, p], st),
        "tde_estimate": ([p, p, i64, p, i64, i32, i64, i64, i32, p, p, p], st),
        "tde_estimate_batch": ([p, ctypes.POINTER(PairDesc), i32, i32, i32, p, p, p, p], st),
        "tde_batch_create": ([p, ctypes.POINTER(PairDesc), i32, i32, i32, p, p, p,
                              ctypes.POINTER(p)], st),
        "tde_batch_run": ([p, p], st),
        "tde_batch_destroy": ([p], st),
        "tde_model_param_count": ([], i64),
        "tde_model_create": ([p, i64, ctypes.c_uint64, ctypes.POINTER(p)], st),
        "tde_model_destroy": ([p], st),
        "tde_model_get": ([p, p, p, p, p, p], st),
        "tde_model_set": ([p, p, p, p, i64], st),
        "tde_train_step": ([p, p, p, i32, p, f32, f32, p, p], st),
        "tde_propose": ([p, p, p, i32, p, p, p], st),
        "tde_estimate_learned": ([p, p, p, p, i32, i32, f32, p, p, p, p], st),
        "tde_synth_pairs": ([p, ctypes.c_uint64, i64, i32, i64, i64, f32, f32, f32, f32, p, p, p,
                             p], st),
        "tde_autotune": ([p, i32, p, p, i32, i32], st),
        "tde_autotune_table": ([p, p, i32, p], st),
        "tde_autotune_load": ([p, p, i32], st),
        "tde_ctx_pick_engine": ([p, i32, i64, i64, i64], i32),
        "tde_xcorr_windows": ([p, p, i64, i32, i32, p, p, p], st),
        "tde_learned_create": ([p, p, p, p, i32, i32, f32, p, p, p, ctypes.POINTER(p)], st),
        "tde_learned_run": ([p, p], st),
        "tde_learned_destroy": ([p], st),
        "tde_refine": ([p, p, i64, p, i64, p, i32, i64, i64, p, p], st),
        "tde_stream_create": ([p, p, i64, i32, i32, i64, p, ctypes.POINTER(p)], st),
        "tde_stream_push": ([p, p, i64, p], st),
        "tde_stream_best": ([p, p, p, ctypes.POINTER(i32), p], st),
        "tde_stream_destroy": ([p], st),
    }
    for name, (args, res) in sig.items():
        fn = getattr(lib, name)
        fn.argtypes, fn.restype = args, res
    _lib = lib
    return lib


def _stream(stream) -> int:
    if stream is None:
        stream = torch.cuda.current_stream()
    return int(stream.cuda_stream) if hasattr(stream, "cuda_stream") else int(stream)


def _need(t: torch.Tensor, dtype, name: str):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


def _engine(e) -> int:
    return ENGINES[e] if isinstance(e, str) else int(e)


class Peaks(ctypes.Structure):
    """tde_peaks: issue rates per SM per SM clock (see tde_measure_peaks)."""
    _fields_ = [("sm_count", ctypes.c_int), ("popc_per_sm_clk", ctypes.c_double),
                ("imad_per_sm_clk", ctypes.c_double), ("e4m3_mac_per_sm_clk", ctypes.c_double),
                ("e2m1_mac_per_sm_clk", ctypes.c_double)]


def measure_peaks(device: int = 0) -> dict:
    """tde_measure_peaks on `device`: POPC, IMAD, E4M3 and E2M1 tensor-core MAC
    rates per SM per clock, and the SM count."""
    pk = Peaks()
    s = load().tde_measure_peaks(int(device), ctypes.addressof(pk))
    if s != TDE_OK:
        raise TdeError(s, "tde_measure_peaks failed")
    return {f: getattr(pk, f) for f, _ in Peaks._fields_}


class Context:
    """Owns a ``tde_ctx`` on one device (workspace, staging, status word)."""

    def __init__(self, device: int | None = None):
        self.lib = load()
        if device is None:
            device = torch.cuda.current_device()
        self.device = int(device)
        h = ctypes.c_void_p()
        s = self.lib.tde_ctx_create(self.device, ctypes.byref(h))
        if s != TDE_OK:
            raise TdeError(s, f"tde_ctx_create(device={device}) failed")
        self.handle = h

    def close(self):
        """Releases the context (its workspace, plans' tables and status word)."""
        if getattr(self, "handle", None):
            self.lib.tde_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def check(self, status: int):
        """Raises TdeError (with the context's last error text) for a non-OK status."""
        if status != TDE_OK:
            msg = self.lib.tde_last_error(self.handle)
            raise TdeError(status, msg.decode() if msg else "")

    # --- methods mirroring the C entry points -----------------------------
    def sync(self, stream=None):
        """Waits for `stream` and raises TdeError if a kernel flagged NaN/Inf
        input, an out-of-range level or a timed-out wait since the last sync."""
        self.check(self.lib.tde_ctx_sync(self.handle, _stream(stream)))

    def set_profiling(self, enable: bool):
        """Brackets every engine-kernel launch with CUDA events (read_profile)."""
        self.check(self.lib.tde_ctx_set_profiling(self.handle, int(bool(enable))))

    def selftest_wait_timeout(self, stream=None):
        """Launches a CTA whose bounded waits run out (about 4 s); the next
        sync raises TdeError with status TDE_ERR_TIMEOUT."""
        self.check(self.lib.tde_selftest_wait_timeout(self.handle, _stream(stream)))

    def set_ntt_primes(self, nprimes: int):
        """0: the NTT engine uses one prime wherever the values fit it; 2: always
        two primes and CRT (for plans made after the call)."""
        self.check(self.lib.tde_ctx_set_ntt_primes(self.handle, int(nprimes)))

    def read_profile(self):
        """(kernel launches, engine-kernel launches, engine ms) since last read."""
        k, e, ms = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_double()
        self.check(self.lib.tde_ctx_read_profile(self.handle, ctypes.byref(k), ctypes.byref(e),
                                                 ctypes.byref(ms)))
        return int(k.value), int(e.value), float(ms.value)

    def quantize(self, x, bits, q_out=None, stream=None):
        """See tde_quantize."""
        return tde_quantize(self, x, bits, q_out, stream)

    def xcorr_int(self, qx, qy, bits, lag_min=None, lag_max=None, engine="auto",
                  dtype=torch.int32, c_out=None, stream=None):
        """See tde_xcorr_int."""
        return tde_xcorr_int(self, qx, qy, bits, lag_min, lag_max, engine, dtype, c_out, stream)

    def argmax(self, c, lag_min, stream=None):
        """See tde_argmax."""
        return tde_argmax(self, c, lag_min, stream)

    def refine(self, x, y, c, lag_min, stream=None):
        """See tde_refine."""
        return tde_refine(self, x, y, c, lag_min, stream)

    def xcorr_fft32(self, x, y, lag_min=None, lag_max=None, c_out=None, stream=None):
        """See tde_xcorr_fft32."""
        return tde_xcorr_fft32(self, x, y, lag_min, lag_max, c_out, stream)

    def estimate(self, x, y, bits, lag_min=None, lag_max=None, engine="auto", stream=None):
        """See tde_estimate."""
        return tde_estimate(self, x, y, bits, lag_min, lag_max, engine, stream)

    def estimate_batch(self, xs, ys, bits, lag_mins=None, lag_maxs=None, engine="auto",
                       c_out=None, stream=None):
        """See tde_estimate_batch."""
        return tde_estimate_batch(self, xs, ys, bits, lag_mins, lag_maxs, engine, c_out, stream)

    # --- autotuner ---------------------------------------------------------
    def autotune(self, bits: int, points, reps: int = 3):
        """Times every exact engine at each (n, lag_count) of ``points`` and
        makes AUTO use the fastest (nearest point in log2 n, log2 lags).
        Returns the context's table (``autotune_table``)."""
        n = (ctypes.c_int64 * len(points))(*[int(p[0]) for p in points])
        lags = (ctypes.c_int64 * len(points))(*[int(p[1]) for p in points])
        self.check(self.lib.tde_autotune(self.handle, int(bits), ctypes.addressof(n),
                                         ctypes.addressof(lags), len(points), int(reps)))
        return self.autotune_table()

    def autotune_table(self):
        """The table as a list of dicts (bits, log2_n, log2_lags, engine,
        ns_per_pair {engine name: ns or None})."""
        cnt = ctypes.c_int()
        self.check(self.lib.tde_autotune_table(self.handle, None, 0, ctypes.byref(cnt)))
        arr = (TuneEntry * max(cnt.value, 1))()
        self.check(self.lib.tde_autotune_table(self.handle, ctypes.addressof(arr), cnt.value,
                                               ctypes.byref(cnt)))
        return [entry_to_dict(arr[i]) for i in range(cnt.value)]

    def pick_engine(self, bits: int, nx: int, ny: int, lag_count: int) -> str:
        """Name of the engine AUTO runs for such a pair on this context."""
        e = self.lib.tde_ctx_pick_engine(self.handle, int(bits), int(nx), int(ny), int(lag_count))
        if e < 0:
            raise ValueError("invalid arguments")
        return ENGINE_NAMES[e]

    def autotune_load(self, table):
        """Installs a table (as returned by ``autotune_table``)."""
        arr = (TuneEntry * max(len(table), 1))()
        for i, d in enumerate(table):
            arr[i] = dict_to_entry(d)
        self.check(self.lib.tde_autotune_load(self.handle, ctypes.addressof(arr), len(table)))


def entry_to_dict(e: TuneEntry) -> dict:
    return {"bits": int(e.bits), "log2_n": int(e.log2_n), "log2_lags": int(e.log2_lags),
            "engine": ENGINE_NAMES[int(e.engine)],
            "ns_per_pair": {ENGINE_NAMES[k]: (float(e.ns_per_pair[k]) if e.ns_per_pair[k] >= 0
                                              else None) for k in (1, 2, 3)}}


def dict_to_entry(d: dict) -> TuneEntry:
    e = TuneEntry()
    e.bits, e.log2_n, e.log2_lags = int(d["bits"]), int(d["log2_n"]), int(d["log2_lags"])
    e.engine = _engine(d["engine"])
    e.ns_per_pair[0] = -1.0
    for name, v in d.get("ns_per_pair", {}).items():
        e.ns_per_pair[ENGINES[name]] = -1.0 if v is None else float(v)
    return e


# Points the default autotune measures: min length 2^k and lag counts from a
# narrow search window up to the full range.
DEFAULT_TUNE_POINTS = tuple((1 << k, min(lags, 2 * (1 << k) - 1))
                            for k in (10, 12, 14, 16, 18, 20)
                            for lags in (256, 2048, 16384, 1 << 17, 1 << 21)
                            if lags <= 2 * (1 << k) - 1 or lags == 1 << 21)


def tune_cache_key(device: int) -> str:
    """Key of a cached table: device name, SM count, CUDA runtime and the
    library digest (a rebuilt library re-tunes)."""
    prop = torch.cuda.get_device_properties(device)
    digest = ""
    stamp = os.path.join(_PKG, "_build", "stamp")
    if os.path.exists(stamp):
        with open(stamp) as f:
            digest = f.read().strip()[:16]
    return f"{prop.name}|sm{prop.multi_processor_count}|cuda{torch.version.cuda}|{digest}"


def autotune_cached(ctx: Context, bits_list=(1, 2, 4), points=DEFAULT_TUNE_POINTS,
                    path: str | None = None, reps: int = 3):
    """Loads the table for this device from the JSON cache at ``path``
    (default: ``$TDE_TUNE_CACHE`` or ~/.cache/tde_autotune.json), or measures
    it with ``Context.autotune`` and stores it there."""
    import json
    path = path or os.environ.get("TDE_TUNE_CACHE",
                                  os.path.join(os.path.expanduser("~"), ".cache",
                                               "tde_autotune.json"))
    key = tune_cache_key(ctx.device)
    cache = {}
    if os.path.exists(path):
        try:
            with open(path) as f:
                cache = json.load(f)
        except (OSError, ValueError):
            cache = {}
    table = cache.get(key)
    if table and {int(t["bits"]) for t in table} >= set(bits_list):
        ctx.autotune_load(table)
        return table
    for b in bits_list:
        ctx.autotune(b, points, reps)
    table = ctx.autotune_table()
    cache[key] = table
    os.makedirs(os.path.dirname(os.path.abspath(path)), exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1)
    os.replace(tmp, path)
    return table


ENGINE_NAMES = {v: k for k, v in ENGINES.items()}


def pick_engine(bits: int, nx: int, ny: int, lag_count: int) -> str:
    """Name of the engine TDE_ENGINE_AUTO runs for such a pair."""
    e = load().tde_pick_engine(int(bits), int(nx), int(ny), int(lag_count))
    if e < 0:
        raise ValueError("invalid arguments")
    return ENGINE_NAMES[e]


def full_lags(nx: int, ny: int):
    """Every lag with a non-empty overlap: (-(nx - 1), ny - 1)."""
    return -(nx - 1), ny - 1


def tde_quantize(ctx: Context, x: torch.Tensor, bits: int, q_out=None, stream=None):
    """Algorithm 1's quantization of one FP32 signal on its device: bits = 1 is
    sign(x) with sign(0) = 0; bits = 2, 4 the sign-magnitude rank quantizer
    (2^bits - 1 levels, thresholds exact order statistics of |x|).  Returns
    int8 levels [n] (or fills q_out); asynchronous on `stream`."""
    _need(x, torch.float32, "x")
    if q_out is None:
        q_out = torch.empty(x.numel(), dtype=torch.int8, device=x.device)
    _need(q_out, torch.int8, "q_out")
    ctx.check(ctx.lib.tde_quantize(ctx.handle, x.data_ptr(), x.numel(), int(bits),
                                   q_out.data_ptr(), _stream(stream)))
    return q_out


def tde_quantize_batch(ctx: Context, x: torch.Tensor, bits: int, q_out=None, stream=None):
    """x: [nsig, n] float32 -> [nsig, n] int8 in one call."""
    _need(x, torch.float32, "x")
    nsig, n = x.shape
    if q_out is None:
        q_out = torch.empty((nsig, n), dtype=torch.int8, device=x.device)
    _need(q_out, torch.int8, "q_out")
    ctx.check(ctx.lib.tde_quantize_batch(ctx.handle, x.data_ptr(), n, nsig, int(bits),
                                         q_out.data_ptr(), _stream(stream)))
    return q_out


NOALLOC_MAX_SIGNALS = 16


def tde_quantize_noalloc(x: torch.Tensor, bits: int, q_out=None, status_out=None, stream=None):
    """Allocation-free quantizer (no context): x is [nsig, n] float32 (nsig <=
    16) or [n]; returns (q [nsig, n] int8, status uint32 tensor of one word,
    bit 0 = NaN/Inf seen).  Output tensors may be passed in preallocated."""
    _need(x, torch.float32, "x")
    if x.dim() not in (1, 2):
        raise ValueError("x must be [n] or [nsig, n]")
    nsig, n = (1, x.numel()) if x.dim() == 1 else (x.shape[0], x.shape[1])
    if q_out is None:
        q_out = torch.empty(x.shape, dtype=torch.int8, device=x.device)
    if status_out is None:
        status_out = torch.empty(1, dtype=torch.int32, device=x.device)
    _need(q_out, torch.int8, "q_out")
    if q_out.shape != x.shape or q_out.device != x.device:
        raise ValueError("q_out must have x's shape and device")
    if status_out.dtype not in (torch.int32, torch.uint32) or status_out.numel() < 1 \
            or status_out.device != x.device:
        raise ValueError("status_out must be a 32-bit integer tensor on x's device")
    with torch.cuda.device(x.device):  # the library runs on the current device
        s = load().tde_quantize_noalloc(x.data_ptr(), int(n), int(nsig), int(bits), q_out.data_ptr(),
                                        status_out.data_ptr(), _stream(stream))
    if s != TDE_OK:
        raise TdeError(s, "tde_quantize_noalloc failed")
    return q_out, status_out


def tde_xcorr_int(ctx: Context, qx, qy, bits, lag_min=None, lag_max=None, engine="auto",
                  dtype=torch.int32, c_out=None, stream=None):
    """Exact integer cross-correlation (Eq. 1) of int8 levels:
    c[i] = sum_n qx[n] qy[n + tau], tau = lag_min + i, over [lag_min, lag_max]
    (default every lag with overlap).  engine: "auto", "popc", "mma" or
    "ntt"; dtype int32 (rejected where it could overflow) or int64.
    Asynchronous on `stream`."""
    _need(qx, torch.int8, "qx")
    _need(qy, torch.int8, "qy")
    lo, hi = full_lags(qx.numel(), qy.numel())
    lag_min = lo if lag_min is None else int(lag_min)
    lag_max = hi if lag_max is None else int(lag_max)
    count = lag_max - lag_min + 1
    if c_out is None:
        c_out = torch.empty(max(count, 0), dtype=dtype, device=qx.device)
    _need(c_out, dtype, "c_out")
    code = TDE_I64 if dtype == torch.int64 else TDE_I32
    ctx.check(ctx.lib.tde_xcorr_int(ctx.handle, qx.data_ptr(), qx.numel(), qy.data_ptr(),
                                    qy.numel(), int(bits), lag_min, lag_max, _engine(engine),
                                    c_out.data_ptr(), code, _stream(stream)))
    return c_out


def tde_argmax(ctx: Context, c, lag_min, stream=None):
    """The maximiser of c (int32 or int64, element i = lag lag_min + i) by
    the tie rule: the largest value, then the smallest |tau|, then the
    smallest tau.  Returns device tensors (lag [1], value [1]) int64."""
    if c.dtype not in (torch.int32, torch.int64):
        raise TypeError("c must be int32 or int64")
    _need(c, c.dtype, "c")
    lag = torch.empty(1, dtype=torch.int64, device=c.device)
    val = torch.empty(1, dtype=torch.int64, device=c.device)
    code = TDE_I64 if c.dtype == torch.int64 else TDE_I32
    ctx.check(ctx.lib.tde_argmax(ctx.handle, c.data_ptr(), code, int(lag_min), c.numel(),
                                 lag.data_ptr(), val.data_ptr(), _stream(stream)))
    return lag, val


REFINED_FIELDS = ("lag", "value", "lag_lo", "lag_hi", "n_int_ties", "n_ties", "r", "frac")


def tde_refine(ctx: Context, x, y, c, lag_min, stream=None) -> dict:
    """Algorithm 1's last steps for c (the integer correlation of the
    quantized x, y; element i = lag lag_min + i): the tied set of maxima
    re-ranked by the real cross-correlation of x and y, its representative,
    bounds and sizes, the real value and the sub-sample offset (synchronises
    the stream to read the result)."""
    _need(x, torch.float32, "x")
    _need(y, torch.float32, "y")
    if c.dtype not in (torch.int32, torch.int64):
        raise TypeError("c must be int32 or int64")
    _need(c, c.dtype, "c")
    out = torch.zeros(8, dtype=torch.int64, device=c.device)  # one tde_refined (64 bytes)
    code = TDE_I64 if c.dtype == torch.int64 else TDE_I32
    ctx.check(ctx.lib.tde_refine(ctx.handle, x.data_ptr(), x.numel(), y.data_ptr(), y.numel(),
                                 c.data_ptr(), code, int(lag_min), c.numel(), out.data_ptr(),
                                 _stream(stream)))
    ctx.sync(stream)
    h = out.cpu()
    ints = [int(v) for v in h[:6]]
    dbl = h[6:].numpy().view(np.float64)
    return dict(zip(REFINED_FIELDS, ints + [float(dbl[0]), float(dbl[1])]))


def tde_xcorr_fft32(ctx: Context, x, y, lag_min=None, lag_max=None, c_out=None, stream=None):
    """FP32 FFT comparator.  x: [npairs, nx], y: [npairs, ny] (float32 or
    int8, or 1-D for one pair); returns [npairs, count] float32."""
    if x.dtype not in (torch.float32, torch.int8) or y.dtype != x.dtype:
        raise TypeError("x and y must both be float32 or both int8")
    _need(x, x.dtype, "x")
    _need(y, y.dtype, "y")
    x2, y2 = (x.view(1, -1), y.view(1, -1)) if x.dim() == 1 else (x, y)
    npairs, nx, ny = x2.shape[0], x2.shape[1], y2.shape[1]
    lo, hi = full_lags(nx, ny)
    lag_min = lo if lag_min is None else int(lag_min)
    lag_max = hi if lag_max is None else int(lag_max)
    if c_out is None:
        c_out = torch.empty((npairs, lag_max - lag_min + 1), dtype=torch.float32, device=x.device)
    _need(c_out, torch.float32, "c_out")
    code = TDE_I8 if x.dtype == torch.int8 else TDE_F32
    ctx.check(ctx.lib.tde_xcorr_fft32(ctx.handle, x2.data_ptr(), y2.data_ptr(), code, nx, ny,
                                      npairs, lag_min, lag_max, c_out.data_ptr(), _stream(stream)))
    return c_out


def tde_estimate(ctx: Context, x, y, bits, lag_min=None, lag_max=None, engine="auto", stream=None):
    """Algorithm 1 for one FP32 pair: quantize both, correlate exactly over
    [lag_min, lag_max] (default every lag), take the tie-ruled argmax.
    Returns device tensors (lag [1], value [1]) int64; asynchronous."""
    _need(x, torch.float32, "x")
    _need(y, torch.float32, "y")
    lo, hi = full_lags(x.numel(), y.numel())
    lag_min = lo if lag_min is None else int(lag_min)
    lag_max = hi if lag_max is None else int(lag_max)
    lag = torch.empty(1, dtype=torch.int64, device=x.device)
    val = torch.empty(1, dtype=torch.int64, device=x.device)
    ctx.check(ctx.lib.tde_estimate(ctx.handle, x.data_ptr(), x.numel(), y.data_ptr(), y.numel(),
                                   int(bits), lag_min, lag_max, _engine(engine), lag.data_ptr(),
                                   val.data_ptr(), _stream(stream)))
    return lag, val


def make_descs(xs, ys, lag_mins=None, lag_maxs=None):
    """Pair descriptors from lists of 1-D float32 CUDA tensors (or the rows of
    two 2-D tensors).  Default lag range: every lag with a nonempty overlap."""
    n = len(xs)
    descs = (PairDesc * n)()
    for i in range(n):
        x, y = xs[i], ys[i]
        _need(x, torch.float32, f"xs[{i}]")
        _need(y, torch.float32, f"ys[{i}]")
        lo, hi = full_lags(x.numel(), y.numel())
        descs[i] = PairDesc(x.data_ptr(), y.data_ptr(), x.numel(), y.numel(),
                            lo if lag_mins is None else int(lag_mins[i]),
                            hi if lag_maxs is None else int(lag_maxs[i]))
    return descs


def tde_estimate_batch(ctx: Context, xs, ys, bits, lag_mins=None, lag_maxs=None, engine="auto",
                       c_out=None, stream=None, descs=None):
    """Returns (lags, values) as int64 CUDA tensors of length npairs."""
    if descs is None:
        descs = make_descs(xs, ys, lag_mins, lag_maxs)
    n = len(descs)
    dev = torch.device("cuda", ctx.device)
    lags = torch.empty(n, dtype=torch.int64, device=dev)
    vals = torch.empty(n, dtype=torch.int64, device=dev)
    cptr = None
    if c_out is not None:
        _need(c_out, torch.int32, "c_out")
        cptr = c_out.data_ptr()
    ctx.check(ctx.lib.tde_estimate_batch(ctx.handle, descs, n, int(bits), _engine(engine), cptr,
                                         lags.data_ptr(), vals.data_ptr(), _stream(stream)))
    return lags, vals


class Batch:
    """A planned batch (tde_batch_create): the whole estimate step for fixed
    descriptors captured in a CUDA graph; run() replays it.  Refill the input
    tensors the descriptors point to between runs; results land in .lags,
    .vals (and c_out if given)."""

    def __init__(self, ctx: Context, xs, ys, bits, lag_mins=None, lag_maxs=None, engine="auto",
                 c_out=None, descs=None):
        self.ctx = ctx
        self.descs = descs if descs is not None else make_descs(xs, ys, lag_mins, lag_maxs)
        n = len(self.descs)
        dev = torch.device("cuda", ctx.device)
        self.lags = torch.empty(n, dtype=torch.int64, device=dev)
        self.vals = torch.empty(n, dtype=torch.int64, device=dev)
        self.c_out = c_out
        cptr = None
        if c_out is not None:
            _need(c_out, torch.int32, "c_out")
            cptr = c_out.data_ptr()
        h = ctypes.c_void_p()
        ctx.check(ctx.lib.tde_batch_create(ctx.handle, self.descs, n, int(bits), _engine(engine),
                                           cptr, self.lags.data_ptr(), self.vals.data_ptr(),
                                           ctypes.byref(h)))
        self.handle = h

    def run(self, stream=None):
        self.ctx.check(self.ctx.lib.tde_batch_run(self.handle, _stream(stream)))
        return self.lags, self.vals

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.tde_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------ learned lag proposal

def synth_pairs(ctx: Context, seed: int, first: int, npairs: int, n: int, dmax: int,
                ar=(0.0, 0.98), snr_db=(-5.0, 30.0), stream=None):
    """Device-generated shifted pairs: (x [npairs, n], y [npairs, n], shift)."""
    dev = torch.device("cuda", ctx.device)
    x = torch.empty((npairs, n), dtype=torch.float32, device=dev)
    y = torch.empty((npairs, n), dtype=torch.float32, device=dev)
    d = torch.empty(npairs, dtype=torch.int64, device=dev)
    ctx.check(ctx.lib.tde_synth_pairs(ctx.handle, int(seed), int(first), int(npairs), int(n),
                                      int(dmax), float(ar[0]), float(ar[1]), float(snr_db[0]),
                                      float(snr_db[1]), x.data_ptr(), y.data_ptr(), d.data_ptr(),
                                      _stream(stream)))
    return x, y, d


def tde_xcorr_windows(ctx: Context, q2: torch.Tensor, bits: int, centres: torch.Tensor,
                      c_out=None, stream=None):
    """Exact correlation in 8 windows per pair.  q2: [2P, n] int8 (pair p at
    rows 2p, 2p+1); centres: [P, 8] int32 (device).  Returns [P, 8, 257]
    int32 with [p, w, i] = c_p[centres[p, w] - 128 + i] (0 outside the lags)."""
    _need(q2, torch.int8, "q2")
    _need(centres, torch.int32, "centres")
    npairs, n = q2.shape[0] // 2, q2.shape[1]
    if centres.shape != (npairs, 8):
        raise ValueError("centres must be [npairs, 8]")
    if c_out is None:
        c_out = torch.empty((npairs, 8, 257), dtype=torch.int32, device=q2.device)
    _need(c_out, torch.int32, "c_out")
    ctx.check(ctx.lib.tde_xcorr_windows(ctx.handle, q2.data_ptr(), n, npairs, int(bits),
                                        centres.data_ptr(), c_out.data_ptr(), _stream(stream)))
    return c_out


class LearnedBatch:
    """tde_learned_create: the learned estimate of fixed x, y buffers ([P, n]
    float32, refilled between runs) captured in a CUDA graph; run() replays
    it.  Results land in .lags, .vals and .fallback."""

    def __init__(self, model, x: torch.Tensor, y: torch.Tensor, bits: int = 2, theta: float = 0.5):
        _need(x, torch.float32, "x")
        _need(y, torch.float32, "y")
        self.model, self.ctx = model, model.ctx
        self.x, self.y = x, y
        npairs = x.shape[0]
        self.lags = torch.empty(npairs, dtype=torch.int64, device=x.device)
        self.vals = torch.empty(npairs, dtype=torch.int64, device=x.device)
        self.fallback = torch.empty(npairs, dtype=torch.int32, device=x.device)
        h = ctypes.c_void_p()
        self.ctx.check(self.ctx.lib.tde_learned_create(
            self.ctx.handle, model.handle, x.data_ptr(), y.data_ptr(), npairs, int(bits),
            float(theta), self.lags.data_ptr(), self.vals.data_ptr(), self.fallback.data_ptr(),
            ctypes.byref(h)))
        self.handle = h

    def run(self, stream=None):
        self.ctx.check(self.ctx.lib.tde_learned_run(self.handle, _stream(stream)))
        return self.lags, self.vals, self.fallback

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.tde_learned_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def interleave_q(qx: torch.Tensor, qy: torch.Tensor) -> torch.Tensor:
    """[P, n] int8 x and y -> [2P, n] with pair p at rows 2p (x), 2p+1 (y)."""
    return torch.stack([qx, qy], dim=1).reshape(-1, qx.shape[1]).contiguous()


class Model:
    """A lag-proposal CNN on the device (tde_model_*)."""

    def __init__(self, ctx: Context, n: int, seed: int = 0):
        self.ctx, self.n = ctx, int(n)
        self.lib = load()
        h = ctypes.c_void_p()
        ctx.check(self.lib.tde_model_create(ctx.handle, self.n, int(seed), ctypes.byref(h)))
        self.handle = h
        self.count = int(self.lib.tde_model_param_count())

    def close(self):
        if getattr(self, "handle", None):
            self.lib.tde_model_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def state(self):
        """Host copies of the parameters, AdamW moments, gradient and step."""
        import numpy as np
        arrs = [np.empty(self.count, np.float32) for _ in range(4)]
        step = ctypes.c_int64()
        s = self.lib.tde_model_get(self.handle, *[a.ctypes.data for a in arrs], ctypes.byref(step))
        if s != TDE_OK:
            raise TdeError(s, "tde_model_get failed")
        return {"params": arrs[0], "adam_m": arrs[1], "adam_v": arrs[2], "grad": arrs[3],
                "step": int(step.value)}

    def load_state(self, st):
        """Sets the parameters (and moments, step when given) from state()."""
        import numpy as np
        ps = np.ascontiguousarray(st["params"], np.float32)
        m = np.ascontiguousarray(st.get("adam_m", np.zeros_like(ps)), np.float32)
        v = np.ascontiguousarray(st.get("adam_v", np.zeros_like(ps)), np.float32)
        s = self.lib.tde_model_set(self.handle, ps.ctypes.data, m.ctypes.data, v.ctypes.data,
                                   int(st.get("step", 0)))
        if s != TDE_OK:
            raise TdeError(s, "tde_model_set failed")

    def save(self, path: str):
        """Parameters, AdamW moments and step count to an .npz (exact resume)."""
        import numpy as np
        st = self.state()
        np.savez(path, n=self.n, **{k: v for k, v in st.items()})

    def load(self, path: str):
        """Restores a checkpoint written by save() for the same signal length."""
        import numpy as np
        z = np.load(path)
        if int(z["n"]) != self.n:
            raise ValueError("checkpoint is for another signal length")
        self.load_state({k: z[k] for k in ("params", "adam_m", "adam_v", "step")})

    def train_step(self, q2: torch.Tensor, labels: torch.Tensor, lr: float, weight_decay=1e-4,
                   stream=None):
        """One deterministic AdamW step on pairs q2 [2P, n] int8 (pair p at rows
        2p, 2p + 1) against label lags [P] int64; returns the per-pair loss."""
        _need(q2, torch.int8, "q")
        _need(labels, torch.int64, "labels")
        npairs = q2.shape[0] // 2
        loss = torch.empty(npairs, dtype=torch.float32, device=q2.device)
        self.ctx.check(self.lib.tde_train_step(self.ctx.handle, self.handle, q2.data_ptr(), npairs,
                                               labels.data_ptr(), float(lr), float(weight_decay),
                                               loss.data_ptr(), _stream(stream)))
        return loss

    def propose(self, q2: torch.Tensor, stream=None):
        """Window centres [P, 8] int32 (lags, best first) and margins [P] (the
        softmax mass of the top 8 bins) for pairs q2 [2P, n] int8."""
        _need(q2, torch.int8, "q")
        npairs = q2.shape[0] // 2
        cent = torch.empty((npairs, 8), dtype=torch.int32, device=q2.device)
        marg = torch.empty(npairs, dtype=torch.float32, device=q2.device)
        self.ctx.check(self.lib.tde_propose(self.ctx.handle, self.handle, q2.data_ptr(), npairs,
                                            cent.data_ptr(), marg.data_ptr(), _stream(stream)))
        return cent, marg

    def estimate(self, x: torch.Tensor, y: torch.Tensor, bits: int = 2, theta: float = 0.5,
                 stream=None):
        """The learned estimate of pairs x, y [P, n] float32: the exact
        tie-ruled maximum over the proposal's 8 windows, or over every lag
        when the margin is below theta.  Returns (lags, values, fallback)."""
        _need(x, torch.float32, "x")
        _need(y, torch.float32, "y")
        npairs = x.shape[0]
        lags = torch.empty(npairs, dtype=torch.int64, device=x.device)
        vals = torch.empty(npairs, dtype=torch.int64, device=x.device)
        fb = torch.empty(npairs, dtype=torch.int32, device=x.device)
        self.ctx.check(self.lib.tde_estimate_learned(self.ctx.handle, self.handle, x.data_ptr(),
                                                     y.data_ptr(), npairs, int(bits), float(theta),
                                                     lags.data_ptr(), vals.data_ptr(),
                                                     fb.data_ptr(), _stream(stream)))
        return lags, vals, fb
