"""ctypes wrapper of ``oracle.c`` -- test infrastructure only (see package doc).

Every function follows the paper (arXiv 2509.19974) literally:
  quantize        Algorithm 1's quantization step (sign with sign(0)=0, Sec. 4.2; or
                  the sign-magnitude rank quantizer, Sec. 3.2 "any scheme").
  xcorr/xcorr_at  Eq. (1) on the quantized sequences, direct int64 sums.
  argmax          Algorithm 1's argmax step, ties -> smallest |tau| then tau.
  real_ccf        Eq. (1) on the original (unquantized) sequences, in float64.
  refine          Algorithm 1's last steps: the tied set of integer maxima,
                  re-ranked by the real cross-correlation when it holds several
                  lags, plus a parabolic sub-sample offset at its representative.
Pinned by tests/test_oracle_pins.py.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (-O2, OpenMP) into oracle/liboracle.so."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        i64, p = ctypes.c_int64, ctypes.c_void_p
        lib.oracle_quantize.argtypes = [p, i64, ctypes.c_int, p]
        lib.oracle_quantize.restype = ctypes.c_int
        lib.oracle_rank_thresholds.argtypes = [p, i64, ctypes.c_int, p]
        lib.oracle_rank_thresholds.restype = ctypes.c_int
        lib.oracle_xcorr.argtypes = [p, i64, p, i64, i64, i64, p]
        lib.oracle_xcorr.restype = None
        lib.oracle_xcorr_at.argtypes = [p, i64, p, i64, p, i64, p]
        lib.oracle_xcorr_at.restype = None
        lib.oracle_argmax.argtypes = [p, i64, i64, p, p]
        lib.oracle_argmax.restype = None
        lib.oracle_num_threads.argtypes = []
        lib.oracle_num_threads.restype = ctypes.c_int
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def full_lag_range(nx: int, ny: int) -> tuple[int, int]:
    """All lags with a nonempty overlap: [-(nx-1), ny-1]."""
    return -(nx - 1), ny - 1


def quantize(x: np.ndarray, bits: int) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    q = np.empty(x.shape[0], dtype=np.int8)
    rc = _load().oracle_quantize(_ptr(x), x.shape[0], int(bits), _ptr(q))
    if rc != 0:
        raise ValueError("oracle_quantize: invalid input (empty, bad bits, NaN or Inf)")
    return q


def rank_thresholds(x: np.ndarray, bits: int) -> np.ndarray:
    x = np.ascontiguousarray(x, dtype=np.float32)
    t = np.empty(8, dtype=np.float32)
    rc = _load().oracle_rank_thresholds(_ptr(x), x.shape[0], int(bits), _ptr(t))
    if rc != 0:
        raise ValueError("oracle_rank_thresholds: invalid input")
    return t[: (1 << (bits - 1)) - 1].copy()


def xcorr(qx: np.ndarray, qy: np.ndarray, lag_min: int | None = None,
          lag_max: int | None = None) -> np.ndarray:
    qx = np.ascontiguousarray(qx, dtype=np.int8)
    qy = np.ascontiguousarray(qy, dtype=np.int8)
    lo, hi = full_lag_range(qx.shape[0], qy.shape[0])
    lag_min = lo if lag_min is None else int(lag_min)
    lag_max = hi if lag_max is None else int(lag_max)
    c = np.empty(lag_max - lag_min + 1, dtype=np.int64)
    _load().oracle_xcorr(_ptr(qx), qx.shape[0], _ptr(qy), qy.shape[0], lag_min, lag_max, _ptr(c))
    return c


def xcorr_at(qx: np.ndarray, qy: np.ndarray, lags) -> np.ndarray:
    qx = np.ascontiguousarray(qx, dtype=np.int8)
    qy = np.ascontiguousarray(qy, dtype=np.int8)
    lags = np.ascontiguousarray(lags, dtype=np.int64)
    c = np.empty(lags.shape[0], dtype=np.int64)
    _load().oracle_xcorr_at(_ptr(qx), qx.shape[0], _ptr(qy), qy.shape[0], _ptr(lags),
                            lags.shape[0], _ptr(c))
    return c


def argmax(c: np.ndarray, lag_min: int) -> tuple[int, int]:
    c = np.ascontiguousarray(c, dtype=np.int64)
    lag = ctypes.c_int64()
    val = ctypes.c_int64()
    _load().oracle_argmax(_ptr(c), int(lag_min), c.shape[0], ctypes.byref(lag), ctypes.byref(val))
    return int(lag.value), int(val.value)


def estimate(x: np.ndarray, y: np.ndarray, bits: int, lag_min: int | None = None,
             lag_max: int | None = None) -> tuple[int, int]:
    """Algorithm 1: quantize both signals, correlate, argmax."""
    qx, qy = quantize(x, bits), quantize(y, bits)
    lo, hi = full_lag_range(qx.shape[0], qy.shape[0])
    lag_min = lo if lag_min is None else lag_min
    lag_max = hi if lag_max is None else lag_max
    return argmax(xcorr(qx, qy, lag_min, lag_max), lag_min)


def real_ccf(x: np.ndarray, y: np.ndarray, tau: int) -> float:
    """(x * y)[tau] = sum_n x[n] y[n + tau] over the overlap, float64 (Eq. (1) on the
    original signals); 0.0 for an empty overlap."""
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    lo, hi = max(0, -tau), min(x.shape[0], y.shape[0] - tau)
    if hi <= lo:
        return 0.0
    return float(np.dot(x[lo:hi], y[lo + tau: hi + tau]))


def refine(x: np.ndarray, y: np.ndarray, c: np.ndarray, lag_min: int) -> dict:
    """Algorithm 1 after the integer correlation c (lags lag_min ..): the set of
    lags where c is maximal; when it holds several, the subset where the real
    cross-correlation of x and y is maximal.  The representative is the set's
    tie-ruled element (smallest |tau|, then tau).  frac is the vertex offset of
    the parabola through the real cross-correlation at the representative and
    its two neighbours (0 when a neighbour has no overlap or the three points
    are not a strict maximum; clamped to [-0.5, 0.5])."""
    c = np.asarray(c, dtype=np.int64)
    vmax = int(c.max())
    tied = [lag_min + int(i) for i in np.nonzero(c == vmax)[0]]
    best = tied
    if len(tied) > 1:
        r = [real_ccf(x, y, t) for t in tied]
        rmax = max(r)
        best = [t for t, v in zip(tied, r) if v == rmax]
    rep = min(best, key=lambda t: (abs(t), t))
    r0 = real_ccf(x, y, rep)
    frac = 0.0
    nx, ny = len(x), len(y)
    if -(nx - 1) <= rep - 1 and rep + 1 <= ny - 1:
        rm, rp = real_ccf(x, y, rep - 1), real_ccf(x, y, rep + 1)
        den = rm - 2.0 * r0 + rp
        if den < 0.0 and r0 >= rm and r0 >= rp:
            frac = min(0.5, max(-0.5, 0.5 * (rm - rp) / den))
    return {"lag": rep, "value": vmax, "r": r0, "frac": frac, "n_int_ties": len(tied),
            "n_ties": len(best), "lag_lo": min(best), "lag_hi": max(best)}
