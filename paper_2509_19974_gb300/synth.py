"""Seeded synthetic workloads for the time-difference estimator.

This module only draws random signals; it holds none of the estimator's
arithmetic (no quantization, no correlation, no argmax), so both the CUDA path
and the CPU oracle can consume its outputs.  The paper's own data (speech
commands over environmental noise, Sec. 4.2) is not available; these
generators stand in for it with the shapes, lengths and shift/SNR structure of
the five workloads below.

Shift construction (Sec. 2.2, Eq. (2)): a source ``s`` is drawn, ``x`` is the
window ``s[D : D+N]`` and ``y`` the window ``s[D-d : D-d+N]``, so that
``x[n] = y[n + d]`` before noise and the correlation peak sits at lag ``d``.
Noise is i.i.d. Gaussian per signal, scaled so that the mean square of the
clean window over that of the noise equals the requested SNR (Sec. 4.2 fixes
SNR as a ratio of squared l2 norms per unit time).

Seeds: numpy PCG64; workload k uses seed 1000 + k unless told otherwise; pair
``i`` of a batch draws from ``SeedSequence(seed).spawn(npairs)[i]``.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
from scipy.signal import lfilter


def _rng(seed) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def ar1(rng: np.random.Generator, length: int, a: float) -> np.ndarray:
    """Stationary AR(1): s[0] = e0 / sqrt(1 - a^2), s[n] = a s[n-1] + e[n]."""
    e = rng.standard_normal(length)
    if a != 0.0:
        e[0] = e[0] / np.sqrt(1.0 - a * a)
        e = lfilter([1.0], [1.0, -a], e)
    return e.astype(np.float32)


def add_noise(rng: np.random.Generator, clean: np.ndarray, snr_db: float) -> np.ndarray:
    p_s = float(np.mean(clean.astype(np.float64) ** 2))
    sigma = np.sqrt(p_s / (10.0 ** (snr_db / 10.0)))
    return (clean.astype(np.float64) + sigma * rng.standard_normal(clean.shape[0])).astype(np.float32)


def shifted_pair(rng, n: int, dmax: int, d: int, snr_db: float, ar: float = 0.0):
    """One pair with x[n] = y[n + d] before noise (peak at lag d)."""
    s = ar1(rng, n + 2 * dmax, ar)
    x = s[dmax: dmax + n]
    y = s[dmax - d: dmax - d + n]
    return add_noise(rng, x, snr_db), add_noise(rng, y, snr_db)


@dataclass
class Batch:
    """A batch of pairs.  ``x``/``y`` are lists of FP32 arrays (ragged allowed)."""
    x: list
    y: list
    shift: np.ndarray                 # true lag d of each pair
    bits: int
    lag_min: np.ndarray               # per-pair lag range, inclusive
    lag_max: np.ndarray
    snr_db: np.ndarray = field(default_factory=lambda: np.zeros(0))
    name: str = ""

    @property
    def npairs(self) -> int:
        return len(self.x)

    def stacked(self):
        """(X, Y) as [npairs, N] float32 arrays when all lengths are equal."""
        return np.stack(self.x), np.stack(self.y)


def single_pair(seed: int = 1001, n: int = 4096, dmax: int = 512, snr_db: float = 20.0,
                bits: int = 1) -> Batch:
    """One white-Gaussian pair, N = 4096, d ~ U[-512, 512], 20 dB, full lags."""
    rng = _rng(seed)
    d = int(rng.integers(-dmax, dmax + 1))
    x, y = shifted_pair(rng, n, dmax, d, snr_db)
    return Batch([x], [y], np.array([d]), bits, np.array([-(n - 1)]), np.array([n - 1]),
                 np.array([snr_db]), f"single pair N={n} b={bits}")


def equal_batch(seed: int = 1002, npairs: int = 256, n: int = 65536, dmax: int = 8192,
                ar: float = 0.95, snr_lo: float = 0.0, snr_hi: float = 30.0,
                bits: int = 2) -> Batch:
    """Equal-length AR(1) pairs, d ~ U[-dmax, dmax], SNR ~ U[lo, hi] dB, full lags."""
    kids = np.random.SeedSequence(seed).spawn(npairs)
    xs, ys, ds, snrs = [], [], [], []
    for k in kids:
        rng = _rng(k)
        d = int(rng.integers(-dmax, dmax + 1))
        snr = float(rng.uniform(snr_lo, snr_hi))
        x, y = shifted_pair(rng, n, dmax, d, snr, ar)
        xs.append(x), ys.append(y), ds.append(d), snrs.append(snr)
    return Batch(xs, ys, np.array(ds), bits, np.full(npairs, -(n - 1)), np.full(npairs, n - 1),
                 np.array(snrs), f"{npairs} pairs N={n} AR({ar}) b={bits}")


def uneven_batch(seed: int = 1003, npairs: int = 4096, n_lo: int = 1024, n_hi: int = 262144,
                 snr_db: float = 10.0, bits: int = 2) -> Batch:
    """Uneven lengths: N log-uniform on [n_lo, n_hi] rounded to a multiple of 64,
    white sources, d ~ U[-N/8, N/8], lags restricted to +-floor(N/8)."""
    kids = np.random.SeedSequence(seed).spawn(npairs)
    xs, ys, ds, lo, hi = [], [], [], [], []
    for k in kids:
        rng = _rng(k)
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        n = int(min(max(64 * round(n / 64), n_lo), n_hi))
        w = n // 8
        d = int(rng.integers(-w, w + 1))
        x, y = shifted_pair(rng, n, w, d, snr_db)
        xs.append(x), ys.append(y), ds.append(d), lo.append(-w), hi.append(w)
    return Batch(xs, ys, np.array(ds), bits, np.array(lo), np.array(hi),
                 np.full(npairs, snr_db), f"{npairs} uneven pairs N in [{n_lo},{n_hi}] b={bits}")


def template_search(seed: int = 1004, nx: int = 1 << 24, ny: int = 1 << 14, ar: float = 0.9,
                    snr_db: float = -5.0, bits: int = 4) -> Batch:
    """Long template search: y (AR(1) segment) embedded in white noise x at a
    uniform offset o; SNR measured over the embedded span.  With
    c[tau] = sum x[n] y[n + tau] the peak is at tau = -o; the valid lags (y fully
    inside x) are tau in [-(nx - ny), 0]."""
    rng = _rng(seed)
    y = ar1(rng, ny, ar)
    o = int(rng.integers(0, nx - ny + 1))
    p_y = float(np.mean(y.astype(np.float64) ** 2))
    sigma = np.sqrt(p_y / (10.0 ** (snr_db / 10.0)))
    x = sigma * rng.standard_normal(nx)
    x[o: o + ny] += y
    return Batch([x.astype(np.float32)], [y], np.array([-o]), bits, np.array([-(nx - ny)]),
                 np.array([0]), np.array([snr_db]), f"template search Nx={nx} Ny={ny} b={bits}")


def proposal_batch(seed: int = 1005, npairs: int = 65536, n: int = 65536, dmax: int = 16384,
                   ar_hi: float = 0.98, snr_lo: float = -5.0, snr_hi: float = 30.0,
                   bits: int = 2) -> Batch:
    """Pairs for the learned lag proposal: d ~ U[-16384, 16384], AR coefficient
    ~ U[0, 0.98], SNR ~ U[-5, 30] dB, full lags."""
    kids = np.random.SeedSequence(seed).spawn(npairs)
    xs, ys, ds, snrs = [], [], [], []
    for k in kids:
        rng = _rng(k)
        d = int(rng.integers(-dmax, dmax + 1))
        a = float(rng.uniform(0.0, ar_hi))
        snr = float(rng.uniform(snr_lo, snr_hi))
        x, y = shifted_pair(rng, n, dmax, d, snr, a)
        xs.append(x), ys.append(y), ds.append(d), snrs.append(snr)
    return Batch(xs, ys, np.array(ds), bits, np.full(npairs, -(n - 1)), np.full(npairs, n - 1),
                 np.array(snrs), f"{npairs} proposal pairs N={n} b={bits}")
