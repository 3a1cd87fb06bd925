"""Accuracy against SNR on synthetic signals, following the paper's accuracy
protocol (Sec. 4.2) with synthetic signals in place of its two datasets.

Per trial, at 16 kHz:

  y   the target: one second (16000 samples) of a speech-like stand-in, white
      noise through a two-pole resonator (poles at radius 0.9, angle 0.1 pi)
      under a Hann envelope over its middle 80 %;
  x   five seconds (80000 samples): the target delayed by nu ~ U[0, 4 s)
      (a sub-sample shift, done as a phase shift of the zero-padded
      spectrum, i.e. band-limited interpolation) plus an environmental-noise
      stand-in, white noise through a one-pole low-pass (a = 0.95), scaled so
      that the target's squared l2 norm per sample over the background's is
      the SNR.

With c[tau] = sum_n x[n] y[n + tau], the target at delay nu in x peaks at
tau = -nu, so the estimate is nu_hat = -tau_hat. Three estimators, all
through the library over every lag:

  proposed        Algorithm 1 with the sign quantizer (b = 1): the integer
                  correlation, its tied maxima re-ranked by the real
                  cross-correlation (tde_refine);
  integer maxima  the set of integer maxima alone (no re-ranking);
  real CCF        the argmax of the unquantized cross-correlation (the FP32
                  FFT comparator).

A trial is correct when every delay of the estimated set satisfies
|nu_hat - nu| < 1. Usage:

    python -m paper_2509_19974_gb300.accuracy_sweep [--trials 1000] [--snrs ...]
"""
from __future__ import annotations

import argparse

import numpy as np
from scipy.signal import lfilter

FS = 16000
NY, NX = FS, 5 * FS
MAX_DELAY = 4 * FS


def make_pair(rng, snr_db: float, nx: int = NX, ny: int = NY, max_delay: int = MAX_DELAY):
    """(x, y, nu): FP32 noisy mixture, FP32 target, true delay in samples."""
    r, w = 0.9, 0.1 * np.pi
    t = lfilter([1.0], [1.0, -2.0 * r * np.cos(w), r * r], rng.standard_normal(ny))
    env = np.zeros(ny)
    m = int(0.8 * ny)
    env[(ny - m) // 2: (ny - m) // 2 + m] = np.hanning(m)
    t *= env
    nu = float(rng.uniform(0.0, max_delay))
    f = np.fft.rfftfreq(2 * nx)
    placed = np.zeros(2 * nx)
    placed[:ny] = t
    delayed = np.fft.irfft(np.fft.rfft(placed) * np.exp(-2j * np.pi * f * nu), 2 * nx)[:nx]
    b = lfilter([1.0], [1.0, -0.95], rng.standard_normal(nx))
    p_t = float(np.sum(t * t)) / ny
    p_b = float(np.sum(b * b)) / nx
    b *= np.sqrt(p_t / (p_b * 10.0 ** (snr_db / 10.0)))
    return (delayed + b).astype(np.float32), t.astype(np.float32), nu


def run(trials: int, snrs, seed: int = 2026):
    import torch

    from . import build, tde

    build.build()
    ctx = tde.Context(0)
    lo = -(NX - 1)
    rows = []
    for snr in snrs:
        rng = np.random.default_rng([seed, int(round(10 * snr)) + 1000])
        ok = {"proposed": 0, "integer maxima": 0, "real CCF": 0}
        for _ in range(trials):
            x, y, nu = make_pair(rng, snr)
            xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
            qx, qy = ctx.quantize(xt, 1), ctx.quantize(yt, 1)
            c = ctx.xcorr_int(qx, qy, 1, dtype=torch.int64)
            r = ctx.refine(xt, yt, c, lo)
            ok["proposed"] += abs(-r["lag_lo"] - nu) < 1 and abs(-r["lag_hi"] - nu) < 1
            tied = -(torch.nonzero(c == c.max()).flatten() + lo)
            ok["integer maxima"] += bool(((tied.double() - nu).abs() < 1).all())
            f = ctx.xcorr_fft32(xt, yt)
            ok["real CCF"] += abs(-(int(torch.argmax(f.flatten())) + lo) - nu) < 1
        rows.append((snr, {k: v / trials for k, v in ok.items()}))
    ctx.close()
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--trials", type=int, default=1000)
    ap.add_argument("--snrs", type=float, nargs="+", default=[-20, -15, -10, -5, 0, 5, 10])
    a = ap.parse_args()
    rows = run(a.trials, a.snrs)
    print(f"| SNR (dB) | proposed | integer maxima | real CCF |  ({a.trials} trials per SNR)")
    print("|---:|---:|---:|---:|")
    for snr, acc in rows:
        print(f"| {snr:g} | {acc['proposed']:.3f} | {acc['integer maxima']:.3f} | {acc['real CCF']:.3f} |")


if __name__ == "__main__":
    main()
