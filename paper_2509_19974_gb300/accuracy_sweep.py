"""Accuracy against SNR on synthetic signals, following the paper's accuracy
protocol (Sec. 4.2) with synthetic signals in place of its datasets.

Per trial: a target burst (white noise low-passed by a one-pole filter,
a = 0.9) of n/2 samples inside a frame of n samples; x = target + background,
y = the target delayed by a fractional nu ~ U[0, n/4) (an FFT phase shift of
the frame) + an independent background; the background is white noise scaled
so that the ratio of the target's squared l2 norm per sample to the
background's is the SNR. Three estimators, all through the library:

  proposed        Algorithm 1 with the sign quantizer (b = 1): the integer
                  correlation, its tied maxima re-ranked by the real
                  cross-correlation (tde_refine);
  until line 4    the set of integer maxima alone;
  real CCF        the argmax of the unquantized cross-correlation (the FP32
                  FFT comparator).

A trial is correct when every lag of the estimated set is within one sample
of nu (|lag - nu| < 1). Usage:

    python -m paper_2509_19974_gb300.accuracy_sweep [--n 16000] [--trials 200]
"""
from __future__ import annotations

import argparse

import numpy as np
import torch
from scipy.signal import lfilter

from . import build, tde


def make_pair(rng, n: int, snr_db: float):
    t = lfilter([1.0], [1.0, -0.9], rng.standard_normal(n // 2))  # one-pole low-pass
    frame = np.zeros(n)
    start = n // 8
    frame[start: start + t.shape[0]] = t
    nu = float(rng.uniform(0.0, n / 4))
    f = np.fft.rfftfreq(2 * n)
    spec = np.fft.rfft(np.concatenate([frame, np.zeros(n)]))
    shifted = np.fft.irfft(spec * np.exp(-2j * np.pi * f * nu), 2 * n)[:n]
    p_sig = float(np.mean(t ** 2))
    sigma = np.sqrt(p_sig / 10 ** (snr_db / 10.0))
    x = frame + sigma * rng.standard_normal(n)
    y = shifted + sigma * rng.standard_normal(n)
    return x.astype(np.float32), y.astype(np.float32), nu


def run(n: int, trials: int, snrs, seed: int = 2026):
    build.build()
    ctx = tde.Context(0)
    lo, hi = -(n - 1), n - 1
    rows = []
    for snr in snrs:
        rng = np.random.default_rng([seed, int(round(10 * snr)) + 1000])
        ok = {"proposed": 0, "until line 4": 0, "real CCF": 0}
        for _ in range(trials):
            x, y, nu = make_pair(rng, n, snr)
            xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
            qx, qy = ctx.quantize(xt, 1), ctx.quantize(yt, 1)
            c = ctx.xcorr_int(qx, qy, 1, lo, hi, dtype=torch.int64)
            r = ctx.refine(xt, yt, c, lo)
            ok["proposed"] += abs(r["lag_lo"] - nu) < 1 and abs(r["lag_hi"] - nu) < 1
            tied = torch.nonzero(c == c.max()).flatten() + lo
            ok["until line 4"] += bool(((tied.double() - nu).abs() < 1).all())
            f = ctx.xcorr_fft32(xt, yt)
            ok["real CCF"] += abs(int(torch.argmax(f.flatten())) + lo - nu) < 1
        rows.append((snr, {k: v / trials for k, v in ok.items()}))
    ctx.close()
    return rows


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=16000)
    ap.add_argument("--trials", type=int, default=200)
    ap.add_argument("--snrs", type=float, nargs="+", default=[-20, -15, -10, -5, 0, 5, 10])
    a = ap.parse_args()
    rows = run(a.n, a.trials, a.snrs)
    print(f"| SNR (dB) | proposed | until line 4 | real CCF |  (n = {a.n}, {a.trials} trials)")
    print("|---:|---:|---:|---:|")
    for snr, acc in rows:
        print(f"| {snr:g} | {acc['proposed']:.3f} | {acc['until line 4']:.3f} | {acc['real CCF']:.3f} |")


if __name__ == "__main__":
    main()
