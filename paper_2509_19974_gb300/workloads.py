"""Timings of the estimator on its other workloads, through the public API.

The bench times the 256-pair, N = 65536 batch. This module times the other
seeded workloads of `synth` on one GPU:

  single     one pair, N = 4096, b = 1, lags +-4095: device time per estimate
             per engine, per call through `estimate` and per replay of a
             one-pair planned batch (graph);
  uneven     4096 pairs, N log-uniform on [1024, 262144], b = 2, lags +-N/8,
             as one planned batch (graph replay), under AUTO and under each
             engine;
  template   a 2^14-sample template in a 2^24-sample signal, b = 4, every
             valid lag, int64: the correlation per engine, and the FP32 FFT
             comparator; the NTT both with one prime and with CRT of two.

Device times are CUDA events on the current stream after warm-up. Usage:

    python -m paper_2509_19974_gb300.workloads [--only single uneven template] [--reps 10]
"""
from __future__ import annotations

import argparse
import time


def _events_ms(fn, reps: int) -> float:
    import torch
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        fn()
    e1.record(st)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def single(ctx, reps: int):
    import torch

    from . import synth, tde
    b = synth.single_pair(bits=1)
    x, y = torch.from_numpy(b.x[0]).cuda(), torch.from_numpy(b.y[0]).cuda()
    rows = []
    for eng in ("auto", "popc", "mma", "ntt"):
        for _ in range(5):
            ctx.estimate(x, y, 1, engine=eng)
        torch.cuda.synchronize()
        ms = _events_ms(lambda: ctx.estimate(x, y, 1, engine=eng), reps)
        rows.append(("single pair 4096, b = 1, estimate()", eng, f"{ms * 1e3:.1f} us",
                     f"{1e3 / ms / 1e3:.1f} K estimates/s"))
    for eng in ("auto", "popc", "mma"):
        bt = tde.Batch(ctx, [x], [y], 1, engine=eng)
        for _ in range(5):
            bt.run()
        torch.cuda.synchronize()
        ms = _events_ms(bt.run, 20 * reps)
        t0 = time.perf_counter()
        for _ in range(20 * reps):
            lags, _ = bt.run()
            int(lags[0].item())
        wall_us = (time.perf_counter() - t0) / (20 * reps) * 1e6
        rows.append(("single pair 4096, b = 1, graph replay", eng,
                     f"{ms * 1e3:.1f} us ({wall_us:.0f} us with the lag read back)",
                     f"{1e3 / ms / 1e3:.1f} K estimates/s"))
        bt.close()
    return rows


def uneven(ctx, reps: int):
    import torch

    from . import synth, tde
    b = synth.uneven_batch()
    xs = [torch.from_numpy(v).cuda() for v in b.x]
    ys = [torch.from_numpy(v).cuda() for v in b.y]
    macs = float(sum(len(x) * (hi - lo + 1) for x, lo, hi in zip(b.x, b.lag_min, b.lag_max)))
    rows = []
    for eng in ("auto", "mma", "popc", "ntt"):
        bt = tde.Batch(ctx, xs, ys, 2, b.lag_min, b.lag_max, engine=eng)
        for _ in range(2):
            bt.run()
        torch.cuda.synchronize()
        ms = _events_ms(bt.run, reps if eng in ("auto", "mma") else max(1, reps // 2))
        rows.append((f"uneven {b.npairs}-pair batch, b = 2", eng, f"{ms:.2f} ms",
                     f"{b.npairs / ms:.1f} K pairs/s, {macs / ms / 1e9:.0f} T MAC/s"))
        bt.close()
    return rows


def template(ctx, reps: int):
    import torch

    from . import synth, tde
    b = synth.template_search()
    lo, hi = int(b.lag_min[0]), int(b.lag_max[0])
    x, y = torch.from_numpy(b.x[0]).cuda(), torch.from_numpy(b.y[0]).cuda()
    qx, qy = ctx.quantize(x, 4), ctx.quantize(y, 4)
    c = torch.empty(hi - lo + 1, dtype=torch.int64, device="cuda")
    macs = float((hi - lo + 1) * len(b.y[0]))
    two = tde.Context(ctx.device)
    two.set_ntt_primes(2)
    rows = []
    for name, cx, eng in (("auto", ctx, "auto"), ("mma", ctx, "mma"), ("ntt, one prime", ctx, "ntt"),
                          ("ntt, two primes + CRT", two, "ntt"), ("popc", ctx, "popc")):
        def run(cx=cx, eng=eng):
            cx.xcorr_int(qx, qy, 4, lo, hi, engine=eng, dtype=torch.int64, c_out=c)
        for _ in range(2):
            run()
        torch.cuda.synchronize()
        ms = _events_ms(run, reps if eng != "popc" else 2)
        lag, _ = ctx.argmax(c, lo)
        rows.append((f"template 2^24 x 2^14, b = 4, int64 (lag {int(lag.item())}, true "
                     f"{int(b.shift[0])})", name, f"{ms:.3f} ms", f"{macs / ms / 1e9:.0f} T MAC/s"))
    f = torch.empty(hi - lo + 1, dtype=torch.float32, device="cuda")
    for _ in range(2):
        ctx.xcorr_fft32(x, y, lo, hi, c_out=f)
    torch.cuda.synchronize()
    ms = _events_ms(lambda: ctx.xcorr_fft32(x, y, lo, hi, c_out=f), reps)
    rows.append(("template 2^24 x 2^14 (FP32 signals)", "FP32 FFT comparator", f"{ms:.3f} ms", ""))
    two.close()
    return rows


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--only", nargs="+", choices=("single", "uneven", "template"),
                    default=["single", "uneven", "template"])
    ap.add_argument("--reps", type=int, default=10)
    a = ap.parse_args()
    from . import build, tde
    build.build()
    ctx = tde.Context(0)
    rows = []
    for w in a.only:
        rows += {"single": single, "uneven": uneven, "template": template}[w](ctx, a.reps)
    ctx.close()
    print("| Workload | Engine | Time | Throughput |")
    print("|---|---|---|---|")
    for r in rows:
        print("| " + " | ".join(r) + " |")


if __name__ == "__main__":
    main()
