"""Throughput of the time-difference estimator on one GB300 (or N, sharded).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Workload (the 65536-sample, 2-bit workload the headline metric is quoted on):
256 pairs per GPU, N = 65536, AR(1) 0.95 sources, shift d ~ U[-8192, 8192],
SNR ~ U[0, 30] dB, 2-bit rank quantizer, every lag (+-65535), full exact
integer correlation, tie-ruled argmax.  One step = quantize all 512 signals,
correlate all 256 pairs, argmax all 256 -- the whole path.  Inputs (134 MB)
and correlations (134 MB) exceed the 129 MB L2, so nothing is flushed between
steps.

Two forms run on the same pairs: the full form (every lag, one planned batch
replayed from its CUDA graph) and the learned-proposal form (the shipped
checkpoint; its whole step, fallback included, replayed from a CUDA graph).
The learned form is timed with --in-flight batches (default 6) in flight on
separate streams, each its own planned graph, and with one stream
(learned_proposal.single_stream); both count every pair of every step.

The JSON line carries: value (device-timed pairs/s over all ranks), e2e
(pairs/s through the public API from pinned host buffers, copies included),
the roofline of the dominant kernel (the correlation engine, timed live with
CUDA events on its own stream by the library), the oracle's throughput on a
bounded sample of the same pairs (cpu_baseline) and a lag-parity check
against it, the SM clocks sampled during the timed region, and the number of
library kernel launches in the timed region.

``--impl reference`` times the CPU oracle (test infrastructure) on the host
cores on the same workload, one bounded sample of pairs per step.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "TDE pairs/s at N=65536, 2-bit: learned-proposal vs full int xcorr (bit-exact lag)"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                  "sm_max_mhz": 2070.0}
# The tensor-core kernels compute in E4M3 (kind::f8f6f4, bits 4) or in packed
# E2M1 (kind::mxf4, bits 1 and 2): their peak is the measured BF16 peak times
# the nominal dense FP8 / BF16 (4.5 / 2.25) or FP4 / BF16 (13.5 / 2.25) ratio.
FP8_OVER_BF16 = 2.0
FP4_OVER_BF16 = 6.0


def probe_peak(probe, key, clk, ops_per_unit=1.0):
    """Per-second peak from the library's issue-rate probe (tde_measure_peaks):
    rate per SM per clock x SMs x the SM clock sampled during the timed region
    (MHz; the maximum clock if none was sampled) x ops per unit."""
    if not probe:
        return None
    mhz = clk.get("sm_mhz") or clk.get("sm_max_mhz") or peaks()[0].get("sm_max_mhz", 2070.0)
    return probe[key] * probe["sm_count"] * mhz * 1e6 * ops_per_unit


def tensor_peak(pk, bits):
    """(burst TFLOP/s, sustained TFLOP/s, operand type, kernel suffix) of the
    tensor-core kernels at `bits`."""
    r, dt, suf = (FP4_OVER_BF16, "e2m1", "4") if bits <= 2 else (FP8_OVER_BF16, "e4m3", "8")
    return (pk["bf16_tflops"] * r, pk.get("bf16_tflops_sustained", pk["bf16_tflops"]) * r, dt, suf)
# dram__bytes_read.sum + dram__bytes_write.sum per launch of the engine kernel
# from one ncu capture of this workload (see profiles/); None once the kernel
# has changed since the capture.
# DRAM bytes (read + write) per launch of each form's dominant kernel, from one
# ncu capture of this bench's workload (profiles/); keyed by (kernel, pairs,
# N, bits).  Cleared whenever the kernel changes.
TRAFFIC = {("k_xcorr_mma4", 256, 65536, 2): 214.2e6, ("k_xcorr_win_pp", 256, 65536, 2): 35.78e6}
CKPT = os.path.join(ROOT, "paper_2509_19974_gb300", "models", "proposal_n65536_b2.npz")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--engine", default="auto")
    ap.add_argument("--npairs", type=int, default=256)
    ap.add_argument("--n", type=int, default=65536)
    ap.add_argument("--bits", type=int, default=2)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-fft", action="store_true")
    ap.add_argument("--in-flight", type=int, default=6,
                    help="learned form: batches in flight on separate streams (1 = one stream)")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--agree-pairs", type=int, default=16384,
                    help="proposal workload: fresh pairs checked against the full form")
    ap.add_argument("--c5-rounds", type=int, default=4,
                    help="proposal workload: timed rounds, each on fresh batches")
    ap.add_argument("--no-proposal-pairs", action="store_true")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the single-pair, uneven-batch and template-search records")
    return ap.parse_args()


def rank_seed(rank: int) -> int:
    """Each rank draws its own pairs (weak scaling: no pair is shared)."""
    return 1002 + 7919 * rank


def workload(args, rank):
    from paper_2509_19974_gb300 import synth
    return synth.equal_batch(seed=rank_seed(rank), npairs=args.npairs, n=args.n, bits=args.bits)


def max_over_ranks(value: float, world: int, device=None) -> float:
    """The slowest rank's time (the bench's cross-rank reductions are this
    and min_over_ranks; no data crosses ranks)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def min_over_ranks(value: float, world: int, device=None) -> float:
    """The smallest value over ranks (a lag agreement, an all-ranks flag)."""
    return -max_over_ranks(-float(value), world, device)


def config(args, world):
    return {"workload": f"{args.npairs} pairs/GPU, N={args.n}, AR(1) 0.95, d~U[-8192,8192], "
                        f"SNR~U[0,30] dB, b={args.bits} rank quantizer, all lags "
                        f"+-{args.n - 1}, full exact integer correlation + tie-ruled argmax",
            "forms": "learned proposal vs full integer correlation, same pairs",
            "global_batch": args.npairs * world, "seq_len": args.n, "bits": args.bits,
            "engine": args.engine, "parallelism": f"pairs sharded over {world} GPU(s)",
            "learned_in_flight": f"{args.in_flight} batches of {args.npairs} pairs in flight on "
                                 "separate streams (each its own planned graph)",
            "l2": "inputs 134 MB + correlations 134 MB per GPU exceed the 129 MB L2; no flush"}


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            return json.load(f), "measured"
    except OSError:
        return FALLBACK_PEAKS, "fallback"


class ClockSampler:
    """nvidia-smi SM clock / throttle-reason samples during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index, tag: str = "full"):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"tde_clocks_{os.getpid()}_{tag}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9 and parts[1].isdigit():
                    rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [int(r[1]) for r in rows]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": int(rows[0][2]),
                "samples": len(rows), "power_w_max": max((float(r[3]) for r in rows
                                                          if r[3].replace(".", "").isdigit()),
                                                         default=None),
                "reasons": reasons}


def overlap_macs(nx, ny, lo, hi):
    """Sum over lags lo..hi of the overlap length min(nx, ny - tau) - max(0, -tau)."""
    taus = np.arange(lo, hi + 1, dtype=np.int64)
    ov = np.minimum(nx, ny - taus) - np.maximum(0, -taus)
    return int(np.clip(ov, 0, None).sum())


def cpu_baseline(b, seconds, max_pairs=64):
    import oracle
    oracle.build()
    lags, t0, k = [], time.perf_counter(), 0
    while k < min(max_pairs, b.npairs):
        lags.append(oracle.estimate(b.x[k], b.y[k], b.bits, int(b.lag_min[k]), int(b.lag_max[k])))
        k += 1
        if time.perf_counter() - t0 >= seconds:
            break
    dt = time.perf_counter() - t0
    return {"value": k / dt, "unit": "pairs/s", "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"first {k} of the {b.npairs} pairs (quantize + direct int64 correlation "
                      f"over all lags + argmax), {dt:.1f} s"}, lags


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    b = workload(args, 0)
    import oracle
    oracle.build()
    per_step = []
    k = 0
    for step in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        oracle.estimate(b.x[k % b.npairs], b.y[k % b.npairs], b.bits)
        dt = time.perf_counter() - t0
        k += 1
        if step >= args.warmup:
            per_step.append(dt)
    secs = float(np.sum(per_step))
    value = args.steps / secs
    out = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
           "data": "synthetic", "impl": "reference", "config": config(args, 1),
           "cpu_baseline": {"value": value, "unit": "pairs/s", "cores": oracle.num_threads(),
                            "kind": "oracle", "sample": "one pair of the workload per step"},
           "e2e": {"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# Pairs of the learned proposal's own workload: N = 65536, 2-bit, shift
# d ~ U[-16384, 16384], AR(1) coefficient ~ U[0, 0.98], SNR ~ U[-5, 30] dB,
# drawn by the device generator from a pair-index range disjoint from the
# checkpoint's training, calibration and test pairs.
PROPOSAL_SEED = 1005
PROPOSAL_DMAX, PROPOSAL_AR, PROPOSAL_SNR = 16384, (0.0, 0.98), (-5.0, 30.0)
PROPOSAL_BENCH_FIRST = 3 << 40


def proposal_pairs_record(ctx, model, theta, args, stream, barrier, world, rank, local):
    """The learned form against the full form on the proposal workload's
    pairs, where low SNR and smooth sources make the proposal fall back:
    lag agreement and fallback rate over --agree-pairs fresh pairs (every
    rank its own), and both forms' throughput over --c5-rounds refills of
    the timed plans' buffers with fresh batches (the fallback decided and run
    on the device inside the timed steps)."""
    import torch
    from paper_2509_19974_gb300 import tde
    P, n = args.npairs, args.n
    first0 = PROPOSAL_BENCH_FIRST + (rank << 32)
    nbuf = max(1, args.in_flight)
    bufs = [(torch.empty((P, n), dtype=torch.float32, device="cuda"),
             torch.empty((P, n), dtype=torch.float32, device="cuda")) for _ in range(nbuf)]
    plans = [tde.LearnedBatch(model, xb, yb, args.bits, theta) for xb, yb in bufs]
    sts = [stream] + [torch.cuda.Stream() for _ in range(nbuf - 1)]
    full = tde.Batch(ctx, None, None, args.bits, engine=args.engine,
                     descs=tde.make_descs(list(bufs[0][0].unbind(0)), list(bufs[0][1].unbind(0))))
    batch_no = [0]

    def fill(k):
        x, y, _ = tde.synth_pairs(ctx, PROPOSAL_SEED, first0 + batch_no[0] * P, P, n,
                                  PROPOSAL_DMAX, PROPOSAL_AR, PROPOSAL_SNR)
        bufs[k][0].copy_(x)
        bufs[k][1].copy_(y)
        batch_no[0] += 1

    # agreement and fallback on fresh pairs, batch after batch through plan 0
    nb = max(1, args.agree_pairs // P)
    agree = fb = 0
    for _ in range(nb):
        fill(0)
        lf, vf = [t.clone() for t in full.run(stream)]
        ll, lv, lfb = plans[0].run(stream)
        agree += int(((ll == lf) & (lv == vf)).sum())
        fb += int(lfb.sum())
    torch.cuda.synchronize()
    # throughput: each round refills every plan's buffers (untimed), then times
    # `steps` steps of each form on them
    for k in range(nbuf):
        fill(k)
    torch.cuda.synchronize()  # the fills (current stream) before other streams read them
    for _ in range(max(3, args.warmup)):
        for pl, st in zip(plans, sts):
            pl.run(st)
        full.run(stream)
    torch.cuda.synchronize()  # no run in flight while the next fills write the buffers
    t_l = t_f = 0.0
    steps_l = steps_f = 0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local, "proposal") as clk:
        for _ in range(args.c5_rounds):
            for k in range(nbuf):
                fill(k)
            barrier()
            e0.record(stream)
            for s_ in sts[1:]:
                s_.wait_event(e0)
            for i in range(args.steps):
                plans[i % nbuf].run(sts[i % nbuf])
            for s_ in sts[1:]:
                ev = torch.cuda.Event()
                ev.record(s_)
                stream.wait_event(ev)
            e1.record(stream)
            barrier()
            t_l += max_over_ranks(e0.elapsed_time(e1), world, device="cuda")
            steps_l += args.steps
            barrier()
            e0.record(stream)
            for _ in range(args.steps):
                full.run(stream)
            e1.record(stream)
            barrier()
            t_f += max_over_ranks(e0.elapsed_time(e1), world, device="cuda")
            steps_f += args.steps
    for pl in plans:
        pl.close()
    full.close()
    checked = nb * P
    a = min_over_ranks(agree / checked, world, device="cuda")
    v_l = P * world * steps_l / (t_l / 1e3)
    v_f = P * world * steps_f / (t_f / 1e3)
    return {"workload": f"{P} pairs/GPU per step, N={n}, b={args.bits}, d~U[-{PROPOSAL_DMAX},"
                        f"{PROPOSAL_DMAX}], AR(1) a~U[0,0.98], SNR~U[-5,30] dB (device generator, "
                        "pairs disjoint from the checkpoint's training/calibration/test pairs), "
                        "all lags",
            "pairs_checked": checked * world, "lag_agreement_with_full": a,
            "fallback_rate": fb / checked, "theta": theta,
            "learned": {"value": v_l, "unit": "pairs/s", "ms_per_step": t_l / steps_l,
                        "in_flight": nbuf, "steps": steps_l,
                        "batches": f"{args.c5_rounds} rounds x {nbuf} fresh batches"},
            "full": {"value": v_f, "unit": "pairs/s", "ms_per_step": t_f / steps_f,
                     "steps": steps_f},
            "speedup_vs_full": v_l / v_f, "target_met": bool(a >= 0.999 and v_l > v_f),
            "clocks": clk.summary()}


def other_workloads(ctx, args, local):
    """The other seeded workloads on this GPU, each through the public API
    with CUDA events on the current stream after warm-up, with the SM clocks
    sampled over its timed region and its results checked against the oracle
    on a stated subset:
      single    one pair, N = 4096, b = 1, lags +-4095 (one-pair planned batch
                replayed from its graph, AUTO);
      uneven    4096 pairs, N log-uniform on [1024, 262144], b = 2, lags
                +-N/8 (one planned batch replayed from its graph, AUTO);
      template  a 2^14-sample template in a 2^24-sample signal, b = 4, every
                valid lag, int64 (AUTO)."""
    import torch
    import oracle
    from paper_2509_19974_gb300 import synth, tde
    oracle.build()
    pk, pk_kind = peaks()
    out = {}

    def timed(fn, reps, tag):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local, tag) as clk:
            st = torch.cuda.current_stream()
            e0.record(st)
            for _ in range(reps):
                fn()
            e1.record(st)
            torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps, clk.summary()

    # single pair
    b = synth.single_pair(bits=1)
    x, y = torch.from_numpy(b.x[0]).cuda(), torch.from_numpy(b.y[0]).cuda()
    bt = tde.Batch(ctx, [x], [y], 1, engine="auto")
    ms, clk = timed(bt.run, 200, "single")
    lags, vals = bt.run()
    want = oracle.estimate(b.x[0], b.y[0], 1)
    macs = overlap_macs(4096, 4096, -4095, 4095)
    out["single_pair"] = {
        "workload": "1 pair, N=4096, b=1 sign, lags +-4095, one-pair planned batch replayed "
                    "from its CUDA graph, AUTO engine",
        "us_per_estimate": ms * 1e3, "estimates_per_s": 1e3 / ms, "mac_per_s": macs / (ms / 1e3),
        "bound": "launch latency (six small launches per replay)",
        "parity": {"checked_pairs": 1, "lag_value_mismatches":
                   int((int(lags[0]), int(vals[0])) != want)}, "clocks": clk}
    bt.close()

    # uneven batch
    b = synth.uneven_batch()
    xs = [torch.from_numpy(v).cuda() for v in b.x]
    ys = [torch.from_numpy(v).cuda() for v in b.y]
    macs = float(sum(overlap_macs(len(xv), len(yv), int(lo), int(hi))
                     for xv, yv, lo, hi in zip(b.x, b.y, b.lag_min, b.lag_max)))
    bt = tde.Batch(ctx, xs, ys, 2, b.lag_min, b.lag_max, engine="auto")
    ms, clk = timed(bt.run, max(3, args.steps // 2), "uneven")
    lags, vals = [t.cpu().numpy() for t in bt.run()]
    order = np.argsort([len(v) for v in b.x], kind="stable")
    subset = list(order[:12]) + list(np.random.default_rng(7).choice(order[:2048], 4, replace=False))
    mism = sum(int((int(lags[i]), int(vals[i])) !=
                   oracle.estimate(b.x[i], b.y[i], 2, int(b.lag_min[i]), int(b.lag_max[i])))
               for i in subset)
    out["uneven_batch"] = {
        "workload": f"{b.npairs} pairs, N log-uniform on [1024, 262144] (x64), b=2, lags +-N/8, "
                    "one planned batch replayed from its CUDA graph, AUTO engine per pair",
        "ms_per_batch": ms, "pairs_per_s": b.npairs / (ms / 1e3), "mac_per_s": macs / (ms / 1e3),
        "roofline": {"bound": "tensor", "achieved": 2 * macs / (ms / 1e3) / 1e12,
                     "peak": tensor_peak(pk, 2)[0], "unit": "TFLOP/s",
                     "frac": 2 * macs / (ms / 1e3) / 1e12 / tensor_peak(pk, 2)[0],
                     "what": "whole replayed step (quantize, every engine, argmax) against the "
                             f"{pk_kind} BF16 burst x 6 (nominal FP4: the tensor-core pairs run on "
                             "E2M1 operands); 2 FLOP per overlap MAC"},
        "parity": {"checked_pairs": len(subset), "lag_value_mismatches": mism,
                   "subset": "the 12 shortest pairs and 4 drawn from the shorter half (seed 7)"},
        "clocks": clk}
    bt.close()
    del xs, ys

    # template search
    b = synth.template_search()
    lo, hi = int(b.lag_min[0]), int(b.lag_max[0])
    x, y = torch.from_numpy(b.x[0]).cuda(), torch.from_numpy(b.y[0]).cuda()
    qx, qy = ctx.quantize(x, 4), ctx.quantize(y, 4)
    c = torch.empty(hi - lo + 1, dtype=torch.int64, device="cuda")
    macs = float((hi - lo + 1) * len(b.y[0]))
    eng = tde.pick_engine(4, len(b.x[0]), len(b.y[0]), hi - lo + 1)

    def run():
        ctx.xcorr_int(qx, qy, 4, lo, hi, engine="auto", dtype=torch.int64, c_out=c)
    ms, clk = timed(run, max(3, args.steps), "template")
    lag, val = ctx.argmax(c, lo)
    lag, val = int(lag.item()), int(val.item())
    qxh, qyh = oracle.quantize(b.x[0], 4), oracle.quantize(b.y[0], 4)
    rng = np.random.default_rng(11)
    sample = np.concatenate([[lo, hi, lag], rng.integers(lo, hi + 1, 61)]).astype(np.int64)
    ch = c.cpu().numpy()
    ref = oracle.xcorr_at(qxh, qyh, sample)
    mism = int(np.sum(ch[sample - lo] != ref)) + int(val != int(ref[2]))
    out["template_search"] = {
        "workload": "x 2^24 white + y 2^14 AR(1) 0.9 embedded at a uniform offset, -5 dB, b=4, "
                    f"every valid lag ({hi - lo + 1}), int64, AUTO engine ({eng})",
        "ms": ms, "mac_per_s": macs / (ms / 1e3),
        "roofline": {"bound": "tensor", "achieved": 2 * macs / (ms / 1e3) / 1e12,
                     "peak": tensor_peak(pk, 4)[0], "unit": "TFLOP/s",
                     "frac": 2 * macs / (ms / 1e3) / 1e12 / tensor_peak(pk, 4)[0],
                     "what": f"the correlation call against the {pk_kind} BF16 burst x 2 (FP8: b = 4 "
                             "runs on E4M3 operands); 2 FLOP per valid-lag MAC"},
        "lag": lag, "true_lag": int(b.shift[0]),
        "parity": {"checked_lags": len(sample), "value_mismatches": mism,
                   "subset": "both ends, the GPU's argmax and 61 seeded lags vs the oracle's "
                             "correlation at those lags"},
        "clocks": clk}
    return out


def pipelined_e2e(make_plan, X, Y, steps, stream, barrier):
    """End to end through the public API: every step copies its inputs from
    pinned host memory and reads its lags back.  Two device input buffers, each
    with its own planned step, let step i's host->device copy (on a copy
    stream) overlap step i-1's compute.  Returns (ms for `steps` steps,
    h2d bytes per step, d2h bytes per step)."""
    import torch
    Xh = torch.from_numpy(X).pin_memory()
    Yh = torch.from_numpy(Y).pin_memory()
    bufs = [(torch.empty(X.shape, dtype=torch.float32, device="cuda"),
             torch.empty(Y.shape, dtype=torch.float32, device="cuda")) for _ in range(2)]
    plans = [make_plan(xb, yb) for xb, yb in bufs]
    lag_h = torch.empty((2, X.shape[0]), dtype=torch.int64).pin_memory()
    copy_stream = torch.cuda.Stream()
    done = [torch.cuda.Event() for _ in range(2)]
    loaded = [torch.cuda.Event() for _ in range(2)]

    def run(nsteps):
        for k in range(2):
            done[k].record(stream)
        for i in range(nsteps):
            k = i % 2
            copy_stream.wait_event(done[k])        # the buffer's previous step is over
            with torch.cuda.stream(copy_stream):
                bufs[k][0].copy_(Xh, non_blocking=True)
                bufs[k][1].copy_(Yh, non_blocking=True)
                loaded[k].record(copy_stream)
            stream.wait_event(loaded[k])
            lags = plans[k](stream)
            lag_h[k].copy_(lags, non_blocking=True)
            done[k].record(stream)

    run(2)
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    run(steps)
    f1.record(stream)
    barrier()
    return f0.elapsed_time(f1), int(X.nbytes + Y.nbytes), int(lag_h[0].numel() * 8)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    import torch
    import torch.distributed as dist
    from paper_2509_19974_gb300 import build, tde

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    ctx = tde.Context(local)
    probe = tde.measure_peaks(local)
    b = workload(args, rank)
    X, Y = b.stacked()
    Xd, Yd = torch.from_numpy(X).cuda(), torch.from_numpy(Y).cuda()
    xs, ys = list(Xd.unbind(0)), list(Yd.unbind(0))
    descs = tde.make_descs(xs, ys, b.lag_min, b.lag_max)
    stream = torch.cuda.current_stream()

    # The production path: the whole step planned once and replayed as one
    # CUDA graph (tde_batch_create / tde_batch_run).
    batch = tde.Batch(ctx, None, None, args.bits, engine=args.engine, descs=descs)

    def step():
        return batch.run()

    def step_nograph():
        return tde.tde_estimate_batch(ctx, None, None, args.bits, engine=args.engine, descs=descs)

    for _ in range(max(args.warmup, 3)):
        lags, vals = step()
        step_nograph()
    ctx.sync()
    ctx.read_profile()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    with ClockSampler(local) as clk:
        barrier()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.steps):
            lags, vals = step()
        e1.record(stream)
        barrier()
        ms = e0.elapsed_time(e1)
        launches, _, _ = ctx.read_profile()
        # Same steps without the graph, the library bracketing the engine
        # kernel with CUDA events on its stream: the roofline's kernel time.
        ctx.set_profiling(True)
        h0, h1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        for _ in range(args.steps):
            step_nograph()
        h1.record(stream)
        barrier()
        ctx.set_profiling(False)
    ms_nograph = h0.elapsed_time(h1)
    _, eng_launches, eng_ms = ctx.read_profile()
    ctx.sync()
    ms_max = max_over_ranks(ms, world, device="cuda")
    value = args.npairs * world * args.steps / (ms_max / 1e3)

    # --- end to end through the public API from pinned host memory
    e2e = None
    if not args.no_e2e:
        def full_plan(xb, yb):
            d = tde.make_descs(list(xb.unbind(0)), list(yb.unbind(0)), b.lag_min, b.lag_max)
            pb = tde.Batch(ctx, None, None, args.bits, engine=args.engine, descs=d)
            return lambda st: pb.run(st)[0]
        t_e2e, h2d, d2h = pipelined_e2e(full_plan, X, Y, args.steps, stream, barrier)
        t_e2e = max_over_ranks(t_e2e, world, device="cuda")
        e2e = {"value": args.npairs * world * args.steps / (t_e2e / 1e3),
               "unit": "pairs/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
               "overlap": "step i's host->device copy overlaps step i-1's compute"}

    gpu_lags = lags.cpu().numpy()
    gpu_vals = vals.cpu().numpy()

    # --- the learned-proposal form on the same pairs (trained checkpoint)
    learned = None
    if not args.no_learned and args.n == 65536 and args.bits == 2 and os.path.exists(CKPT):
        z = np.load(CKPT)
        theta = float(z["theta"])
        model = tde.Model(ctx, args.n)
        model.load(CKPT)
        # the whole learned step (fallback decided on the device) as a CUDA graph
        lb = tde.LearnedBatch(model, Xd, Yd, args.bits, theta)
        for _ in range(max(3, args.warmup)):
            lb.run(stream)
        torch.cuda.synchronize()
        ctx.read_profile()
        clk_l = ClockSampler(local, "learned")
        clk_l.__enter__()
        k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        barrier()
        k0.record(stream)
        for _ in range(args.steps):
            lb.run(stream)
        k1.record(stream)
        barrier()
        launches_l, _, _ = ctx.read_profile()
        ms_l1 = k0.elapsed_time(k1) / args.steps
        ll, lv, lf = lb.lags, lb.vals, lb.fallback
        # two batches in flight: a second plan (own workspace and graph) on a
        # second stream, steps alternating, so one batch's small launches
        # overlap the other's heavy kernels
        ms_l, in_flight = ms_l1, 1
        if args.in_flight > 1:
            lbs = [lb] + [tde.LearnedBatch(model, Xd, Yd, args.bits, theta) for _ in range(args.in_flight - 1)]
            sts = [stream] + [torch.cuda.Stream() for _ in range(args.in_flight - 1)]
            for _ in range(max(3, args.warmup)):
                for b_, s_ in zip(lbs, sts):
                    b_.run(s_)
            barrier()
            k0.record(stream)
            for s_ in sts[1:]:
                s_.wait_event(k0)
            for i in range(args.steps):
                lbs[i % len(lbs)].run(sts[i % len(lbs)])
            for s_ in sts[1:]:
                ev = torch.cuda.Event()
                ev.record(s_)
                stream.wait_event(ev)
            k1.record(stream)
            barrier()
            ms_n = k0.elapsed_time(k1) / args.steps
            same = all(bool(((b_.lags == ll) & (b_.vals == lv)).all()) for b_ in lbs[1:])
            # every rank uses the in-flight figure only if every rank's plans agree
            if min_over_ranks(1.0 if same else 0.0, world, device="cuda") == 1.0:
                ms_l, in_flight = ms_n, len(lbs)
        ms_l1 = max_over_ranks(ms_l1, world, device="cuda")
        ms_l = max_over_ranks(ms_l, world, device="cuda")
        agree = min_over_ranks(float(((ll == lags) & (lv == vals)).float().mean()), world,
                               device="cuda")
        # the window kernel, timed by the library on its stream
        ctx.read_profile()
        ctx.set_profiling(True)
        for _ in range(args.steps):
            model.estimate(Xd, Yd, args.bits, theta)
        torch.cuda.synchronize()
        ctx.set_profiling(False)
        _, wl, wms = ctx.read_profile()
        # exact window MACs from the proposal's centres (deterministic)
        q2 = tde.tde_quantize_batch(ctx, torch.stack([Xd, Yd], dim=1).reshape(-1, args.n)
                                    .contiguous(), args.bits)
        cent, _ = model.propose(q2)
        cent = cent.cpu().numpy()
        win_macs = 0
        for p in range(args.npairs):
            for c in cent[p]:
                lo, hi = max(int(c) - 128, -(args.n - 1)), min(int(c) + 128, args.n - 1)
                win_macs += overlap_macs(args.n, args.n, lo, hi) if hi >= lo else 0
        # the MACs the polyphase windows kernel issues: per pair the distinct
        # 128-lag blocks its windows need, 128 x 128 entries each over the
        # 128-sample rows of the signal
        blocks = 0
        for p in range(args.npairs):
            bl = set()
            for c in cent[p]:
                lo, hi = max(int(c) - 128, -(args.n - 1)), min(int(c) + 128, args.n - 1)
                if hi >= lo:
                    bl.update(range(lo // 128, (hi + 127) // 128 + 1))
            blocks += len(bl)
        issued_macs = blocks * 128 * 128 * (-(-args.n // 128))
        pk, pk_kind = peaks()
        pb, ps_ = pk["bf16_tflops"] * FP8_OVER_BF16, pk.get("bf16_tflops_sustained", pk["bf16_tflops"]) * FP8_OVER_BF16
        ach = 2.0 * win_macs / (wms / max(wl, 1) / 1e3) if wl else None
        wname = "k_xcorr_win_pp"
        roof_l = None if ach is None else {
            "bound": "tensor", "kernel": wname, "achieved": ach / 1e12,
            "peak": pb, "unit": "TFLOP/s", "frac": ach / 1e12 / pb,
            "frac_of_sustained": ach / 1e12 / ps_,
            "traffic": TRAFFIC.get((wname, args.npairs, args.n, args.bits)),
            "peak_source": f"{pk_kind} dense BF16 burst (bf16_tflops) x 2 (nominal dense FP8 / BF16): the "
                           "kernel's operands are e4m3 at every b; achieved counts 2 FLOP per overlap MAC of "
                           "the 257-lag windows (algorithmic); the kernel issues macs_issued_per_launch "
                           "(the windows' 128-lag blocks, shared by neighbouring windows)",
            "ms_per_launch": wms / wl, "macs_per_launch": win_macs,
            "macs_issued_per_launch": issued_macs, "launches": wl}
        if roof_l is not None:
            pp = probe_peak(probe, "e4m3_mac_per_sm_clk", clk_l.summary(), 2.0)
            roof_l["frac_of_probe"] = ach / pp if pp else None
            roof_l["probe_peak"] = pp / 1e12 if pp else None
        # end to end: inputs from pinned host memory, lags back, every step
        e2e_l = None
        if not args.no_e2e:
            def learned_plan(xb, yb):
                pl = tde.LearnedBatch(model, xb, yb, args.bits, theta)
                return lambda st: pl.run(st)[0]
            t_l, h2d, d2h = pipelined_e2e(learned_plan, X, Y, args.steps, stream, barrier)
            t_l = max_over_ranks(t_l, world, device="cuda")
            e2e_l = {"value": args.npairs * world * args.steps / (t_l / 1e3), "unit": "pairs/s",
                     "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                     "overlap": "step i's host->device copy overlaps step i-1's compute"}
        clk_l.__exit__(None, None, None)  # sampled over the learned form's timed regions
        meta = json.loads(str(z["meta"]))
        learned = {"value": args.npairs * world / (ms_l / 1e3), "unit": "pairs/s",
                   "ms_per_step": ms_l, "in_flight": in_flight, "clocks": clk_l.summary(),
                   "single_stream": {"value": args.npairs * world / (ms_l1 / 1e3),
                                     "ms_per_step": ms_l1},
                   "e2e": e2e_l, "roofline": roof_l, "gpu_launches": int(launches_l),
                   "lag_agreement_with_full": agree, "fallback_rate": float(lf.float().mean()),
                   "theta": theta, "full_form_value": args.npairs * world * args.steps / (ms_max / 1e3),
                   "speedup_vs_full": (ms_max / args.steps) / ms_l,
                   "what": "quantize -> 16x decimate -> CNN (BF16 weights; tensor-core conv, "
                           "FP32 accumulation) -> top-8 257-lag windows -> exact tensor-core "
                           "correlation in the windows -> tie-ruled argmax; full correlation "
                           "when margin < theta, decided and run on the device; the whole step "
                           "replayed from a CUDA graph",
                   "checkpoint": {"train_pairs": meta.get("train_pairs"),
                                  "train_seconds": meta.get("train_seconds"),
                                  "calibration": meta.get("calibration"),
                                  "test": meta.get("test")}}
        if not args.no_proposal_pairs:
            learned["proposal_pairs"] = proposal_pairs_record(ctx, model, theta, args, stream,
                                                              barrier, world, rank, local)
        model.close()

    # --- FP32 FFT comparator beside it: the same quantized pairs, timed alone
    fft = None
    if not args.no_fft:
        qX = torch.stack([ctx.quantize(x, args.bits) for x in xs])
        qY = torch.stack([ctx.quantize(y, args.bits) for y in ys])
        c_exact = torch.empty(args.npairs * (2 * args.n - 1), dtype=torch.int32, device="cuda")
        tde.tde_estimate_batch(ctx, None, None, args.bits, engine=args.engine, descs=descs,
                               c_out=c_exact)
        c_fft = ctx.xcorr_fft32(qX, qY)
        for _ in range(2):
            ctx.xcorr_fft32(qX, qY, c_out=c_fft)
        torch.cuda.synchronize()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        reps = max(3, args.steps // 4)
        for _ in range(reps):
            ctx.xcorr_fft32(qX, qY, c_out=c_fft)
        g1.record(stream)
        torch.cuda.synchronize()
        ms_fft = g0.elapsed_time(g1) / reps
        ce = c_exact.view(args.npairs, -1)
        err = ((c_fft.double() - ce.double()).abs().amax(dim=1) / ce.abs().amax(dim=1).double())
        am = c_fft.argmax(dim=1, keepdim=True)
        agree = (ce.gather(1, am).squeeze(1) == ce.amax(dim=1)).float().mean()
        fft = {"pairs_per_s": args.npairs / (ms_fft / 1e3), "ms_per_batch": ms_fft,
               "what": "cuFFT R2C/C2R FP32 correlation of the same quantized pairs (int8 in)",
               "max_err_over_max_abs_c": float(err.max()), "bound": 1e-4,
               "lag_is_exact_maximiser_frac": float(agree)}
        del qX, qY, c_exact, c_fft
    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    # --- roofline of the correlation engine kernel
    pk, pk_kind = peaks()
    macs = sum(overlap_macs(args.n, args.n, int(b.lag_min[i]), int(b.lag_max[i]))
               for i in range(args.npairs))
    per_launch_ms = eng_ms / max(eng_launches, 1)
    engine = args.engine
    if engine == "auto":
        engine = tde.pick_engine(args.bits, args.n, args.n, int(b.lag_max[0] - b.lag_min[0] + 1))
    roof = None
    if eng_launches:
        macs_launch = macs * args.steps / eng_launches
        achieved_mac = macs_launch / (per_launch_ms / 1e3)
        if engine == "popc":
            popc_per_mac = (2.0 if args.bits <= 2 else 18.0) / 32.0
            peak_mac = probe_peak(probe, "popc_per_sm_clk", clk.summary(), 1.0 / popc_per_mac)
            roof = {"bound": "alu", "kernel": "k_xcorr_popc", "achieved": achieved_mac / 1e12,
                    "peak": peak_mac / 1e12, "unit": "TMAC/s", "frac": achieved_mac / peak_mac,
                    "traffic": None,
                    "peak_source": f"POPC pipe: {probe['sm_count']} SMs x "
                                   f"{probe['popc_per_sm_clk']:.1f} POPC/clk (tde_measure_peaks) x the "
                                   f"sampled SM clock; {popc_per_mac * 32:.0f} POPC per 32 MACs"}
        elif engine == "mma":
            tflops = 2.0 * achieved_mac / 1e12
            peak, peak_s, dt, suf = tensor_peak(pk, args.bits)
            kname = "k_xcorr_mma" + suf
            pp = probe_peak(probe, "e2m1_mac_per_sm_clk" if args.bits <= 2 else "e4m3_mac_per_sm_clk",
                            clk.summary(), 2.0)
            roof = {"bound": "tensor", "kernel": kname, "achieved": tflops, "peak": peak,
                    "unit": "TFLOP/s", "frac": tflops / peak,
                    "frac_of_sustained": tflops / peak_s,
                    "probe_peak": pp / 1e12 if pp else None,
                    "frac_of_probe": tflops * 1e12 / pp if pp else None,
                    "traffic": TRAFFIC.get((kname, args.npairs, args.n, args.bits)),
                    "peak_source": f"{pk_kind} dense BF16 burst (bf16_tflops) x {peak / pk['bf16_tflops']:.0f} "
                                   f"(nominal dense {'FP4' if args.bits <= 2 else 'FP8'} / BF16): the "
                                   f"kernel's operands are {dt}; achieved counts 2 FLOP per overlap MAC "
                                   "(algorithmic)"}
        if roof is not None:
            roof.update({"ms_per_launch": per_launch_ms, "macs_per_launch": macs_launch,
                         "launches": eng_launches})

    out = {"metric": METRIC, "value": value, "unit": "pairs/s", "n_gpus": world,
           "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms_max / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": tensor_peak(peaks()[0], args.bits)[2],
           "data": "synthetic", "config": config(args, world), "e2e": e2e,
           "gpu_launches": int(launches), "roofline": roof,
           "no_graph": {"value": args.npairs * world * args.steps / (ms_nograph / 1e3),
                        "ms_per_step": ms_nograph / args.steps},
           "mac_per_s": macs * world * args.steps / (ms_max / 1e3),
           "clocks": clk.summary(), "fft32_comparator": fft, "learned_proposal": learned,
           "peaks_probe": dict(probe, what="tde_measure_peaks: issue rates per SM per SM clock "
                                           "(POPC, IMAD, tcgen05 E4M3 and E2M1 MACs, M=128 N=256)")}
    # Headline: the metric compares the learned-proposal form with the full
    # integer correlation; the learned form leads when its lags agree with the
    # full form's on >= 99.9% of this run's pairs, the full form is kept beside.
    if learned is not None and learned["lag_agreement_with_full"] >= 0.999:
        out["full_form"] = {"value": out["value"], "ms_per_step": out["ms_per_step"],
                            "e2e": out["e2e"], "roofline": out["roofline"],
                            "gpu_launches": out["gpu_launches"], "clocks": out["clocks"]}
        out["form"] = "learned proposal (windows + exact tensor-core correlation, full fallback)"
        out["value"] = learned["value"]
        out["ms_per_step"] = learned["ms_per_step"]
        out["e2e"] = learned["e2e"]
        out["roofline"] = learned["roofline"]
        out["full_form"]["dtype"] = out["dtype"]
        out["dtype"] = "e4m3"  # the windows kernel's operands (the CNN is BF16, the fallback the full form's)
        out["gpu_launches"] = learned["gpu_launches"]
        if learned["clocks"].get("sm_mhz") is not None:
            out["clocks"] = learned["clocks"]
    else:
        out["form"] = "full integer correlation"
    if not args.no_cpu_baseline and world == 1:
        cb, ref = cpu_baseline(b, args.cpu_seconds)
        out["cpu_baseline"] = cb
        mism = sum(1 for k, (l, v) in enumerate(ref) if (int(gpu_lags[k]), int(gpu_vals[k])) != (l, v))
        out["parity"] = {"checked_pairs": len(ref), "lag_value_mismatches": mism}
    out["true_shift_hit_rate"] = float(np.mean(gpu_lags == b.shift))
    if not args.no_workloads and world == 1:
        out["workloads"] = other_workloads(ctx, args, local)
    print(json.dumps(out))
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
