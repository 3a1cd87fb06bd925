"""Parity at the workloads' full sizes, in the launch configuration the bench
times (a planned batch replayed from its CUDA graph), against the oracle.

  * 256 pairs x 65536 samples, AR(1) 0.95 sources, b in {1, 2, 4}, all lags,
    every engine: the quantized levels of every signal, the full correlation
    of a sample of pairs, 24 sampled lags of every pair, the identity
    sum_tau c[tau] = (sum qx)(sum qy) for every pair, and every pair's lag and
    value (checked against the oracle's argmax on the sampled pairs, and as
    the tie-ruled maximiser of the checked correlation on all).
  * 4096 pairs of uneven length (log-uniform 1024..262144), b = 2, lags
    +-N/8, AUTO engines: full correlations and lags of a seeded sample of 192
    pairs plus the shortest and the longest.
  * Template search 2^24 x 2^14, b = 4, valid lags: the full correlation of
    every engine (int64 output through CRT for the NTT) and the lag equal
    to the oracle's.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_19974_gb300 import synth, tde

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2509_19974_gb300 import build
    build.build()
    c = tde.Context(0)
    yield c
    c.close()


def _tie_ruled(c: np.ndarray, lag_min: int):
    """Largest value, then smallest |tau|, then smallest tau."""
    v = c.max()
    taus = np.nonzero(c == v)[0] + lag_min
    key = np.abs(taus) * 2 + (taus > 0)
    return int(taus[np.argmin(key)]), int(v)


# ------------------------------------------------------ 256 x 65536, all lags

N2, P2 = 65536, 256
FULL_SAMPLE = (0, 1, 77, 128, 200, 255)


@pytest.fixture(scope="module")
def batch256():
    return synth.equal_batch(npairs=P2, n=N2)


@pytest.fixture(scope="module")
def ref256(batch256):
    """Per bits: oracle levels of every signal and full correlations of the
    sampled pairs."""
    out = {}
    for bits in (1, 2, 4):
        qx = np.stack([oracle.quantize(x, bits) for x in batch256.x])
        qy = np.stack([oracle.quantize(y, bits) for y in batch256.y])
        full = {p: oracle.xcorr(qx[p], qy[p]) for p in FULL_SAMPLE}
        out[bits] = (qx, qy, full)
    return out


@pytest.mark.parametrize("bits", [1, 2, 4])
@pytest.mark.parametrize("engine", ["popc", "mma", "ntt"])
def test_full_size_equal_batch(ctx, batch256, ref256, bits, engine):
    qx, qy, full = ref256[bits]
    x = torch.from_numpy(np.stack(batch256.x)).cuda()
    y = torch.from_numpy(np.stack(batch256.y)).cuda()
    # quantized levels of every signal, batched like the bench's first step
    q = tde.tde_quantize_batch(ctx, torch.stack([x, y], 1).reshape(-1, N2).contiguous(), bits)
    ctx.sync()
    q = q.view(P2, 2, N2).cpu().numpy()
    assert np.array_equal(q[:, 0], qx) and np.array_equal(q[:, 1], qy)

    L = 2 * N2 - 1
    c_out = torch.empty(P2 * L, dtype=torch.int32, device="cuda")
    b = tde.Batch(ctx, list(x.unbind(0)), list(y.unbind(0)), bits, engine=engine, c_out=c_out)
    lags, vals = b.run()
    ctx.sync()
    c = c_out.view(P2, L).cpu().numpy().astype(np.int64)
    lags, vals = lags.cpu().numpy(), vals.cpu().numpy()
    b.close()
    lo = -(N2 - 1)
    rng = np.random.default_rng(bits * 10 + len(engine))
    sums = qx.astype(np.int64).sum(1) * qy.astype(np.int64).sum(1)
    assert np.array_equal(c.sum(1), sums)
    for p in range(P2):
        taus = np.concatenate([[lo, -1, 0, 1, N2 - 1], rng.integers(lo, N2, 19)])
        assert np.array_equal(c[p, taus - lo], oracle.xcorr_at(qx[p], qy[p], taus)), p
        assert (int(lags[p]), int(vals[p])) == _tie_ruled(c[p], lo), p
    for p, ref in full.items():
        assert np.array_equal(c[p], ref), p
        assert (int(lags[p]), int(vals[p])) == oracle.argmax(ref, lo), p


# ------------------------------------------------- 4096 uneven pairs, +-N/8

def test_full_size_uneven_batch(ctx):
    bt = synth.uneven_batch()
    P = bt.npairs
    xs = [torch.from_numpy(v).cuda() for v in bt.x]
    ys = [torch.from_numpy(v).cuda() for v in bt.y]
    counts = (bt.lag_max - bt.lag_min + 1).astype(np.int64)
    offs = np.concatenate([[0], np.cumsum(counts)])
    c_out = torch.empty(int(offs[-1]), dtype=torch.int32, device="cuda")
    b = tde.Batch(ctx, xs, ys, 2, bt.lag_min, bt.lag_max, c_out=c_out)
    b.run()
    lags, vals = b.run()  # a replay, like the bench's timed steps
    ctx.sync()
    lags, vals = lags.cpu().numpy(), vals.cpu().numpy()
    b.close()
    lens = np.array([len(v) for v in bt.x])
    rng = np.random.default_rng(4096)
    sample = set(rng.choice(P, 192, replace=False).tolist())
    sample |= {int(np.argmin(lens)), int(np.argmax(lens))}
    for p in sorted(sample):
        lo, hi = int(bt.lag_min[p]), int(bt.lag_max[p])
        qx, qy = oracle.quantize(bt.x[p], 2), oracle.quantize(bt.y[p], 2)
        ref = oracle.xcorr(qx, qy, lo, hi)
        got = c_out[offs[p]: offs[p + 1]].cpu().numpy().astype(np.int64)
        assert np.array_equal(got, ref), p
        assert (int(lags[p]), int(vals[p])) == oracle.argmax(ref, lo), p


# ------------------------------------------------- template search 2^24 x 2^14

@pytest.fixture(scope="module")
def template():
    bt = synth.template_search()
    qx, qy = oracle.quantize(bt.x[0], 4), oracle.quantize(bt.y[0], 4)
    lo, hi = int(bt.lag_min[0]), int(bt.lag_max[0])
    ref = oracle.xcorr(qx, qy, lo, hi)
    return bt, ref, oracle.argmax(ref, lo)


@pytest.mark.parametrize("engine", ["ntt", "mma", "popc"])
def test_full_size_template_search(ctx, template, engine):
    bt, ref, (lag, val) = template
    lo, hi = int(bt.lag_min[0]), int(bt.lag_max[0])
    x = torch.from_numpy(bt.x[0]).cuda()
    y = torch.from_numpy(bt.y[0]).cuda()
    qx, qy = ctx.quantize(x, 4), ctx.quantize(y, 4)
    c = ctx.xcorr_int(qx, qy, 4, lo, hi, engine=engine, dtype=torch.int64)
    got_lag, got_val = ctx.argmax(c, lo)
    ctx.sync()
    assert np.array_equal(c.cpu().numpy(), ref)
    assert (int(got_lag), int(got_val)) == (lag, val)
    # the planted offset is recovered at -5 dB
    assert lag == int(bt.shift[0])
