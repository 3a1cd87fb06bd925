"""Learned lag proposal on the GPU: the generator, the CNN's loss and
gradient against the float64 reference, AdamW, and the learned estimator's
lag against the exact correlation (windows only, and with full fallback)."""
import numpy as np
import pytest
import torch

import oracle
from oracle import cnn_ref
from paper_2509_19974_gb300 import tde

pytestmark = pytest.mark.gpu
N = 16384


@pytest.fixture(scope="module")
def ctx():
    from paper_2509_19974_gb300 import build
    build.build()
    c = tde.Context(0)
    yield c
    c.close()


def test_synth_pairs_deterministic_and_shifted(ctx):
    x, y, d = tde.synth_pairs(ctx, 7, 100, 6, N, 2000, ar=(0.5, 0.5), snr_db=(40.0, 40.0))
    x2, y2, d2 = tde.synth_pairs(ctx, 7, 100, 6, N, 2000, ar=(0.5, 0.5), snr_db=(40.0, 40.0))
    torch.cuda.synchronize()
    assert torch.equal(x, x2) and torch.equal(y, y2) and torch.equal(d, d2)
    d = d.cpu().numpy()
    assert np.all(np.abs(d) <= 2000)
    xs, ys = x.cpu().numpy().astype(np.float64), y.cpu().numpy().astype(np.float64)
    for p in range(6):      # x[n] = y[n + d] up to 40 dB noise
        k = int(d[p])
        a = xs[p][max(0, -k): N - max(0, k)]
        b = ys[p][max(0, k): N - max(0, -k)]
        assert np.corrcoef(a, b)[0, 1] > 0.99


def _quantized_pairs(ctx, P, seed, snr=(10.0, 30.0)):
    x, y, d = tde.synth_pairs(ctx, seed, 0, P, N, 2000, ar=(0.0, 0.9), snr_db=snr)
    q2 = tde.tde_quantize_batch(ctx, torch.stack([x, y], dim=1).reshape(-1, N).contiguous(), 2)
    return x, y, d, q2


def test_loss_and_gradient_match_float64_reference(ctx):
    m = tde.Model(ctx, N, seed=3)
    x, y, d, q2 = _quantized_pairs(ctx, 4, 11)
    labels = d.clone()
    p0 = m.state()["params"]
    loss = m.train_step(q2, labels, lr=0.0, weight_decay=0.0)
    st = m.state()
    torch.cuda.synchronize()
    ref_params = p0.astype(np.float64)
    lay, a_off = cnn_ref.layout()
    for (wo, bo, cin) in lay:       # the device's forward pass uses BF16 weights
        ref_params[wo:bo] = cnn_ref.bf16_round(p0[wo:bo]).astype(np.float64)
    ref_loss, ref_grad = cnn_ref.loss_and_grad(ref_params, q2.cpu().numpy(), labels.cpu().numpy())
    assert np.allclose(loss.cpu().numpy(), ref_loss, rtol=2e-4, atol=2e-4)
    g = st["grad"].astype(np.float64)
    assert np.linalg.norm(g - ref_grad) <= 2e-3 * np.linalg.norm(ref_grad)
    m.close()


def test_adamw_step(ctx):
    m = tde.Model(ctx, N, seed=4)
    x, y, d, q2 = _quantized_pairs(ctx, 2, 12)
    p0 = m.state()["params"].astype(np.float64)
    lr, wd = 1e-3, 1e-2
    m.train_step(q2, d, lr=lr, weight_decay=wd)
    st = m.state()
    g = st["grad"].astype(np.float64)
    mm = 0.1 * g
    vv = 0.001 * g * g
    is_w = np.zeros_like(p0, bool)
    for (wo, bo, cin) in cnn_ref.layout()[0]:
        is_w[wo:bo] = True
    want = p0 - lr * ((mm / 0.1) / (np.sqrt(vv / 0.001) + 1e-8) + np.where(is_w, wd * p0, 0.0))
    assert st["step"] == 1
    assert np.allclose(st["params"], want, rtol=1e-5, atol=1e-6)
    m.close()


def test_training_reduces_loss(ctx):
    m = tde.Model(ctx, N, seed=5)
    losses = []
    for it in range(60):
        x, y, d, q2 = _quantized_pairs(ctx, 32, 1000 + it, snr=(20.0, 30.0))
        losses.append(float(m.train_step(q2, d, lr=3e-3).mean()))
    assert np.mean(losses[-10:]) < 0.7 * np.mean(losses[:5]), losses
    m.close()


def _window_reference(qx, qy, centres):
    """Tie-ruled argmax of the exact correlation over the union of windows."""
    lags = set()
    for c in centres:
        lags.update(range(max(int(c) - 128, -(N - 1)), min(int(c) + 128, N - 1) + 1))
    lags = np.array(sorted(lags), np.int64)
    vals = oracle.xcorr_at(qx, qy, lags)
    best = None
    for t, v in zip(lags.tolist(), vals.tolist()):
        key = (v, -abs(t), -t)
        if best is None or key > best[0]:
            best = (key, t, v)
    return best[1], best[2]


def test_learned_estimate_windows_and_fallback(ctx):
    m = tde.Model(ctx, N, seed=6)
    x, y, d, q2 = _quantized_pairs(ctx, 6, 21)
    cent, marg = m.propose(q2)
    lags, vals, fb = m.estimate(x, y, bits=2, theta=0.0)       # windows only
    torch.cuda.synchronize()
    assert int(fb.sum()) == 0
    xs, ys = x.cpu().numpy(), y.cpu().numpy()
    cent = cent.cpu().numpy()
    for p in range(6):
        qx, qy = oracle.quantize(xs[p], 2), oracle.quantize(ys[p], 2)
        assert (int(lags[p]), int(vals[p])) == _window_reference(qx, qy, cent[p])
    lags, vals, fb = m.estimate(x, y, bits=2, theta=2.0)       # all fall back
    torch.cuda.synchronize()
    assert int(fb.sum()) == 6
    for p in range(6):
        assert (int(lags[p]), int(vals[p])) == oracle.estimate(xs[p], ys[p], 2)
    m.close()


def test_inference_proposal_matches_reference_top_bin(ctx):
    """The inference forward (tensor cores, BF16 activations) proposes the same
    best bin as the float64 reference of the trained model, and its margin is
    within 1e-2 of the reference's."""
    import os
    ck = os.path.join(os.path.dirname(tde.__file__), "models", "proposal_n65536_b2.npz")
    z = np.load(ck)
    n = 65536
    m = tde.Model(ctx, n)
    m.load(ck)
    x, y, d = tde.synth_pairs(ctx, 31, 0, 4, n, 16384, (0.5, 0.9), (10.0, 30.0))
    q2 = tde.tde_quantize_batch(ctx, torch.stack([x, y], dim=1).reshape(-1, n).contiguous(), 2)
    cent, marg = m.propose(q2)
    torch.cuda.synchronize()
    params = z["params"].astype(np.float64)
    for (wo, bo, cin) in cnn_ref.layout()[0]:
        params[wo:bo] = cnn_ref.bf16_round(z["params"][wo:bo]).astype(np.float64)
    _, s = cnn_ref.forward(torch.tensor(params), q2.cpu().numpy())
    s = s.numpy()
    Lf = n // 256
    for p in range(4):
        top = np.argsort(-s[p], kind="stable")[:8]
        assert int(cent[p, 0]) == 256 * (int(top[0]) - (Lf - 1))
        e = np.exp(s[p] - s[p].max())
        assert abs(float(marg[p]) - e[top].sum() / e.sum()) < 1e-2
    m.close()


@pytest.mark.parametrize("bits", [1, 2, 4])
@pytest.mark.parametrize("n", [100, 4096 + 37, 65536])
def test_xcorr_windows_match_oracle_at_edges(ctx, bits, n):
    """The tensor-core windows against the oracle's correlation at the same
    lags: centres at both ends of the lag range, partly and wholly outside
    it, duplicated, and random; lags outside [-(n-1), n-1] read 0."""
    import oracle
    rng = np.random.default_rng(n * 7 + bits)
    P = 3
    k = 7 if bits == 4 else 1
    q = rng.integers(-k, k + 1, size=(2 * P, n)).astype(np.int8)
    q[rng.random((2 * P, n)) < 0.2] = 0
    cent = np.empty((P, 8), np.int32)
    for p in range(P):
        cent[p] = [-(n - 1), n - 1, -(n - 1) - 100, n + 300, 0, 0,
                   rng.integers(-(n - 1), n), rng.integers(-(n - 1), n)]
    c = tde.tde_xcorr_windows(ctx, torch.from_numpy(q).cuda(), bits,
                              torch.from_numpy(cent).cuda())
    ctx.sync()
    c = c.cpu().numpy().astype(np.int64)
    for p in range(P):
        for w in range(8):
            lags = np.arange(cent[p, w] - 128, cent[p, w] + 129)
            inr = (lags >= -(n - 1)) & (lags <= n - 1)
            ref = np.zeros(257, np.int64)
            if inr.any():
                ref[inr] = oracle.xcorr_at(q[2 * p], q[2 * p + 1], lags[inr])
            assert np.array_equal(c[p, w], ref), (p, w)


def _window_lags(cent):
    return cent[..., None].astype(np.int64) + np.arange(-128, 129)


@pytest.mark.parametrize("bits,n,P,lev", [(4, 1 << 20, 320, 7), (2, (1 << 22) + 4133, 320, 1)])
def test_xcorr_windows_exact_on_long_pairs(ctx, bits, n, P, lev):
    """Eq. (1) in the windows stays exact where one CTA's share of a pair sums
    more samples than FP32 holds exactly: every level at +lev (the largest
    magnitude of the bits), so c[tau] = lev^2 (n - |tau|) reaches
    49 * 2^20 > 2^24 at b = 4, with enough pairs that a CTA's run covers
    whole pairs.  The closed form is checked against the oracle at sampled
    lags, then every window value against the closed form."""
    import oracle
    rng = np.random.default_rng(n + bits)
    q = torch.full((2 * P, n), lev, dtype=torch.int8, device="cuda")
    cent = np.empty((P, 8), np.int32)
    cent[:, 0] = 0
    cent[:, 1] = -(n - 1)
    cent[:, 2] = n - 1
    cent[:, 3:] = rng.integers(-(n - 1), n, size=(P, 5))
    c = tde.tde_xcorr_windows(ctx, q, bits, torch.from_numpy(cent).cuda())
    ctx.sync()
    c = c.cpu().numpy().astype(np.int64)
    lags = _window_lags(cent)
    inr = np.abs(lags) <= n - 1
    closed = np.where(inr, lev * lev * (n - np.abs(lags)), 0)
    assert int(closed.max()) == lev * lev * n
    ones = np.full(n, lev, np.int8)
    sample = np.array([0, 1, -1, n - 1, -(n - 1), 12345, -777777 % n, n // 2])
    assert np.array_equal(oracle.xcorr_at(ones, ones, sample), lev * lev * (n - np.abs(sample)))
    bad = np.argwhere(c != closed)
    assert bad.size == 0, (bad[:5], c[tuple(bad[0])], closed[tuple(bad[0])])


def test_xcorr_windows_exact_random_b4_long(ctx):
    """Random b = 4 levels, y a shifted copy of x, n = 2^20, 320 pairs: the
    matched lag sums about 19.6e6 > 2^24; two pairs' windows (around the shift
    and elsewhere) are compared with the oracle lag by lag."""
    import oracle
    n, P = 1 << 20, 320
    g = torch.Generator(device="cuda").manual_seed(5)
    x = torch.randint(-7, 8, (P, n + 8192), dtype=torch.int8, device="cuda", generator=g)
    d = np.random.default_rng(9).integers(-4000, 4001, size=P)
    q = torch.empty((2 * P, n), dtype=torch.int8, device="cuda")
    q[0::2] = x[:, 4096:4096 + n]
    for p in range(P):  # x[n] = y[n + d]
        q[2 * p + 1] = x[p, 4096 - int(d[p]):4096 - int(d[p]) + n]
    cent = np.empty((P, 8), np.int32)
    cent[:, 0] = d
    cent[:, 1:] = np.random.default_rng(10).integers(-(n - 1), n, size=(P, 7))
    c = tde.tde_xcorr_windows(ctx, q, 4, torch.from_numpy(cent).cuda())
    ctx.sync()
    c = c.cpu().numpy().astype(np.int64)
    qh = q.cpu().numpy()
    for p in (0, P - 1):
        lags = _window_lags(cent[p])
        want = oracle.xcorr_at(qh[2 * p], qh[2 * p + 1], lags.reshape(-1)).reshape(8, 257)
        assert want[0, 128] > (1 << 24)
        assert np.array_equal(c[p], want), p


def test_xcorr_windows_int32_overflow_refused(ctx):
    """n * (2^(bits-1))^2 >= 2^31 cannot be held in the int32 windows: the call
    is refused on the host with TDE_ERR_OVERFLOW (b = 4, n = 2^25)."""
    n = 1 << 25
    q = torch.zeros((2, n), dtype=torch.int8, device="cuda")
    cent = torch.zeros((1, 8), dtype=torch.int32, device="cuda")
    with pytest.raises(tde.TdeError) as e:
        tde.tde_xcorr_windows(ctx, q, 4, cent)
    assert e.value.status == tde.TDE_ERR_OVERFLOW
    tde.tde_xcorr_windows(ctx, q[:, : n // 2].contiguous(), 4, cent)  # 2^24 * 64 = 2^30 fits
    ctx.sync()


def test_xcorr_windows_level_outside_bits_flagged(ctx):
    """A level outside the bits' range (3 with bits = 2) is flagged on the
    device: the next sync returns TDE_ERR_INVALID, and the context is then
    usable again."""
    q = torch.ones((2, 4096), dtype=torch.int8, device="cuda")
    q[0, 17] = 3
    cent = torch.zeros((1, 8), dtype=torch.int32, device="cuda")
    tde.tde_xcorr_windows(ctx, q, 2, cent)
    with pytest.raises(tde.TdeError) as e:
        ctx.sync()
    assert e.value.status == tde.TDE_ERR_INVALID
    q[0, 17] = 1
    c = tde.tde_xcorr_windows(ctx, q, 2, cent)
    ctx.sync()
    assert int(c[0, 0, 128]) == 4096


def test_learned_batch_graph_mixed_fallback(ctx):
    """The graph-captured learned estimate: with theta between the pairs'
    margins some pairs fall back (decided on the device); every lag is the
    window reference or the full estimate accordingly, and a replay on refilled
    inputs gives the same as a direct call."""
    m = tde.Model(ctx, N, seed=6)
    x, y, d, q2 = _quantized_pairs(ctx, 8, 31)
    cent, marg = m.propose(q2)
    theta = float(torch.median(marg).item())
    xb, yb = x.clone(), y.clone()
    lb = tde.LearnedBatch(m, xb, yb, bits=2, theta=theta)
    lags, vals, fb = lb.run()
    torch.cuda.synchronize()
    fbn = fb.cpu().numpy()
    margn = marg.cpu().numpy()
    assert np.array_equal(fbn, (margn < theta).astype(np.int32))
    assert 0 < fbn.sum() < 8
    xs, ys = x.cpu().numpy(), y.cpu().numpy()
    cent = cent.cpu().numpy()
    for p in range(8):
        qx, qy = oracle.quantize(xs[p], 2), oracle.quantize(ys[p], 2)
        want = oracle.estimate(xs[p], ys[p], 2) if fbn[p] else _window_reference(qx, qy, cent[p])
        assert (int(lags[p]), int(vals[p])) == want, p
    # refill with other pairs and replay; compare with the direct (uncaptured) call
    x2, y2, _, _ = _quantized_pairs(ctx, 8, 32)
    xb.copy_(x2), yb.copy_(y2)
    lags2, vals2, fb2 = [t.clone() for t in lb.run()]
    l3, v3, f3 = m.estimate(x2, y2, bits=2, theta=theta)
    torch.cuda.synchronize()
    assert torch.equal(lags2, l3) and torch.equal(vals2, v3) and torch.equal(fb2, f3)
    lb.close()
    m.close()


def test_xcorr_windows_many_pairs_mixed_patterns(ctx):
    """Enough pairs that every CTA of the windows kernel walks several
    visits (its plan ring and both slot rings lap), with every window
    pattern the proposal or a caller gives: 8 adjacent bins, scattered bins,
    centres on no 128-lag boundary, 8 identical centres, windows partly or
    wholly outside the lag range.  48 pairs, every pattern among them, are
    compared with the oracle lag by lag."""
    import oracle
    n, P = 8192 + 77, 600
    rng = np.random.default_rng(21)
    q = rng.integers(-1, 2, size=(2 * P, n)).astype(np.int8)
    lf = n // 256
    cent = np.empty((P, 8), np.int32)
    for p in range(P):
        kind = p % 5
        if kind == 0:
            b0 = rng.integers(-lf + 5, lf - 5)
            cent[p] = 256 * (b0 + np.arange(-4, 4))
        elif kind == 1:
            cent[p] = 256 * rng.choice(np.arange(-lf + 1, lf), 8, replace=False)
        elif kind == 2:
            cent[p] = rng.integers(-(n - 1), n, 8)
        elif kind == 3:
            cent[p] = rng.integers(-(n - 1), n)
        else:
            cent[p] = [-(n - 1), n - 1, -(n + 200), n + 500, 0, 128, 129, rng.integers(-(n - 1), n)]
    c = tde.tde_xcorr_windows(ctx, torch.from_numpy(q).cuda(), 2, torch.from_numpy(cent).cuda())
    ctx.sync()
    c = c.cpu().numpy().astype(np.int64)
    for p in list(range(10)) + list(rng.choice(np.arange(10, P), 38, replace=False)):
        lags = _window_lags(cent[p])
        inr = np.abs(lags) <= n - 1
        want = np.zeros((8, 257), np.int64)
        want[inr] = oracle.xcorr_at(q[2 * p], q[2 * p + 1], lags[inr])
        assert np.array_equal(c[p], want), (p, p % 5)
