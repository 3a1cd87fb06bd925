"""Pins of the float64 CNN reference (oracle/cnn_ref.py) to things other than
itself: central finite differences of its loss agree with its autograd
gradient; swapping x and y mirrors the scores (score_yx[l] = score_xy[-l]);
its forward equals the architecture restated as explicit sums (no conv
routine) with np.correlate for the scores; and with pass-through weights the
features and scores have a closed form.  CPU only."""
import numpy as np
import torch

from oracle import cnn_ref


def _setup(seed=0, P=2, n=4096):
    rng = np.random.default_rng(seed)
    lay, a_off = cnn_ref.layout()
    params = np.zeros(a_off + 1)
    for (wo, bo, cin) in lay:
        params[wo:bo] = rng.uniform(-1, 1, bo - wo) * np.sqrt(6.0 / (cin * 9))
        params[bo:bo + 32] = rng.uniform(-0.1, 0.1, 32)
    params[a_off] = 0.01
    q2 = rng.integers(-1, 2, (2 * P, n)).astype(np.int8)
    labels = rng.integers(-(n - 1), n, P)
    return params, q2, labels


def test_gradient_matches_finite_differences():
    params, q2, labels = _setup()
    _, g = cnn_ref.loss_and_grad(params, q2, labels)
    rng = np.random.default_rng(1)
    idx = np.concatenate([rng.choice(len(params) - 1, 24, replace=False), [len(params) - 1]])

    def loss(p):
        return float(cnn_ref.loss_and_grad(p, q2, labels)[0].mean())
    for i in idx:
        h = 1e-6 * max(1.0, abs(params[i]))
        pp, pm = params.copy(), params.copy()
        pp[i] += h
        pm[i] -= h
        fd = (loss(pp) - loss(pm)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 + 1e-4 * abs(fd), (i, fd, g[i])


def test_swapping_signals_mirrors_scores():
    params, q2, _ = _setup(P=3)
    p = torch.tensor(params)
    _, s = cnn_ref.forward(p, q2)
    swapped = q2.reshape(-1, 2, q2.shape[1])[:, ::-1].reshape(q2.shape).copy()
    _, s2 = cnn_ref.forward(p, swapped)
    assert torch.allclose(s, s2.flip(1), rtol=1e-12, atol=1e-12)


def _forward_by_sums(params, q2):
    """The architecture written out with explicit sums (no conv routine):
    d[j] = sum of levels 16 j .. 16 j + 15, over 4; per layer
    z[co][p] = b[co] + sum_ci sum_k W[co][ci][k] h[ci][p + k - 4] (h zero
    outside), y[co][p] = max(relu z[co][2p], relu z[co][2p + 1]); then
    score[l] = alpha sum_c sum_i fx[c][i] fy[c][i + l] by np.correlate per
    channel."""
    lay, a_off = cnn_ref.layout()
    S, n = q2.shape
    feats = []
    for s in range(S):
        h = np.array([[q2[s, 16 * j:16 * j + 16].astype(np.float64).sum() / 4.0 for j in range(n // 16)]])
        for (wo, bo, cin) in lay:
            W = params[wo:bo].reshape(32, cin, 9)
            b = params[bo:bo + 32]
            L = h.shape[1]
            z = np.tile(b[:, None], (1, L))
            for k in range(9):
                sh = k - 4  # input position p + sh
                lo, hi = max(0, -sh), min(L, L - sh)
                z[:, lo:hi] += W[:, :, k] @ h[:, lo + sh:hi + sh]
            r = np.maximum(z, 0.0)
            h = np.maximum(r[:, 0::2], r[:, 1::2])
        feats.append(h)
    Lf = feats[0].shape[1]
    out = []
    for p in range(S // 2):
        fx, fy = feats[2 * p], feats[2 * p + 1]
        # np.correlate(fy, fx, 'full')[m] = sum_i fy[i + m - (Lf - 1)] fx[i]
        sc = sum(np.correlate(fy[c], fx[c], mode="full") for c in range(32))
        out.append(params[a_off] * sc)
    return np.stack(feats), np.stack(out)


def test_forward_matches_the_architecture_written_as_sums():
    """cnn_ref.forward (torch conv1d / max_pool1d / padded slices) equals the
    architecture restated as explicit sums and np.correlate, features and
    scores, on random weights and levels."""
    params, q2, _ = _setup(seed=3, P=2, n=2048)
    f, s = cnn_ref.forward(torch.tensor(params), q2)
    f2, s2 = _forward_by_sums(params, q2)
    assert np.allclose(f.numpy(), f2, rtol=1e-12, atol=1e-12)
    assert np.allclose(s.numpy(), s2, rtol=1e-10, atol=1e-10)


def test_forward_with_pass_through_weights_is_pooled_decimation():
    """Closed form: with every layer passing channel 0 through its centre tap
    (W[0][0][4] = 1, all else 0, zero biases), the features are channel 0 =
    the 16-fold max-pool of relu(d) (relu is idempotent on the pooled
    non-negative values), the other channels zero, and score[l] = alpha
    sum_i g_x[i] g_y[i + l] for those pooled decimations g."""
    lay, a_off = cnn_ref.layout()
    params = np.zeros(a_off + 1)
    for (wo, bo, cin) in lay:
        params[wo + 4] = 1.0  # W[0][0][4]
    params[a_off] = 0.5
    rng = np.random.default_rng(6)
    n = 4096
    q2 = rng.integers(-1, 2, (2, n)).astype(np.int8)
    f, s = cnn_ref.forward(torch.tensor(params), q2)
    d = q2.astype(np.float64).reshape(2, n // 16, 16).sum(-1) / 4.0
    g = np.maximum(d, 0.0).reshape(2, n // 256, 16).max(-1)
    assert np.allclose(f.numpy()[:, 0], g, rtol=0, atol=0)
    assert np.all(f.numpy()[:, 1:] == 0)
    Lf = n // 256
    want = np.array([0.5 * sum(g[0, i] * g[1, i + l] for i in range(Lf) if 0 <= i + l < Lf)
                     for l in range(-(Lf - 1), Lf)])
    assert np.allclose(s.numpy()[0], want, rtol=0, atol=1e-12)
