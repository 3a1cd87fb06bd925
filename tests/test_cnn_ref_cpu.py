"""Pins of the float64 CNN reference (oracle/cnn_ref.py) to things other than
itself: central finite differences of its loss agree with its autograd
gradient, and swapping x and y mirrors the scores (score_yx[l] = score_xy[-l]).
CPU only."""
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
