"""Float64 CPU reference of the lag-proposal CNN -- test infrastructure only.

Plain PyTorch CPU ops in float64 (conv1d, ReLU, max-pool, a correlation of
the feature maps, softmax cross-entropy) written from the architecture the
library documents (include/tde.h: 16x block-sum decimation / 4, four
[conv k9 pad 4, 32 channels, bias, ReLU, max-pool 2] layers shared by x and
y, score[l] = alpha sum_c sum_i fx[c][i] fy[c][i + l]).  The proposal is not
part of the paper's method; these are the definitions its kernels must match.
Parity: this file is the reference; its pins (tests/test_cnn_ref_cpu.py) are a
finite-difference check of its gradient, the forward restated as explicit
sums, and a closed form with pass-through weights.
"""
from __future__ import annotations

import numpy as np
import torch

C, K, LAYERS, DEC, BIN = 32, 9, 4, 16, 256


def layout():
    """[(w_off, b_off, cin)] per layer and the alpha offset."""
    out, off = [], 0
    for l in range(LAYERS):
        cin = 1 if l == 0 else C
        out.append((off, off + C * cin * K, cin))
        off += C * cin * K + C
    return out, off


def bf16_round(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest BF16 (ties to even)."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def forward(params, q2: np.ndarray):
    """params: float64 tensor (requires_grad allowed); q2: [2P, n] int8.
    Returns (features [2P, 32, n/256], scores [P, 2 Lf - 1])."""
    lay, a_off = layout()
    x = torch.from_numpy(q2.astype(np.float64))
    S, n = x.shape
    h = x.view(S, 1, n // DEC, DEC).sum(-1) * 0.25
    for (wo, bo, cin) in lay:
        W = params[wo: bo].view(C, cin, K)
        b = params[bo: bo + C]
        h = torch.nn.functional.conv1d(h, W, b, padding=K // 2)
        h = torch.nn.functional.max_pool1d(torch.relu(h), 2)
    f = h  # [S, 32, Lf]
    Lf = f.shape[-1]
    fx, fy = f[0::2], f[1::2]
    fyp = torch.nn.functional.pad(fy, (Lf - 1, Lf - 1))
    scores = []
    for b in range(2 * Lf - 1):      # lag l = b - (Lf - 1): fy[i + l] = fyp[i + b]
        scores.append((fx * fyp[..., b: b + Lf]).sum(dim=(1, 2)))
    return f, params[a_off] * torch.stack(scores, dim=1)


def label_bins(labels: np.ndarray, Lf: int) -> np.ndarray:
    b = np.floor((labels.astype(np.int64) + BIN // 2) / BIN).astype(np.int64)
    return np.clip(b, -(Lf - 1), Lf - 1) + Lf - 1


def loss_and_grad(params_np: np.ndarray, q2: np.ndarray, labels: np.ndarray):
    """Mean softmax cross-entropy over pairs and its gradient (float64), with
    the conv weights taken as given (pass BF16-rounded values to mirror the
    device's forward pass)."""
    p = torch.tensor(params_np, dtype=torch.float64, requires_grad=True)
    f, s = forward(p, q2)
    t = torch.from_numpy(label_bins(labels, f.shape[-1]))
    per = torch.nn.functional.cross_entropy(s, t, reduction="none")
    per.mean().backward()
    return per.detach().numpy(), p.grad.numpy()
