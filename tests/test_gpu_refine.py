"""Algorithm 1's last steps on the device (tde_refine) against the oracle: the
tied set of integer maxima re-ranked by the real cross-correlation, its
representative, bounds and sizes, the real value and the sub-sample offset."""
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


def _run(ctx, x, y, bits, lo, hi, dtype=torch.int64):
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    qx, qy = ctx.quantize(xt, bits), ctx.quantize(yt, bits)
    c = ctx.xcorr_int(qx, qy, bits, lo, hi, dtype=dtype)
    got = ctx.refine(xt, yt, c, lo)
    want = oracle.refine(x, y, oracle.xcorr(oracle.quantize(x, bits), oracle.quantize(y, bits), lo, hi), lo)
    return got, want


def _check(got, want, x, y):
    for k in ("value", "n_int_ties"):
        assert got[k] == want[k], k
    scale = float(np.abs(x.astype(np.float64)).sum() * np.abs(y.astype(np.float64)).max()) + 1.0
    tol = 1e-12 * scale
    if got["lag"] == want["lag"]:
        assert abs(got["r"] - want["r"]) <= tol
        assert abs(got["frac"] - want["frac"]) <= 1e-6
        if want["n_ties"] == 1 or got["n_ties"] == want["n_ties"]:
            assert (got["lag_lo"], got["lag_hi"], got["n_ties"]) == (want["lag_lo"], want["lag_hi"],
                                                                     want["n_ties"])
    else:
        # only real values within FP64 rounding of each other may be ordered differently
        assert abs(oracle.real_ccf(x, y, got["lag"]) - want["r"]) <= tol


def test_hand_worked_cases(ctx):
    cases = [
        (np.array([1, 0, 2], np.float32), np.array([1, 0, 1, 0, 3], np.float32)),  # tie -> {2}
        (np.array([1, 0, 2], np.float32), np.array([1, 0, 3, 0, 1], np.float32)),  # tie -> {0}
        (np.array([1, 0, 1], np.float32), np.array([1, 0, 1, 0, 1], np.float32)),  # real tie {0, 2}
        (np.array([1, 2], np.float32), np.array([2, 1, 0], np.float32)),           # vertex -0.5
    ]
    for x, y in cases:
        lo, hi = oracle.full_lag_range(len(x), len(y))
        for dt in (torch.int32, torch.int64):
            got, want = _run(ctx, x, y, 1, lo, hi, dt)
            assert got == want


@pytest.mark.parametrize("n", [5, 17, 64, 300])
def test_random_short_sign_pairs(ctx, n):
    rng = np.random.default_rng(n)
    for trial in range(12):
        nx, ny = n, n + int(rng.integers(0, 9))
        x = rng.integers(-3, 4, nx).astype(np.float32)  # integers: many ties, exact reals
        y = rng.integers(-3, 4, ny).astype(np.float32)
        lo, hi = oracle.full_lag_range(nx, ny)
        if trial % 3 == 2:  # a sub-range of lags
            lo, hi = lo // 2, hi // 2
        got, want = _run(ctx, x, y, 1, lo, hi, torch.int32 if trial % 2 else torch.int64)
        assert got == want, (trial, got, want)


@pytest.mark.parametrize("bits", [1, 2])
def test_random_real_valued_pairs(ctx, bits):
    rng = np.random.default_rng(77 + bits)
    for nx, ny in ((200, 230), (1000, 1000), (4096, 3000)):
        x = rng.standard_normal(nx).astype(np.float32)
        y = rng.standard_normal(ny).astype(np.float32)
        lo, hi = oracle.full_lag_range(nx, ny)
        got, want = _run(ctx, x, y, bits, lo, hi)
        _check(got, want, x, y)


def test_full_size_pair_no_ties(ctx):
    bt = synth.equal_batch(npairs=1, n=65536)
    x, y = bt.x[0], bt.y[0]
    lo, hi = oracle.full_lag_range(65536, 65536)
    got, want = _run(ctx, x, y, 2, lo, hi, torch.int32)
    _check(got, want, x, y)
    assert got["n_int_ties"] >= 1 and got["lag_lo"] <= got["lag"] <= got["lag_hi"]


def test_refine_rejects_bad_arguments(ctx):
    x = torch.zeros(8, device="cuda")
    c = torch.zeros(15, dtype=torch.int32, device="cuda")
    with pytest.raises(tde.TdeError):
        ctx.refine(x, x, c, -8)  # lag -8 has no overlap
    with pytest.raises(TypeError):
        ctx.refine(x, x, c.float(), -7)
