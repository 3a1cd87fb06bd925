"""FP32 FFT comparator (the real-valued FFT baseline of Sec. 2.3 on the GPU):
within 1e-4 * max|c| of the exact correlation, and its argmax is one of the
exact maximisers (FP32 values near tied integer maxima may reorder, so that is
the agreement that is fixed; equality with the tie-ruled lag is not)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_19974_gb300 import tde

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2509_19974_gb300 import build
    build.build()
    c = tde.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("bits", [1, 2, 4])
@pytest.mark.parametrize("shape", [(3, 1000, 1000), (2, 777, 1500), (1, 65536, 65536)])
def test_fft32_on_levels_against_exact(ctx, bits, shape):
    npairs, nx, ny = shape
    rng = np.random.default_rng(bits * 100 + nx)
    k = 1 if bits <= 2 else 7
    qx = rng.integers(-k, k + 1, (npairs, nx)).astype(np.int8)
    qy = rng.integers(-k, k + 1, (npairs, ny)).astype(np.int8)
    # plant a shifted copy so that each pair has a clear peak
    qy[:, 10: 10 + min(nx, ny) // 2] = qx[:, : min(nx, ny) // 2]
    c = ctx.xcorr_fft32(torch.from_numpy(qx).cuda(), torch.from_numpy(qy).cuda())
    torch.cuda.synchronize()
    c = c.cpu().numpy().astype(np.float64)
    for p in range(npairs):
        ref = oracle.xcorr(qx[p], qy[p]).astype(np.float64)
        assert np.abs(c[p] - ref).max() <= 1e-4 * np.abs(ref).max()
        assert ref[int(np.argmax(c[p]))] == ref.max()


def test_fft32_on_floats_restricted_lags(ctx):
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 3000)).astype(np.float32)
    y = rng.standard_normal((2, 2500)).astype(np.float32)
    lo, hi = -1200, 800
    c = ctx.xcorr_fft32(torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda(), lo, hi)
    torch.cuda.synchronize()
    c = c.cpu().numpy().astype(np.float64)
    for p in range(2):
        full = np.correlate(y[p].astype(np.float64), x[p].astype(np.float64), "full")
        ref = full[lo + 2999: hi + 2999 + 1]
        assert np.abs(c[p] - ref).max() <= 1e-4 * np.abs(full).max()
