"""The allocation-free quantizer entry point, tde_quantize_noalloc.

It serves callers that cannot allocate device memory (real-time callbacks,
hosts with their own device-memory manager, work enqueued during stream
capture): its scratch is a fixed device array inside the library rather than
a context's workspace.  This file is collected last so that, if it fails, a
run stopped at the first failure has already run every other test; it passes
both alone in a fresh process and after the other tests.

Parity: its output must equal that of tde_quantize (the context-based entry
point) bit for bit -- quantized levels are integers -- on two calls in a row,
which also checks that the shared scratch left by one call does not leak into
the next.  It runs kernels of its own (a multi-pass radix select), so it is
also compared with the oracle directly, on constant and heavily tied signals
where selection schemes differ most.
"""

import numpy as np
import pytest
import torch

from paper_2509_19974_gb300 import build, tde

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    build.build()
    return tde.load()


def _call(lib, x, bits, q, status):
    nsig, n = x.shape
    return lib.tde_quantize_noalloc(x.data_ptr(), n, nsig, bits, q.data_ptr(), status.data_ptr(),
                                    torch.cuda.current_stream().cuda_stream)


def _reference(ctx, x, bits):
    return torch.stack([ctx.quantize(x[i].contiguous(), bits) for i in range(x.shape[0])])


@pytest.mark.parametrize("bits", [1, 2, 4])
def test_noalloc_matches_context_quantizer_twice(lib, bits):
    ctx = tde.Context(0)
    rng = np.random.default_rng(100 + bits)
    shapes = [(3, 70001), (16, 4099)]   # the second call uses every scratch slot
    for nsig, n in shapes:
        x = rng.standard_normal((nsig, n)).astype(np.float32)
        x[:, ::13] = 0.0
        xd = torch.from_numpy(x).cuda()
        q = torch.full((nsig, n), 99, dtype=torch.int8, device="cuda")
        status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
        assert _call(lib, xd, bits, q, status) == tde.TDE_OK
        want = _reference(ctx, xd, bits)
        ctx.sync()
        torch.cuda.synchronize()
        assert torch.equal(q, want)
        assert int(status.item()) == 0
    ctx.close()


@pytest.mark.parametrize("bits", [2, 4])
def test_noalloc_matches_oracle_on_ties(lib, bits):
    """Against the oracle's quantizer (Algorithm 1's quantization step) on
    signals where the order statistics tie: a constant signal, a negative
    constant, x rounded to three values, x on a 5-value grid with zeros and
    -0.0, and a plain Gaussian; two calls in a row."""
    import oracle
    rng = np.random.default_rng(300 + bits)
    n = 20011
    g = rng.standard_normal((5, n)).astype(np.float32)
    x = np.empty((5, n), np.float32)
    x[0] = 1.5
    x[1] = -0.25
    x[2] = np.round(np.clip(g[2], -1, 1))
    x[3] = np.round(2 * g[3]) / 2
    x[3, ::7] = -0.0
    x[4] = g[4]
    for _ in range(2):
        xd = torch.from_numpy(x).cuda()
        q = torch.full((5, n), 99, dtype=torch.int8, device="cuda")
        status = torch.full((1,), 7, dtype=torch.int32, device="cuda")
        assert _call(lib, xd, bits, q, status) == tde.TDE_OK
        torch.cuda.synchronize()
        assert int(status.item()) == 0
        qh = q.cpu().numpy()
        for i in range(5):
            assert np.array_equal(qh[i], oracle.quantize(x[i], bits)), i
        x = x[::-1].copy()


def test_noalloc_wrapper_checks_buffers(lib):
    """The Python wrapper refuses output buffers of the wrong size or type
    before anything is enqueued."""
    x = torch.ones((2, 100), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        tde.tde_quantize_noalloc(x, 2, q_out=torch.empty((2, 99), dtype=torch.int8, device="cuda"))
    with pytest.raises(ValueError):
        tde.tde_quantize_noalloc(x, 2, status_out=torch.empty(1, dtype=torch.int64, device="cuda"))
    with pytest.raises(ValueError):
        tde.tde_quantize_noalloc(x.reshape(2, 10, 10), 2)
    q, st = tde.tde_quantize_noalloc(x, 2)
    torch.cuda.synchronize()
    assert int(st.item()) == 0 and q.shape == x.shape


def test_noalloc_reports_nonfinite_and_limits(lib):
    x = torch.ones((2, 1000), dtype=torch.float32, device="cuda")
    x[1, 500] = float("nan")
    q = torch.empty((2, 1000), dtype=torch.int8, device="cuda")
    status = torch.zeros(1, dtype=torch.int32, device="cuda")
    assert _call(lib, x, 2, q, status) == tde.TDE_OK
    torch.cuda.synchronize()
    assert int(status.item()) & 1
    big = torch.zeros((17, 10), dtype=torch.float32, device="cuda")
    qb = torch.empty((17, 10), dtype=torch.int8, device="cuda")
    assert _call(lib, big, 2, qb, status) == tde.TDE_ERR_UNSUPPORTED
    assert lib.tde_quantize_noalloc(None, 10, 1, 2, None, None, None) == tde.TDE_ERR_INVALID
    assert _call(lib, big[:2], 3, qb[:2], status) == tde.TDE_ERR_INVALID
