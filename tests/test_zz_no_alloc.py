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
the next.
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
