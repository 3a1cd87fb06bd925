"""Streaming template search (overlap-save over chunks) against the oracle:
after every chunk the running answer equals Algorithm 1 on the prefix seen so
far (the template wholly inside), whatever the chunk sizes."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_19974_gb300 import stream, tde

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2509_19974_gb300 import build
    build.build()
    c = tde.Context(0)
    yield c
    c.close()


def _prefix_answer(qx, qy, m):
    ny = qy.shape[0]
    lo = -(m - ny)
    return oracle.argmax(oracle.xcorr(qx[:m], qy, lo, 0), lo)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_stream_matches_prefix_oracle(ctx, seed):
    rng = np.random.default_rng(900 + seed)
    nx, ny, off = 20000, 300, int(rng.integers(0, 19700))
    x = rng.standard_normal(nx).astype(np.float32)
    y = (x[off: off + ny] + 0.7 * rng.standard_normal(ny)).astype(np.float32)
    qx, qy = oracle.quantize(x, 1), oracle.quantize(y, 1)
    ts = stream.TemplateStream(ctx, torch.from_numpy(y).cuda())
    m = 0
    while m < nx:
        step = int(rng.choice([1, 7, 299, 300, 301, 1000, 4096]))
        step = min(step, nx - m)
        got = ts.push(torch.from_numpy(x[m: m + step]).cuda())
        m += step
        if m < ny:
            assert got is None
        else:
            assert got == _prefix_answer(qx, qy, m), m
    assert ts.best[0] == _prefix_answer(qx, qy, nx)[0]


def test_stream_long_signal_finds_the_template(ctx):
    rng = np.random.default_rng(77)
    nx, ny, off = 1 << 20, 4096, 654321
    x = rng.standard_normal(nx).astype(np.float32)
    y = x[off: off + ny].copy()
    ts = stream.TemplateStream(ctx, torch.from_numpy(y).cuda())
    xt = torch.from_numpy(x).cuda()
    for a in range(0, nx, 100000):
        ts.push(xt[a: a + 100000])
    qx, qy = oracle.quantize(x, 1), oracle.quantize(y, 1)
    assert ts.best == _prefix_answer(qx, qy, nx)
    assert ts.best[0] == -off  # noiseless copy: the true position (Theorem 1)


def test_stream_rejects_rank_quantizer(ctx):
    with pytest.raises(ValueError):
        stream.TemplateStream(ctx, torch.ones(8, device="cuda"), bits=2)
    import ctypes
    h = ctypes.c_void_p()
    y = torch.ones(8, device="cuda")
    assert ctx.lib.tde_stream_create(ctx.handle, y.data_ptr(), 8, 2, 0, 64, 0,
                                     ctypes.byref(h)) == tde.TDE_ERR_UNSUPPORTED


def test_stream_async_pushes_and_split_chunks(ctx):
    """Pushes enqueued without host synchronisation, chunks longer than
    max_chunk split into pieces, and several engines: the answer read at the
    end equals the oracle's on the whole signal; a chunk longer than
    max_chunk is refused by the C entry point itself."""
    rng = np.random.default_rng(55)
    nx, ny, off = 60000, 700, 31415
    x = rng.standard_normal(nx).astype(np.float32)
    y = (x[off: off + ny] + 0.5 * rng.standard_normal(ny)).astype(np.float32)
    qx, qy = oracle.quantize(x, 1), oracle.quantize(y, 1)
    want = _prefix_answer(qx, qy, nx)
    xt = torch.from_numpy(x).cuda()
    for eng in ("auto", "popc", "mma", "ntt"):
        ts = stream.TemplateStream(ctx, torch.from_numpy(y).cuda(), engine=eng, max_chunk=1000)
        assert ts.read() is None
        for a in range(0, nx, 4096):
            ts.push_async(xt[a: a + 4096])
        assert ts.read() == want, eng
        ts.close()
    ts = stream.TemplateStream(ctx, torch.from_numpy(y).cuda(), max_chunk=16)
    assert ctx.lib.tde_stream_push(ts.handle, xt.data_ptr(), 17, 0) == tde.TDE_ERR_INVALID
    ts.close()


def test_stream_fold_tie_order(ctx):
    """The device fold's order: a later chunk's equal maximum does not replace
    an earlier position (smaller |tau|), a larger value does."""
    y = torch.ones(2, device="cuda")
    ts = stream.TemplateStream(ctx, y)
    x1 = torch.tensor([-1, -1, 1, 1, -1, 1, 1], dtype=torch.float32, device="cuda")
    assert ts.push(x1) == (-2, 2)          # positions 2 and 5 tie at 2: the earlier
    x2 = torch.tensor([-1, 1, 1], dtype=torch.float32, device="cuda")
    assert ts.push(x2) == (-2, 2)          # position 8 ties again: still 2
    ts.close()
    y3 = torch.ones(3, device="cuda")
    ts = stream.TemplateStream(ctx, y3)
    assert ts.push(torch.tensor([1, 1, -1, 1], dtype=torch.float32, device="cuda")) == (0, 1)
    assert ts.push(torch.tensor([1, 1, 1], dtype=torch.float32, device="cuda")) == (-3, 3)  # 3 and 4 tie
    ts.close()

