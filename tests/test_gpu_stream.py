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
