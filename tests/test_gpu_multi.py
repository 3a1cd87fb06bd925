"""The lag-sharded template search through the library's kernels: every
emulated rank's shard (sequentially, on one GPU) combined by the cross-rank
rule equals the oracle's unsharded answer; the one-rank entry point too."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_19974_gb300 import multi, tde

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_2509_19974_gb300 import build
    build.build()
    c = tde.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("bits", [1, 2, 4])
def test_sharded_template_search_equals_oracle(ctx, bits):
    rng = np.random.default_rng(40 + bits)
    nx, ny, off = 40000, 3000, 12345
    x = rng.standard_normal(nx).astype(np.float32)
    y = (x[off: off + ny] + 0.5 * rng.standard_normal(ny)).astype(np.float32)
    lo, hi = -(nx - ny), 0  # y wholly inside x
    qx, qy = oracle.quantize(x, bits), oracle.quantize(y, bits)
    want = oracle.argmax(oracle.xcorr(qx, qy, lo, hi), lo)
    assert want[0] == -off
    xt, yt = torch.from_numpy(x).cuda(), torch.from_numpy(y).cuda()
    assert multi.template_search(ctx, xt, yt, bits, lo, hi) == want
    gqx, gqy = ctx.quantize(xt, bits), ctx.quantize(yt, bits)
    for world in (2, 3, 8):
        locs = [multi.shard_argmax(ctx, gqx, gqy, bits, a, b)
                for a, b in multi.lag_shards(lo, hi, world)]
        assert multi.combine_argmax(locs) == want


def test_sharded_search_ties_across_shards(ctx):
    # constant signals: every full-overlap lag ties; the answer is lag 0
    x = torch.ones(257, device="cuda")
    y = torch.ones(257, device="cuda")
    gqx, gqy = ctx.quantize(x, 1), ctx.quantize(y, 1)
    locs = [multi.shard_argmax(ctx, gqx, gqy, 1, a, b) for a, b in multi.lag_shards(-256, 256, 4)]
    assert multi.combine_argmax(locs) == (0, 257)
