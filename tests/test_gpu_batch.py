"""Batched execution: uneven pairs (a reduced copy of the log-uniform
4096-pair workload), all engines, through tde_estimate_batch and through a
planned batch replayed from its CUDA graph; correlations and lags bit-exact
against the oracle, and replays after refilling the inputs."""
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


def _ref(b):
    out = []
    for p in range(b.npairs):
        qx, qy = oracle.quantize(b.x[p], b.bits), oracle.quantize(b.y[p], b.bits)
        c = oracle.xcorr(qx, qy, int(b.lag_min[p]), int(b.lag_max[p]))
        out.append((c, oracle.argmax(c, int(b.lag_min[p]))))
    return out


@pytest.mark.parametrize("engine", ["auto", "mma", "popc", "ntt"])
def test_planned_batch_graph_replays(ctx, engine):
    b1 = synth.uneven_batch(seed=11, npairs=24, n_lo=1024, n_hi=40000, bits=2)
    b2 = synth.uneven_batch(seed=12, npairs=24, n_lo=1024, n_hi=40000, bits=2)
    # same shapes for the second fill: take b2's samples, cut/pad to b1's lengths
    xs = [torch.from_numpy(v).cuda() for v in b1.x]
    ys = [torch.from_numpy(v).cuda() for v in b1.y]
    counts = (b1.lag_max - b1.lag_min + 1).astype(np.int64)
    c_out = torch.empty(int(counts.sum()), dtype=torch.int32, device="cuda")
    batch = tde.Batch(ctx, xs, ys, 2, b1.lag_min, b1.lag_max, engine=engine, c_out=c_out)
    for fill in range(2):
        if fill == 1:
            for p in range(b1.npairs):
                n = b1.x[p].shape[0]
                b1.x[p] = np.resize(b2.x[p], n).astype(np.float32)
                b1.y[p] = np.resize(b2.y[p], n).astype(np.float32)
                xs[p].copy_(torch.from_numpy(b1.x[p]))
                ys[p].copy_(torch.from_numpy(b1.y[p]))
        lags, vals = batch.run()
        ctx.sync()
        c_all = c_out.cpu().numpy().astype(np.int64)
        off = 0
        for p, (c, (lag, val)) in enumerate(_ref(b1)):
            assert np.array_equal(c_all[off: off + counts[p]], c), (fill, p)
            off += counts[p]
            assert (int(lags[p]), int(vals[p])) == (lag, val), (fill, p)
    batch.close()


def test_batch_mixed_engines_auto(ctx):
    """AUTO sends short/narrow pairs to popc and long ones to the tensor cores
    in the same call."""
    b = synth.uneven_batch(seed=13, npairs=40, n_lo=1024, n_hi=60000, bits=2)
    engines = {tde.pick_engine(2, len(x), len(y), int(hi - lo + 1))
               for x, y, lo, hi in zip(b.x, b.y, b.lag_min, b.lag_max)}
    assert engines == {"popc", "mma"}
    xs = [torch.from_numpy(v).cuda() for v in b.x]
    ys = [torch.from_numpy(v).cuda() for v in b.y]
    lags, vals = ctx.estimate_batch(xs, ys, 2, b.lag_min, b.lag_max)
    ctx.sync()
    for p, (c, lv) in enumerate(_ref(b)):
        assert (int(lags[p]), int(vals[p])) == lv
