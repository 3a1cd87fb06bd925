"""The NTT engine's two arithmetics (Sec. 3.2's multimodular route): one prime
(the default wherever the values fit its centred residues) and two primes
recombined by CRT (forced on a second context).  Both against the oracle,
bit-exact, on ragged lengths, every bit width, the largest values the levels
allow, the longest template the engine takes, and a planned batch."""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_19974_gb300 import synth, tde

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctxs():
    from paper_2509_19974_gb300 import build
    build.build()
    one, two = tde.Context(0), tde.Context(0)
    two.set_ntt_primes(2)
    yield {1: one, 2: two}
    one.close()
    two.close()


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _levels(rng, n, bits):
    k = (1 << (bits - 1)) - 1 if bits > 1 else 1
    return rng.integers(-k, k + 1, size=n).astype(np.int8)


@pytest.mark.parametrize("nprimes", [1, 2])
@pytest.mark.parametrize("bits", [1, 2, 4])
@pytest.mark.parametrize("nx,ny,lags", [(1, 1, None), (1000, 3001, None), (4097, 4097, None),
                                        (70001, 2049, (-70000, 0)), (20000, 20000, (-5, 7))])
def test_both_arithmetics_match_oracle(ctxs, nprimes, bits, nx, ny, lags):
    rng = np.random.default_rng(nx + 3 * ny + bits)
    qx, qy = _levels(rng, nx, bits), _levels(rng, ny, bits)
    lo, hi = lags if lags else (-(nx - 1), ny - 1)
    c = ctxs[nprimes].xcorr_int(_gpu(qx), _gpu(qy), bits, lo, hi, engine="ntt", dtype=torch.int64)
    ctxs[nprimes].sync()
    assert np.array_equal(c.cpu().numpy(), oracle.xcorr(qx, qy, lo, hi))


@pytest.mark.parametrize("nprimes", [1, 2])
def test_extremes_at_the_longest_template(ctxs, nprimes):
    """The longest template the engine takes (7/8 of 2^19 samples) with every
    level at +-7: |c| reaches 458752 * 49, the largest value one prime must
    hold; sampled lags plus the ends against the oracle."""
    nt = 458752
    qx = np.full(nt, 7, np.int8)
    qy = np.full(nt + 1000, -7, np.int8)
    qy[::997] = 7
    lo, hi = -(nt - 1), nt + 999
    c = ctxs[nprimes].xcorr_int(_gpu(qx), _gpu(qy), 4, lo, hi, engine="ntt", dtype=torch.int64)
    ctxs[nprimes].sync()
    got = c.cpu().numpy()
    rng = np.random.default_rng(9)
    lags = np.concatenate([np.arange(lo, lo + 50), rng.integers(lo, hi + 1, 400),
                           np.arange(-60, 1100), np.arange(hi - 50, hi + 1)])
    assert np.array_equal(got[lags - lo], oracle.xcorr_at(qx, qy, lags))
    assert got.min() < -49 * nt * 99 // 100  # near the bound the one prime must hold


@pytest.mark.parametrize("bits", [2, 4])
def test_batch_graph_both_arithmetics(ctxs, bits):
    b = synth.uneven_batch(npairs=10, n_lo=1024, n_hi=40000, bits=bits)
    xs, ys = [_gpu(v) for v in b.x], [_gpu(v) for v in b.y]
    out = {}
    for nq, ctx in ctxs.items():
        lags, vals = ctx.estimate_batch(xs, ys, bits, b.lag_min, b.lag_max, engine="ntt")
        ctx.sync()
        out[nq] = [(int(l), int(v)) for l, v in zip(lags, vals)]
    assert out[1] == out[2]
    for p in range(b.npairs):
        qx, qy = oracle.quantize(b.x[p], bits), oracle.quantize(b.y[p], bits)
        ref = oracle.xcorr(qx, qy, int(b.lag_min[p]), int(b.lag_max[p]))
        assert out[1][p] == oracle.argmax(ref, int(b.lag_min[p]))


def test_bad_prime_count_is_rejected(ctxs):
    for bad in (-1, 1, 3):
        with pytest.raises(tde.TdeError):
            ctxs[1].set_ntt_primes(bad)
