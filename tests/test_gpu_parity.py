"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Bit-exact everywhere: quantized levels, correlations and the tie-ruled lag are
integers.  Sizes span several CTA tiles of each engine with ragged tails; the
edge cases cover N = 1, nx != ny, restricted lag ranges touching +-(N-1),
exact zeros and -0.0, constant signals (massive ties), the largest values the
levels allow, and the host-side and device-side error paths.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2509_19974_gb300 import synth, tde

pytestmark = pytest.mark.gpu

ENGINES = ["popc", "mma", "ntt"]


@pytest.fixture(scope="module")
def ctx():
    from paper_2509_19974_gb300 import build
    build.build()
    c = tde.Context(0)
    yield c
    c.close()


def _gpu(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _levels(rng, n, bits, p_zero=0.2):
    k = (1 << (bits - 1)) - 1 if bits > 1 else 1
    q = rng.integers(-k, k + 1, size=n).astype(np.int8)
    q[rng.random(n) < p_zero] = 0
    return q


# ------------------------------------------------------------------ step A

@pytest.mark.parametrize("bits", [1, 2, 4])
@pytest.mark.parametrize("n", [1, 2, 3, 31, 1000, 4097, 65536 + 123])
def test_quantize_matches_oracle(ctx, bits, n):
    rng = np.random.default_rng(n * 7 + bits)
    x = rng.standard_normal(n).astype(np.float32)
    x[rng.random(n) < 0.05] = 0.0
    if n > 5:
        x[3] = -0.0
        x[4] = x[5]           # a tie in |x|
        x[1] = -x[2]
    got = ctx.quantize(_gpu(x), bits)
    ctx.sync()
    assert np.array_equal(got.cpu().numpy(), oracle.quantize(x, bits))


@pytest.mark.parametrize("bits", [2, 4])
def test_quantize_heavy_ties_and_scales(ctx, bits):
    rng = np.random.default_rng(11)
    # many equal magnitudes (few distinct values), huge and tiny exponents
    x = rng.choice(np.array([0.0, 1.0, -1.0, 2.5, -2.5, 1e-38, -3e38, 7.0], np.float32), 20001)
    got = ctx.quantize(_gpu(x), bits)
    ctx.sync()
    assert np.array_equal(got.cpu().numpy(), oracle.quantize(x, bits))
    # constant signal
    x = np.full(5000, -3.25, np.float32)
    got = ctx.quantize(_gpu(x), bits)
    ctx.sync()
    assert np.array_equal(got.cpu().numpy(), oracle.quantize(x, bits))


@pytest.mark.parametrize("bits", [2, 4])
@pytest.mark.parametrize("xoff,qoff", [(1, 0), (0, 3), (3, 1)])
def test_quantize_unaligned_buffers(ctx, bits, xoff, qoff):
    """x not 16-byte aligned or q not 4-byte aligned: the one-launch
    quantizer takes its per-sample path for the whole signal."""
    rng = np.random.default_rng(31 * xoff + qoff + bits)
    n = 9000 + 7
    x = rng.standard_normal(n).astype(np.float32)
    x[::13] = 0.0
    xb = torch.zeros(n + 4, dtype=torch.float32, device="cuda")
    xb[xoff:xoff + n] = _gpu(x)
    qb = torch.zeros(n + 4, dtype=torch.int8, device="cuda")
    got = ctx.quantize(xb[xoff:xoff + n], bits, q_out=qb[qoff:qoff + n])
    ctx.sync()
    assert np.array_equal(got.cpu().numpy(), oracle.quantize(x, bits))
    assert int(qb[:qoff].abs().sum()) == 0 and int(qb[qoff + n:].abs().sum()) == 0


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf])
@pytest.mark.parametrize("bits", [1, 2, 4])
def test_quantize_nonfinite_is_reported(ctx, bits, bad):
    x = np.ones(777, np.float32)
    x[500] = bad
    ctx.quantize(_gpu(x), bits)
    with pytest.raises(tde.TdeError) as e:
        ctx.sync()
    assert e.value.status == tde.TDE_ERR_INVALID
    ctx.sync()  # the status word was cleared


# ------------------------------------------------------------------ step B

CASES = [
    # nx, ny, lag range (None = full)
    (1, 1, None),
    (1, 77, None),
    (77, 1, None),
    (33, 65, None),
    (5000, 4097, None),
    (4096, 4096, None),
    (20000 + 37, 19000 + 5, None),
    (20000, 20000, (-19999, -19000)),
    (20000, 20000, (18500, 19999)),
    (20000, 20000, (-1, 1)),
    (20000, 20000, (0, 0)),
    (9000, 30000, (-8999, 29999)),
]


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("bits", [1, 2, 4])
@pytest.mark.parametrize("case", CASES, ids=[f"{a}x{b}-{r}" for a, b, r in CASES])
def test_xcorr_matches_oracle(ctx, engine, bits, case):
    nx, ny, rng_lags = case
    rng = np.random.default_rng(nx * 31 + ny + bits)
    qx, qy = _levels(rng, nx, bits), _levels(rng, ny, bits)
    lo, hi = rng_lags if rng_lags else (-(nx - 1), ny - 1)
    for dtype in (torch.int32, torch.int64):
        c = ctx.xcorr_int(_gpu(qx), _gpu(qy), bits, lo, hi, engine=engine, dtype=dtype)
        ctx.sync()
        ref = oracle.xcorr(qx, qy, lo, hi)
        assert np.array_equal(c.cpu().numpy().astype(np.int64), ref)


@pytest.mark.parametrize("engine", ENGINES)
def test_xcorr_long_pair_restricted_lags(ctx, engine):
    """The longest pairs of the uneven batch: 262144 samples, lags +-32768
    (the NTT needs a 2^19 transform here)."""
    n, w = 262144, 32768
    rng = np.random.default_rng(5)
    qx, qy = _levels(rng, n, 2), _levels(rng, n, 2)
    c = ctx.xcorr_int(_gpu(qx), _gpu(qy), 2, -w, w, engine=engine)
    ctx.sync()
    got = c.cpu().numpy().astype(np.int64)
    lags = np.concatenate([np.arange(-w, -w + 300), rng.integers(-w, w + 1, 2000),
                           np.arange(w - 300, w + 1)])
    assert np.array_equal(got[lags + w], oracle.xcorr_at(qx, qy, lags))
    assert got.sum() == int(oracle.xcorr(qx, qy, -w, w).sum())


@pytest.mark.parametrize("engine", ENGINES)
def test_xcorr_extreme_values(ctx, engine):
    """All +7 against all +7 (the largest |c|), and alternating signs."""
    n = 30011
    q = np.full(n, 7, np.int8)
    c = ctx.xcorr_int(_gpu(q), _gpu(q), 4, engine=engine)
    ctx.sync()
    assert np.array_equal(c.cpu().numpy().astype(np.int64), oracle.xcorr(q, q))
    q = np.where(np.arange(n) % 2 == 0, 1, -1).astype(np.int8)
    c = ctx.xcorr_int(_gpu(q), _gpu(q), 2, engine=engine)
    ctx.sync()
    assert np.array_equal(c.cpu().numpy().astype(np.int64), oracle.xcorr(q, q))


def test_xcorr_host_errors(ctx):
    q = _gpu(np.ones(100, np.int8))
    with pytest.raises(tde.TdeError) as e:
        ctx.xcorr_int(q, q, 3)
    assert e.value.status == tde.TDE_ERR_INVALID
    with pytest.raises(tde.TdeError) as e:
        ctx.xcorr_int(q, q, 1, -100, 0)
    assert e.value.status == tde.TDE_ERR_INVALID
    with pytest.raises(tde.TdeError) as e:
        ctx.xcorr_int(q, q, 1, 5, 4)
    assert e.value.status == tde.TDE_ERR_INVALID
    big = torch.zeros(40_000_000, dtype=torch.int8, device="cuda")
    with pytest.raises(tde.TdeError) as e:
        ctx.xcorr_int(big, big, 4, 0, 0)
    assert e.value.status == tde.TDE_ERR_OVERFLOW
    del big


def test_xcorr_level_out_of_range_is_reported(ctx):
    q = np.ones(300, np.int8)
    q[7] = 2
    ctx.xcorr_int(_gpu(q), _gpu(q), 2, engine="popc")
    with pytest.raises(tde.TdeError):
        ctx.sync()


# ------------------------------------------------------------------ step C

def test_argmax_tie_cases(ctx):
    cases = [
        (np.full(9, 5), -4),
        (np.array([0, 0, 7, 0, 0, 0, 0, 0, 7, 0, 0]), -5),
        (np.array([0, 0, 7, 0, 0, 0, 0, 7, 0, 0, 0]), -5),
        (np.array([1, 4, 4, 4]), 10),
        (np.array([4, 4, -9]), -10),
        (np.array([-8, -2, -5]), 0),
        (np.array([-8]), 77),
        (np.array([-(2**31), -(2**31)]), -1),
        (np.array([2**31 - 1, 2**31 - 1, 0]), -1),
    ]
    for c, lag_min in cases:
        want = oracle.argmax(c.astype(np.int64), lag_min)
        for dt in (np.int32, np.int64):
            lag, val = ctx.argmax(_gpu(c.astype(dt)), lag_min)
            assert (int(lag.item()), int(val.item())) == want, (c, lag_min, dt)


def test_argmax_large_random(ctx):
    rng = np.random.default_rng(5)
    for n in (1, 1000, 1 << 20, (1 << 22) + 3):
        c = rng.integers(-50, 50, size=n)
        lag_min = int(rng.integers(-n, 1))
        want = oracle.argmax(c, lag_min)
        for dt in (np.int32, np.int64):
            lag, val = ctx.argmax(_gpu(c.astype(dt)), lag_min)
            assert (int(lag.item()), int(val.item())) == want


# --------------------------------------------------------- steps A-C together

@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("bits", [1, 2, 4])
def test_estimate_single_pair(ctx, engine, bits):
    b = synth.single_pair(bits=bits)
    lag, val = ctx.estimate(_gpu(b.x[0]), _gpu(b.y[0]), bits, engine=engine)
    assert (int(lag.item()), int(val.item())) == oracle.estimate(b.x[0], b.y[0], bits)


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("bits", [1, 2, 4])
def test_estimate_batch_uneven(ctx, engine, bits):
    """Uneven lengths and lag ranges (a reduced copy of the 4096-pair
    log-uniform workload), correlations and lags against the oracle."""
    b = synth.uneven_batch(npairs=12, n_lo=64, n_hi=12000, bits=bits)
    xs = [_gpu(v) for v in b.x]
    ys = [_gpu(v) for v in b.y]
    counts = (b.lag_max - b.lag_min + 1).astype(np.int64)
    c_out = torch.empty(int(counts.sum()), dtype=torch.int32, device="cuda")
    lags, vals = ctx.estimate_batch(xs, ys, bits, b.lag_min, b.lag_max, engine=engine,
                                    c_out=c_out)
    ctx.sync()
    c_all = c_out.cpu().numpy().astype(np.int64)
    off = 0
    for p in range(b.npairs):
        qx, qy = oracle.quantize(b.x[p], bits), oracle.quantize(b.y[p], bits)
        ref = oracle.xcorr(qx, qy, int(b.lag_min[p]), int(b.lag_max[p]))
        assert np.array_equal(c_all[off: off + counts[p]], ref), p
        off += counts[p]
        assert (int(lags[p]), int(vals[p])) == oracle.argmax(ref, int(b.lag_min[p]))


def test_estimate_constant_signals_tie_to_zero(ctx):
    x = np.full(3000, 0.5, np.float32)
    lag, val = ctx.estimate(_gpu(x), _gpu(x), 1)
    assert (int(lag.item()), int(val.item())) == (0, 3000)


@pytest.mark.parametrize("bits", [2, 4])
def test_quantize_many_signals_batched(ctx, bits):
    """512 signals in one batched call (one CTA per signal per select pass):
    every signal's levels equal the oracle's, on two calls in a row."""
    rng = np.random.default_rng(77 + bits)
    X = rng.standard_normal((512, 65536)).astype(np.float32)
    X[:, ::50] = 0.0
    xd = torch.from_numpy(X).cuda()
    q1 = tde.tde_quantize_batch(ctx, xd, bits)
    q2 = tde.tde_quantize_batch(ctx, xd, bits)
    ctx.sync()
    assert torch.equal(q1, q2)
    q1 = q1.cpu().numpy()
    for i in range(512):
        assert np.array_equal(q1[i], oracle.quantize(X[i], bits)), i
