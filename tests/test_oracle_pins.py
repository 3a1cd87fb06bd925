"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand, an off-by-one threshold, a wrong
tie rule) fails at least one of them.  CPU only.
"""
import itertools

import numpy as np
import pytest

import oracle
from paper_2509_19974_gb300 import synth
from tests._golden import read_cases


def _ints(rng, n, k):
    return rng.integers(-k, k + 1, size=n).astype(np.int8)


# ---------------------------------------------------------------- Eq. (1)

def _ccf_by_pairs(x, y):
    """Eq. (1) as a sum over the outer product binned by index difference:
    every pair (m, m') contributes x[m] y[m'] to lag m' - m."""
    out = {}
    for m, xv in enumerate(x.tolist()):
        for mp, yv in enumerate(y.tolist()):
            out[mp - m] = out.get(mp - m, 0) + xv * yv
    return out


def test_ccf_golden_hand_computed():
    for case in read_cases("ccf_small.txt"):
        x = np.array(case["x"], dtype=np.int8)
        y = np.array(case["y"], dtype=np.int8)
        lag_min = int(case["lag_min"][0])
        want = np.array(case["c"], dtype=np.int64)
        got = oracle.xcorr(x, y, lag_min, lag_min + len(want) - 1)
        assert np.array_equal(got, want)
        assert oracle.argmax(got, lag_min) == tuple(int(v) for v in case["argmax"])


def test_ccf_exhaustive_ternary_tiny():
    """Brute force over every x, y in {-1,0,1}^n, 1 <= n <= 3 (and 4 x 2)."""
    shapes = [(1, 1), (1, 3), (2, 2), (3, 1), (3, 3), (4, 2), (2, 4)]
    for nx, ny in shapes:
        for xv in itertools.product((-1, 0, 1), repeat=nx):
            x = np.array(xv, dtype=np.int8)
            for yv in itertools.product((-1, 0, 1), repeat=ny):
                y = np.array(yv, dtype=np.int8)
                c = oracle.xcorr(x, y)
                ref = _ccf_by_pairs(x, y)
                assert [ref[t] for t in range(-(nx - 1), ny)] == c.tolist()


def test_ccf_onehot_lag_convention():
    """x = e_i, y = e_j: x[n] = y[n + (j - i)], so by Eq. (2)-(3) the only
    nonzero lag is j - i (positive lag means y is later)."""
    for nx, ny in [(5, 7), (7, 5), (1, 6)]:
        for i in range(nx):
            for j in range(ny):
                x = np.zeros(nx, np.int8)
                y = np.zeros(ny, np.int8)
                x[i] = 1
                y[j] = 1
                c = oracle.xcorr(x, y)
                lags = np.arange(-(nx - 1), ny)
                assert np.array_equal(c, (lags == j - i).astype(np.int64))


def test_ccf_matches_numpy_correlate():
    """Library correlation: numpy.correlate(y, x, 'full')[tau + nx - 1]; the
    index map is the one the one-hot test fixes."""
    rng = np.random.default_rng(1)
    for nx, ny, k in [(1, 1, 1), (17, 33, 1), (64, 63, 7), (300, 129, 1), (1000, 1000, 7)]:
        x, y = _ints(rng, nx, k), _ints(rng, ny, k)
        ref = np.correlate(y.astype(np.int64), x.astype(np.int64), "full")
        assert np.array_equal(oracle.xcorr(x, y), ref)


def _ks_correlation(x, y, k):
    """Kronecker substitution (Sec. 3.2, complexity paragraph): correlation is
    the convolution of x with the reversed y; evaluate both polynomials at 2^L
    with 2^L > 2 N K^2, multiply as integers, recover signed base-2^L digits."""
    n = max(len(x), len(y))
    L = int(np.floor(np.log2(n * k * k))) + 2
    yr = y[::-1]
    U = sum(int(v) << (L * i) for i, v in enumerate(x.tolist()))
    V = sum(int(v) << (L * i) for i, v in enumerate(yr.tolist()))
    W = U * V
    coeffs = []
    half, mask = 1 << (L - 1), (1 << L) - 1
    for _ in range(len(x) + len(y) - 1):
        d = W & mask
        if d >= half:
            d -= 1 << L
        coeffs.append(d)
        W = (W - d) >> L
    assert W == 0
    # (x conv yr)[p] = c[ny - 1 - p]
    return np.array(coeffs[::-1], dtype=np.int64)


def test_ccf_matches_kronecker_substitution():
    rng = np.random.default_rng(2)
    for nx, ny, k in [(8, 8, 1), (31, 40, 1), (128, 128, 7), (2048, 1500, 1), (4096, 4096, 7)]:
        x, y = _ints(rng, nx, k), _ints(rng, ny, k)
        assert np.array_equal(oracle.xcorr(x, y), _ks_correlation(x, y, k))


def test_ccf_sum_identity_and_symmetry():
    rng = np.random.default_rng(3)
    for nx, ny in [(1, 9), (50, 50), (513, 77), (4096, 4096)]:
        x, y = _ints(rng, nx, 7), _ints(rng, ny, 7)
        c = oracle.xcorr(x, y)
        assert c.sum() == int(x.astype(np.int64).sum()) * int(y.astype(np.int64).sum())
        # c_xy[tau] = c_yx[-tau]
        assert np.array_equal(c, oracle.xcorr(y, x)[::-1])


def test_ccf_restricted_range_and_at():
    rng = np.random.default_rng(4)
    x, y = _ints(rng, 700, 1), _ints(rng, 500, 1)
    full = oracle.xcorr(x, y)
    lo = -(700 - 1)
    assert np.array_equal(oracle.xcorr(x, y, -10, 25), full[-10 - lo: 26 - lo])
    lags = np.array([-699, -1, 0, 3, 499, -250])
    assert np.array_equal(oracle.xcorr_at(x, y, lags), full[lags - lo])
    # lags outside the overlap are empty sums
    assert np.array_equal(oracle.xcorr(x, y, 500, 502), np.zeros(3, np.int64))


# -------------------------------------------------- Algorithm 1's quantization step

def test_quantize_golden_hand_computed():
    for case in read_cases("quantize_small.txt"):
        x = np.array([float(v) for v in case["x"]], dtype=np.float32)
        want = np.array(case["q"], dtype=np.int8)
        assert np.array_equal(oracle.quantize(x, int(case["bits"][0])), want)


def test_quantize_sign_closed_form():
    x = np.array([3.5, -1e-30, 0.0, -0.0, 1e30, -2.0, 1.4e-45], np.float32)
    assert oracle.quantize(x, 1).tolist() == [1, -1, 0, 0, 1, -1, 1]


@pytest.mark.parametrize("bits", [2, 4])
@pytest.mark.parametrize("n", [1, 2, 3, 14, 15, 16, 1000, 4097])
def test_rank_quantizer_level_populations(bits, n):
    """With distinct |x|, #{|q| >= m} = n - min(n-1, floor((2m-1) n / L))."""
    rng = np.random.default_rng(n * 10 + bits)
    mag = rng.permutation(n).astype(np.float32) + 1.0        # distinct, nonzero
    x = mag * np.where(rng.random(n) < 0.5, -1.0, 1.0).astype(np.float32)
    q = oracle.quantize(x, bits)
    L = (1 << bits) - 1
    for m in range(1, (1 << (bits - 1))):
        idx = min(n - 1, ((2 * m - 1) * n) // L)
        assert int((np.abs(q.astype(np.int32)) >= m).sum()) == n - idx
    assert np.abs(q).max() <= (1 << (bits - 1)) - 1


@pytest.mark.parametrize("bits", [1, 2, 4])
def test_quantizer_monotone_odd_and_zero(bits):
    """phi is non-decreasing with phi(0) = 0 (Theorem 1's hypotheses), and the
    sign-magnitude construction is odd."""
    rng = np.random.default_rng(bits)
    x = rng.standard_normal(3001).astype(np.float32)
    x[::97] = 0.0
    x[5] = -0.0
    q = oracle.quantize(x, bits)
    order = np.argsort(x, kind="stable")
    assert np.all(np.diff(q[order].astype(np.int32)) >= 0)
    assert np.all(q[x == 0] == 0)
    assert np.array_equal(oracle.quantize(-x, bits), -q)


def test_rank_thresholds_are_order_statistics():
    rng = np.random.default_rng(9)
    x = rng.standard_normal(999).astype(np.float32)
    a = np.sort(np.abs(x))
    for bits in (2, 4):
        L = (1 << bits) - 1
        want = [a[min(998, ((2 * m - 1) * 999) // L)] for m in range(1, 1 << (bits - 1))]
        assert np.array_equal(oracle.rank_thresholds(x, bits), np.array(want, np.float32))


def test_quantize_rejects_nonfinite():
    for bad in (np.nan, np.inf, -np.inf):
        x = np.array([1.0, bad, 2.0], np.float32)
        for bits in (1, 2, 4):
            with pytest.raises(ValueError):
                oracle.quantize(x, bits)


# -------------------------------------------------- Algorithm 1's argmax step

def test_argmax_tie_rule_cases():
    # constant: every lag ties -> 0 when 0 is in range
    assert oracle.argmax(np.full(9, 5, np.int64), -4) == (0, 5)
    # symmetric tie at +-3 -> -3
    c = np.zeros(11, np.int64)
    c[5 - 3] = c[5 + 3] = 7
    assert oracle.argmax(c, -5) == (-3, 7)
    # tie between +2 and -3 -> +2 (smaller |tau| wins over smaller tau)
    c = np.zeros(11, np.int64)
    c[5 + 2] = c[5 - 3] = 7
    assert oracle.argmax(c, -5) == (2, 7)
    # all lags positive, tie -> smallest tau
    assert oracle.argmax(np.array([1, 4, 4, 4]), 10) == (11, 4)
    # all lags negative, tie -> largest tau (smallest |tau|)
    assert oracle.argmax(np.array([4, 4, -9]), -10) == (-9, 4)
    # negative values, single count
    assert oracle.argmax(np.array([-8, -2, -5]), 0) == (1, -2)
    assert oracle.argmax(np.array([-8]), 77) == (77, -8)


# -------------------------------------------------- Theorem 1 / its proof

def _shift_construction(rng, n, support, nu, a):
    """Zero-padded y with finite support and x[m] = a * y[m + nu] exactly in
    the index range, so Eq. (2) holds on all of Z."""
    y = np.zeros(n, np.float32)
    start = max(0, nu) + rng.integers(0, n - support - abs(nu) + 1)
    y[start: start + support] = rng.standard_normal(support).astype(np.float32)
    x = np.zeros(n, np.float32)
    for m in range(n):
        if 0 <= m + nu < n:
            x[m] = np.float32(a) * y[m + nu]
    assert np.count_nonzero(x) == np.count_nonzero(y)
    return x, y


@pytest.mark.parametrize("bits", [1, 2, 4])
def test_theorem1_invariance(bits):
    """Theorem 1: for x[n] = a y[n + nu] and monotone phi, psi with
    phi(0) = psi(0) = 0, the quantized correlation is maximal at nu (Remark 1:
    possibly among other maximisers, so c[nu] == max c is what is fixed)."""
    rng = np.random.default_rng(100 + bits)
    for trial in range(40):
        n = int(rng.integers(40, 400))
        support = int(rng.integers(1, n // 2))
        nu = int(rng.integers(-(n - support) // 2, (n - support) // 2 + 1))
        a = float(rng.uniform(0.01, 50.0))
        x, y = _shift_construction(rng, n, support, nu, a)
        qx, qy = oracle.quantize(x, bits), oracle.quantize(y, bits)
        c = oracle.xcorr(qx, qy)
        lo = -(n - 1)
        assert c[nu - lo] == c.max()
        lag, val = oracle.argmax(c, lo)
        assert val == c[nu - lo]


def test_rearrangement_bound():
    """Proof of Theorem 1: for every lag, c[tau] is at most the sum of products
    of the descending sorts over the index set; equality at nu."""
    rng = np.random.default_rng(7)
    for trial in range(10):
        n = int(rng.integers(20, 60))
        support = int(rng.integers(3, n // 2))
        nu = int(rng.integers(-(n - support) // 2, (n - support) // 2 + 1))
        x, y = _shift_construction(rng, n, support, nu, 1.7)
        qx = oracle.quantize(x, 4).astype(np.int64)
        qy = oracle.quantize(y, 4).astype(np.int64)
        c = oracle.xcorr(qx.astype(np.int8), qy.astype(np.int8))
        for tau in range(-(n - 1), n):
            ms = [m for m in range(-n, 2 * n) if (0 <= m < n and qx[m] != 0)
                  or (0 <= m + tau < n and qy[m + tau] != 0)]
            u = sorted([qx[m] if 0 <= m < n else 0 for m in ms], reverse=True)
            v = sorted([qy[m + tau] if 0 <= m + tau < n else 0 for m in ms], reverse=True)
            bound = int(np.dot(u, v)) if ms else 0
            ct = int(c[tau + n - 1])
            assert ct <= bound
            if tau == nu:
                assert ct == bound


def test_estimate_on_synthetic_shift():
    """End to end on the 4096-sample, 20 dB shifted pair: the sign estimator
    lands on the planted shift (a statistic at this SNR, not a theorem)."""
    b = synth.single_pair()
    lag, _ = oracle.estimate(b.x[0], b.y[0], 1)
    assert lag == int(b.shift[0])


# ---- Algorithm 1's last steps (re-ranking the tied set) and the sub-sample offset

def test_refine_hand_worked_tie():
    """x = [1, 0, 2] and y = [1, 0, 1, 0, 3] quantize (sign) to [1, 0, 1] and
    [1, 0, 1, 0, 1]: the integer correlation is 2 at lags 0 and 2 (a tie).  The
    real one is 1*1 + 2*1 = 3 at lag 0 and 1*1 + 2*3 = 7 at lag 2, so
    Algorithm 1 returns {2} although the integer tie rule alone says 0."""
    x = np.array([1.0, 0.0, 2.0], dtype=np.float32)
    y = np.array([1.0, 0.0, 1.0, 0.0, 3.0], dtype=np.float32)
    qx, qy = oracle.quantize(x, 1), oracle.quantize(y, 1)
    lo, hi = oracle.full_lag_range(3, 5)
    c = oracle.xcorr(qx, qy, lo, hi)
    assert oracle.argmax(c, lo) == (0, 2)
    r = oracle.refine(x, y, c, lo)
    assert (r["lag"], r["value"], r["n_int_ties"], r["n_ties"]) == (2, 2, 2, 1)
    assert r["r"] == 7.0 and (r["lag_lo"], r["lag_hi"]) == (2, 2)
    # swapping the weights flips the choice: 1*1 + 2*3 = 7 at lag 0
    y2 = np.array([1.0, 0.0, 3.0, 0.0, 1.0], dtype=np.float32)
    assert oracle.refine(x, y2, oracle.xcorr(qx, oracle.quantize(y2, 1), lo, hi), lo)["lag"] == 0


def test_refine_real_tie_keeps_the_set():
    """x = [1, 0, 1], y = [1, 0, 1, 0, 1]: integer and real correlations both
    tie at lags 0 and 2 (value 2), so the set stays {0, 2}; representative 0."""
    x = np.array([1.0, 0.0, 1.0], dtype=np.float32)
    y = np.array([1.0, 0.0, 1.0, 0.0, 1.0], dtype=np.float32)
    lo, hi = oracle.full_lag_range(3, 5)
    c = oracle.xcorr(oracle.quantize(x, 1), oracle.quantize(y, 1), lo, hi)
    r = oracle.refine(x, y, c, lo)
    assert (r["lag"], r["n_int_ties"], r["n_ties"], r["lag_lo"], r["lag_hi"]) == (0, 2, 2, 0, 2)


def test_refine_parabola_vertex():
    """x = [1, 2], y = [2, 1, 0]: the real correlation is 4, 4, 1 at lags -1,
    0, 1 (integer: 1, 2, 1, so lag 0).  The parabola through (-1, 4), (0, 4),
    (1, 1) is -1.5 t^2 - 1.5 t + 4 with its vertex at t = -0.5."""
    x = np.array([1.0, 2.0], dtype=np.float32)
    y = np.array([2.0, 1.0, 0.0], dtype=np.float32)
    lo, hi = oracle.full_lag_range(2, 3)
    c = oracle.xcorr(oracle.quantize(x, 1), oracle.quantize(y, 1), lo, hi)
    r = oracle.refine(x, y, c, lo)
    assert r["lag"] == 0 and r["r"] == 4.0 and r["frac"] == -0.5
    # a symmetric peak has its vertex on the lag: autocorrelation of [1, 1]
    z = np.array([1.0, 1.0], dtype=np.float32)
    cz = oracle.xcorr(oracle.quantize(z, 1), oracle.quantize(z, 1), -1, 1)
    assert oracle.refine(z, z, cz, -1)["frac"] == 0.0


def test_real_ccf_matches_numpy_correlate():
    rng = np.random.default_rng(12)
    x = rng.standard_normal(37).astype(np.float32)
    y = rng.standard_normal(23).astype(np.float32)
    full = np.correlate(y.astype(np.float64), x.astype(np.float64), mode="full")
    # numpy's full correlate of (y, x) at output k is sum_n y[n + k - (len(x) - 1)] x[n]
    for tau in range(-(37 - 1), 23):
        assert abs(oracle.real_ccf(x, y, tau) - full[tau + 36]) < 1e-9
