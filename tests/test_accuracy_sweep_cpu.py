"""The accuracy sweep's synthetic pairs (Sec. 4.2 protocol): the delay sign
convention, the SNR scaling and the band-limited sub-sample shift, checked on
the CPU with numpy alone."""
import numpy as np
import pytest

from paper_2509_19974_gb300.accuracy_sweep import MAX_DELAY, NX, NY, make_pair


def _ccf(x, y):
    # c[tau] = sum_n x[n] y[n + tau] for tau in [-(nx - 1), ny - 1]
    return np.correlate(y.astype(np.float64), x.astype(np.float64), "full")


def test_shapes_and_delay_range():
    rng = np.random.default_rng(1)
    for _ in range(5):
        x, y, nu = make_pair(rng, 0.0)
        assert x.shape == (NX,) and y.shape == (NY,) and x.dtype == np.float32
        assert 0.0 <= nu < MAX_DELAY


def test_clean_peak_is_at_minus_nu():
    # at a very high SNR the real CCF's argmax tau is the rounded -nu
    rng = np.random.default_rng(2)
    for _ in range(3):
        x, y, nu = make_pair(rng, 60.0, nx=8000, ny=1600, max_delay=6400)
        tau = int(np.argmax(_ccf(x, y))) - (x.size - 1)
        assert abs(-tau - nu) < 1


def test_integer_delay_is_a_plain_shift():
    # an integer nu makes the band-limited shift an exact copy of the target
    class R:
        def __init__(self, g):
            self.g = g

        def standard_normal(self, n):
            return self.g.standard_normal(n)

        def uniform(self, a, b):
            return 1234.0

    x, y, nu = make_pair(R(np.random.default_rng(3)), 300.0, nx=8000, ny=1600, max_delay=6400)
    assert nu == 1234.0
    np.testing.assert_allclose(x[1234:1234 + 1600], y, atol=1e-4 * np.abs(y).max())


@pytest.mark.parametrize("snr", [-10.0, 0.0, 10.0])
def test_snr_is_the_power_ratio(snr):
    # background alone = x minus the delayed target; power per sample ratio = SNR
    class R:
        def __init__(self, g):
            self.g = g

        def standard_normal(self, n):
            return self.g.standard_normal(n)

        def uniform(self, a, b):
            return 100.0

    x, y, _ = make_pair(R(np.random.default_rng(4)), snr)
    b = x.astype(np.float64).copy()
    b[100:100 + NY] -= y
    got = 10 * np.log10((np.sum(y.astype(np.float64) ** 2) / NY) / (np.sum(b ** 2) / NX))
    assert abs(got - snr) < 1e-3
