"""Pins of the seeded input generators: the Eq. (47) random chi field has the
stated mean, standard deviation and Gaussian correlation exp(-d^2/(2 l_c^2))
(the self-convolution of exp(-d^2/l_c^2)); the uniform and Box-Muller draws
have the textbook moments; everything is reproducible from the seed."""
import numpy as np

from paper_1904_03808_gb300 import inputs as I


def test_uniform_moments_and_reproducible():
    u = I.uniform01(7, 200000)
    assert abs(u.mean() - 0.5) < 4e-3 and abs(u.var() - 1 / 12) < 2e-3
    assert u.min() >= 0 and u.max() < 1
    assert np.array_equal(u[1000:1010], I.uniform01(7, 10, offset=1000))
    assert not np.array_equal(u[:10], I.uniform01(8, 10))


def test_box_muller_moments():
    z = I.normal_noise(3, 400000)
    assert abs(z.mean()) < 6e-3 and abs(z.var() - 1) < 1e-2
    assert abs(np.mean(z ** 4) - 3) < 5e-2


def test_chi_field_statistics_and_correlation():
    n, lc = 64, 1.5
    chi = I.chi_field(5, n, n, n, 600.0, 30.0, lc)
    assert chi.shape == (n, n, n)
    assert abs(chi.mean() - 600.0) < 1.5
    assert abs(chi.std() - 30.0) < 1.5
    d = (chi - chi.mean()) / chi.std()
    for lag in (1, 2, 3):
        rho_x = np.mean(d * np.roll(d, lag, axis=2))
        rho_y = np.mean(d * np.roll(d, lag, axis=1))
        rho_z = np.mean(d[lag:] * d[:-lag])
        want = np.exp(-lag * lag / (2 * lc * lc))
        for r in (rho_x, rho_y, rho_z):
            assert abs(r - want) < 0.03, (lag, r, want)
    assert np.array_equal(chi, I.chi_field(5, n, n, n, 600.0, 30.0, lc))


def test_rhs_field_range_and_walls():
    b = I.rhs_field(1, 8, 8, 8)
    assert b.shape == (3, 9, 8, 8)
    assert np.all(b[:, 0] == 0) and np.all(b[:, 8] == 0)
    inner = b[:, 1:8]
    assert inner.min() >= -1 and inner.max() < 1 and abs(inner.mean()) < 0.05
