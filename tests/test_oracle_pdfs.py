"""Pins of the oracle's basic shapes and closed-form integrals (oracle/pdfs.py)."""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.special
import scipy.stats
import torch

from oracle import pdfs

T = lambda v: torch.tensor(v, dtype=torch.float64)  # noqa: E731


def quad(fn, lo, hi, points=None):
    v, _ = scipy.integrate.quad(lambda x: float(fn(T(x))), lo, hi, epsabs=0, epsrel=1e-13,
                                limit=500, points=points)
    return v


@pytest.mark.parametrize("lo,hi,mu,sigma", [(0, 10, 5.0, 0.4), (5.2, 5.3, 5.279, 0.003),
                                            (-0.2, 0.2, 0.0, 0.02), (0, 1, 1.7, 0.3), (-3, 2, -1, 2.5)])
def test_gauss_integral_vs_quad(lo, hi, mu, sigma):
    ref = quad(lambda x: pdfs.gauss_shape(x, mu, sigma), lo, hi, points=[mu] if lo < mu < hi else None)
    got = float(pdfs.gauss_integral(lo, hi, T(mu), T(sigma)))
    assert got == pytest.approx(ref, rel=1e-12)


def test_gauss_shape_is_scaled_normal_pdf():
    x = np.linspace(-3, 7, 101)
    ref = scipy.stats.norm.pdf(x, 2.0, 1.3) * 1.3 * math.sqrt(2 * math.pi)
    got = pdfs.gauss_shape(T(x), 2.0, 1.3).numpy()
    np.testing.assert_allclose(got, ref, rtol=1e-14)


@pytest.mark.parametrize("lo,hi,lam", [(0, 10, -0.3), (0, 10, -1 / 1.5), (0, 10, -1.25), (1, 3, 0.7), (0, 10, 1e-9)])
def test_expo_integral_vs_quad(lo, hi, lam):
    ref = quad(lambda x: pdfs.expo_shape(x, lam), lo, hi)
    got = float(pdfs.expo_integral(lo, hi, T(lam)))
    assert got == pytest.approx(ref, rel=1e-9 if abs(lam) < 1e-6 else 1e-12)


def test_expo_integral_zero_rate_is_range_length():
    assert float(pdfs.expo_integral(2.0, 5.0, T(0.0))) == 3.0


def test_truncated_exponential_matches_scipy():
    x = np.linspace(0, 10, 41)
    lam = -0.3
    got = pdfs.expo_shape(T(x), lam).numpy() / float(pdfs.expo_integral(0.0, 10.0, T(lam)))
    ref = scipy.stats.truncexpon.pdf(x, b=10 * 0.3, scale=1 / 0.3)
    np.testing.assert_allclose(got, ref, rtol=1e-13)


@pytest.mark.parametrize("lo,hi,a1,a2", [(-0.2, 0.2, -1.0, 0.5), (0, 3, 0.3, -0.05), (-1, 1, 0, 0)])
def test_poly2_integral_vs_quad(lo, hi, a1, a2):
    ref = quad(lambda x: pdfs.poly2_shape(x, a1, a2), lo, hi)
    got = float(pdfs.poly2_integral(lo, hi, T(a1), T(a2)))
    assert got == pytest.approx(ref, rel=1e-13)


def test_poly2_shape_matches_numpy_polyval():
    x = np.linspace(-0.2, 0.2, 17)
    np.testing.assert_allclose(pdfs.poly2_shape(T(x), -1.0, 0.5).numpy(),
                               np.polynomial.polynomial.polyval(x, [1.0, -1.0, 0.5]), rtol=1e-15)


@pytest.mark.parametrize("m0,c,p", [(5.29, -20.0, 0.5), (5.29, -5.0, 1.0), (1.0, -2.0, 0.5), (5.29, -40, 2.0)])
def test_argus_full_range_integral_incomplete_gamma(m0, c, p):
    # With u = 1 - m^2/m0^2:  m dm = -(m0^2/2) du, so
    #   int_0^m0 m u^p e^{c u} dm = (m0^2/2) int_0^1 u^p e^{c u} du
    #                             = (m0^2/2) gamma_lower(p+1, -c) / (-c)^(p+1)      (c < 0)
    ref = 0.5 * m0 ** 2 * scipy.special.gammainc(p + 1, -c) * scipy.special.gamma(p + 1) / (-c) ** (p + 1)
    got = quad(lambda m: pdfs.argus_shape(m, T(m0), T(c), T(p)), 0.0, m0)
    assert got == pytest.approx(ref, rel=1e-9)


def test_argus_zero_above_endpoint():
    m = T([5.2899, 5.29, 5.295, 5.3])
    v = pdfs.argus_shape(m, T(5.29), T(-20.0), T(0.5))
    assert float(v[0]) > 0 and float(v[1]) == 0 and float(v[2]) == 0 and float(v[3]) == 0
