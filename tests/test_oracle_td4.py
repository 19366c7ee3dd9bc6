"""Pins of the time-dependent four-body oracle (oracle/td4.py) against quadrature, library
routines, closed forms, finite differences and an independent route to the normalisation."""
import math

import numpy as np
import pytest
from scipy import integrate, stats
from scipy.special import eval_legendre

import synth
from oracle import td4


def _conv_quad(g, t, s):
    """int_0^inf e^{-g u} N(t - u; 0, s) du by adaptive quadrature (real and imaginary parts)."""
    def f(u, part):
        v = np.exp(-g * u) * math.exp(-(t - u) ** 2 / (2 * s * s)) / (s * math.sqrt(2 * math.pi))
        return v.real if part == 0 else v.imag
    lo, hi = max(0.0, t - 12 * s), max(t + 12 * s, 0.0) + 40.0 / max(g.real, 1e-3)
    re = integrate.quad(f, lo, hi, args=(0,), limit=400, epsabs=1e-15, epsrel=1e-12)[0]
    im = integrate.quad(f, lo, hi, args=(1,), limit=400, epsabs=1e-15, epsrel=1e-12)[0]
    return re + 1j * im


@pytest.mark.parametrize("g", [2.4, 2.43 - 0.01j, 2.4 - 0.3j, 0.7 + 0.0j])
@pytest.mark.parametrize("t", [-0.3, -0.05, 0.0, 0.004, 0.1, 1.3, 6.0])
@pytest.mark.parametrize("s", [0.05, 0.2])
def test_convolution_against_quadrature(g, t, s):
    E = td4.conv_exp(g, np.array([t]), s)[0]
    ref = _conv_quad(complex(g), t, s)
    assert abs(E - ref) <= 1e-9 * max(abs(ref), 1e-12) + 1e-15


def test_real_rate_is_the_exponentially_modified_gaussian():
    t = np.linspace(-0.4, 8.0, 301)
    for G, s in ((1 / 0.41, 0.05), (0.9, 0.3)):
        E = td4.conv_exp(G, t, s).real
        ref = stats.exponnorm.pdf(t, K=1.0 / (s * G), loc=0.0, scale=s) / G
        np.testing.assert_allclose(E, ref, rtol=1e-11, atol=1e-300)


def test_convolution_integrates_to_one_over_g():
    for g in (2.44, 2.44 - 0.2j):
        for part in (0, 1):
            f = lambda t: (td4.conv_exp(g, np.array([t]), 0.05)[0]).real if part == 0 else \
                (td4.conv_exp(g, np.array([t]), 0.05)[0]).imag
            val = integrate.quad(f, -1.0, 30.0, points=[0.0], limit=400, epsabs=1e-13)[0]
            ref = (1.0 / g).real if part == 0 else (1.0 / g).imag
            assert abs(val - ref) < 1e-9


def test_time_integrals_match_quadrature_of_the_time_terms():
    x, y, tau, s = 0.3, 0.2, 0.41, 0.05   # large mixing so every term matters
    I = td4.time_integrals(x, y, tau)
    for j in range(4):
        f = lambda t: td4.time_terms(np.array([t]), x, y, tau, s)[j][0]
        val = integrate.quad(f, -1.0, 40.0, points=[0.0], limit=500, epsabs=1e-13)[0]
        assert abs(val - I[j]) < 1e-9, (j, val, I[j])


def test_time_derivatives_by_finite_differences():
    t = np.array([-0.07, 0.02, 0.3, 2.0])
    p0 = np.array([0.05, 0.03, 0.41, 0.06])
    _, d = td4.time_terms(t, *p0, derivs=True)
    for i in range(4):
        h = 1e-6 * max(abs(p0[i]), 0.01)
        pp, pm = p0.copy(), p0.copy()
        pp[i] += h
        pm[i] -= h
        Tp, Tm = td4.time_terms(t, *pp), td4.time_terms(t, *pm)
        for j in range(4):
            fd = (Tp[j] - Tm[j]) / (2 * h)
            np.testing.assert_allclose(d[i][j], fd, rtol=1e-6, atol=1e-8)


def test_angular_factors_are_legendre_and_orthogonal():
    c = np.linspace(-1, 1, 11)
    one = np.ones_like(c)
    np.testing.assert_allclose(td4.angular("TS0", c, one, 0 * c).real, eval_legendre(2, c), rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(td4.angular("VS0", c, one, 0 * c).real, eval_legendre(1, c), rtol=1e-14)
    np.testing.assert_allclose(td4.angular("SV0", one, c, 0 * c).real, eval_legendre(1, c), rtol=1e-14)
    # Gauss-Legendre x Gauss-Legendre x uniform-phi quadrature over the angles
    xs, ws = np.polynomial.legendre.leggauss(12)
    ph = np.linspace(-np.pi, np.pi, 16, endpoint=False)
    C1, C2, PH = np.meshgrid(xs, xs, ph, indexing="ij")
    W = np.einsum("i,j->ij", ws, ws)[:, :, None] * (2 * np.pi / ph.size)
    kinds = td4.ANGULAR
    vals = {k: td4.angular(k, C1, C2, PH) for k in kinds}
    gram = np.array([[np.sum(W * vals[a] * np.conj(vals[b])) for b in kinds] for a in kinds])
    # helicity-basis norms: int P_j^2 dc = 2/(2j+1); int s^2 dc = 4/3; int cos^2 / sin^2 dphi = pi
    norms = {"SS": 8 * np.pi, "VS0": 8 * np.pi / 3, "SV0": 8 * np.pi / 3, "VV0": 8 * np.pi / 9,
             "VVpar": 16 * np.pi / 9, "VVperp": 16 * np.pi / 9, "TS0": 8 * np.pi / 5, "TV0": 8 * np.pi / 15}
    for i, a in enumerate(kinds):
        assert abs(gram[i, i] - norms[a]) < 1e-12
    # different helicity structures of the same spins are orthogonal
    idx = {k: i for i, k in enumerate(kinds)}
    for a, b in (("VV0", "VVpar"), ("VV0", "VVperp"), ("VVpar", "VVperp"), ("SS", "TS0"), ("VS0", "TV0")):
        assert abs(gram[idx[a], idx[b]]) < 1e-12


def test_lineshape_at_the_pole_mass():
    for (m0, g0), L in (((0.8955, 0.0473), 1), ((1.4324, 0.109), 2), ((0.99, 0.07), 0)):
        F = td4.lineshape(np.array([m0]), m0, g0, L, 0.494, 0.140, 1.5)[0]
        assert abs(abs(F) ** 2 - 1.0 / (m0 * g0) ** 2) <= 1e-12 / (m0 * g0) ** 2


def test_phase_space_mass_marginal():
    kin = synth.TD4_MASSES
    M, m1, m2, m3, m4 = (kin[k] for k in ("M", "m1", "m2", "m3", "m4"))
    n = 400_000
    ps = synth.four_body_phase_space(n, 4, M, m1, m2, m3, m4)
    edges = np.linspace(m1 + m2, M - m3 - m4, 21)
    counts, _ = np.histogram(ps["m12"], edges)
    w = lambda b, a: td4._ps_weight(np.array([a]), np.array([b]), dict(kin))[0]
    expect = np.array([integrate.dblquad(w, lo, hi, m3 + m4, M - m1 - m2, epsrel=1e-6)[0]
                       for lo, hi in zip(edges[:-1], edges[1:])])
    expect *= n / expect.sum()
    chi2 = np.sum((counts - expect) ** 2 / np.maximum(expect, 1))
    assert chi2 / (len(counts) - 1) < 2.5, chi2
    # angles uniform
    for k, (lo, hi) in (("c12", (-1, 1)), ("c34", (-1, 1)), ("phi", (-np.pi, np.pi))):
        assert stats.kstest(ps[k], "uniform", args=(lo, hi - lo)).pvalue > 1e-3


@pytest.fixture(scope="module")
def small():
    spec = synth.c4_spec()
    theta = np.array(synth.param_values(spec))
    m = td4.TD4Model(spec)
    mc = synth.four_body_phase_space(20_000, 1710014, **synth.TD4_MASSES)
    data = td4.generate(spec, theta, 3000, 41)
    return spec, theta, m, m.amplitudes(mc), data


def test_norm_through_gram_equals_direct_average(small):
    spec, theta, m, mca, _ = small
    th = theta.copy()
    th[m.tp[0]], th[m.tp[1]] = 0.2, 0.1   # visible mixing
    N = m.norm(m.gram(mca), th)
    c, b = m.coefficients(th), m.b
    A, B = mca @ c, mca @ b
    I = td4.time_integrals(th[m.tp[0]], th[m.tp[1]], th[m.tp[2]])
    direct = np.mean(0.5 * (abs(A) ** 2 + abs(B) ** 2) * I[0] + 0.5 * (abs(A) ** 2 - abs(B) ** 2) * I[2]
                     + (A * B.conj()).real * I[1] + (A * B.conj()).imag * I[3])
    assert abs(N - direct) <= 1e-12 * abs(direct)


def test_nll_gradient_by_finite_differences(small):
    spec, theta, m, mca, data = small
    th = theta * 1.02
    nll, g = m.nll_grad(data, mca, th)
    a = m.amplitudes(data)
    f = lambda t: m.nll(data, mca, t, a=a)
    for i in range(len(th)):
        # fourth-order central differences: truncation ~h^4, round-off ~eps |NLL| / h
        h = 1e-4 * max(abs(th[i]), 0.01)
        e = np.zeros_like(th)
        e[i] = h
        fd = (8 * (f(th + e) - f(th - e)) - (f(th + 2 * e) - f(th - 2 * e))) / (12 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1.0), (i, fd, g[i])


def test_no_mixing_reduces_to_exponential_times_amplitude(small):
    spec, theta, m, mca, data = small
    th = theta.copy()
    th[m.tp[0]] = th[m.tp[1]] = 0.0
    a = m.amplitudes(data)
    R = m.rate(a, data["t"], th)
    A = a @ m.coefficients(th)
    tau, s = th[m.tp[2]], th[m.tp[3]]
    ref = np.abs(A) ** 2 * stats.exponnorm.pdf(data["t"], K=tau / s, scale=s) * tau
    np.testing.assert_allclose(R, ref, rtol=1e-11)


def test_generated_times_have_the_lifetime(small):
    _, theta, m, _, data = small
    t = data["t"]
    tau = theta[m.tp[2]]
    # mixing is small: <t> = tau (the resolution has zero mean) within the sample's error
    assert abs(t.mean() - tau) < 4 * t.std() / math.sqrt(t.size)
