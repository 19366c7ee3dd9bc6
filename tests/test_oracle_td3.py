"""Pins of the time-dependent three-body oracle (oracle/td3.py): the CP-image amplitudes,
the no-mixing and non-resonant limits, the normalisation through the three Gram matrices
against a direct MC average, finite differences of the NLL, and the generated lifetime."""
import math

import numpy as np
import pytest
from scipy import stats

import synth
from oracle import dalitz as od
from oracle import td3

KIN = synth.TD3_MASSES


def _cands(n, seed):
    return synth.dalitz_candidates(n, seed, KIN["M"], KIN["m1"], KIN["m2"], KIN["m3"])


@pytest.fixture(scope="module")
def small():
    spec = synth.td3_spec()
    theta = np.array(synth.param_values(spec))
    m = td3.TD3Model(spec)
    mc = _cands(20_000, 1710015)
    data = td3.generate(spec, theta, 3000, 51, _cands)
    return spec, theta, m, mc, data


def test_dalitz_region_is_symmetric_and_abar_is_the_exchanged_amplitude(small):
    spec, theta, m, mc, data = small
    # the exchanged point of an inside point is inside (equal charged-pion masses)
    sw = {"s12": mc["s13"], "s13": mc["s12"]}
    kin = spec["pdf"][1]
    assert bool(od.inside(sw["s12"], sw["s13"], kin).all())
    a, ab = m.amplitudes(mc, theta)
    a_sw, ab_sw = m.amplitudes(sw, theta)
    np.testing.assert_allclose(ab, a_sw, rtol=1e-13, atol=0)
    np.testing.assert_allclose(a, ab_sw, rtol=1e-13, atol=0)
    # a rho+ in (12) at the exchanged point is the rho- in (13) at the original point
    names = [a_[3] for a_ in spec["pdf"][2][:-1]]
    k_p, k_m = names.index("m0_rho770_p"), names.index("m0_rho770_m")
    np.testing.assert_allclose(ab[:, k_p], a[:, k_m], rtol=1e-12)


def test_no_mixing_rate_is_the_amplitude_times_the_resolved_exponential(small):
    spec, theta, m, mc, data = small
    th = theta.copy()
    th[m.tp[0]] = th[m.tp[1]] = 0.0
    amps = m.amplitudes(data, th)
    R = m.rate(amps, data["t"], th)
    A = amps[0] @ m.coefficients(th)
    tau, s = th[m.tp[2]], th[m.tp[3]]
    ref = np.abs(A) ** 2 * stats.exponnorm.pdf(data["t"], K=tau / s, scale=s) * tau
    np.testing.assert_allclose(R, ref, rtol=1e-11)


def test_non_resonant_only_is_a_resolved_exponential_of_rate_G_1_minus_y(small):
    # A = B = c_NR: R = |c|^2 E(G(1 - y)) and N = |c|^2 / (G(1 - y)); f is the Dalitz-flat,
    # exponentially modified Gaussian density with rate G(1 - y)
    spec, theta, m, mc, data = small
    th = theta.copy()
    names = synth.param_names(spec)
    for i, n in enumerate(names):
        if n.startswith(("re_", "im_")) and not n.endswith("NR"):
            th[i] = 0.0
    th[m.tp[0]], th[m.tp[1]] = 0.02, 0.3
    x, y, tau, s = (th[i] for i in m.tp)
    rate = (1.0 - y) / tau
    nll = m.nll(data, mc, th)
    ref = -np.sum(np.log(stats.exponnorm.pdf(data["t"], K=1.0 / (rate * s), scale=s)))
    assert nll == pytest.approx(ref, rel=1e-11)


def test_norm_through_grams_equals_direct_average(small):
    spec, theta, m, mc, data = small
    th = theta.copy()
    th[m.tp[0]], th[m.tp[1]] = 0.2, 0.1   # visible mixing
    N = m.norm(m.grams(mc, th), th)
    a, ab = m.amplitudes(mc, th)
    c = m.coefficients(th)
    A, B = a @ c, ab @ c
    I = td3.time_integrals(th[m.tp[0]], th[m.tp[1]], th[m.tp[2]])
    direct = np.mean(0.5 * (abs(A) ** 2 + abs(B) ** 2) * I[0] + 0.5 * (abs(A) ** 2 - abs(B) ** 2) * I[2]
                     + (A * B.conj()).real * I[1] + (A * B.conj()).imag * I[3])
    assert abs(N - direct) <= 1e-12 * abs(direct)


def test_nll_gradient_by_finite_differences(small):
    spec, theta, m, mc, data = small
    th = theta * 1.02
    th[m.tp[0]], th[m.tp[1]] = 0.05, 0.03
    grams = m.grams(mc, th)
    amps = m.amplitudes(data, th)
    nll, g = m.nll_grad(data, mc, th, amps=amps, grams=grams)
    f = lambda t: m.nll(data, mc, t, amps=amps, grams=grams)
    for i, p in enumerate(spec["params"]):
        if p[0].startswith(("m0_", "w_")):
            continue  # lineshapes are constants of this model's cached amplitudes
        h = 1e-4 * max(abs(th[i]), 0.01)
        e = np.zeros_like(th)
        e[i] = h
        fd = (8 * (f(th + e) - f(th - e)) - (f(th + 2 * e) - f(th - 2 * e))) / (12 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1.0), (p[0], fd, g[i])


def test_generated_times_have_the_lifetime(small):
    spec, theta, m, mc, data = small
    t = data["t"]
    tau = theta[m.tp[2]]
    assert abs(t.mean() - tau) < 4 * t.std() / math.sqrt(t.size)


def test_polar_coefficients(small):
    spec, theta, m, mc, data = small
    ps = synth.to_polar(spec)
    mp = td3.TD3Model(ps)
    tp = np.array(synth.param_values(ps))
    grams, amps = m.grams(mc, theta), m.amplitudes(data, theta)
    assert mp.nll(data, mc, tp, amps=amps, grams=grams) == pytest.approx(
        m.nll(data, mc, theta, amps=amps, grams=grams), rel=1e-13)
    names = synth.param_names(ps)
    tp2 = tp.copy()
    for i, n in enumerate(names):
        if n.startswith("phase_") and i not in (names.index("phase_rho770_p"),):
            tp2[i] += 0.2
    _, g = mp.nll_grad(data, mc, tp2, amps=amps, grams=grams)
    f = lambda t: mp.nll(data, mc, t, amps=amps, grams=grams)
    for i, n in enumerate(names):
        if not n.startswith(("mag_", "phase_")):
            continue
        h = 1e-4 * max(abs(tp2[i]), 0.1)   # fourth-order stencil: truncation ~h^4
        e = np.zeros_like(tp2)
        e[i] = h
        fd = (8 * (f(tp2 + e) - f(tp2 - e)) - (f(tp2 + 2 * e) - f(tp2 - 2 * e))) / (12 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1.0), (n, fd, g[i])
