"""Pins of the three-body amplitude oracle (oracle/dalitz.py)."""
import numpy as np
import pytest
import torch

import synth
from oracle import dalitz as od
from oracle import model as om

KIN = dict(synth.DALITZ_MASSES, r_res=1.5, r_par=5.0)
MASS = {1: KIN["m1"], 2: KIN["m2"], 3: KIN["m3"]}
T = lambda v: torch.tensor(v, dtype=torch.float64)  # noqa: E731


# ---- explicit four-vector kinematics (independent of the oracle's invariant formulas) ----
def _boost(p, beta):
    """Boost four-vectors p (..., 4) = (E, px, py, pz) by velocity beta (..., 3)."""
    b2 = np.sum(beta * beta, axis=-1, keepdims=True)
    g = 1.0 / np.sqrt(1.0 - b2)
    bp = np.sum(beta * p[..., 1:], axis=-1, keepdims=True)
    E = g * (p[..., :1] + bp)
    vec = p[..., 1:] + ((g - 1.0) * bp / np.where(b2 > 0, b2, 1.0) + g * p[..., :1]) * beta
    return np.concatenate([E, vec], axis=-1)


def _iso(rng, n):
    c = rng.uniform(-1, 1, n)
    ph = rng.uniform(0, 2 * np.pi, n)
    s = np.sqrt(1 - c * c)
    return np.stack([s * np.cos(ph), s * np.sin(ph), c], axis=-1)


def _decay_events(n, seed):
    """Explicit parent-frame four-momenta of M -> (12) 3, (12) -> 1 2 with random angles."""
    rng = np.random.default_rng(seed)
    M, m1, m2, m3 = KIN["M"], KIN["m1"], KIN["m2"], KIN["m3"]
    m12 = rng.uniform(m1 + m2 + 1e-3, M - m3 - 1e-3, n)
    lam = lambda a, b, c: a * a + b * b + c * c - 2 * a * b - 2 * a * c - 2 * b * c  # noqa: E731
    pst = np.sqrt(lam(M * M, m12 ** 2, m3 * m3)) / (2 * M)
    n1 = _iso(rng, n)
    pR = np.concatenate([np.sqrt(m12 ** 2 + pst ** 2)[:, None], pst[:, None] * n1], axis=1)
    p3 = np.concatenate([np.sqrt(m3 ** 2 + pst ** 2)[:, None], -pst[:, None] * n1], axis=1)
    q = np.sqrt(lam(m12 ** 2, m1 * m1, m2 * m2)) / (2 * m12)
    n2 = _iso(rng, n)
    p1r = np.concatenate([np.sqrt(m1 ** 2 + q ** 2)[:, None], q[:, None] * n2], axis=1)
    p2r = np.concatenate([np.sqrt(m2 ** 2 + q ** 2)[:, None], -q[:, None] * n2], axis=1)
    beta = pR[:, 1:] / pR[:, :1]
    return {1: _boost(p1r, beta), 2: _boost(p2r, beta), 3: p3}


def _mass2(p):
    return p[:, 0] ** 2 - np.sum(p[:, 1:] ** 2, axis=1)


def _helicity_explicit(P, a, b, c):
    pab = P[a] + P[b]
    beta = -pab[:, 1:] / pab[:, :1]
    A = _boost(P[a], beta)
    C = _boost(P[c], beta)
    qa = np.linalg.norm(A[:, 1:], axis=1)
    kc = np.linalg.norm(C[:, 1:], axis=1)
    cos = np.sum(A[:, 1:] * C[:, 1:], axis=1) / (qa * kc)
    return qa, kc, cos


@pytest.mark.parametrize("pair", ["12", "13", "23"])
def test_helicity_quantities_match_explicit_boosts(pair):
    P = _decay_events(2000, seed=int(pair))
    s = {"12": _mass2(P[1] + P[2]), "13": _mass2(P[1] + P[3]), "23": _mass2(P[2] + P[3])}
    a, b, c = od.PAIRS[pair]
    s_ab = s[f"{min(a, b)}{max(a, b)}"]
    s_ac = s[f"{min(a, c)}{max(a, c)}"]
    q, k, cos = od.helicity_frame(T(s_ab), T(s_ac), KIN["M"], MASS[a], MASS[b], MASS[c])
    qe, ke, cose = _helicity_explicit(P, a, b, c)
    np.testing.assert_allclose(q.numpy(), qe, rtol=1e-9)
    np.testing.assert_allclose(k.numpy(), ke, rtol=1e-9)
    np.testing.assert_allclose(cos.numpy(), cose, atol=1e-8)
    # s23 from the oracle's invariant sum rule
    inv = od.invariants(T(s["12"]), T(s["13"]), KIN["M"], KIN["m1"], KIN["m2"], KIN["m3"])
    np.testing.assert_allclose(inv["23"].numpy(), s["23"], rtol=1e-11)


@pytest.mark.parametrize("pair", ["12", "13", "23"])
def test_spin_factor_invariant_form(pair):
    # -4 q k cos(theta) = s_AC - s_BC - (mA^2 - mB^2)(M^2 - mC^2)/s_AB (momentum conservation)
    P = _decay_events(500, seed=10 + int(pair))
    s = {"12": _mass2(P[1] + P[2]), "13": _mass2(P[1] + P[3]), "23": _mass2(P[2] + P[3])}
    a, b, c = od.PAIRS[pair]
    key = lambda i, j: f"{min(i, j)}{max(i, j)}"  # noqa: E731
    mA, mB, mC, M = MASS[a], MASS[b], MASS[c], KIN["M"]
    z1 = s[key(a, c)] - s[key(b, c)] - (mA ** 2 - mB ** 2) * (M ** 2 - mC ** 2) / s[key(a, b)]
    q, k, cos = od.helicity_frame(T(s[key(a, b)]), T(s[key(a, c)]), M, mA, mB, mC)
    np.testing.assert_allclose(od.spin_factor(1, q, k, cos).numpy(), z1, rtol=1e-8, atol=1e-10)
    lam = lambda x, y, z: x * x + y * y + z * z - 2 * x * y - 2 * x * z - 2 * y * z  # noqa: E731
    sab = s[key(a, b)]
    z2 = z1 ** 2 - lam(sab, mA ** 2, mB ** 2) * lam(M ** 2, sab, mC ** 2) / (3 * sab ** 2)
    np.testing.assert_allclose(od.spin_factor(2, q, k, cos).numpy(), z2, rtol=1e-7, atol=1e-10)


def test_explicit_decays_are_inside_both_boundaries():
    P = _decay_events(3000, seed=5)
    s12, s13 = _mass2(P[1] + P[2]), _mass2(P[1] + P[3])
    assert bool(od.inside(T(s12), T(s13), KIN).all())
    from synth.gen import _inside_dalitz
    assert bool(_inside_dalitz(s12, s13, KIN["M"], KIN["m1"], KIN["m2"], KIN["m3"]).all())


def test_boundary_agrees_with_synth_formula():
    rng = np.random.default_rng(4)
    lo12, hi12, lo13, hi13 = synth.dalitz_box(KIN["M"], KIN["m1"], KIN["m2"], KIN["m3"])
    a = rng.uniform(lo12, hi12, 200000)
    b = rng.uniform(lo13, hi13, 200000)
    from synth.gen import _inside_dalitz
    x = od.inside(T(a), T(b), KIN).numpy()
    y = _inside_dalitz(a, b, KIN["M"], KIN["m1"], KIN["m2"], KIN["m3"])
    assert (x == y).mean() > 1 - 1e-4
    assert 0.3 < x.mean() < 0.7


@pytest.mark.parametrize("L", [0, 1, 2])
def test_breit_wigner_pole_and_barrier_ratio(L):
    m0, g0, r = 0.8955, 0.0473, 1.5
    mA, mB = KIN["m1"], KIN["m2"]
    s = T([m0 * m0])
    q0 = torch.sqrt(od.kallen(s, mA ** 2, mB ** 2)) / (2 * m0)
    bw = od.breit_wigner(s, T(m0), T(g0), L, q0, q0, r)
    assert float(bw.abs() ** 2) == pytest.approx(1.0 / (m0 * g0) ** 2, rel=1e-13)
    assert float(od.running_width(s, T(m0), T(g0), L, q0, q0, r)) == pytest.approx(g0, rel=1e-14)


def test_barrier_factors_published_forms():
    z = T(np.linspace(0, 10, 11))
    np.testing.assert_allclose(od.barrier(1, z).numpy() ** 2, 1 / (1 + z.numpy()), rtol=1e-15)
    np.testing.assert_allclose(od.barrier(2, z).numpy() ** 2, 9 / (9 + 3 * z.numpy() + z.numpy() ** 2), rtol=1e-15)


def _small_c3(n_mc=20000):
    spec = synth.c3_spec(n_mc=n_mc)
    mc = synth.dalitz_candidates(n_mc, 1710013, KIN["M"], KIN["m1"], KIN["m2"], KIN["m3"])
    data = synth.dalitz_candidates(3000, 77, KIN["M"], KIN["m1"], KIN["m2"], KIN["m3"])
    return spec, od.DalitzModel(spec), mc, data


def test_flat_phase_space_nll_is_zero():
    spec, m, mc, data = _small_c3()
    th = np.array(synth.param_values(spec))
    names = synth.param_names(spec)
    for i, n in enumerate(names):
        if n.startswith(("re_", "im_")) and not n.endswith("NR"):
            th[i] = 0.0
    assert m.nll(data, mc, th) == pytest.approx(0.0, abs=1e-9)


def test_homogeneity_and_gradient():
    spec, m, mc, data = _small_c3()
    th = np.array(synth.param_values(spec))
    names = synth.param_names(spec)
    coef = np.array([n.startswith(("re_", "im_")) for n in names])
    f0, g = m.nll_grad(data, mc, th)
    th2 = th.copy()
    th2[coef] *= 1.7
    assert m.nll(data, mc, th2) == pytest.approx(f0, rel=1e-12)
    # Euler: sum over all coefficient parameters of theta_j dNLL/dtheta_j = 0
    assert abs(float(np.sum(th[coef] * g[coef]))) < 1e-8 * float(np.sum(np.abs(th[coef] * g[coef])))
    steps = [1e-6 if c else 0.0 for c in coef]
    idx = np.flatnonzero(coef)
    fd = om.fd_grad(lambda t: m.nll(data, mc, t), th, [s if s else 1e-7 for s in steps])
    np.testing.assert_allclose(g[idx], np.array(fd)[idx], rtol=2e-5, atol=1e-4)


def test_gram_quadratic_form_equals_mc_mean():
    spec, m, mc, data = _small_c3()
    th = torch.as_tensor(synth.param_values(spec), dtype=torch.float64)
    G = m.gram(mc, th)
    c = m.coefficients(th)
    quad_form = float((c @ G @ c.conj()).real)
    mean = float(m.intensity(m.amplitude_matrix(mc, th), th).mean())
    assert quad_form == pytest.approx(mean, rel=1e-12)
    assert torch.allclose(G, G.conj().T, rtol=0, atol=1e-14)


def test_lineshape_gradient_by_finite_differences():
    # d NLL / d m0 and d NLL / d Gamma0 of every resonance: the oracle's autograd gradient
    # against fourth-order central differences of its NLL (the masses and widths enter
    # through q0, the barrier ratio, the running width and the pole)
    spec, m, mc, data = _small_c3()
    th = np.array(synth.param_values(spec))
    names = synth.param_names(spec)
    _, g = m.nll_grad(data, mc, th)
    f = lambda t: m.nll(data, mc, t)
    for i, n in enumerate(names):
        if not n.startswith(("m0_", "w_")):
            continue
        h = 1e-5 * th[i]
        e = np.zeros_like(th)
        e[i] = h
        fd = (8 * (f(th + e) - f(th - e)) - (f(th + 2 * e) - f(th - 2 * e))) / (12 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(g[i]), 1.0), (n, fd, g[i])


def test_polar_coefficients():
    # magnitude/phase parameters: the same NLL as the Cartesian point c = r e^{i phi}, and the
    # autograd gradient against central differences in (r, phi)
    spec, m, mc, data = _small_c3()
    ps = synth.to_polar(spec)
    mp = od.DalitzModel(ps)
    th = np.array(synth.param_values(spec))
    tp = np.array(synth.param_values(ps))
    assert mp.nll(data, mc, tp) == pytest.approx(m.nll(data, mc, th), rel=1e-13)
    tp2 = tp.copy()
    names = synth.param_names(ps)
    for i, n in enumerate(names):
        if n.startswith("phase_") and not n.endswith("NR"):
            tp2[i] += 0.3
    _, g = mp.nll_grad(data, mc, tp2)
    f = lambda t: mp.nll(data, mc, t)
    for i, n in enumerate(names):
        if not n.startswith(("mag_", "phase_")):
            continue
        h = 1e-6
        e = np.zeros_like(tp2)
        e[i] = h
        fd = (f(tp2 + e) - f(tp2 - e)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-5 * max(abs(g[i]), 1.0), (n, fd, g[i])
