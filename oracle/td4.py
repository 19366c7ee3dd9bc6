"""Time-dependent four-body amplitude model (float64 / complex128 numpy, CPU).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper adds a time-dependent amplitude analysis of four-body decays, used for a mixing
measurement, to GooFit's amplitude PDFs (Sec. 5), with phase-space MC samples for the
normalisation (Sec. 5).  It prints no formula, so this file writes out a standard model:

Kinematics.  A parent of mass M decays to particles 1, 2 (the pair "12", e.g. K pi) and
3, 4 (the pair "34", pi pi).  Observables: the pair masses m12, m34, the helicity cosines
c12 = cos th12, c34 = cos th34 (angle of particle 1 / 3 in its pair's rest frame relative to
the pair's flight direction), the angle phi between the two decay planes, and the decay
time t (ps).  Four-body phase space in these variables has density p q12 q34 (uniform in
c12, c34, phi); p is the momentum of the pairs in the parent frame, q12, q34 the daughter
momenta in the pair frames.

Amplitudes.  a_k = F_1(m12) F_2(m34) W_k(c12, c34, phi), with the lineshape of a resonance
(m0, G0, spin L) in a pair whose daughters have momentum q (q0 at m = m0)
    F(m) = BW(m^2) (q/q0)^L B_L(r q)/B_L(r q0),   BW(s) = 1/(m0^2 - s - i m0 G(m)),
    G(m) = G0 (q/q0)^(2L+1) (m0/m) (B_L(r q)/B_L(r q0))^2,
    B_0 = 1, B_1 = sqrt(1/(1+z)), B_2 = sqrt(9/(9+3z+z^2)), z = (r q)^2,
and the angular structure W_k of the spins (L1, L2) (helicity form, d^j_00 = P_j):
    SS 1;  VS0 c12;  SV0 c34;  VV0 c12 c34;  VVpar s12 s34 cos phi;  VVperp i s12 s34 sin phi;
    TS0 P2(c12);  TV0 P2(c12) c34       (s = sin th, P2(c) = (3c^2 - 1)/2).
A = sum_k c_k a_k (free, doubly-Cabibbo-suppressed coefficients), B = sum_k b_k a_k (fixed,
Cabibbo-favoured coefficients; the same amplitude basis).

Decay-time dependence (Gamma = 1/tau, mixing parameters x, y) for t >= 0:
    R_true = e^{-Gamma t} [ (|A|^2+|B|^2)/2 cosh(y Gamma t) + (|A|^2-|B|^2)/2 cos(x Gamma t)
                            + Re(A B*) sinh(y Gamma t) + Im(A B*) sin(x Gamma t) ],
convolved with a Gaussian resolution of width sigma_t.  Writing each term through
e^{-g t} with g = Gamma(1 -+ y) (cosh, sinh) and g = Gamma(1 - i x) (cos + i sin), the
convolution of e^{-g t} (t >= 0) with the resolution is
    E(g; t, s) = 1/2 exp(g^2 s^2/2 - g t) erfc(u),  u = (g s^2 - t)/(s sqrt 2),
evaluated through the Faddeeva function w(z) = exp(-z^2) erfc(-i z):
    Re u >= 0:  E = 1/2 exp(-t^2/(2 s^2)) w(i u)
    Re u <  0:  E = exp(g^2 s^2/2 - g t) - 1/2 exp(-t^2/(2 s^2)) w(-i u)
(both arguments in the upper half plane).  Then
    T_ch = (E(G(1-y)) + E(G(1+y)))/2,  T_sh = (E(G(1-y)) - E(G(1+y)))/2,
    T_c + i T_s = E(G(1 - i x)),
    R = (|A|^2+|B|^2)/2 T_ch + (|A|^2-|B|^2)/2 T_c + Re(A B*) T_sh + Im(A B*) T_s.

Normalisation over phase space and all t (the resolution keeps the integral over t):
    int e^{-Gt} cosh = 1/(G(1-y^2)), sinh -> y/(G(1-y^2)), cos -> 1/(G(1+x^2)), sin -> x/(G(1+x^2));
    N = <|A|^2+|B|^2>/2 I_ch + <|A|^2-|B|^2>/2 I_c + Re<A B*> I_sh + Im<A B*> I_s,
    <.> = mean over a uniform phase-space MC sample, <a_k a_l*> = G_kl (the Gram matrix).
f = R / N;  NLL = - sum_i log f(x_i, t_i).

The gradient is written out analytically (tests pin it against finite differences):
    dR/dRe c_k = Re(a_k V), dR/dIm c_k = -Im(a_k V),  V = (T_ch + T_c) A* + (T_sh - i T_s) B*,
    dE/dg = (g s^2 - t) E - s/sqrt(2 pi) exp(-t^2/(2 s^2)),
    dE/ds = g^2 s E - (g s^2 + t)/(s^2 sqrt(2 pi)) exp(-t^2/(2 s^2)).
"""
import math

import numpy as np
from scipy.special import wofz

ANGULAR = ("SS", "VS0", "SV0", "VV0", "VVpar", "VVperp", "TS0", "TV0")
SPINS = {"SS": (0, 0), "VS0": (1, 0), "SV0": (0, 1), "VV0": (1, 1), "VVpar": (1, 1), "VVperp": (1, 1),
         "TS0": (2, 0), "TV0": (2, 1)}
OBS = ("m12", "m34", "c12", "c34", "phi", "t")


def two_body_momentum(M, ma, mb):
    lam = (M * M - (ma + mb) ** 2) * (M * M - (ma - mb) ** 2)
    return np.sqrt(np.clip(lam, 0.0, None)) / (2.0 * M)


def barrier(L, z):
    if L == 0:
        return np.ones_like(z)
    if L == 1:
        return np.sqrt(1.0 / (1.0 + z))
    if L == 2:
        return np.sqrt(9.0 / (9.0 + 3.0 * z + z * z))
    raise ValueError("spin > 2")


def lineshape(m, m0, g0, L, ma, mb, r):
    """F(m) = BW(m^2) (q/q0)^L B_L(r q)/B_L(r q0) for a resonance decaying to (ma, mb)."""
    q = two_body_momentum(m, ma, mb)
    q0 = two_body_momentum(m0, ma, mb)
    bratio = barrier(L, (r * q) ** 2) / barrier(L, (r * q0) ** 2)
    width = g0 * (q / q0) ** (2 * L + 1) * (m0 / m) * bratio ** 2
    bw = 1.0 / (m0 * m0 - m * m - 1j * m0 * width)
    return bw * (q / q0) ** L * bratio


def angular(kind, c12, c34, phi):
    s12 = np.sqrt(np.clip(1.0 - c12 * c12, 0.0, None))
    s34 = np.sqrt(np.clip(1.0 - c34 * c34, 0.0, None))
    p2 = 0.5 * (3.0 * c12 * c12 - 1.0)
    out = {
        "SS": np.ones_like(c12),
        "VS0": c12,
        "SV0": c34,
        "VV0": c12 * c34,
        "VVpar": s12 * s34 * np.cos(phi),
        "VVperp": 1j * s12 * s34 * np.sin(phi),
        "TS0": p2,
        "TV0": p2 * c34,
    }[kind]
    return np.asarray(out, dtype=np.complex128)


def conv_exp(g, t, s):
    """E(g; t, s): e^{-g t'} (t' >= 0) convolved with a Gaussian of width s, at t (g complex ok)."""
    g = np.asarray(g, dtype=np.complex128)
    t = np.asarray(t, dtype=np.float64)
    g, t = np.broadcast_arrays(g, t)
    u = (g * s * s - t) / (s * math.sqrt(2.0))
    gauss = np.exp(-t * t / (2.0 * s * s))
    E = np.empty(t.shape, dtype=np.complex128)
    pos = u.real >= 0.0
    E[pos] = 0.5 * gauss[pos] * wofz(1j * u[pos])
    neg = ~pos
    E[neg] = np.exp(g[neg] * g[neg] * s * s / 2.0 - g[neg] * t[neg]) - 0.5 * gauss[neg] * wofz(-1j * u[neg])
    return E


def conv_exp_derivs(g, t, s, E):
    """(dE/dg, dE/ds) of conv_exp at the same arguments."""
    g = np.asarray(g, dtype=np.complex128)
    gauss = np.exp(-t * t / (2.0 * s * s))
    dg = (g * s * s - t) * E - s / math.sqrt(2.0 * math.pi) * gauss
    ds = g * g * s * E - (g * s * s + t) / (s * s * math.sqrt(2.0 * math.pi)) * gauss
    return dg, ds


def time_terms(t, x, y, tau, s, derivs=False):
    """(T_ch, T_sh, T_c, T_s) at the observed times; with derivs also d/d(x, y, tau, s)."""
    G = 1.0 / tau
    gp, gm, gc = G * (1.0 - y), G * (1.0 + y), G * (1.0 - 1j * x)
    Ep, Em, Ec = conv_exp(gp, t, s), conv_exp(gm, t, s), conv_exp(gc, t, s)
    T = (0.5 * (Ep + Em).real, 0.5 * (Ep - Em).real, Ec.real, Ec.imag)
    if not derivs:
        return T
    dgp, dsp = conv_exp_derivs(gp, t, s, Ep)
    dgm, dsm = conv_exp_derivs(gm, t, s, Em)
    dgc, dsc = conv_exp_derivs(gc, t, s, Ec)
    # parameter -> (dT_ch, dT_sh, dT_c, dT_s); dg/dy = -+G, dg/dtau = -g/tau, dgc/dx = -iG
    zero = np.zeros_like(t)
    dx = (zero, zero, (dgc * (-1j * G)).real, (dgc * (-1j * G)).imag)
    dy = (0.5 * (dgp * (-G) + dgm * G).real, 0.5 * (dgp * (-G) - dgm * G).real, zero, zero)
    dtau = (0.5 * (dgp * (-gp / tau) + dgm * (-gm / tau)).real, 0.5 * (dgp * (-gp / tau) - dgm * (-gm / tau)).real,
            (dgc * (-gc / tau)).real, (dgc * (-gc / tau)).imag)
    ds = (0.5 * (dsp + dsm).real, 0.5 * (dsp - dsm).real, dsc.real, dsc.imag)
    return T, (dx, dy, dtau, ds)


def time_integrals(x, y, tau, derivs=False):
    """(I_ch, I_sh, I_c, I_s): integrals over t of the four terms; with derivs d/d(x, y, tau)."""
    I = (tau / (1 - y * y), y * tau / (1 - y * y), tau / (1 + x * x), x * tau / (1 + x * x))
    if not derivs:
        return I
    dx = (0.0, 0.0, -2 * x * tau / (1 + x * x) ** 2, tau * (1 - x * x) / (1 + x * x) ** 2)
    dy = (2 * y * tau / (1 - y * y) ** 2, tau * (1 + y * y) / (1 - y * y) ** 2, 0.0, 0.0)
    dtau = (1 / (1 - y * y), y / (1 - y * y), 1 / (1 + x * x), x / (1 + x * x))
    return I, (dx, dy, dtau)


class TD4Model:
    def __init__(self, spec):
        kind, kin, amps, tpar = spec["pdf"]
        assert kind == "td4"
        self.kin = kin
        self.amps = amps
        self.pidx = {p[0]: i for i, p in enumerate(spec["params"])}
        self.P = len(spec["params"])
        self.re = [self.pidx[a[3]] for a in amps]
        self.im = [self.pidx[a[4]] for a in amps]
        self.b = np.array([complex(*a[5]) for a in amps])
        self.tp = [self.pidx[n] for n in tpar]  # x, y, tau, sigma_t

    def amplitudes(self, cols):
        """(n, K) complex128 amplitudes a_k at the events' phase-space coordinates."""
        k = self.kin
        m12, m34 = np.asarray(cols["m12"], float), np.asarray(cols["m34"], float)
        c12, c34, phi = (np.asarray(cols[n], float) for n in ("c12", "c34", "phi"))
        out = np.empty((m12.size, len(self.amps)), dtype=np.complex128)
        for j, (ang, (m01, g01), (m02, g02), _, _, _) in enumerate(self.amps):
            L1, L2 = SPINS[ang]
            f1 = lineshape(m12, m01, g01, L1, k["m1"], k["m2"], k["r_res"])
            f2 = lineshape(m34, m02, g02, L2, k["m3"], k["m4"], k["r_res"])
            out[:, j] = f1 * f2 * angular(ang, c12, c34, phi)
        return out

    def coefficients(self, theta):
        th = np.asarray(theta, dtype=np.float64)
        return th[self.re] + 1j * th[self.im]

    def gram(self, mc_amps):
        return mc_amps.T @ mc_amps.conj() / mc_amps.shape[0]   # G_kl = <a_k conj(a_l)>

    def norm(self, G, theta, derivs=False):
        th = np.asarray(theta, dtype=np.float64)
        c, b = self.coefficients(th), self.b
        x, y, tau = th[self.tp[0]], th[self.tp[1]], th[self.tp[2]]
        AA = np.real(c @ G @ c.conj())
        BB = np.real(b @ G @ b.conj())
        AB = c @ G @ b.conj()
        res = time_integrals(x, y, tau, derivs)
        I = res[0] if derivs else res
        N = 0.5 * (AA + BB) * I[0] + 0.5 * (AA - BB) * I[2] + AB.real * I[1] + AB.imag * I[3]
        if not derivs:
            return N
        dI = res[1]
        g = np.zeros(self.P)
        VN = (I[0] + I[2]) * (G @ c.conj()) + (I[1] - 1j * I[3]) * (G @ b.conj())  # <a_k V_N>
        g[self.re] += VN.real
        g[self.im] += -VN.imag
        for j, d in enumerate(dI):
            g[self.tp[j]] += 0.5 * (AA + BB) * d[0] + 0.5 * (AA - BB) * d[2] + AB.real * d[1] + AB.imag * d[3]
        return N, g

    def rate(self, a, t, theta, derivs=False):
        """R at each event (amplitude rows a, observed times t); with derivs dR/dtheta (n, P)."""
        th = np.asarray(theta, dtype=np.float64)
        c = self.coefficients(th)
        A, B = a @ c, a @ self.b
        x, y, tau, s = (th[i] for i in self.tp)
        res = time_terms(np.asarray(t, float), x, y, tau, s, derivs)
        T = res[0] if derivs else res
        AA, BB, AB = np.abs(A) ** 2, np.abs(B) ** 2, A * B.conj()
        R = 0.5 * (AA + BB) * T[0] + 0.5 * (AA - BB) * T[2] + AB.real * T[1] + AB.imag * T[3]
        if not derivs:
            return R
        dR = np.zeros((R.size, self.P))
        V = (T[0] + T[2]) * A.conj() + (T[1] - 1j * T[3]) * B.conj()
        aV = a * V[:, None]
        dR[:, self.re] += aV.real
        dR[:, self.im] += -aV.imag
        for j, d in enumerate(res[1]):
            dR[:, self.tp[j]] += 0.5 * (AA + BB) * d[0] + 0.5 * (AA - BB) * d[2] + AB.real * d[1] + AB.imag * d[3]
        return R, dR

    def nll(self, cols, mc_amps, theta, a=None):
        a = self.amplitudes(cols) if a is None else a
        R = self.rate(a, cols["t"], theta)
        N = self.norm(self.gram(mc_amps), theta)
        return float(-np.sum(np.log(R)) + R.size * math.log(N))

    def nll_grad(self, cols, mc_amps, theta, a=None):
        a = self.amplitudes(cols) if a is None else a
        R, dR = self.rate(a, cols["t"], theta, derivs=True)
        N, dN = self.norm(self.gram(mc_amps), theta, derivs=True)
        nll = float(-np.sum(np.log(R)) + R.size * math.log(N))
        g = -(dR / R[:, None]).sum(axis=0) + R.size * dN / N
        return nll, g

    def true_rate(self, a, t_true, theta):
        """R without resolution at true times t >= 0 (generation)."""
        th = np.asarray(theta, dtype=np.float64)
        c = self.coefficients(th)
        A, B = a @ c, a @ self.b
        x, y, tau = (th[i] for i in self.tp[:3])
        G = 1.0 / tau
        e = np.exp(-G * t_true)
        AA, BB, AB = np.abs(A) ** 2, np.abs(B) ** 2, A * B.conj()
        return e * (0.5 * (AA + BB) * np.cosh(y * G * t_true) + 0.5 * (AA - BB) * np.cos(x * G * t_true)
                    + AB.real * np.sinh(y * G * t_true) + AB.imag * np.sin(x * G * t_true))


def _ps_weight(m12, m34, kin):
    """Four-body phase-space density in (m12, m34) (uniform in the angles): p q12 q34."""
    M = kin["M"]
    inside = m12 + m34 < M
    w = (two_body_momentum(M, m12, np.where(inside, m34, 0.0)) * two_body_momentum(m12, kin["m1"], kin["m2"])
         * two_body_momentum(m34, kin["m3"], kin["m4"]))
    return np.where(inside, w, 0.0)


def envelope_cells(spec, theta, seed, cells=48, scan=1_000_000, safety=1.5):
    """Per-cell upper bounds of w_PS (|A| + |B|)^2 on a cells x cells grid over (m12, m34).

    The bound of a cell is `safety` times the largest value found by a uniform scan of the
    cell and its neighbours (uniform angles).  R_true e^{G(1-|y|) t} <= (|A| + |B|)^2 for
    every t, so these also bound the time-dependent acceptance weight.
    """
    m = TD4Model(spec)
    (lo12, hi12), (lo34, hi34) = [o[1:] for o in spec["observables"][:2]]
    rng = np.random.Generator(np.random.PCG64(seed))
    th = np.asarray(theta, dtype=np.float64)
    c = m.coefficients(th)
    pts = {"m12": rng.uniform(lo12, hi12, scan), "m34": rng.uniform(lo34, hi34, scan),
           "c12": rng.uniform(-1, 1, scan), "c34": rng.uniform(-1, 1, scan), "phi": rng.uniform(-np.pi, np.pi, scan)}
    a = m.amplitudes(pts)
    v = _ps_weight(pts["m12"], pts["m34"], m.kin) * (np.abs(a @ c) + np.abs(a @ m.b)) ** 2
    i = np.minimum(((pts["m12"] - lo12) / (hi12 - lo12) * cells).astype(int), cells - 1)
    j = np.minimum(((pts["m34"] - lo34) / (hi34 - lo34) * cells).astype(int), cells - 1)
    cmax = np.zeros((cells, cells))
    np.maximum.at(cmax, (i, j), v)
    padded = np.pad(cmax, 1)
    nb = np.max([padded[1 + di:cells + 1 + di, 1 + dj:cells + 1 + dj] for di in (-1, 0, 1) for dj in (-1, 0, 1)],
                axis=0)
    return safety * nb


def _generate_part(spec, theta, n, seed, bounds, chunk):
    m = TD4Model(spec)
    th = np.asarray(theta, dtype=np.float64)
    x, y, tau, s = (th[i] for i in m.tp)
    rate = (1.0 - abs(y)) / tau
    (lo12, hi12), (lo34, hi34) = [o[1:] for o in spec["observables"][:2]]
    tlo, thi = [o for o in spec["observables"] if o[0] == "t"][0][1:]
    cells = bounds.shape[0]
    flat = bounds.ravel()
    prob = flat / flat.sum()
    rng = np.random.Generator(np.random.PCG64(seed))
    out = {k: np.empty(n) for k in OBS}
    filled, worst = 0, 0.0
    while filled < n:
        # proposal: a cell with probability proportional to its bound, a point uniform in it
        k = rng.choice(flat.size, size=chunk, p=prob)
        ci, cj = k // cells, k % cells
        cand = {"m12": lo12 + (ci + rng.uniform(0, 1, chunk)) * (hi12 - lo12) / cells,
                "m34": lo34 + (cj + rng.uniform(0, 1, chunk)) * (hi34 - lo34) / cells,
                "c12": rng.uniform(-1, 1, chunk), "c34": rng.uniform(-1, 1, chunk),
                "phi": rng.uniform(-np.pi, np.pi, chunk)}
        t_true = rng.exponential(1.0 / rate, chunk)
        a = m.amplitudes(cand)
        target = _ps_weight(cand["m12"], cand["m34"], m.kin) * m.true_rate(a, t_true, th) * np.exp(rate * t_true)
        ratio = target / flat[k]
        worst = max(worst, float(ratio.max()))
        keep = rng.uniform(0.0, 1.0, chunk) < ratio
        t_obs = t_true + rng.normal(0.0, s, chunk)
        keep &= (t_obs >= tlo) & (t_obs <= thi)
        take = min(n - filled, int(keep.sum()))
        for key in OBS[:5]:
            out[key][filled:filled + take] = cand[key][keep][:take]
        out["t"][filled:filled + take] = t_obs[keep][:take]
        filled += take
    return out, worst


def generate(spec, theta, n, seed, workers=1, chunk=200_000):
    """n events of the model: accept--reject on the true rate, then resolution smearing.

    Proposal: (m12, m34) uniform inside a cell of a 48 x 48 grid chosen with probability
    proportional to the cell's envelope bound, uniform angles, true times from
    Exp(G(1-|y|)); acceptance w_PS R_true e^{G(1-|y|) t} / bound.  The result does not
    depend on `workers` (each worker draws its own seeded share).  Raises if a candidate
    exceeded its envelope.
    """
    bounds = envelope_cells(spec, theta, seed + 17)
    if workers <= 1:
        out, worst = _generate_part(spec, theta, n, seed, bounds, chunk)
    else:
        import multiprocessing as mp
        sizes = [n // workers + (1 if w < n % workers else 0) for w in range(workers)]
        with mp.get_context("spawn").Pool(workers) as pool:
            parts = pool.starmap(_generate_part, [(spec, theta, sizes[w], seed * 1000 + w, bounds, chunk)
                                                  for w in range(workers)])
        out = {k: np.concatenate([p[0][k] for p in parts]) for k in OBS}
        worst = max(p[1] for p in parts)
    if worst > 1.0:
        raise RuntimeError(f"accept-reject envelope exceeded ({worst:.3f})")
    return out
