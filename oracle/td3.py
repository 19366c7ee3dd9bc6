"""Time-dependent three-body amplitude model (float64 / complex128 numpy, CPU).

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

The paper lists time-dependent amplitude analyses of three-body decays among GooFit's
amplitude PDFs (Sec. 5) and times a time-dependent D0 -> pi+ pi- pi0 fit (Table 2).  It
prints no formula; this file writes out the model (a reading):

Kinematics.  Particle 1 is the neutral pion, 2 and 3 the charged pions (m2 = m3), so the
Dalitz plot in s12 = m^2(1 2), s13 = m^2(1 3) is symmetric under s12 <-> s13.  Observables
s12, s13 and the decay time t.

Amplitudes.  a_k(s12, s13) are the three-body isobar amplitudes of oracle/dalitz.py
(relativistic Breit--Wigner with running width, Blatt--Weisskopf factors, Zemach spin
factors; a constant non-resonant amplitude).  CP conjugation exchanges the charged pions,
i.e. the two Dalitz coordinates, so the anti-particle's amplitudes are
    abar_k(s12, s13) = a_k(s13, s12).
With no CP violation (q/p = 1, the same coefficients):
    A = sum_k c_k a_k,   B = sum_k c_k abar_k.

Decay time.  R is the four-body model's mixing rate (oracle/td4.py) with these A and B:
    R = (|A|^2+|B|^2)/2 T_ch + (|A|^2-|B|^2)/2 T_c + Re(A B*) T_sh + Im(A B*) T_s,
the T's being the resolution-convolved exponentials of td4.time_terms.

Normalisation over phase space (uniform MC) and all t:
    N = <|A|^2+|B|^2>/2 I_ch + <|A|^2-|B|^2>/2 I_c + Re<A B*> I_sh + Im<A B*> I_s,
    <|A|^2> = c^T G_aa c*,  <|B|^2> = c^T G_bb c*,  <A B*> = c^T G_ab c*,
    G_aa = <a_k a_l*>, G_bb = <abar_k abar_l*>, G_ab = <a_k abar_l*> (MC means).

Gradient (analytic; tests pin it against finite differences):
    dR/dRe c_k = Re(a_k V_A + abar_k V_B),  dR/dIm c_k = -Im(a_k V_A + abar_k V_B),
    V_A = (T_ch + T_c) A* + (T_sh - i T_s) B*,  V_B = (T_ch - T_c) B* + (T_sh + i T_s) A*.
"""
import math

import numpy as np
import torch

from . import dalitz as od
from .td4 import time_integrals, time_terms


class TD3Model:
    def __init__(self, spec):
        kind, kin, amps, tpar = spec["pdf"]
        assert kind == "td3"
        self.kin = kin
        self.amps = amps
        self.pidx = {p[0]: i for i, p in enumerate(spec["params"])}
        self.P = len(spec["params"])
        self.re = [self.pidx[a[-2]] for a in amps]
        self.im = [self.pidx[a[-1]] for a in amps]
        self.tp = [self.pidx[n] for n in tpar]  # x, y, tau, sigma_t
        self.polar = spec.get("coef") == "polar"
        self._dz = od.DalitzModel(dict(spec, pdf=("coherent", kin, amps)))

    def amplitudes(self, cols, theta):
        """(a, abar): (n, K) complex128 amplitudes at (s12, s13) and at the exchanged point."""
        th = torch.as_tensor(np.asarray(theta, dtype=np.float64))
        s12 = np.asarray(cols["s12"], dtype=np.float64)
        s13 = np.asarray(cols["s13"], dtype=np.float64)
        with torch.no_grad():
            a = self._dz.amplitude_matrix({"s12": s12, "s13": s13}, th).numpy()
            ab = self._dz.amplitude_matrix({"s12": s13, "s13": s12}, th).numpy()
        return a, ab

    def coefficients(self, theta):
        """c_k: (Re, Im) parameters, or with spec["coef"] == "polar" (r, phi): r e^{i phi}."""
        th = np.asarray(theta, dtype=np.float64)
        if self.polar:
            return th[self.re] * np.exp(1j * th[self.im])
        return th[self.re] + 1j * th[self.im]

    def _to_params(self, g, theta):
        """Map a gradient over (Re c, Im c) to the coefficient parameters (chain rule; polar:
        d/dr = cos(phi) d/dRe + sin(phi) d/dIm, d/dphi = -r sin(phi) d/dRe + r cos(phi) d/dIm)."""
        if not self.polar:
            return g
        th = np.asarray(theta, dtype=np.float64)
        r, ph = th[self.re], th[self.im]
        gre, gim = g[..., self.re].copy(), g[..., self.im].copy()
        out = g.copy()
        out[..., self.re] = np.cos(ph) * gre + np.sin(ph) * gim
        out[..., self.im] = -r * np.sin(ph) * gre + r * np.cos(ph) * gim
        return out

    def grams(self, mc_cols, theta):
        a, ab = self.amplitudes(mc_cols, theta)
        n = a.shape[0]
        return a.T @ a.conj() / n, ab.T @ ab.conj() / n, a.T @ ab.conj() / n

    def norm(self, grams, theta, derivs=False):
        Gaa, Gbb, Gab = grams
        th = np.asarray(theta, dtype=np.float64)
        c = self.coefficients(th)
        x, y, tau = th[self.tp[0]], th[self.tp[1]], th[self.tp[2]]
        PA = float(np.real(c @ Gaa @ c.conj()))
        PB = float(np.real(c @ Gbb @ c.conj()))
        X = complex(c @ Gab @ c.conj())
        res = time_integrals(x, y, tau, derivs)
        I = res[0] if derivs else res
        N = 0.5 * (PA + PB) * I[0] + 0.5 * (PA - PB) * I[2] + X.real * I[1] + X.imag * I[3]
        if not derivs:
            return N
        dN = np.zeros(self.P)
        va, vb = Gaa @ c.conj(), Gbb @ c.conj()          # d<|A|^2>/dRe c = 2 Re va, /dIm c = -2 Im va
        u, w = Gab @ c.conj(), Gab.T @ c                  # dX/dRe c = u + w, dX/dIm c = i (u - w)
        dPA = (2 * va.real, -2 * va.imag)
        dPB = (2 * vb.real, -2 * vb.imag)
        dX = (u + w, 1j * (u - w))
        for part, idx in ((0, self.re), (1, self.im)):
            dN[idx] += (0.5 * (dPA[part] + dPB[part]) * I[0] + 0.5 * (dPA[part] - dPB[part]) * I[2]
                        + dX[part].real * I[1] + dX[part].imag * I[3])
        for j, d in enumerate(res[1]):
            dN[self.tp[j]] += 0.5 * (PA + PB) * d[0] + 0.5 * (PA - PB) * d[2] + X.real * d[1] + X.imag * d[3]
        return N, self._to_params(dN, th)

    def rate(self, amps, t, theta, derivs=False):
        a, ab = amps
        th = np.asarray(theta, dtype=np.float64)
        c = self.coefficients(th)
        A, B = a @ c, ab @ c
        x, y, tau, s = (th[i] for i in self.tp)
        res = time_terms(np.asarray(t, float), x, y, tau, s, derivs)
        T = res[0] if derivs else res
        AA, BB, AB = np.abs(A) ** 2, np.abs(B) ** 2, A * B.conj()
        R = 0.5 * (AA + BB) * T[0] + 0.5 * (AA - BB) * T[2] + AB.real * T[1] + AB.imag * T[3]
        if not derivs:
            return R
        dR = np.zeros((R.size, self.P))
        VA = (T[0] + T[2]) * A.conj() + (T[1] - 1j * T[3]) * B.conj()
        VB = (T[0] - T[2]) * B.conj() + (T[1] + 1j * T[3]) * A.conj()
        q = a * VA[:, None] + ab * VB[:, None]
        np.add.at(dR, (slice(None), self.re), q.real)
        np.add.at(dR, (slice(None), self.im), -q.imag)
        for j, d in enumerate(res[1]):
            dR[:, self.tp[j]] += 0.5 * (AA + BB) * d[0] + 0.5 * (AA - BB) * d[2] + AB.real * d[1] + AB.imag * d[3]
        return R, self._to_params(dR, th)

    def nll(self, cols, mc_cols, theta, amps=None, grams=None):
        amps = self.amplitudes(cols, theta) if amps is None else amps
        grams = self.grams(mc_cols, theta) if grams is None else grams
        R = self.rate(amps, cols["t"], theta)
        return float(-np.sum(np.log(R)) + R.size * math.log(self.norm(grams, theta)))

    def nll_grad(self, cols, mc_cols, theta, amps=None, grams=None):
        amps = self.amplitudes(cols, theta) if amps is None else amps
        grams = self.grams(mc_cols, theta) if grams is None else grams
        R, dR = self.rate(amps, cols["t"], theta, derivs=True)
        N, dN = self.norm(grams, theta, derivs=True)
        nll = float(-np.sum(np.log(R)) + R.size * math.log(N))
        return nll, -(dR / R[:, None]).sum(axis=0) + R.size * dN / N

    def true_rate(self, amps, t_true, theta):
        """R without resolution at true times t >= 0 (generation)."""
        a, ab = amps
        th = np.asarray(theta, dtype=np.float64)
        c = self.coefficients(th)
        A, B = a @ c, ab @ c
        x, y, tau = (th[i] for i in self.tp[:3])
        G = 1.0 / tau
        AA, BB, AB = np.abs(A) ** 2, np.abs(B) ** 2, A * B.conj()
        return np.exp(-G * t_true) * (0.5 * (AA + BB) * np.cosh(y * G * t_true)
                                      + 0.5 * (AA - BB) * np.cos(x * G * t_true)
                                      + AB.real * np.sinh(y * G * t_true) + AB.imag * np.sin(x * G * t_true))


def generate(spec, theta, n, seed, candidates, chunk=100_000, safety=1.3):
    """n events of the model: Dalitz points from `candidates(k, seed)` (uniform phase space),
    true times from Exp(G (1 - |y|)), accepted with probability R_true / (e^{-G(1-|y|)t} F),
    F = safety x the largest (|A| + |B|)^2 on a scan sample (which bounds the bracket), then a
    Gaussian resolution.  Returns the columns s12, s13, t (observed)."""
    m = TD3Model(spec)
    th = np.asarray(theta, dtype=np.float64)
    x, y, tau, s = (th[i] for i in m.tp)
    G = 1.0 / tau
    gmin = G * (1.0 - abs(y))
    scan = candidates(200_000, seed + 7919)
    a, ab = m.amplitudes(scan, th)
    c = m.coefficients(th)
    F = safety * float(np.max((np.abs(a @ c) + np.abs(ab @ c)) ** 2))
    rng = np.random.default_rng(seed)
    out = {"s12": [], "s13": [], "t": []}
    have, k = 0, 0
    while have < n:
        cand = candidates(chunk, seed + 1 + k)
        k += 1
        tt = rng.exponential(1.0 / gmin, chunk)
        amps = m.amplitudes(cand, th)
        w = m.true_rate(amps, tt, th) / (np.exp(-gmin * tt) * F)
        assert np.all(w <= 1.0), float(w.max())
        acc = rng.uniform(size=chunk) < w
        for key, v in (("s12", cand["s12"][acc]), ("s13", cand["s13"][acc]), ("t", tt[acc])):
            out[key].append(v)
        have += int(acc.sum())
    cols = {key: np.concatenate(v)[:n] for key, v in out.items()}
    cols["t"] = cols["t"] + rng.normal(0.0, s, n)
    return cols
