"""Seeded (numpy PCG64) event-sample generators for the synthetic workloads.

Every sampler uses numpy's own distribution samplers (normal, exponential, gamma,
uniform) and rejects draws outside the observable range.  No density of the fitted
model is evaluated here, except through a caller-supplied function in
``accept_reject``.
"""
import math

import numpy as np


def _truncated(draw, lo, hi, n, rng):
    """Draw n values from ``draw(rng, k)`` restricted to [lo, hi] by rejection."""
    out = np.empty(n, dtype=np.float64)
    filled = 0
    while filled < n:
        k = max(1024, int((n - filled) * 1.2) + 16)
        v = draw(rng, k)
        v = v[(v >= lo) & (v <= hi)]
        take = min(n - filled, v.size)
        out[filled:filled + take] = v[:take]
        filled += take
    return out


def gen_c1(n=100_000, seed=1710001):
    """x in [0, 10]: 0.3 Gaussian(5.0, 0.4) + 0.7 exponential with rate 0.3, truncated."""
    rng = np.random.Generator(np.random.PCG64(seed))
    n_sig = int(rng.binomial(n, 0.3))
    sig = _truncated(lambda r, k: r.normal(5.0, 0.4, k), 0.0, 10.0, n_sig, rng)
    bkg = _truncated(lambda r, k: r.exponential(1.0 / 0.3, k), 0.0, 10.0, n - n_sig, rng)
    x = np.concatenate([sig, bkg])
    rng.shuffle(x)
    return {"x": x}


def gen_c2(n=10_000_000, seed=1710002):
    """(m, dE, t) on [5.2,5.3] x [-0.2,0.2] x [0,10]: 20% signal, 80% background.

    Signal: m ~ N(5.279, 0.003), dE ~ N(0, 0.02), t ~ exponential(mean 1.5).
    Background: m from the Argus shape with endpoint 5.29, curvature -20, power 0.5 --
    drawn as u = 1 - m^2/m0^2 ~ Gamma(shape 1.5, scale 1/20), m = m0 sqrt(1 - u) --
    dE from the quadratic 1 - dE + 0.5 dE^2 by accept--reject against a flat envelope,
    and t ~ exponential(mean 0.8).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n_sig = int(rng.binomial(n, 0.2))
    n_bkg = n - n_sig
    m_s = _truncated(lambda r, k: r.normal(5.279, 0.003, k), 5.2, 5.3, n_sig, rng)
    d_s = _truncated(lambda r, k: r.normal(0.0, 0.02, k), -0.2, 0.2, n_sig, rng)
    t_s = _truncated(lambda r, k: r.exponential(1.5, k), 0.0, 10.0, n_sig, rng)

    m0 = 5.29
    u_max = 1.0 - (5.2 / m0) ** 2
    u = _truncated(lambda r, k: r.gamma(1.5, 1.0 / 20.0, k), 1e-300, u_max, n_bkg, rng)
    m_b = m0 * np.sqrt(1.0 - u)

    coeffs = [1.0, -1.0, 0.5]                    # 1 + a1 x + a2 x^2 at the truth values
    env = np.polynomial.polynomial.polyval(-0.2, coeffs)   # its maximum on [-0.2, 0.2]
    d_b = np.empty(n_bkg)
    filled = 0
    while filled < n_bkg:
        k = int((n_bkg - filled) * 1.3) + 1024
        x = rng.uniform(-0.2, 0.2, k)
        keep = x[rng.uniform(0.0, env, k) < np.polynomial.polynomial.polyval(x, coeffs)]
        take = min(n_bkg - filled, keep.size)
        d_b[filled:filled + take] = keep[:take]
        filled += take
    t_b = _truncated(lambda r, k: r.exponential(0.8, k), 0.0, 10.0, n_bkg, rng)

    cols = {"m": np.concatenate([m_s, m_b]), "dE": np.concatenate([d_s, d_b]),
            "t": np.concatenate([t_s, t_b])}
    perm = rng.permutation(n)
    return {k: v[perm] for k, v in cols.items()}


def round_to_f32(cols, spec=None):
    """Round every column to the nearest float32 value (kept as float64 arrays).

    With a spec, a value whose rounding leaves its observable's [lo, hi] is replaced by the
    nearest float32 inside the range.
    """
    lims = {o[0]: (o[1], o[2]) for o in spec["observables"]} if spec else {}
    out = {}
    for k, v in cols.items():
        r = np.asarray(v, dtype=np.float32)
        if k in lims:
            lo, hi = lims[k]
            lo32 = np.float32(lo)
            hi32 = np.float32(hi)
            if float(lo32) < lo:
                lo32 = np.nextafter(lo32, np.float32(np.inf))
            if float(hi32) > hi:
                hi32 = np.nextafter(hi32, np.float32(-np.inf))
            r = np.clip(r, lo32, hi32)
        out[k] = r.astype(np.float64)
    return out


def dalitz_box(M, m1, m2, m3):
    """Bounding box of the Dalitz plot in (s12, s13)."""
    return (m1 + m2) ** 2, (M - m3) ** 2, (m1 + m3) ** 2, (M - m2) ** 2


def _inside_dalitz(s12, s13, M, m1, m2, m3):
    # s13 range at fixed s12 from the energies of particles 1 and 3 in the (12) rest frame.
    r = np.sqrt(s12)
    e1 = (s12 + m1 * m1 - m2 * m2) / (2 * r)
    e3 = (M * M - s12 - m3 * m3) / (2 * r)
    p1 = np.sqrt(np.clip(e1 * e1 - m1 * m1, 0.0, None))
    p3 = np.sqrt(np.clip(e3 * e3 - m3 * m3, 0.0, None))
    lo = (e1 + e3) ** 2 - (p1 + p3) ** 2
    hi = (e1 + e3) ** 2 - (p1 - p3) ** 2
    return (s13 > lo) & (s13 < hi) & (e3 > m3)


def dalitz_candidates(n, seed, M, m1, m2, m3):
    """n points uniform over the Dalitz region (uniform in the box, outside points rejected)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    lo12, hi12, lo13, hi13 = dalitz_box(M, m1, m2, m3)
    s12 = np.empty(n)
    s13 = np.empty(n)
    filled = 0
    while filled < n:
        k = int((n - filled) * 2.0) + 1024
        a = rng.uniform(lo12, hi12, k)
        b = rng.uniform(lo13, hi13, k)
        ok = _inside_dalitz(a, b, M, m1, m2, m3)
        a, b = a[ok], b[ok]
        take = min(n - filled, a.size)
        s12[filled:filled + take] = a[:take]
        s13[filled:filled + take] = b[:take]
        filled += take
    return {"s12": s12, "s13": s13}


def accept_reject(candidates, density, fmax, n, seed, chunk=1_000_000):
    """Keep n candidate points by accept--reject against ``density`` with envelope ``fmax``.

    ``candidates(k, seed)`` returns a dict of k columns drawn uniformly over the support;
    ``density(cols)`` returns the (unnormalised) density at those points and is supplied
    by the caller.  Returns the accepted columns and the largest density/fmax seen.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    out = None
    filled = 0
    worst = 0.0
    sub = 0
    while filled < n:
        cols = candidates(chunk, seed * 1000 + sub)
        sub += 1
        f = np.asarray(density(cols), dtype=np.float64)
        worst = max(worst, float(f.max() / fmax))
        keep = rng.uniform(0.0, fmax, f.size) < f
        if out is None:
            out = {k: np.empty(n) for k in cols}
        take = min(n - filled, int(keep.sum()))
        for k, v in cols.items():
            out[k][filled:filled + take] = v[keep][:take]
        filled += take
    return out, worst


def toy_sizes(n_toys=4096, lo=1e3, hi=1e6, seed=1710099):
    """Event counts log-uniform on [lo, hi] for a toy-MC study."""
    rng = np.random.Generator(np.random.PCG64(seed))
    u = rng.uniform(math.log(lo), math.log(hi), n_toys)
    return np.floor(np.exp(u)).astype(np.int64)


def _two_body_momentum(M, ma, mb):
    """Momentum of either daughter in the rest frame of a mass-M system (0 below threshold)."""
    lam = (M * M - (ma + mb) ** 2) * (M * M - (ma - mb) ** 2)
    return np.sqrt(np.clip(lam, 0.0, None)) / (2.0 * M)


def four_body_phase_space(n, seed, M, m1, m2, m3, m4):
    """n points of four-body phase space in (m12, m34, cos th12, cos th34, phi).

    Four-body phase space factorises into the parent's two-body decay to the (12) and (34)
    systems and their two-body decays; in these variables its density is proportional to
    p(M; m12, m34) q(m12; m1, m2) q(m34; m3, m4), uniform in both helicity cosines and in the
    angle phi between the decay planes.  (m12, m34) are drawn uniformly over their box and
    kept by accept--reject on that weight (zero where m12 + m34 > M).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    lo12, hi12 = m1 + m2, M - m3 - m4
    lo34, hi34 = m3 + m4, M - m1 - m2

    def weight(a, b):
        inside = a + b < M
        w = (_two_body_momentum(M, a, np.where(inside, b, 0.0)) * _two_body_momentum(a, m1, m2)
             * _two_body_momentum(b, m3, m4))
        return np.where(inside, w, 0.0)

    ga, gb = np.meshgrid(np.linspace(lo12, hi12, 801), np.linspace(lo34, hi34, 801))
    wmax = 1.05 * float(weight(ga, gb).max())
    m12 = np.empty(n)
    m34 = np.empty(n)
    filled = 0
    while filled < n:
        k = int((n - filled) * 3.0) + 4096
        a = rng.uniform(lo12, hi12, k)
        b = rng.uniform(lo34, hi34, k)
        ok = rng.uniform(0.0, wmax, k) < weight(a, b)
        a, b = a[ok], b[ok]
        take = min(n - filled, a.size)
        m12[filled:filled + take] = a[:take]
        m34[filled:filled + take] = b[:take]
        filled += take
    return {"m12": m12, "m34": m34, "c12": rng.uniform(-1.0, 1.0, n), "c34": rng.uniform(-1.0, 1.0, n),
            "phi": rng.uniform(-math.pi, math.pi, n)}


def gen_c4_candidates(n, seed, kin, rate):
    """Phase-space points plus true decay times t_true ~ Exp(rate) (the envelope in time of an
    accept--reject against the time-dependent rate, which the caller supplies)."""
    cols = four_body_phase_space(n, seed, kin["M"], kin["m1"], kin["m2"], kin["m3"], kin["m4"])
    rng = np.random.Generator(np.random.PCG64(seed + 7_000_001))
    cols["t_true"] = rng.exponential(1.0 / rate, n)
    return cols


def smear_times(t_true, sigma, seed):
    """Observed decay times: t_true plus Gaussian resolution N(0, sigma)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return t_true + rng.normal(0.0, sigma, t_true.size)
