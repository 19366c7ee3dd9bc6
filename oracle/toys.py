"""Toy pseudo-experiments drawn with the counter-based generator (reference for the device).

Candidate j of a toy with seed s takes the Philox4x64-10 outputs w0, w1, w2 at counter
(j, 0, 0, 0) and key (s, 0x6f6f67) (oracle/philox.py); the float32 uniforms
u = (w >> 40) 2^-24 place the candidate uniformly in the Dalitz box,
    s12 = lo12 + u0 * (hi12 - lo12),   s13 = lo13 + u1 * (hi13 - lo13)   (float32 arithmetic),
and it is accepted when it lies inside the kinematic region and u2 * fmax < |S(s12, s13)|^2.
The toy is the first n accepted candidates in candidate order.  The acceptance decision is
taken in float32, the precision of the device generator, with this oracle's own amplitude
formulas (helicity-angle form, oracle/dalitz.py).
"""
import numpy as np
import torch

from . import dalitz as od
from . import philox as ph


def _u24(w):
    return np.float32(int(w) >> 40) * np.float32(2.0 ** -24)


def generate_toy(spec, theta, fmax, seed, n, chunk=8192, max_candidates=50_000_000):
    model = od.DalitzModel(spec)
    kin = model.kin
    M, m1, m2, m3 = kin["M"], kin["m1"], kin["m2"], kin["m3"]
    lo12, hi12 = (m1 + m2) ** 2, (M - m3) ** 2
    lo13, hi13 = (m1 + m3) ** 2, (M - m2) ** 2
    f = np.float32
    lo12f, w12f, lo13f, w13f = f(lo12), f(hi12 - lo12), f(lo13), f(hi13 - lo13)
    th32 = torch.as_tensor(np.asarray(theta, dtype=np.float64)).to(torch.float32)
    fmax32 = f(fmax)
    out12, out13, idx = [], [], []
    j = 0
    while len(out12) < n and j < max_candidates:
        us = [[_u24(w) for w in ph.philox4x64((jj, 0, 0, 0), (seed, ph.TOY_KEY1))[:3]] for jj in range(j, j + chunk)]
        us = np.array(us, dtype=np.float32)
        s12 = (lo12f + (us[:, 0] * w12f).astype(np.float32)).astype(np.float32)
        s13 = (lo13f + (us[:, 1] * w13f).astype(np.float32)).astype(np.float32)
        t12 = torch.from_numpy(s12)
        t13 = torch.from_numpy(s13)
        ok12 = (t12 > f(lo12)) & (t12 < f(hi12))
        t12c = torch.clamp(t12, f(lo12) * f(1.0000001), f(hi12) * f(0.9999999))
        _, _, cos = od.helicity_frame(t12c, t13, f(M), f(m1), f(m2), f(m3))
        inside = (ok12 & (cos.abs() <= 1.0)).numpy()
        with torch.no_grad():
            A = model.amplitude_matrix({"s12": s12, "s13": s13}, th32, dtype=torch.float32)
            S2 = model.intensity(A, th32).numpy().astype(np.float32)
        acc = inside & ((us[:, 2] * fmax32).astype(np.float32) < S2)
        for k in np.flatnonzero(acc):
            if len(out12) < n:
                out12.append(s12[k])
                out13.append(s13[k])
                idx.append(j + k)
        j += chunk
    return np.array(out12, dtype=np.float32), np.array(out13, dtype=np.float32), np.array(idx)
