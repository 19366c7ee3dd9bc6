"""Toy pseudo-experiments drawn with the counter-based generator (reference for the device).

TEST INFRASTRUCTURE: used only by the tests, the smoke check and the benchmark's CPU legs.

Candidate j of a toy with seed s takes the Philox4x64-10 outputs w0..w3 at counter
(j, 0, 0, 0) and key (s, 0x6f6f67) (oracle/philox.py).  The proposal is importance-sampled
over an envelope grid of n12 x n13 cells covering the Dalitz box, with per-cell bounds B_c on
|S|^2 (accept--reject, Section 4's toy studies):
  * cell choice: the top 32 bits of w0 against cumulative thresholds
    thr_c = floor(S_c / W * 2^32) (S_c = B_0 + ... + B_c and W the total, summed in FP64 in
    cell order; the last threshold is 2^32); the chosen cell is the first with top < thr_c,
    so cell c is drawn with probability (thr_c - thr_{c-1}) / 2^32, proportional to B_c;
  * the point, uniform in cell (i, j), with float32 uniforms u = (w >> 40) 2^-24:
        s12 = lo12 + (i + u(w1)) * cw12,   s13 = lo13 + (j + u(w2)) * cw13   (float32 steps);
  * acceptance: inside the kinematic region and u(w3) * B_c < |S(s12, s13)|^2.
The toy is the first n accepted candidates in candidate order.  Accepted points have density
proportional to min(|S|^2, B) over the region, i.e. exactly |S|^2 where B bounds it.  The
acceptance decision is taken in float32, the precision of the device generator, with this
oracle's own amplitude formulas (helicity-angle form, oracle/dalitz.py).
"""
import math

import numpy as np
import torch

from . import dalitz as od
from . import philox as ph


def _u24(w):
    return np.float32(int(w) >> 40) * np.float32(2.0 ** -24)


def _box(kin):
    M, m1, m2, m3 = kin["M"], kin["m1"], kin["m2"], kin["m3"]
    return (m1 + m2) ** 2, (M - m3) ** 2, (m1 + m3) ** 2, (M - m2) ** 2


def thresholds(bound):
    """Cumulative cell thresholds thr_c = floor(S_c / W * 2^32), the last one 2^32."""
    b = np.asarray(bound, dtype=np.float32).reshape(-1)
    W = 0.0
    for v in b:
        W += float(v)
    thr = np.zeros(b.size, dtype=np.uint64)
    S = 0.0
    for c, v in enumerate(b):
        S += float(v)
        thr[c] = int(math.floor(S / W * 4294967296.0))
    thr[-1] = 1 << 32
    return thr


def envelope(spec, theta, n12=96, n13=96, sub=6, factor=1.2):
    """A per-cell bound on |S|^2: factor x the largest FP64 intensity on a sub x sub lattice
    (edges included) of the cell and its eight neighbours.  Returns (n12, n13, float32 bounds)."""
    model = od.DalitzModel(spec)
    lo12, hi12, lo13, hi13 = _box(model.kin)
    cw12, cw13 = (hi12 - lo12) / n12, (hi13 - lo13) / n13
    f = np.arange(sub) / (sub - 1)
    a = (lo12 + cw12 * (np.arange(n12)[:, None] + f[None, :])).reshape(-1)
    b = (lo13 + cw13 * (np.arange(n13)[:, None] + f[None, :])).reshape(-1)
    A, B = np.meshgrid(a, b, indexing="ij")
    A, B = torch.from_numpy(A.reshape(-1)), torch.from_numpy(B.reshape(-1))
    ok = od.inside(A, B, model.kin)
    th = torch.as_tensor(np.asarray(theta, dtype=np.float64))
    I = torch.zeros(A.numel(), dtype=torch.float64)
    with torch.no_grad():
        I[ok] = model.intensity(model.amplitude_matrix({"s12": A[ok], "s13": B[ok]}, th), th)
    cmax = I.numpy().reshape(n12, sub, n13, sub).max(axis=(1, 3))
    pad = np.pad(cmax, 1)
    nb = np.max([pad[1 + di:1 + di + n12, 1 + dj:1 + dj + n13] for di in (-1, 0, 1) for dj in (-1, 0, 1)], axis=0)
    return n12, n13, (factor * nb).astype(np.float32)


def generate_toy(spec, theta, env, seed, n, chunk=8192, max_candidates=50_000_000):
    """The first n accepted candidates of the toy with this seed: (s12, s13, candidate index).

    env = (n12, n13, per-cell float32 bounds in row-major (s12, s13) cell order)."""
    model = od.DalitzModel(spec)
    kin = model.kin
    M, m1, m2, m3 = kin["M"], kin["m1"], kin["m2"], kin["m3"]
    lo12, hi12, lo13, hi13 = _box(kin)
    n12, n13, bound = env
    bound = np.asarray(bound, dtype=np.float32).reshape(-1)
    thr = thresholds(bound)
    f = np.float32
    lo12f, lo13f = f(lo12), f(lo13)
    cw12f, cw13f = f((hi12 - lo12) / n12), f((hi13 - lo13) / n13)
    th32 = torch.as_tensor(np.asarray(theta, dtype=np.float64)).to(torch.float32)
    out12, out13, idx = [], [], []
    j = 0
    while len(out12) < n and j < max_candidates:
        w = np.array([ph.philox4x64((jj, 0, 0, 0), (seed, ph.TOY_KEY1)) for jj in range(j, j + chunk)],
                     dtype=np.uint64)
        cell = np.searchsorted(thr, w[:, 0] >> np.uint64(32), side="right")
        ci, cj = (cell // n13).astype(np.float32), (cell % n13).astype(np.float32)
        u = [((w[:, k] >> np.uint64(40)).astype(np.float32) * f(2.0 ** -24)).astype(np.float32) for k in (1, 2, 3)]
        s12 = (lo12f + ((ci + u[0]).astype(np.float32) * cw12f).astype(np.float32)).astype(np.float32)
        s13 = (lo13f + ((cj + u[1]).astype(np.float32) * cw13f).astype(np.float32)).astype(np.float32)
        ub = (u[2] * bound[cell]).astype(np.float32)
        t12 = torch.from_numpy(s12)
        t13 = torch.from_numpy(s13)
        ok12 = (t12 > f(lo12)) & (t12 < f(hi12))
        t12c = torch.clamp(t12, f(lo12) * f(1.0000001), f(hi12) * f(0.9999999))
        _, _, cos = od.helicity_frame(t12c, t13, f(M), f(m1), f(m2), f(m3))
        inside = (ok12 & (cos.abs() <= 1.0)).numpy()
        with torch.no_grad():
            A = model.amplitude_matrix({"s12": s12, "s13": s13}, th32, dtype=torch.float32)
            S2 = model.intensity(A, th32).numpy().astype(np.float32)
        acc = inside & (ub < S2)
        for k in np.flatnonzero(acc):
            if len(out12) < n:
                out12.append(s12[k])
                out13.append(s13[k])
                idx.append(j + k)
        j += chunk
    return np.array(out12, dtype=np.float32), np.array(out13, dtype=np.float32), np.array(idx)
