"""Basic one-dimensional shapes and their integrals over a finite range (float64).

Each basic PDF of the paper's model language (Fig. 1; Sec. 1: basic shapes that
combination PDFs put together) is represented by an unnormalised shape u(x) and, where one
exists, the closed-form integral of u over the observable's range [lo, hi].  The paper
names no formulas; these are the standard definitions:

  Gaussian     u = exp(-(x - mu)^2 / (2 sigma^2))
               I = sigma sqrt(pi/2) [erf((hi - mu)/(sqrt2 sigma)) - erf((lo - mu)/(sqrt2 sigma))]
  Exponential  u = exp(lam x)
               I = (exp(lam hi) - exp(lam lo)) / lam        (lam = 0: hi - lo),
               evaluated as exp(lam lo) expm1(lam (hi - lo)) / lam
  Polynomial   u = 1 + a1 x + a2 x^2   (constant term fixed to 1: it is degenerate with
               the normalisation)
               I = (hi - lo) + a1 (hi^2 - lo^2)/2 + a2 (hi^3 - lo^3)/3
  Argus        u = m (1 - m^2/m0^2)^p exp(c (1 - m^2/m0^2))  for m < m0, else 0
               no closed form on a sub-range: normalised on a grid.

Parity: pinned in tests/test_oracle_pdfs.py against scipy quadrature and, for the Argus
shape, against the incomplete-gamma closed form of its integral over [0, m0].
"""
import math

import torch


def gauss_shape(x, mu, sigma):
    z = (x - mu) / sigma
    return torch.exp(-0.5 * z * z)


def gauss_integral(lo, hi, mu, sigma):
    r2 = math.sqrt(2.0)
    return sigma * math.sqrt(math.pi / 2.0) * (
        torch.special.erf((hi - mu) / (r2 * sigma)) - torch.special.erf((lo - mu) / (r2 * sigma)))


def expo_shape(x, lam):
    return torch.exp(lam * x)


def expo_integral(lo, hi, lam):
    if float(torch.as_tensor(lam).detach()) == 0.0:
        return torch.as_tensor(hi - lo, dtype=torch.float64) + 0.0 * lam
    # (exp(lam hi) - exp(lam lo)) / lam, written with expm1 so that it stays accurate
    # as lam -> 0.
    return torch.exp(lam * lo) * torch.expm1(lam * (hi - lo)) / lam


def poly2_shape(x, a1, a2):
    return 1.0 + a1 * x + a2 * x * x


def poly2_integral(lo, hi, a1, a2):
    return (hi - lo) + a1 * (hi ** 2 - lo ** 2) / 2.0 + a2 * (hi ** 3 - lo ** 3) / 3.0


def argus_shape(m, m0, c, p):
    u = 1.0 - (m / m0) ** 2
    inside = u > 0
    u_safe = torch.where(inside, u, torch.ones_like(u))
    val = m * u_safe ** p * torch.exp(c * u_safe)
    return torch.where(inside, val, torch.zeros_like(val))
