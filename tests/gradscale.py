"""Per-component scale of gradient errors for the full-size parity tests.

A gradient error dg_i moves the minimum of the likelihood in parameter i by about
dg_i sigma_i^2, i.e. by dg_i sigma_i standard deviations, with sigma_i^2 the inverse of the
curvature d^2 NLL / d theta_i^2.  The full-size tests bound dg_i sigma_i for every component,
next to the stated 1e-4 of the largest component, so that a small component cannot be wrong
by a large fraction of itself unnoticed.
"""
import numpy as np


def sigmas(model, ds, theta, idx, precision="f64", rel=1e-4):
    """1 / sqrt(d^2 NLL / d theta_i^2) for i in idx, by central differences of the adjoint
    gradient of the given path (the FP64 path is itself pinned to the oracle)."""
    theta = np.asarray(theta, dtype=np.float64)
    out = np.full(len(theta), np.nan)
    for i in idx:
        h = rel * max(abs(theta[i]), 1e-2)
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        H = (model.nll_grad(ds, tp, precision)[1][i] - model.nll_grad(ds, tm, precision)[1][i]) / (2 * h)
        out[i] = 1.0 / np.sqrt(abs(H))
    return out
