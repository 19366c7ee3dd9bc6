"""Reference minimiser for fit-level parity (float64, CPU).

The paper's FitManager drives Minuit 2 on the NLL (Fig. 1; Sec. 4).  Minuit's exact
rules are not needed for parity: what is compared is the location of the minimum and
the parameter errors.  This oracle finds the minimum with scipy's BFGS on the free
parameters (using the oracle's autograd gradient), polishes it with Newton steps on a
finite-difference Hessian of that gradient, and takes the errors from the inverse of
that Hessian (the usual large-sample covariance of a maximum-likelihood estimate).
"""
import numpy as np
import scipy.optimize


def hessian_fd(grad_fn, theta, free, steps):
    """Symmetrised central-difference Hessian of grad_fn over the free parameters."""
    theta = np.asarray(theta, dtype=np.float64)
    idx = np.flatnonzero(free)
    H = np.zeros((idx.size, idx.size))
    for a, i in enumerate(idx):
        tp = theta.copy()
        tm = theta.copy()
        tp[i] += steps[i]
        tm[i] -= steps[i]
        H[a] = (np.asarray(grad_fn(tp))[idx] - np.asarray(grad_fn(tm))[idx]) / (2 * steps[i])
    return 0.5 * (H + H.T)


def fit(nll_grad_fn, theta0, free, scale, max_newton=4):
    """Minimise nll_grad_fn(theta) -> (nll, grad) over the free parameters.

    Returns (theta_hat, errors, nll_min, edm) with errors from the inverse Hessian.
    ``scale`` gives a typical step per parameter (used for conditioning and FD steps).
    """
    theta0 = np.asarray(theta0, dtype=np.float64)
    free = np.asarray(free, dtype=bool)
    scale = np.asarray(scale, dtype=np.float64)
    idx = np.flatnonzero(free)

    def unpack(x):
        th = theta0.copy()
        th[idx] = theta0[idx] + x * scale[idx]
        return th

    def fun(x):
        f, g = nll_grad_fn(unpack(x))
        return f, np.asarray(g)[idx] * scale[idx]

    res = scipy.optimize.minimize(fun, np.zeros(idx.size), jac=True, method="BFGS",
                                  options={"gtol": 1e-7, "maxiter": 2000})
    theta = unpack(res.x)
    grad_only = lambda th: nll_grad_fn(th)[1]  # noqa: E731
    for _ in range(max_newton):
        steps = np.where(free, 1e-3 * scale, 0.0)
        H = hessian_fd(grad_only, theta, free, steps)
        g = np.asarray(grad_only(theta))[idx]
        dx = np.linalg.solve(H, g)
        edm = 0.5 * float(g @ dx)
        if edm < 1e-10:
            break
        theta[idx] -= dx
    steps = np.where(free, 1e-3 * scale, 0.0)
    H = hessian_fd(grad_only, theta, free, steps)
    cov = np.linalg.inv(H)
    g = np.asarray(grad_only(theta))[idx]
    edm = 0.5 * float(g @ cov @ g)
    err = np.zeros_like(theta)
    err[idx] = np.sqrt(np.diag(cov))
    return theta, err, float(nll_grad_fn(theta)[0]), edm
