"""Pins of the composite-model semantics, normalisation, NLL and gradient (oracle/model.py)."""
import math

import numpy as np
import pytest
import scipy.integrate
import scipy.stats
import torch

import synth
from oracle import model as om
from oracle import pdfs

T = lambda v: torch.tensor(v, dtype=torch.float64)  # noqa: E731


def test_c1_density_is_scipy_truncated_mixture():
    spec = synth.c1_spec()
    m = om.TreeModel(spec)
    x = np.linspace(0.0, 10.0, 57)
    th = [5.1, 0.45, -0.27, 0.33]
    got = m.density({"x": x}, th).numpy()
    a, b = (0 - 5.1) / 0.45, (10 - 5.1) / 0.45
    ref = 0.33 * scipy.stats.truncnorm.pdf(x, a, b, loc=5.1, scale=0.45) + \
        0.67 * scipy.stats.truncexpon.pdf(x, b=10 * 0.27, scale=1 / 0.27)
    np.testing.assert_allclose(got, ref, rtol=1e-12)


def test_c1_nll_is_scipy_logpdf_sum():
    spec = synth.c1_spec()
    m = om.TreeModel(spec)
    x = synth.gen_c1(n=2000, seed=7)["x"]
    th = synth.param_values(spec)
    a, b = (0 - 5.0) / 0.4, (10 - 5.0) / 0.4
    ref = -np.sum(np.log(0.3 * scipy.stats.truncnorm.pdf(x, a, b, loc=5.0, scale=0.4)
                         + 0.7 * scipy.stats.truncexpon.pdf(x, b=3.0, scale=1 / 0.3)))
    assert m.nll({"x": x}, th) == pytest.approx(ref, rel=1e-12)


def test_c1_density_integrates_to_one():
    m = om.TreeModel(synth.c1_spec())
    th = [4.0, 0.9, -0.8, 0.6]
    v, _ = scipy.integrate.quad(lambda x: float(m.density({"x": np.array([x])}, th)[0]), 0, 10,
                                epsrel=1e-12, points=[4.0])
    assert v == pytest.approx(1.0, rel=1e-10)


def _small_grid_spec(bins):
    spec = synth.c2_spec(bins=bins)
    return spec


def test_grid_equals_product_of_1d_grid_sums():
    # For a product of single-observable shapes the midpoint sum over the full grid
    # factorises into the product of the 1D midpoint sums.
    spec = _small_grid_spec(128)
    m = om.TreeModel(spec)
    th = torch.as_tensor(synth.param_values(spec), dtype=torch.float64)
    for comp in spec["pdf"][2]:
        full = float(m.grid_integral(comp, th, spec["norm"][1], {}))
        prod = 1.0
        for leaf in comp[1]:
            lo_hi = {o[0]: (o[1], o[2]) for o in spec["observables"]}[leaf[1]]
            n = 128
            h = (lo_hi[1] - lo_hi[0]) / n
            xs = lo_hi[0] + (np.arange(n) + 0.5) * h
            prod *= float(m.shape(leaf, {leaf[1]: T(xs)}, th, {}).sum()) * h
        assert full == pytest.approx(prod, rel=1e-12)


def test_grid_signal_norm_close_to_closed_form():
    spec = _small_grid_spec(128)
    m = om.TreeModel(spec)
    th = synth.param_values(spec)
    sig = spec["pdf"][2][0]
    grid = float(m.grid_integral(sig, torch.as_tensor(th), spec["norm"][1], {}))
    exact = float(pdfs.gauss_integral(5.2, 5.3, T(th[0]), T(th[1])) *
                  pdfs.gauss_integral(-0.2, 0.2, T(th[2]), T(th[3])) *
                  pdfs.expo_integral(0.0, 10.0, T(th[4])))
    # midpoint rule: relative error O(h^2) on the exponential factor, ~1e-4 here
    assert grid == pytest.approx(exact, rel=3e-4)


def test_grid_argus_converges_to_quadrature():
    # The grid error of the Argus component shrinks with the bin count (reported, not parity).
    spec = synth.c2_spec()
    m = om.TreeModel(spec)
    th = torch.as_tensor(synth.param_values(spec), dtype=torch.float64)
    leaf = ("argus", "m", "m0", "c", "p")
    ref, _ = scipy.integrate.quad(lambda v: float(pdfs.argus_shape(T(v), th[5], th[6], th[7])),
                                  5.2, 5.29, epsrel=1e-12, limit=200)
    errs = []
    for n in (128, 1024, 8192):
        h = 0.1 / n
        xs = 5.2 + (np.arange(n) + 0.5) * h
        errs.append(abs(float(m.shape(leaf, {"m": T(xs)}, th, {}).sum()) * h / ref - 1))
    assert errs[0] < 2e-3 and errs[1] < errs[0] and errs[2] < errs[1]


def test_analytic_3d_density_is_scipy_product():
    # An analytic-normalised 3D sum of products checked against scipy's truncated densities.
    spec = dict(
        name="t3",
        observables=[("m", 5.2, 5.3), ("dE", -0.2, 0.2), ("t", 0.0, 10.0)],
        params=[("mu", 5.28, False, 0), ("s", 0.004, False, 0), ("mu2", 0.01, False, 0),
                ("s2", 0.03, False, 0), ("l", -0.5, False, 0), ("mu3", 5.25, False, 0),
                ("s3", 0.03, False, 0), ("l2", -1.2, False, 0), ("f", 0.35, False, 0)],
        pdf=("add", ["f"], [
            ("prod", [("gauss", "m", "mu", "s"), ("gauss", "dE", "mu2", "s2"), ("expo", "t", "l")]),
            ("prod", [("gauss", "m", "mu3", "s3"), ("expo", "t", "l2")]),
        ]),
        norm=("analytic",),
    )
    m = om.TreeModel(spec)
    rng = np.random.default_rng(3)
    cols = {"m": rng.uniform(5.2, 5.3, 50), "dE": rng.uniform(-0.2, 0.2, 50), "t": rng.uniform(0, 10, 50)}
    th = [p[1] for p in spec["params"]]
    tn = lambda x, lo, hi, mu, s: scipy.stats.truncnorm.pdf(x, (lo - mu) / s, (hi - mu) / s, loc=mu, scale=s)  # noqa: E731
    te = lambda x, l: scipy.stats.truncexpon.pdf(x, b=10 * -l, scale=1 / -l)  # noqa: E731
    ref = 0.35 * tn(cols["m"], 5.2, 5.3, 5.28, 0.004) * tn(cols["dE"], -0.2, 0.2, 0.01, 0.03) * te(cols["t"], -0.5) + \
        0.65 * tn(cols["m"], 5.2, 5.3, 5.25, 0.03) * te(cols["t"], -1.2)
    # the second component does not depend on dE: the model is a density in (m, t) there
    np.testing.assert_allclose(m.density(cols, th).numpy(), ref, rtol=1e-12)


def test_nested_tree_normalised():
    # PROD(ADD(gauss(x), expo(x)), gauss(y)) integrates to one over the box.
    spec = dict(
        name="nested", observables=[("x", 0.0, 4.0), ("y", -1.0, 1.0)],
        params=[("a", 1.5, False, 0), ("b", 0.6, False, 0), ("l", -0.4, False, 0), ("f", 0.4, False, 0),
                ("c", 0.2, False, 0), ("d", 0.5, False, 0)],
        pdf=("prod", [("add", ["f"], [("gauss", "x", "a", "b"), ("expo", "x", "l")]),
                      ("gauss", "y", "c", "d")]),
        norm=("analytic",))
    m = om.TreeModel(spec)
    th = [p[1] for p in spec["params"]]
    f = lambda y, x: float(m.density({"x": np.array([x]), "y": np.array([y])}, th)[0])  # noqa: E731
    v, _ = scipy.integrate.dblquad(f, 0.0, 4.0, -1.0, 1.0, epsrel=1e-10)
    assert v == pytest.approx(1.0, rel=1e-8)


def fd4(fn, theta, steps):
    """Fourth-order central differences (the Argus endpoint makes 2nd-order FD too coarse)."""
    out = []
    for i, h in enumerate(steps):
        def at(k):
            t = list(theta)
            t[i] += k * h
            return fn(t)
        out.append((-at(2) + 8 * at(1) - 8 * at(-1) + at(-2)) / (12 * h))
    return out


@pytest.mark.parametrize("which", ["c1", "c2"])
def test_autograd_gradient_vs_finite_differences(which):
    if which == "c1":
        spec = synth.c1_spec()
        cols = synth.gen_c1(n=3000, seed=11)
        th = [5.05, 0.42, -0.31, 0.29]
    else:
        spec = synth.c2_spec(bins=32)
        cols = synth.gen_c2(n=3000, seed=12)
        th = [5.2792, 0.0031, 0.001, 0.021, -0.66, 5.2903, -19.0, 0.52, -0.9, 0.4, -1.2, 0.21]
    m = om.TreeModel(spec)
    nll, g = m.nll_grad(cols, th)
    steps = [1e-6 * max(abs(t), 1e-3) for t in th]
    fd = fd4(lambda t: m.nll(cols, t), th, steps)
    scale = np.abs(g).max()
    np.testing.assert_allclose(g, fd, rtol=1e-5, atol=1e-6 * scale)
    assert nll == pytest.approx(m.nll(cols, th), rel=1e-14)


def test_fraction_gradient_sign():
    # Moving the fraction towards the value that generated the data lowers the NLL.
    spec = synth.c1_spec()
    cols = synth.gen_c1(n=20000, seed=5)
    m = om.TreeModel(spec)
    _, g_lo = m.nll_grad(cols, [5.0, 0.4, -0.3, 0.2])
    _, g_hi = m.nll_grad(cols, [5.0, 0.4, -0.3, 0.4])
    assert g_lo[3] < 0 < g_hi[3]


def test_sampler_matches_density_chi2():
    # The C2 generator's background m (gamma transform) and dE (accept--reject) marginals
    # follow the oracle's Argus and polynomial shapes.
    cols = synth.gen_c2(n=400_000, seed=99)
    spec = synth.c2_spec()
    m = om.TreeModel(spec)
    th = torch.as_tensor(synth.param_values(spec), dtype=torch.float64)
    # background-dominated region: m < 5.26 (signal is 6 sigma away)
    sel = cols["m"] < 5.26
    mm = cols["m"][sel]
    edges = np.linspace(5.2, 5.26, 31)
    counts, _ = np.histogram(mm, edges)
    fine = np.linspace(5.2, 5.26, 30 * 200 + 1)
    dens = pdfs.argus_shape(T(fine), th[5], th[6], th[7]).numpy()
    cell = np.array([np.trapezoid(dens[i * 200:(i + 1) * 200 + 1], fine[i * 200:(i + 1) * 200 + 1]) for i in range(30)])
    expect = cell / cell.sum() * counts.sum()
    chi2 = float(((counts - expect) ** 2 / expect).sum())
    assert chi2 < 30 + 5 * math.sqrt(60)


def test_weighted_nll_equals_repeated_events():
    # a dataset with integer weights is the dataset with each event repeated w times
    spec = synth.c2_spec(bins=16)
    m = om.TreeModel(spec)
    cols = synth.gen_c2(n=500, seed=31)
    w = np.random.default_rng(5).integers(0, 4, 500).astype(np.float64)
    rep = {k: np.repeat(v, w.astype(int)) for k, v in cols.items()}
    th = np.array(synth.param_values(spec)) * 1.01
    n1, g1 = m.nll_grad(cols, th, weights=w)
    n2, g2 = m.nll_grad(rep, th)
    assert n1 == pytest.approx(n2, rel=1e-12)
    np.testing.assert_allclose(g1, g2, rtol=1e-10, atol=1e-9)


def test_binned_nll_is_the_multinomial_likelihood_of_the_bin_contents():
    # bin centres weighted by their counts: sum_b n_b log(f(x_b) h) is the log of the
    # multinomial probability of the contents with p_b = f(x_b) h, up to a theta-free term
    spec = synth.c1_spec()
    m = om.TreeModel(spec)
    x = synth.gen_c1(n=5000, seed=9)["x"]
    counts, edges = np.histogram(x, bins=50, range=(0.0, 10.0))
    centres = 0.5 * (edges[:-1] + edges[1:])
    h = edges[1] - edges[0]
    th = np.array(synth.param_values(spec))
    nll = m.nll({"x": centres}, th, weights=counts.astype(float))
    p = m.density({"x": centres}, th).numpy() * h
    logmult = scipy.stats.multinomial.logpmf(counts, n=counts.sum(), p=p / p.sum())
    const = math.lgamma(counts.sum() + 1) - np.sum([math.lgamma(c + 1) for c in counts])
    # logpmf normalises p to sum 1; the midpoint probabilities sum to 1 within O(h^2)
    assert -nll + counts.sum() * math.log(h) - counts.sum() * math.log(p.sum()) + const == pytest.approx(
        logmult, rel=1e-12)
