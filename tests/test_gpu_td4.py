"""GPU parity of the time-dependent four-body path (amplitude cache, Gram matrix, NLL +
gradient with mixing and resolution, per-event log f, shards, fits) against the oracle."""
import numpy as np
import pytest

import synth
from oracle import td4 as ot

pytestmark = pytest.mark.gpu

TOL_NLL = {"f64": 1e-9, "f32": 1e-6}
TOL_GRAD = {"f64": 1e-6, "f32": 1e-4}
OBS = ot.OBS


@pytest.fixture(scope="module")
def goo():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1710_08826_gb300 import goo as g
    return g


@pytest.fixture(scope="module")
def ctx(goo):
    return goo.Context(0)


def _mc_cols(n, seed=1710014):
    mc = synth.four_body_phase_space(n, seed, **synth.TD4_MASSES)
    mc["t"] = np.zeros(n)   # the normalisation ignores the MC's time column
    return mc


@pytest.fixture(scope="module")
def sample():
    spec = synth.c4_spec()
    theta = np.array(synth.param_values(spec))
    data = ot.generate(spec, theta, 20_000, 91)
    mc = _mc_cols(40_000)
    return spec, theta, data, mc


def _prep(spec, data, mc, precision):
    if precision == "f32":
        return synth.round_to_f32(data, spec), synth.round_to_f32(mc, spec)
    return data, mc


def _build(goo, ctx, spec, data, mc):
    ds = goo.Dataset.from_spec(ctx, spec, data)
    mcds = goo.Dataset.from_spec(ctx, spec, mc)
    return ds, mcds, goo.Model(ctx, spec, mc=mcds)


def _ref(spec, data, mc, theta):
    m = ot.TD4Model(spec)
    return m.nll_grad(data, m.amplitudes(mc), theta)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("shift", ["truth", "off", "mixing"])
def test_nll_grad_matches_oracle(goo, ctx, sample, precision, shift):
    spec, theta, data, mc = sample
    m = ot.TD4Model(spec)
    th = theta.copy()
    if shift == "off":
        th = th * 1.03
    elif shift == "mixing":   # large mixing: every time term carries weight
        th[m.tp[0]], th[m.tp[1]], th[m.tp[3]] = 0.3, 0.2, 0.08
    d, c = _prep(spec, data, mc, precision)
    ds, mcds, model = _build(goo, ctx, spec, d, c)
    nll, g = model.nll_grad(ds, th, precision)
    rnll, rg = _ref(spec, d, c, th)
    assert abs(nll - rnll) <= TOL_NLL[precision] * abs(rnll), (nll, rnll)
    scale = np.max(np.abs(rg))
    assert np.max(np.abs(g - rg)) <= TOL_GRAD[precision] * scale, (g, rg)
    assert model.nll(ds, th, precision) == pytest.approx(nll, rel=1e-12)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_gram_and_norm(goo, ctx, sample, precision):
    spec, theta, data, mc = sample
    d, c = _prep(spec, data, mc, precision)
    _, mcds, model = _build(goo, ctx, spec, d, c)
    G = model.gram(theta, precision)
    m = ot.TD4Model(spec)
    Gr = m.gram(m.amplitudes(c))
    tol = 1e-12 if precision == "f64" else 2e-6
    assert G.shape == (10, 10)
    assert np.max(np.abs(G - Gr)) <= tol * np.max(np.abs(Gr))
    N = model.normalise(theta, precision)[0]
    assert N == pytest.approx(m.norm(Gr, theta), rel=1e-11 if precision == "f64" else 2e-6)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_per_event_logf(goo, ctx, sample, precision):
    import torch
    spec, theta, data, mc = sample
    d, c = _prep(spec, data, mc, precision)
    ds, _, model = _build(goo, ctx, spec, d, c)
    lf = model.eval_logf(ds, theta, precision)
    m = ot.TD4Model(spec)
    a = m.amplitudes(d)
    ref = np.log(m.rate(a, d["t"], theta)) - np.log(m.norm(m.gram(m.amplitudes(c)), theta))
    lf = lf.cpu().numpy() if isinstance(lf, torch.Tensor) else np.asarray(lf)
    tol = 1e-11 if precision == "f64" else 2e-5
    assert np.max(np.abs(lf - ref)) <= tol * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_ragged_sizes_and_shards(goo, ctx, sample, precision):
    spec, theta, data, mc = sample
    d, c = _prep(spec, data, mc, precision)
    th = theta * 1.01
    for n in (1, 255, 257, 1000, 4099):
        sub = {k: v[:n] for k, v in d.items()}
        ds, _, model = _build(goo, ctx, spec, sub, c)
        nll, g = model.nll_grad(ds, th, precision)
        rnll, rg = _ref(spec, sub, c, th)
        assert abs(nll - rnll) <= TOL_NLL[precision] * max(abs(rnll), 1.0) * 10, (n, nll, rnll)
    ds, _, model = _build(goo, ctx, spec, d, c)
    full, gfull = model.nll_grad(ds, th, precision)
    edges = [0, 1, 257, 5000, 11111, len(d["t"])]
    parts = [model.nll_partial(ds, a, b, th, precision) for a, b in zip(edges[:-1], edges[1:])]
    tot = goo.combine_partials(parts, model.n_params)
    assert tot[2] == len(d["t"])
    assert abs(tot[0] + tot[1] - full) <= (1e-12 if precision == "f64" else 1e-8) * abs(full)


def test_no_mixing_limit(goo, ctx, sample):
    # x = y = 0: R = |A|^2 x (exponential convolved with the resolution), independent of B
    spec, theta, data, mc = sample
    m = ot.TD4Model(spec)
    th = theta.copy()
    th[m.tp[0]] = th[m.tp[1]] = 0.0
    ds, _, model = _build(goo, ctx, spec, data, mc)
    nll, g = model.nll_grad(ds, th, "f64")
    rnll, rg = _ref(spec, data, mc, th)
    assert abs(nll - rnll) <= 1e-9 * abs(rnll)
    assert np.max(np.abs(g - rg)) <= 1e-6 * np.max(np.abs(rg))


def test_fit_matches_oracle_fit(goo, ctx, sample):
    # coefficients and the lifetime free; x, y, sigma_t and the first coefficient fixed: with
    # B fixed the overall scale of A is set only through O(x, y) interference terms, which
    # 20k events do not constrain
    from oracle import fit as of
    spec, theta, data, mc = sample
    m = ot.TD4Model(spec)
    free = [True] * len(theta)
    for i in (m.tp[0], m.tp[1], m.tp[3], m.re[0], m.im[0]):
        free[i] = False
    start = theta.copy()
    start[m.re + m.im] *= 1.05
    d, c = _prep(spec, data, mc, "f32")
    ds, _, model = _build(goo, ctx, spec, d, c)
    steps = np.array([p[3] if p[3] > 0 else 1.0 for p in spec["params"]])
    th_gpu, err_gpu, info = model.fit(ds, start, free, steps, precision="f32", gradient="adjoint")
    mca = m.amplitudes(c)
    a = m.amplitudes(d)
    th_ref, err_ref, _, redm = of.fit(lambda t: m.nll_grad(d, mca, t, a=a), start, free, steps)
    assert redm < 1e-6
    idx = [i for i in range(len(theta)) if free[i]]
    pulls = np.abs(th_gpu[idx] - th_ref[idx]) / err_ref[idx]
    assert np.max(pulls) < 0.01, pulls
    np.testing.assert_allclose(err_gpu[idx], err_ref[idx], rtol=0.02)


def test_full_size_configuration(goo, ctx):
    # 2,000,000 events and 3,000,000 MC points, the sizes and launch configuration the
    # benchmark times (phase-space events with Exp(tau) (x) N(0, sigma_t) decay times)
    spec = synth.c4_spec()
    theta = np.array(synth.param_values(spec))
    kin = dict(synth.TD4_MASSES)
    tau, sig = synth.TD4_TIME["tau"], synth.TD4_TIME["sigma_t"]
    data = synth.gen_c4_candidates(2_000_000, 1710004, kin, 1.0 / tau)
    data["t"] = np.clip(synth.smear_times(data.pop("t_true"), sig, 1710005), *spec["observables"][5][1:])
    mc = _mc_cols(3_000_000)
    m = ot.TD4Model(spec)
    th = theta * 1.01
    for precision in ("f64", "f32"):
        d, c = _prep(spec, data, mc, precision)
        ds, _, model = _build(goo, ctx, spec, d, c)
        nll, g = model.nll_grad(ds, th, precision)
        a = m.amplitudes(d)
        rnll, rg = m.nll_grad(d, m.amplitudes(c), th, a=a)
        assert abs(nll - rnll) <= TOL_NLL[precision] * abs(rnll), (precision, nll, rnll)
        err = np.abs(g - rg)
        assert np.max(err) <= TOL_GRAD[precision] * np.max(np.abs(rg)), (precision, np.max(err) / np.max(np.abs(rg)))
        # every component against its own value as well (measured FP32 worst: 4e-6; the decay-time
        # terms are summed as moment series, so no cancelling difference of convolved
        # exponentials limits them)
        assert np.all(err <= TOL_GRAD[precision] * np.abs(rg)), (precision, err / np.abs(rg))
