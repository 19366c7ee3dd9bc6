"""GPU parity of the polar (magnitude, phase) coefficient form of the three-body models
(cached, floating lineshapes, time-dependent) against the oracle, and a polar fit."""
import numpy as np
import pytest
import torch

import synth
from oracle import dalitz as od
from oracle import fit as ofit
from oracle import td3 as ot3

pytestmark = pytest.mark.gpu

KIN = dict(synth.DALITZ_MASSES)
TOL_NLL = {"f64": 1e-9, "f32": 1e-6}
TOL_GRAD = {"f64": 1e-6, "f32": 1e-4}


@pytest.fixture(scope="module")
def goo():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1710_08826_gb300 import goo as g
    return g


@pytest.fixture(scope="module")
def ctx(goo):
    return goo.Context(0)


def _cands(n, seed, kin=KIN):
    return synth.dalitz_candidates(n, seed, kin["M"], kin["m1"], kin["m2"], kin["m3"])


@pytest.fixture(scope="module")
def c3():
    spec = synth.c3_spec(n_mc=40_000)
    ref = od.DalitzModel(spec)
    theta = np.array(synth.param_values(spec))
    fmax = 1.2 * od.max_intensity_scan(ref, theta, n=300)

    def dens(cols):
        with torch.no_grad():
            th = torch.as_tensor(theta, dtype=torch.float64)
            return ref.intensity(ref.amplitude_matrix(cols, th), th).numpy()
    data, _ = synth.accept_reject(lambda k, s: _cands(k, s), dens, fmax, 20_000, 83, chunk=200_000)
    ps = synth.to_polar(spec)
    tp = np.array(synth.param_values(ps))
    names = synth.param_names(ps)
    for i, n in enumerate(names):   # move the phases and magnitudes off the generating point
        if n.startswith("phase_") and not n.endswith("NR"):
            tp[i] += 0.1
        elif n.startswith("mag_") and not n.endswith("NR"):
            tp[i] *= 1.04
    return ps, tp, data, _cands(40_000, 1710013)


def _prep(spec, data, mc, precision):
    if precision == "f32":
        return synth.round_to_f32(data, spec), synth.round_to_f32(mc, spec)
    return data, mc


def _build(goo, ctx, spec, data, mc):
    ds = goo.Dataset.from_spec(ctx, spec, data)
    mcds = goo.Dataset.from_spec(ctx, spec, mc)
    return ds, mcds, goo.Model(ctx, spec, mc=mcds)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("mode", ["cached", "floating"])
def test_polar_three_body(goo, ctx, c3, precision, mode):
    spec, tp, data, mc = c3
    d, c = _prep(spec, data, mc, precision)
    ds, mcds, model = _build(goo, ctx, spec, d, c)
    model.set_lineshapes(mode)
    nll, g = model.nll_grad(ds, tp, precision)
    rnll, rg = od.DalitzModel(spec).nll_grad(d, c, tp)
    assert abs(nll - rnll) <= TOL_NLL[precision] * abs(rnll), (nll, rnll)
    names = synth.param_names(spec)
    use = np.array([n.startswith(("mag_", "phase_")) or mode == "floating" for n in names])
    scale = np.max(np.abs(rg[use]))
    assert np.max(np.abs(g[use] - rg[use])) <= TOL_GRAD[precision] * scale, (g - rg) / scale


def test_polar_normalisation_equals_cartesian(goo, ctx, c3):
    spec, tp, data, mc = c3
    cart = synth.c3_spec(n_mc=40_000)
    names_p, names_c = synth.param_names(spec), synth.param_names(cart)
    th = np.array(synth.param_values(cart))
    for i, n in enumerate(names_p):
        if n.startswith("mag_"):
            r, ph = tp[i], tp[names_p.index("phase_" + n[4:])]
            th[names_c.index("re_" + n[4:])] = r * np.cos(ph)
            th[names_c.index("im_" + n[4:])] = r * np.sin(ph)
    _, mcds, mp = _build(goo, ctx, spec, data, mc)
    _, _, mcart = _build(goo, ctx, cart, data, mc)
    assert mp.normalise(tp, "f64")[0] == pytest.approx(mcart.normalise(th, "f64")[0], rel=1e-13)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_polar_time_dependent_three_body(goo, ctx, precision):
    spec = synth.to_polar(synth.td3_spec())
    k3 = synth.TD3_MASSES
    cart = synth.td3_spec()
    data = ot3.generate(cart, np.array(synth.param_values(cart)), 10_000, 62, lambda n, s: _cands(n, s, k3))
    mc = _cands(30_000, 1710015, k3)
    mc["t"] = np.zeros(30_000)
    tp = np.array(synth.param_values(spec))
    names = synth.param_names(spec)
    for i, n in enumerate(names):
        if n.startswith("phase_") and n != "phase_rho770_p":
            tp[i] += 0.1
    d, c = _prep(spec, data, mc, precision)
    ds, _, model = _build(goo, ctx, spec, d, c)
    nll, g = model.nll_grad(ds, tp, precision)
    rnll, rg = ot3.TD3Model(spec).nll_grad(d, c, tp)
    assert abs(nll - rnll) <= TOL_NLL[precision] * abs(rnll), (nll, rnll)
    scale = np.max(np.abs(rg))
    assert np.max(np.abs(g - rg)) <= TOL_GRAD[precision] * scale, (g - rg) / scale


def test_polar_fit_matches_oracle_fit(goo, ctx, c3):
    spec, tp, data, mc = c3
    free = np.array([not p[2] for p in spec["params"]])
    steps = np.array([p[3] if p[3] > 0 else 1.0 for p in spec["params"]])
    d, c = _prep(spec, data, mc, "f32")
    ds, _, model = _build(goo, ctx, spec, d, c)
    th_gpu, err_gpu, info = model.fit(ds, tp, free, steps, precision="f32", gradient="adjoint")
    ref = od.DalitzModel(spec)
    th_ref, err_ref, _, redm = ofit.fit(lambda t: ref.nll_grad(d, c, t), tp, free, steps)
    assert redm < 1e-6
    idx = np.flatnonzero(free)
    pulls = np.abs(th_gpu[idx] - th_ref[idx]) / err_ref[idx]
    assert np.max(pulls) < 0.01, pulls
    np.testing.assert_allclose(err_gpu[idx], err_ref[idx], rtol=0.03)
