"""GPU parity of the three-body amplitude path (cache, Gram, coherent NLL + gradient)."""
import numpy as np
import pytest
import torch

import synth
from oracle import dalitz as od

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


def _cands(n, seed):
    return synth.dalitz_candidates(n, seed, KIN["M"], KIN["m1"], KIN["m2"], KIN["m3"])


def _model_data(n_data, n_mc, seed=77, precision="f64"):
    spec = synth.c3_spec(n_mc=n_mc)
    ref = od.DalitzModel(spec)
    theta = synth.param_values(spec)
    fmax = 1.2 * od.max_intensity_scan(ref, theta, n=300)

    def dens(cols):
        with torch.no_grad():
            th = torch.as_tensor(theta, dtype=torch.float64)
            return ref.intensity(ref.amplitude_matrix(cols, th), th).numpy()
    data, worst = synth.accept_reject(lambda k, s: _cands(k, s), dens, fmax, n_data, seed, chunk=200_000)
    assert worst < 1.0
    mc = _cands(n_mc, 1710013)
    if precision == "f32":
        data = synth.round_to_f32(data, spec)
        mc = synth.round_to_f32(mc, spec)
    return spec, ref, theta, data, mc


def _upload(goo, ctx, spec, data, mc):
    ds = goo.Dataset.from_spec(ctx, spec, data)
    mcds = goo.Dataset.from_spec(ctx, spec, mc)
    return ds, mcds, goo.Model(ctx, spec, mc=mcds)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_amplitude_cache_matches_oracle(goo, ctx, precision):
    spec = synth.c3_spec(n_mc=1000)
    data = _cands(20_001, 5)
    if precision == "f32":
        data = synth.round_to_f32(data, spec)
    ds, mcds, model = _upload(goo, ctx, spec, data, data)
    theta = synth.param_values(spec)
    got = model.amplitudes(ds, theta, precision)
    ref = od.DalitzModel(spec).amplitude_matrix(data, theta).numpy()[:, :8]
    scale = np.abs(ref).max(axis=0)
    err = np.abs(got - ref) / scale
    assert err.max() < (1e-12 if precision == "f64" else 3e-5), err.max(axis=0)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_gram_matches_oracle(goo, ctx, precision):
    spec = synth.c3_spec(n_mc=50_000)
    mc = _cands(50_000, 1710013)
    if precision == "f32":
        mc = synth.round_to_f32(mc, spec)
    ds, mcds, model = _upload(goo, ctx, spec, mc, mc)
    theta = synth.param_values(spec)
    G = model.gram(theta, precision)
    R = od.DalitzModel(spec).gram(mc, theta).numpy()
    tol = 1e-12 if precision == "f64" else 2e-6
    assert np.abs(G - R).max() <= tol * np.abs(R).max()
    assert np.allclose(G, G.conj().T, rtol=0, atol=1e-12 * np.abs(R).max())


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("offset", [1.0, 1.1])
def test_coherent_nll_grad(goo, ctx, precision, offset):
    spec, ref, theta, data, mc = _model_data(40_000, 60_000, precision=precision)
    ds, mcds, model = _upload(goo, ctx, spec, data, mc)
    th = np.array(theta)
    names = synth.param_names(spec)
    coef = np.array([n.startswith(("re_", "im_")) and not n.endswith("NR") for n in names])
    th[coef] *= offset
    nll, g = model.nll_grad(ds, th, precision)
    rnll, rg = ref.nll_grad(data, mc, th)
    assert abs(nll - rnll) <= TOL_NLL[precision] * abs(rnll)
    idx = np.flatnonzero(coef)
    scale = np.abs(rg[idx]).max()
    assert np.abs(g[idx] - rg[idx]).max() <= TOL_GRAD[precision] * max(scale, 1.0), (g[idx], rg[idx])
    # lineshape parameters are constants of the cached path: gradient entries are zero
    fixed_ls = np.array([n.startswith(("m0_", "w_")) for n in names])
    assert np.all(g[fixed_ls] == 0)


def test_flat_phase_space_and_homogeneity(goo, ctx):
    spec, ref, theta, data, mc = _model_data(5_000, 20_000, seed=78)
    ds, mcds, model = _upload(goo, ctx, spec, data, mc)
    names = synth.param_names(spec)
    th = np.array(theta)
    flat = th.copy()
    for i, n in enumerate(names):
        if n.startswith(("re_", "im_")) and not n.endswith("NR"):
            flat[i] = 0.0
    assert abs(model.nll(ds, flat, "f64")) < 1e-9
    allc = np.array([n.startswith(("re_", "im_")) for n in names])
    f0, g = model.nll_grad(ds, th, "f64")
    th2 = th.copy()
    th2[allc] *= 1.7
    assert model.nll(ds, th2, "f64") == pytest.approx(f0, rel=1e-12)
    euler = float(np.sum(th[allc] * g[allc]))
    assert abs(euler) < 1e-8 * float(np.sum(np.abs(th[allc] * g[allc])))


def test_lineshape_change_rebuilds_cache(goo, ctx):
    spec, ref, theta, data, mc = _model_data(8_000, 20_000, seed=79)
    ds, mcds, model = _upload(goo, ctx, spec, data, mc)
    names = synth.param_names(spec)
    th = np.array(theta)
    a = model.nll(ds, th, "f64")
    th2 = th.copy()
    th2[names.index("m0_Kst892_12")] = 0.90
    th2[names.index("w_rho770_23")] = 0.155
    b = model.nll(ds, th2, "f64")
    assert abs(b - ref.nll(data, mc, th2)) <= 1e-9 * abs(b)
    assert abs(a - b) > 1.0
    assert model.nll(ds, th, "f64") == a


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_shards_and_empty(goo, ctx, precision):
    spec, ref, theta, data, mc = _model_data(20_000, 20_000, seed=80, precision=precision)
    ds, mcds, model = _upload(goo, ctx, spec, data, mc)
    full, g = model.nll_grad(ds, theta, precision)
    edges = [0, 7, 9_999, 20_000]
    parts = [model.nll_partial(ds, a, b, theta, precision) for a, b in zip(edges[:-1], edges[1:])]
    tot = goo.combine_partials(parts, model.n_params)
    assert abs(tot[0] + tot[1] - full) <= (1e-12 if precision == "f64" else 1e-9) * abs(full)
    np.testing.assert_allclose(tot[3:], g, rtol=1e-9 if precision == "f64" else 1e-5, atol=1e-6)
    empty = goo.Dataset.from_spec(ctx, spec, {"s12": np.zeros(0), "s13": np.zeros(0)})
    assert model.nll(empty, theta, precision) == 0.0


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_c3_full_size(goo, ctx, precision):
    # 5M events, 1M MC points: the sizes of the three-body workload (uniform phase-space data)
    spec = synth.c3_spec()
    data = _cands(5_000_000, 1710003)
    mc = _cands(1_000_000, 1710013)
    if precision == "f32":
        data = synth.round_to_f32(data, spec)
        mc = synth.round_to_f32(mc, spec)
    ds, mcds, model = _upload(goo, ctx, spec, data, mc)
    theta = synth.param_values(spec)
    nll = model.nll(ds, theta, precision)
    rnll = od.DalitzModel(spec).nll(data, mc, theta)
    assert abs(nll - rnll) <= TOL_NLL[precision] * abs(rnll)
