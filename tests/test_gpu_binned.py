"""GPU parity of weighted and binned datasets for the sum/product likelihood path: weighted
NLL + gradient against the oracle, the repeated-events identity, a binned fit against the
oracle's binned fit, shards, and the argument checks."""
import numpy as np
import pytest

import synth
from oracle import fit as ofit
from oracle import model as om

pytestmark = pytest.mark.gpu

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


def _data(spec, cols, precision):
    return synth.round_to_f32(cols, spec) if precision == "f32" else cols


def _weights(n, seed):
    # multiples of 1/2 up to 3, a quarter of them 0: exact in float32, so both sides weigh
    # every event identically
    return np.random.default_rng(seed).integers(0, 7, n).astype(np.float64) * 0.5 * \
        (np.random.default_rng(seed + 1).uniform(size=n) > 0.25)


def _weighted(goo, ctx, spec, cols, w):
    ds = goo.Dataset.from_spec(ctx, spec, cols)
    ds.set_weights(w)
    return ds, goo.Model(ctx, spec)


def _hist_c1(n_bins, n_events=50_000, seed=9):
    spec = synth.c1_spec()
    x = synth.gen_c1(n=n_events, seed=seed)["x"]
    counts, edges = np.histogram(x, bins=n_bins, range=(0.0, 10.0))
    return spec, {"x": 0.5 * (edges[:-1] + edges[1:])}, counts.astype(np.float64)


def _hist_c2(bins, n_events=200_000, seed=21):
    spec = synth.c2_spec()
    cols = synth.gen_c2(n=n_events, seed=seed)
    names = [o[0] for o in spec["observables"]]
    rng = [(o[1], o[2]) for o in spec["observables"]]
    counts, edges = np.histogramdd(np.stack([cols[k] for k in names], axis=1), bins=bins, range=rng)
    centres = [0.5 * (e[:-1] + e[1:]) for e in edges]
    grid = np.meshgrid(*centres, indexing="ij")
    return spec, {k: g.ravel() for k, g in zip(names, grid)}, counts.ravel().astype(np.float64)


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("which", ["c1", "c2"])
def test_weighted_nll_grad_matches_oracle(goo, ctx, precision, which):
    if which == "c1":
        spec, cols = synth.c1_spec(), synth.gen_c1()
    else:
        spec, cols = synth.c2_spec(), synth.gen_c2(n=100_000, seed=22)
    cols = _data(spec, cols, precision)
    n = len(next(iter(cols.values())))
    w = _weights(n, 5)
    theta = np.array(synth.param_values(spec)) * 1.004
    ds, model = _weighted(goo, ctx, spec, cols, w)
    nll, g = model.nll_grad(ds, theta, precision)
    rnll, rg = om.TreeModel(spec).nll_grad(cols, theta, weights=w)
    assert abs(nll - rnll) <= TOL_NLL[precision] * abs(rnll), (nll, rnll)
    assert np.max(np.abs(g - rg)) <= TOL_GRAD[precision] * np.max(np.abs(rg)), (g, rg)
    assert model.nll(ds, theta, precision) == pytest.approx(nll, rel=1e-12)
    # removing the weights gives the unweighted likelihood back
    ds.set_weights(None)
    assert model.nll(ds, theta, precision) == pytest.approx(om.TreeModel(spec).nll(cols, theta),
                                                            rel=TOL_NLL[precision])


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_integer_weights_equal_repeated_events(goo, ctx, precision):
    spec = synth.c2_spec()
    cols = _data(spec, synth.gen_c2(n=30_000, seed=24), precision)
    w = np.random.default_rng(6).integers(0, 4, 30_000).astype(np.float64)
    rep = {k: np.repeat(v, w.astype(int)) for k, v in cols.items()}
    theta = np.array(synth.param_values(spec)) * 0.997
    ds, model = _weighted(goo, ctx, spec, cols, w)
    n1, g1 = model.nll_grad(ds, theta, precision)
    n2, g2 = model.nll_grad(goo.Dataset.from_spec(ctx, spec, rep), theta, precision)
    assert abs(n1 - n2) <= (1e-12 if precision == "f64" else 1e-6) * abs(n2)
    assert np.max(np.abs(g1 - g2)) <= (1e-9 if precision == "f64" else 1e-4) * np.max(np.abs(g2))


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_binned_three_dimensional_matches_oracle(goo, ctx, precision):
    # 40 x 40 x 40 bins (64,000 bin centres, many empty) of the 3-D model
    spec, cols, counts = _hist_c2([40, 40, 40])
    cols = _data(spec, cols, precision)
    theta = np.array(synth.param_values(spec)) * 1.002
    ds, model = _weighted(goo, ctx, spec, cols, counts)
    nll, g = model.nll_grad(ds, theta, precision)
    rnll, rg = om.TreeModel(spec).nll_grad(cols, theta, weights=counts)
    assert abs(nll - rnll) <= TOL_NLL[precision] * abs(rnll), (nll, rnll)
    assert np.max(np.abs(g - rg)) <= TOL_GRAD[precision] * np.max(np.abs(rg))


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_weighted_shards_and_edge_cases(goo, ctx, precision):
    spec, cols, counts = _hist_c1(1000)
    cols = _data(spec, cols, precision)
    theta = np.array(synth.param_values(spec)) * 1.01
    ds, model = _weighted(goo, ctx, spec, cols, counts)
    full, g = model.nll_grad(ds, theta, precision)
    edges = [0, 1, 255, 257, 999, 1000]
    parts = [model.nll_partial(ds, a, b, theta, precision) for a, b in zip(edges[:-1], edges[1:])]
    tot = goo.combine_partials(parts, model.n_params)
    assert tot[2] == 1000
    assert abs(tot[0] + tot[1] - full) <= (1e-12 if precision == "f64" else 1e-9) * abs(full)
    np.testing.assert_allclose(tot[3:], g, rtol=1e-9 if precision == "f64" else 1e-5, atol=1e-9 * np.abs(g).max())
    # every bin empty: nothing is summed
    ds.set_weights(np.zeros(1000))
    nll0, g0 = model.nll_grad(ds, theta, precision)
    assert nll0 == 0.0 and np.all(g0 == 0.0)
    # one bin: -w log f(x)
    one = np.zeros(1000)
    one[417] = 3.0
    ds.set_weights(one)
    ref = om.TreeModel(spec)
    x417 = {"x": cols["x"][417:418]}
    assert model.nll(ds, theta, precision) == pytest.approx(3.0 * ref.nll(x417, theta), rel=TOL_NLL[precision] * 10)


def test_weight_checks(goo, ctx):
    spec, cols, counts = _hist_c1(100)
    ds = goo.Dataset.from_spec(ctx, spec, cols)
    for bad in (-1.0, np.nan, np.inf):
        w = counts.copy()
        w[7] = bad
        with pytest.raises(goo.GooError):
            ds.set_weights(w)
    with pytest.raises(ValueError):
        ds.set_weights(counts[:-1])
    # a refused call leaves the dataset unweighted
    model = goo.Model(ctx, spec)
    theta = np.array(synth.param_values(spec))
    assert model.nll(ds, theta, "f64") == pytest.approx(om.TreeModel(spec).nll(cols, theta), rel=1e-12)
    # amplitude models refuse weighted datasets
    c3 = synth.c3_spec(n_mc=4_000)
    k = synth.DALITZ_MASSES
    pts = synth.dalitz_candidates(4_000, 3, k["M"], k["m1"], k["m2"], k["m3"])
    mcds = goo.Dataset.from_spec(ctx, c3, pts)
    dz = goo.Model(ctx, c3, mc=mcds)
    dds = goo.Dataset.from_spec(ctx, c3, pts)
    dds.set_weights(np.ones(4_000))
    with pytest.raises(goo.GooError):
        dz.nll(dds, np.array(synth.param_values(c3)), "f64")


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_binned_fit_matches_oracle_fit(goo, ctx, precision):
    # 200 bins of the 1-D model, every parameter free; the GPU fit (adjoint gradient)
    # against the oracle's FP64 fit of the same bin contents
    spec, cols, counts = _hist_c1(200)
    cols = _data(spec, cols, precision)
    start = np.array(synth.param_values(spec)) * 1.05
    steps = np.array([p[3] for p in spec["params"]])
    free = np.ones(4, bool)
    ref = om.TreeModel(spec)
    rth, rerr, _, redm = ofit.fit(lambda t: ref.nll_grad(cols, t, weights=counts), start, free, steps)
    assert 0 <= redm < 1e-8
    ds, model = _weighted(goo, ctx, spec, cols, counts)
    th, err, info = model.fit(ds, start, free, steps, precision=precision, gradient="adjoint")
    assert info["status"] == 0, info
    pulls = np.abs(th - rth) / rerr
    assert np.all(pulls < 0.01), pulls
    np.testing.assert_allclose(err, rerr, rtol=0.03)
