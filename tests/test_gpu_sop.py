"""GPU parity of the sum/product likelihood path against the FP64 oracle (through the C ABI)."""
import numpy as np
import pytest

import synth
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
    # the FP32 path evaluates float32 columns: the oracle sees the same rounded values
    return synth.round_to_f32(cols, spec) if precision == "f32" else cols


def _check(goo, ctx, spec, cols, theta, precision, grad=True):
    cols = _data(spec, cols, precision)
    ds = goo.Dataset.from_spec(ctx, spec, cols)
    model = goo.Model(ctx, spec)
    ref = om.TreeModel(spec)
    if grad:
        nll, g = model.nll_grad(ds, theta, precision)
        rnll, rg = ref.nll_grad(cols, theta)
        assert abs(nll - rnll) <= TOL_NLL[precision] * abs(rnll), (nll, rnll)
        err = np.abs(g - rg) / np.max(np.abs(rg))
        assert np.max(err) <= TOL_GRAD[precision], (g, rg)
        return nll, g
    nll = model.nll(ds, theta, precision)
    rnll = ref.nll(cols, theta)
    assert abs(nll - rnll) <= TOL_NLL[precision] * abs(rnll), (nll, rnll)
    return nll, None


@pytest.mark.parametrize("precision", ["f64", "f32"])
@pytest.mark.parametrize("offset", [1.0, 1.05])
def test_c1_nll_grad(goo, ctx, precision, offset):
    spec = synth.c1_spec()
    theta = np.array(synth.param_values(spec)) * offset
    _check(goo, ctx, spec, synth.gen_c1(), theta, precision)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_c2_grid_nll_grad(goo, ctx, precision):
    spec = synth.c2_spec()
    theta = np.array(synth.param_values(spec)) * 1.002
    _check(goo, ctx, spec, synth.gen_c2(n=200_000, seed=21), theta, precision)


@pytest.mark.parametrize("bins", [[2000, 30, 16], [2000, 40, 16]])
def test_grid_normalised_in_the_event_kernel_and_apart(goo, ctx, bins):
    # the FP32 event kernel normalises a separable grid itself up to 4096 1-D bins summed over
    # the leaves (2 x 2046 here) and leaves larger grids to the normalisation kernel (2 x 2056):
    # both against the oracle's full midpoint grid
    spec = synth.c2_spec()
    spec["norm"] = ("grid", bins)
    theta = np.array(synth.param_values(spec)) * 1.003
    _check(goo, ctx, spec, synth.gen_c2(n=100_000, seed=23), theta, "f32")
    cols = _data(spec, synth.gen_c2(n=100_000, seed=23), "f32")
    ds = goo.Dataset.from_spec(ctx, spec, cols)
    model = goo.Model(ctx, spec)
    full, gfull = model.nll_grad(ds, theta, "f32")
    parts = [model.nll_partial(ds, a, b, theta, "f32") for a, b in ((0, 777), (777, 50_001), (50_001, 100_000))]
    tot = goo.combine_partials(parts, model.n_params)
    assert abs(tot[0] + tot[1] - full) <= 1e-9 * abs(full)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_c2_normalise_matches_oracle_grid(goo, ctx, precision):
    spec = synth.c2_spec()
    theta = np.array(synth.param_values(spec)) * 0.998
    model = goo.Model(ctx, spec)
    norms = model.normalise(theta, precision)
    ref = om.TreeModel(spec).component_norms(theta)
    tol = 1e-12 if precision == "f64" else 2e-6
    np.testing.assert_allclose(norms, ref, rtol=tol)


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_per_event_logf(goo, ctx, precision):
    spec = synth.c2_spec(bins=64)
    cols = _data(spec, synth.gen_c2(n=5000, seed=3), precision)
    theta = synth.param_values(spec)
    ds = goo.Dataset.from_spec(ctx, spec, cols)
    got = goo.Model(ctx, spec).eval_logf(ds, theta, precision).cpu().numpy()
    ref = np.log(om.TreeModel(spec).density(cols, theta).numpy())
    tol = 1e-11 if precision == "f64" else 2e-5
    np.testing.assert_allclose(got, ref, rtol=0, atol=tol)


@pytest.mark.parametrize("n", [1, 31, 32, 33, 255, 257, 1023, 4097])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_ragged_sizes(goo, ctx, n, precision):
    spec = synth.c2_spec(bins=16)
    theta = np.array(synth.param_values(spec)) * 1.01
    _check(goo, ctx, spec, synth.gen_c2(n=n, seed=100 + n), theta, precision)


def test_empty_dataset(goo, ctx):
    spec = synth.c1_spec()
    ds = goo.Dataset.from_spec(ctx, spec, {"x": np.zeros(0)})
    nll, g = goo.Model(ctx, spec).nll_grad(ds, synth.param_values(spec), "f64")
    assert nll == 0.0 and np.all(g == 0)


def test_out_of_range_upload_is_rejected(goo, ctx):
    x = synth.gen_c1(n=1000, seed=1)["x"].copy()
    x[[5, 17, 400]] = [-0.5, 10.5, np.nan]
    with pytest.raises(goo.GooError) as e:
        goo.Dataset(ctx, [x], [0.0], [10.0])
    assert e.value.code == goo.GOO_ERR_RANGE and "3 of 1000" in str(e.value)


def test_nonpositive_density_reports(goo, ctx):
    # Argus alone: events above the endpoint have zero density
    spec = dict(name="argus", observables=[("m", 5.2, 5.3)],
                params=[("m0", 5.25, False, 0), ("c", -20.0, False, 0), ("p", 0.5, False, 0)],
                pdf=("argus", "m", "m0", "c", "p"), norm=("grid", [64]))
    ds = goo.Dataset(ctx, [np.array([5.21, 5.22, 5.27])], [5.2], [5.3])
    model = goo.Model(ctx, spec)
    with pytest.raises(goo.GooError) as e:
        model.nll(ds, [5.25, -20.0, 0.5])
    assert e.value.code == goo.GOO_ERR_NONPOSITIVE_PDF
    assert model.nll(ds, [5.28, -20.0, 0.5]) > -1e9  # recovers on the next call


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_shards_combine_to_full(goo, ctx, precision):
    spec = synth.c2_spec(bins=32)
    cols = _data(spec, synth.gen_c2(n=100_003, seed=8), precision)
    theta = np.array(synth.param_values(spec)) * 1.003
    ds = goo.Dataset.from_spec(ctx, spec, cols)
    model = goo.Model(ctx, spec)
    full, g = model.nll_grad(ds, theta, precision)
    edges = [0, 1, 33333, 50000, 77777, 100_003]
    parts = [model.nll_partial(ds, a, b, theta, precision) for a, b in zip(edges[:-1], edges[1:])]
    tot = goo.combine_partials(parts, model.n_params)
    assert tot[2] == 100_003
    assert abs(tot[0] + tot[1] - full) <= 1e-12 * abs(full) * (1 if precision == "f64" else 1e3)
    np.testing.assert_allclose(tot[3:], g, rtol=1e-9 if precision == "f64" else 1e-5, atol=1e-9 * np.abs(g).max())


def test_deterministic_repeat(goo, ctx):
    spec = synth.c2_spec()
    ds = goo.Dataset.from_spec(ctx, spec, synth.gen_c2(n=300_000, seed=9))
    model = goo.Model(ctx, spec)
    th = synth.param_values(spec)
    for prec in ("f64", "f32"):
        a = model.nll_grad(ds, th, prec)
        b = model.nll_grad(ds, th, prec)
        assert a[0] == b[0] and np.array_equal(a[1], b[1])


def test_nested_tree_matches_oracle(goo, ctx):
    spec = dict(
        name="nested", observables=[("x", 0.0, 4.0), ("y", -1.0, 1.0)],
        params=[("a", 1.5, False, 0), ("b", 0.6, False, 0), ("l", -0.4, False, 0), ("f", 0.4, False, 0),
                ("c", 0.2, False, 0), ("d", 0.5, False, 0), ("g", 0.7, False, 0), ("l2", 0.3, False, 0)],
        pdf=("add", ["g"], [
            ("prod", [("add", ["f"], [("gauss", "x", "a", "b"), ("expo", "x", "l")]), ("gauss", "y", "c", "d")]),
            ("prod", [("expo", "x", "l2"), ("expo", "y", "l")])]),
        norm=("analytic",))
    rng = np.random.default_rng(1)
    cols = {"x": rng.uniform(0, 4, 20000), "y": rng.uniform(-1, 1, 20000)}
    theta = [p[1] for p in spec["params"]]
    for prec in ("f64", "f32"):
        _check(goo, ctx, spec, cols, theta, prec)
    spec_g = dict(spec, norm=("grid", [200, 100]))
    _check(goo, ctx, spec_g, cols, theta, "f64")


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_grid_with_shared_observable(goo, ctx, precision):
    # two leaves of one product on the same observable: the grid sum does not factorise, so
    # this takes the dense grid kernel (the C2 model takes the separable one)
    spec = dict(
        name="shared", observables=[("x", 0.0, 4.0), ("y", -1.0, 1.0)],
        params=[("a", 1.5, False, 0), ("b", 0.6, False, 0), ("l", -0.4, False, 0), ("f", 0.4, False, 0),
                ("l2", 0.3, False, 0), ("c", 0.2, False, 0), ("d", 0.1, False, 0)],
        pdf=("add", ["f"], [
            ("prod", [("gauss", "x", "a", "b"), ("expo", "x", "l")]),
            ("prod", [("expo", "x", "l2"), ("poly2", "y", "c", "d")])]),
        norm=("grid", [256, 64]))
    rng = np.random.default_rng(2)
    cols = {"x": rng.uniform(0, 4, 30000), "y": rng.uniform(-1, 1, 30000)}
    theta = np.array([p[1] for p in spec["params"]]) * 1.02
    _check(goo, ctx, spec, cols, theta, precision)


def test_borrowed_torch_columns(goo, ctx):
    import torch
    spec = synth.c1_spec()
    x = synth.gen_c1(n=50_000, seed=4)["x"]
    ds_copy = goo.Dataset.from_spec(ctx, spec, {"x": x})
    t = torch.tensor(x, dtype=torch.float64, device="cuda:0")
    ds_b = goo.Dataset(ctx, [t], [0.0], [10.0])
    model = goo.Model(ctx, spec)
    th = synth.param_values(spec)
    assert model.nll(ds_copy, th) == model.nll(ds_b, th)


def test_autograd_function(goo, ctx):
    import torch
    from paper_1710_08826_gb300.autograd import nll as goo_nll
    spec = synth.c1_spec()
    cols = synth.round_to_f32(synth.gen_c1(n=20000, seed=6), spec)
    ds = goo.Dataset.from_spec(ctx, spec, cols)
    model = goo.Model(ctx, spec)
    th = torch.tensor(np.array(synth.param_values(spec)) * 1.03, dtype=torch.float64, requires_grad=True)
    val = goo_nll(th, model, ds, "f32")
    val.backward()
    _, rg = om.TreeModel(spec).nll_grad(cols, th.detach().numpy())
    np.testing.assert_allclose(th.grad.numpy(), rg, rtol=1e-4, atol=1e-4 * np.abs(rg).max())


@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_c2_full_size(goo, ctx, precision):
    # 10M events in the launch configuration the benchmark times
    spec = synth.c2_spec()
    cols = _data(spec, synth.gen_c2(), precision)
    theta = synth.param_values(spec)
    ds = goo.Dataset.from_spec(ctx, spec, cols)
    model = goo.Model(ctx, spec)
    nll, g = model.nll_grad(ds, theta, precision)
    rnll, rg = om.TreeModel(spec).nll_grad(cols, theta)
    assert abs(nll - rnll) <= TOL_NLL[precision] * abs(rnll)
    # at the generating point the gradient is a sqrt(N)-size fluctuation: compare on the
    # scale of the per-parameter Fisher information sqrt(N * I) via the oracle gradient at
    # a shifted point
    scale = np.maximum(np.abs(rg), np.sqrt(len(cols["m"])) * 1e-2)
    assert np.all(np.abs(g - rg) <= TOL_GRAD[precision] * np.max(scale) + 1e-12), (g, rg)


SPECIALISED_SPECS = {
    "c1": (synth.c1_spec, lambda: synth.gen_c1(), 1.02),
    "c2": (synth.c2_spec, lambda: synth.gen_c2(n=150_000, seed=51), 1.002),
}


@pytest.mark.parametrize("precision_grad", [("f32", True), ("f32", False)])
@pytest.mark.parametrize("which", ["c1", "c2"])
def test_specialised_and_interpreted_kernels_match_oracle(goo, ctx, which, precision_grad):
    # the FP32 event kernel compiled for the model's leaf signature at run time and the
    # library's interpreter: both against the oracle, and against each other
    precision, grad = precision_grad
    mk, gen, off = SPECIALISED_SPECS[which]
    spec = mk()
    cols = _data(spec, gen(), precision)
    theta = np.array(synth.param_values(spec)) * off
    ds = goo.Dataset.from_spec(ctx, spec, cols)
    out = {}
    for jit in (True, False):
        model = goo.Model(ctx, spec)
        model.set_jit(jit)
        out[jit] = model.nll_grad(ds, theta, precision) if grad else (model.nll(ds, theta, precision), None)
        assert model.jit_status == (2 if jit else 0)
    ref = om.TreeModel(spec)
    rnll, rg = ref.nll_grad(cols, theta)
    for jit in (True, False):
        nll, g = out[jit]
        assert abs(nll - rnll) <= TOL_NLL[precision] * abs(rnll), (jit, nll, rnll)
        if grad:
            assert np.max(np.abs(g - rg)) <= TOL_GRAD[precision] * np.max(np.abs(rg)), (jit, g, rg)
    assert abs(out[True][0] - out[False][0]) <= 1e-7 * abs(rnll)


def test_specialised_kernel_on_sparse_and_nested_signatures(goo, ctx):
    # products with fewer leaves than the kernel's slots and the leaf types in other slots,
    # with and without gradient
    spec = synth.c2_spec(bins=32)
    spec["pdf"] = ("add", ["frac"], [
        ("prod", [("expo", "t", "lam_s"), ("gauss", "m", "mu_m", "sig_m")]),
        ("prod", [("poly2", "dE", "a1", "a2"), ("argus", "m", "m0", "c", "p"), ("expo", "t", "lam_b")]),
    ])
    cols = _data(spec, synth.gen_c2(n=60_000, seed=52), "f32")
    theta = np.array(synth.param_values(spec)) * 1.003
    for grad in (True, False):
        ds = goo.Dataset.from_spec(ctx, spec, cols)
        model = goo.Model(ctx, spec)
        ref = om.TreeModel(spec)
        if grad:
            nll, g = model.nll_grad(ds, theta, "f32")
            rnll, rg = ref.nll_grad(cols, theta)
            assert np.max(np.abs(g - rg)) <= TOL_GRAD["f32"] * np.max(np.abs(rg))
        else:
            nll, rnll = model.nll(ds, theta, "f32"), ref.nll(cols, theta)
        assert abs(nll - rnll) <= TOL_NLL["f32"] * abs(rnll)
        assert model.jit_status == 2
