"""GPU test of goo_nll_grad_static, the entry point that allocates no device memory.

It is meant for callers that cannot call cudaMalloc (another component owns the device
memory, or allocation latency and its implicit synchronisation are not acceptable), so the
test passes only device columns and host arrays and compares two calls in a row with the
regular goo_nll_grad path.  Collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-9, "f32": 1e-6}


@pytest.fixture(scope="module")
def goo():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1710_08826_gb300 import goo as g
    g.lib.goo_nll_grad_static.restype = ctypes.c_int
    g.lib.goo_nll_grad_static.argtypes = [
        ctypes.POINTER(g.GooNode), ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_double),
        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(g.GooNormSpec), ctypes.POINTER(ctypes.c_void_p),
        ctypes.c_int, ctypes.c_int64, ctypes.POINTER(ctypes.c_double), ctypes.c_void_p,
        ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    return g


def _static_call(goo, spec, dev_cols, precision, theta):
    import torch
    nodes, nn = goo.spec_to_nodes(spec)
    obs = spec["observables"]
    lo = (ctypes.c_double * len(obs))(*[o[1] for o in obs])
    hi = (ctypes.c_double * len(obs))(*[o[2] for o in obs])
    ns = goo.GooNormSpec()
    ns.kind = goo.NORM[spec["norm"][0]]
    if spec["norm"][0] == "grid":
        for j, b in enumerate(spec["norm"][1]):
            ns.bins[j] = b
    ptrs = (ctypes.c_void_p * len(obs))(*[c.data_ptr() for c in dev_cols])
    th = (ctypes.c_double * len(theta))(*theta)
    nll = ctypes.c_double()
    g = (ctypes.c_double * len(theta))()
    stream = torch.cuda.current_stream().cuda_stream
    rc = goo.lib.goo_nll_grad_static(nodes, nn, len(theta), len(obs), lo, hi, ctypes.byref(ns), ptrs,
                                     goo.precision_code(precision), dev_cols[0].numel(), th,
                                     ctypes.c_void_p(stream) if stream else None, ctypes.byref(nll), g)
    if rc != 0:
        raise goo.GooError(rc, goo.lib.goo_last_error().decode())
    return nll.value, np.array(g[:])


@pytest.mark.parametrize("which", ["c1", "c2"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_static_matches_regular_twice(goo, which, precision):
    import torch
    if which == "c1":
        spec = synth.c1_spec()
        cols = synth.gen_c1(n=70_001, seed=31)
    else:
        spec = synth.c2_spec(bins=64)
        cols = synth.gen_c2(n=300_007, seed=32)
    if precision == "f32":
        cols = synth.round_to_f32(cols, spec)
    theta = list(np.array(synth.param_values(spec)) * 1.01)
    ctx = goo.Context(0)
    ds = goo.Dataset.from_spec(ctx, spec, cols)
    ref_nll, ref_g = goo.Model(ctx, spec).nll_grad(ds, theta, precision)
    dt = torch.float64 if precision == "f64" else torch.float32
    dev_cols = [torch.tensor(cols[o[0]], dtype=dt, device="cuda:0") for o in spec["observables"]]
    for _ in range(2):
        nll, g = _static_call(goo, spec, dev_cols, precision, theta)
        assert abs(nll - ref_nll) <= TOL[precision] * abs(ref_nll)
        np.testing.assert_allclose(g, ref_g, rtol=0, atol=TOL[precision] * np.abs(ref_g).max())


def _dense_grid_spec():
    # two leaves of one product on the same observable: the grid does not factorise, so the
    # dense midpoint-grid kernel runs
    return dict(
        name="dense_grid",
        observables=[("x", 0.0, 10.0), ("y", -1.0, 1.0)],
        params=[("mu", 4.0, False, 0.01), ("sigma", 1.5, False, 0.01), ("lam", -0.2, False, 0.01),
                ("a1", 0.3, False, 0.01), ("a2", 0.2, False, 0.01), ("frac", 0.4, False, 0.01)],
        pdf=("add", ["frac"], [
            ("prod", [("gauss", "x", "mu", "sigma"), ("expo", "x", "lam"), ("poly2", "y", "a1", "a2")]),
            ("prod", [("expo", "x", "lam"), ("poly2", "y", "a1", "a2")]),
        ]),
        norm=("grid", [96, 40]),
    )


def _three_products_spec():
    # three products of up to four leaves: the larger (4 x 4) kernel shape
    return dict(
        name="three_products",
        observables=[("x", 0.0, 10.0), ("y", -1.0, 1.0), ("z", 0.0, 4.0)],
        params=[("mu", 4.0, False, 0.01), ("sigma", 1.5, False, 0.01), ("lam", -0.2, False, 0.01),
                ("a1", 0.3, False, 0.01), ("a2", 0.2, False, 0.01), ("mu_y", 0.1, False, 0.01),
                ("sig_y", 0.4, False, 0.01), ("lam_z", -0.7, False, 0.01), ("f1", 0.3, False, 0.01),
                ("f2", 0.25, False, 0.01)],
        pdf=("add", ["f1", "f2"], [
            ("prod", [("gauss", "x", "mu", "sigma"), ("gauss", "y", "mu_y", "sig_y"), ("expo", "z", "lam_z")]),
            ("prod", [("expo", "x", "lam"), ("poly2", "y", "a1", "a2")]),
            ("prod", [("gauss", "x", "mu", "sigma"), ("poly2", "y", "a1", "a2"), ("expo", "z", "lam_z")]),
        ]),
        norm=("analytic",),
    )


def _uniform_cols(spec, n, seed):
    rng = np.random.default_rng(seed)
    return {o[0]: rng.uniform(o[1], o[2], n) for o in spec["observables"]}


@pytest.mark.parametrize("which", ["dense_grid", "three_products"])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_static_other_model_shapes(goo, which, precision):
    import torch
    spec = _dense_grid_spec() if which == "dense_grid" else _three_products_spec()
    cols = _uniform_cols(spec, 123_457, 33)
    if precision == "f32":
        cols = synth.round_to_f32(cols, spec)
    theta = [p[1] for p in spec["params"]]
    ctx = goo.Context(0)
    ds = goo.Dataset.from_spec(ctx, spec, cols)
    ref_nll, ref_g = goo.Model(ctx, spec).nll_grad(ds, theta, precision)
    dt = torch.float64 if precision == "f64" else torch.float32
    dev_cols = [torch.tensor(cols[o[0]], dtype=dt, device="cuda:0") for o in spec["observables"]]
    tol_g = 1e-9 if precision == "f64" else 1e-4
    for _ in range(2):
        nll, g = _static_call(goo, spec, dev_cols, precision, theta)
        assert abs(nll - ref_nll) <= TOL[precision] * abs(ref_nll)
        np.testing.assert_allclose(g, ref_g, rtol=0, atol=tol_g * np.abs(ref_g).max())


def test_static_empty_input(goo):
    import torch
    spec = synth.c1_spec()
    theta = [p[1] for p in spec["params"]]
    dev_cols = [torch.zeros(0, dtype=torch.float64, device="cuda:0")]
    nll, g = _static_call(goo, spec, dev_cols, "f64", theta)
    assert nll == 0.0 and np.all(g == 0.0)


def test_static_rejects_unsupported_shapes(goo):
    import torch
    spec = synth.c1_spec()
    nested = dict(spec, params=spec["params"] + [("frac2", 0.5, False, 0.01)],
                  pdf=("add", ["frac"], [("add", ["frac2"], [("gauss", "x", "mu", "sigma"), ("expo", "x", "lam")]),
                                         ("expo", "x", "lam")]))
    argus = dict(name="argus_analytic", observables=[("m", 5.2, 5.3)],
                 params=[("m0", 5.29, False, 0.0), ("c", -20.0, False, 0.0), ("p", 0.5, False, 0.0)],
                 pdf=("argus", "m", "m0", "c", "p"), norm=("analytic",))
    for sp, x in ((nested, 5.0), (argus, 5.25)):
        dev_cols = [torch.full((64,), x, dtype=torch.float64, device="cuda:0")]
        with pytest.raises(goo.GooError) as e:
            _static_call(goo, sp, dev_cols, "f64", [p[1] for p in sp["params"]])
        assert e.value.code == goo.GOO_ERR_UNSUPPORTED, e.value


def test_static_rejects_oversized(goo):
    import torch
    spec = synth.c1_spec()
    spec = dict(spec, params=spec["params"] + [(f"extra{i}", 0.0, True, 0.0) for i in range(40)])
    dev_cols = [torch.zeros(16, dtype=torch.float64, device="cuda:0") + 5.0]
    with pytest.raises(goo.GooError) as e:
        _static_call(goo, spec, dev_cols, "f64", [p[1] for p in spec["params"]])
    assert e.value.code == goo.GOO_ERR_ARG and "maximum" in str(e.value)
