"""Dataset ingest on the GPU: copy-engine and mapped (zero-copy) uploads, the fused
conversion and range check (vector and scalar paths), and goo_dataset_update (buffer reuse,
range failures, invalidation of weights, amplitude caches and MC Gram matrices)."""
import numpy as np
import pytest
import torch

import synth
from oracle import dalitz as od
from oracle import model as om

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def goo():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1710_08826_gb300 import goo as g
    return g


@pytest.fixture(scope="module")
def ctx(goo):
    return goo.Context(0)


def _pinned(a, dtype):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).pin_memory()


class _DevArray:
    """A device column exposed through the CUDA array interface (read by torch.as_tensor)."""

    def __init__(self, ptr, n, dtype):
        self.__cuda_array_interface__ = {"shape": (n,), "typestr": "<f4" if dtype == "f32" else "<f8",
                                         "data": (int(ptr), False), "version": 3, "strides": None}


def _col_values(ds, col, n, dtype):
    """A host copy of the first n values of a device column."""
    torch.cuda.synchronize()
    return torch.as_tensor(_DevArray(ds.column_ptr(col, dtype), n, dtype), device="cuda:0").cpu().numpy()


@pytest.mark.parametrize("dtype", ["f32", "f64"])
@pytest.mark.parametrize("n", [1, 3, 4, 1027, 100_003])
def test_copy_and_mapped_uploads_store_the_same_columns(goo, ctx, dtype, n):
    spec = synth.c2_spec(bins=16)
    cols = synth.round_to_f32(synth.gen_c2(n=n, seed=300 + n), spec)
    names = [o[0] for o in spec["observables"]]
    lo = [o[1] for o in spec["observables"]]
    hi = [o[2] for o in spec["observables"]]
    npdt = np.float32 if dtype == "f32" else np.float64
    host = [np.ascontiguousarray(cols[k], dtype=npdt) for k in names]
    d_copy = goo.Dataset(ctx, host, lo, hi, dtype=dtype)
    d_map = goo.Dataset(ctx, [_pinned(h, npdt) for h in host], lo, hi, dtype=dtype, mapped=True)
    for c, h in enumerate(host):
        for prec in ("f32", "f64"):
            want = h.astype(np.float32 if prec == "f32" else np.float64)
            np.testing.assert_array_equal(_col_values(d_copy, c, n, prec), want)
            np.testing.assert_array_equal(_col_values(d_map, c, n, prec), want)


@pytest.mark.parametrize("mapped", [False, True])
def test_range_check_counts_every_bad_event(goo, ctx, mapped):
    # unaligned sources (offset by one element) take the scalar path
    x = synth.gen_c1(n=10_001, seed=2)["x"].astype(np.float32)
    x[[0, 5, 17, 400, 9_999, 10_000]] = [-0.5, 10.5, np.nan, np.inf, -np.inf, 11.0]
    pinned = _pinned(x, np.float32)
    for src, pin in ((x, pinned), (x[1:], pinned[1:])):
        nbad = int(np.sum(~((src >= 0.0) & (src <= 10.0))))
        col = pin if mapped else src
        with pytest.raises(goo.GooError) as e:
            goo.Dataset(ctx, [col], [0.0], [10.0], dtype="f32", mapped=mapped)
        assert e.value.code == goo.GOO_ERR_RANGE and f"{nbad} of {src.size}" in str(e.value)


def test_mapped_upload_needs_pinned_memory(goo, ctx):
    x = np.linspace(1.0, 9.0, 1000, dtype=np.float32)
    with pytest.raises(goo.GooError):
        goo.Dataset(ctx, [x], [0.0], [10.0], dtype="f32", mapped=True)


@pytest.mark.parametrize("mapped", [False, True])
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_update_matches_a_fresh_upload(goo, ctx, mapped, precision):
    spec = synth.c2_spec()
    names = [o[0] for o in spec["observables"]]
    theta = np.array(synth.param_values(spec)) * 1.003
    model = goo.Model(ctx, spec)
    first = synth.round_to_f32(synth.gen_c2(n=50_000, seed=31), spec)
    ds = goo.Dataset.from_spec(ctx, spec, first, dtype="f32")
    ds.set_weights(np.full(50_000, 2.0))
    for n, seed in ((50_000, 32), (12_345, 33), (0, 34), (7, 35)):
        cols = synth.round_to_f32(synth.gen_c2(n=n, seed=seed), spec)
        src = [_pinned(cols[k], np.float32) if mapped else cols[k] for k in names]
        ds.update(src, mapped=mapped)
        assert ds.n == n
        fresh = goo.Dataset.from_spec(ctx, spec, cols, dtype="f32")
        a = model.nll_grad(ds, theta, precision)
        b = model.nll_grad(fresh, theta, precision)
        assert a[0] == b[0] and np.array_equal(a[1], b[1])   # same events, same result (weights gone)
        if n:
            rnll = om.TreeModel(spec).nll(cols, theta)
            assert abs(a[0] - rnll) <= (1e-9 if precision == "f64" else 1e-6) * abs(rnll)


def test_update_errors(goo, ctx):
    spec = synth.c1_spec()
    x = synth.gen_c1(n=1000, seed=3)["x"]
    ds = goo.Dataset.from_spec(ctx, spec, {"x": x})
    with pytest.raises(goo.GooError):          # more events than the buffers hold
        ds.update([np.concatenate([x, x])])
    bad = x.copy()
    bad[[3, 4]] = [-1.0, np.nan]
    with pytest.raises(goo.GooError) as e:
        ds.update([bad])
    assert e.value.code == goo.GOO_ERR_RANGE and ds.n_bad == 2 and ds.n == 0
    model = goo.Model(ctx, spec)
    th = synth.param_values(spec)
    assert model.nll(ds, th, "f64") == 0.0     # a failed update leaves no events
    ds.update([x])
    assert model.nll(ds, th, "f64") == pytest.approx(om.TreeModel(spec).nll({"x": x}, th), rel=1e-12)
    t = torch.tensor(x, dtype=torch.float64, device="cuda:0")
    borrowed = goo.Dataset(ctx, [t], [0.0], [10.0])
    with pytest.raises(goo.GooError) as e:
        borrowed.update([x])
    assert e.value.code == -7   # GOO_ERR_STATE


def test_update_invalidates_amplitude_caches_and_gram(goo, ctx):
    spec = synth.c3_spec(n_mc=20_000)
    k = synth.DALITZ_MASSES

    def pts(n, seed):
        return synth.dalitz_candidates(n, seed, k["M"], k["m1"], k["m2"], k["m3"])
    theta = np.array(synth.param_values(spec))
    # float32-representable points, so both precisions evaluate the same events as the oracle
    mc1, mc2, ev1, ev2 = (synth.round_to_f32(pts(n, s), spec) for n, s in
                          ((20_000, 41), (20_000, 42), (10_000, 43), (10_000, 44)))
    mcds = goo.Dataset.from_spec(ctx, spec, mc1)
    model = goo.Model(ctx, spec, mc=mcds)
    ds = goo.Dataset.from_spec(ctx, spec, ev1)
    for prec in ("f64", "f32"):
        model.nll_grad(ds, theta, prec)        # builds the caches and the Gram matrix
    ds.update([ev2[o[0]] for o in spec["observables"]])
    mcds.update([mc2[o[0]] for o in spec["observables"]])
    ref = od.DalitzModel(spec)
    for prec in ("f64", "f32"):
        nll = model.nll(ds, theta, prec)
        rnll = ref.nll_grad(ev2, mc2, theta)[0]
        assert abs(nll - rnll) <= (1e-9 if prec == "f64" else 1e-6) * abs(rnll), (prec, nll, rnll)
