"""GOO_BORROW_HOST: float32 columns kept in pinned host memory and read over the host link by
every FP32 evaluation of a sum-of-product model.

The event kernel stores each thread's pairs of a tile in its own slots of the stage buffer and
evaluates them exactly as the staged path does, so the results must equal, bit for bit, those
of a device dataset holding the same float32 values (interpreted and specialised kernels, with
and without the gradient, whole and partial ranges with ragged ends).  The host columns may be
rewritten between evaluations; events outside the observable limits (or NaN) make the
evaluation fail with GOO_ERR_RANGE, and the next evaluation of valid events is unaffected.
"""
import numpy as np
import pytest

import synth
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


def _pinned(cols, spec):
    import torch
    return [torch.from_numpy(np.ascontiguousarray(cols[o[0]], dtype=np.float32)).pin_memory()
            for o in spec["observables"]]


def _limits(spec):
    return [o[1] for o in spec["observables"]], [o[2] for o in spec["observables"]]


@pytest.mark.parametrize("jit", [True, False])
def test_equals_device_dataset_bit_for_bit(goo, ctx, jit):
    spec = synth.c2_spec(bins=64)
    n = 1_000_003  # a ragged head and tail around the 8-aligned core
    cols = synth.round_to_f32(synth.gen_c2(n=n, seed=61), spec)
    theta = np.array(synth.param_values(spec)) * 1.01
    host = _pinned(cols, spec)
    lo, hi = _limits(spec)
    hb = goo.Dataset(ctx, host, lo, hi, dtype="f32", borrow_host=True)
    dev = goo.Dataset.from_spec(ctx, spec, cols)
    model = goo.Model(ctx, spec)
    model.set_jit(jit)
    n1, g1 = model.nll_grad(hb, theta, "f32")
    n2, g2 = model.nll_grad(dev, theta, "f32")
    assert n1 == n2 and np.array_equal(g1, g2)
    assert model.nll(hb, theta, "f32") == model.nll(dev, theta, "f32")
    # partial ranges with odd ends
    for b, e in [(3, 999_997), (1, 9), (123_457, 654_321)]:
        p1 = model.nll_partial(hb, b, e, theta, "f32")
        p2 = model.nll_partial(dev, b, e, theta, "f32")
        assert np.array_equal(p1, p2), (b, e)
    rnll, rg = om.TreeModel(spec).nll_grad(cols, theta)
    assert abs(n1 - rnll) <= 1e-6 * abs(rnll)
    assert np.max(np.abs(g1 - rg)) <= 1e-4 * np.max(np.abs(rg))


def test_host_columns_rewritten_between_evaluations(goo, ctx):
    spec = synth.c2_spec(bins=64)
    n = 300_001
    a = synth.round_to_f32(synth.gen_c2(n=n, seed=62), spec)
    b = synth.round_to_f32(synth.gen_c2(n=n, seed=63), spec)
    theta = np.array(synth.param_values(spec))
    host = _pinned(a, spec)
    lo, hi = _limits(spec)
    hb = goo.Dataset(ctx, host, lo, hi, dtype="f32", borrow_host=True)
    model = goo.Model(ctx, spec)
    na, ga = model.nll_grad(hb, theta, "f32")
    for t, o in zip(host, spec["observables"]):
        t.copy_(__import__("torch").from_numpy(np.ascontiguousarray(b[o[0]], dtype=np.float32)))
    nb_, gb_ = model.nll_grad(hb, theta, "f32")
    ref = model.nll_grad(goo.Dataset.from_spec(ctx, spec, b), theta, "f32")
    assert nb_ == ref[0] and np.array_equal(gb_, ref[1])
    assert nb_ != na


def test_out_of_range_events_fail_the_evaluation(goo, ctx):
    import torch
    spec = synth.c2_spec(bins=64)
    n = 200_003
    cols = synth.round_to_f32(synth.gen_c2(n=n, seed=64), spec)
    theta = np.array(synth.param_values(spec))
    host = _pinned(cols, spec)
    lo, hi = _limits(spec)
    hb = goo.Dataset(ctx, host, lo, hi, dtype="f32", borrow_host=True)
    model = goo.Model(ctx, spec)
    good = model.nll_grad(hb, theta, "f32")
    saved = [host[1][70_001].item(), host[0][n - 1].item(), host[2][5].item()]
    host[1][70_001] = 0.5            # dE outside [-0.2, 0.2], in the core
    host[0][n - 1] = float("nan")    # in the ragged tail
    host[2][5] = -1.0                # t below 0, in the first tile
    for grad in (True, False):
        with pytest.raises(goo.GooError) as e:
            if grad:
                model.nll_grad(hb, theta, "f32")
            else:
                model.nll(hb, theta, "f32")
        assert e.value.code == goo.GOO_ERR_RANGE
        assert "3 events" in str(e.value), str(e.value)
    # events exactly at the limits of t (0 and 10, both float32 values) are inside; the float32
    # value nearest 0.2 lies above the limit 0.2 of dE and is outside
    host[1][70_001] = saved[0]
    host[0][n - 1] = saved[1]
    host[2][5] = 0.0
    host[2][6] = 10.0
    saved6 = cols["t"][6]
    model.nll_grad(hb, theta, "f32")
    host[1][70_001] = float(np.float32(0.2))
    with pytest.raises(goo.GooError) as e:
        model.nll_grad(hb, theta, "f32")
    assert e.value.code == goo.GOO_ERR_RANGE and "1 events" in str(e.value)
    host[1][70_001] = saved[0]
    host[2][5] = saved[2]
    host[2][6] = float(saved6)
    again = model.nll_grad(hb, theta, "f32")
    assert again[0] == good[0] and np.array_equal(again[1], good[1])


def test_unsupported_uses_are_refused(goo, ctx):
    spec = synth.c2_spec(bins=64)
    cols = synth.round_to_f32(synth.gen_c2(n=10_000, seed=65), spec)
    host = _pinned(cols, spec)
    lo, hi = _limits(spec)
    hb = goo.Dataset(ctx, host, lo, hi, dtype="f32", borrow_host=True)
    model = goo.Model(ctx, spec)
    theta = np.array(synth.param_values(spec))
    with pytest.raises(goo.GooError) as e:
        model.nll_grad(hb, theta, "f64")
    assert e.value.code == goo.GOO_ERR_UNSUPPORTED
    with pytest.raises(goo.GooError) as e:
        hb.update([np.asarray(c) for c in host])
    assert e.value.code == goo.GOO_ERR_STATE
    with pytest.raises(ValueError):
        goo.Dataset(ctx, host, lo, hi, dtype="f64", borrow_host=True)
    # unpinned host memory has no device mapping
    with pytest.raises(goo.GooError) as e:
        goo.Dataset(ctx, [np.asarray(cols[o[0]], dtype=np.float32) for o in spec["observables"]], lo, hi,
                    dtype="f32", borrow_host=True)
    assert e.value.code == goo.GOO_ERR_ARG
