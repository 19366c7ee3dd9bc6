"""goo_nll_grad_streamed: host columns copied chunk by chunk while earlier chunks are evaluated.

The result must be the FP32 NLL and gradient of the same events (against the regular path
after goo_dataset_update, and against the oracle), for any chunk count, and the dataset must
afterwards hold the events in both precisions; out-of-range events are refused as at upload.
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


@pytest.mark.parametrize("n_chunks", [1, 3, 8])
def test_streamed_matches_regular_and_oracle(goo, ctx, n_chunks):
    spec = synth.c2_spec(bins=64)
    n = 1_000_003
    cols = synth.round_to_f32(synth.gen_c2(n=n, seed=47), spec)
    theta = np.array(synth.param_values(spec)) * 1.01
    host = _pinned(cols, spec)
    model = goo.Model(ctx, spec)
    # a dataset of the right capacity holding other events first
    other = synth.round_to_f32(synth.gen_c2(n=n, seed=48), spec)
    ds = goo.Dataset.from_spec(ctx, spec, other)
    nll, g = model.nll_grad_streamed(ds, host, theta, n_chunks=n_chunks)
    assert ds.n == n
    ref = goo.Dataset.from_spec(ctx, spec, cols)
    rnll, rg = model.nll_grad(ref, theta, "f32")
    assert abs(nll - rnll) <= 1e-9 * abs(rnll), (nll, rnll)
    np.testing.assert_allclose(g, rg, rtol=0, atol=1e-7 * np.abs(rg).max())
    onll, og = om.TreeModel(spec).nll_grad(cols, theta)
    assert abs(nll - onll) <= 1e-6 * abs(onll)
    assert np.max(np.abs(g - og)) <= 1e-4 * np.max(np.abs(og))
    # the dataset now holds these events in both precisions
    assert abs(model.nll(ds, theta, "f64") - om.TreeModel(spec).nll(cols, theta)) <= 1e-9 * abs(onll)


def test_streamed_refuses_out_of_range(goo, ctx):
    spec = synth.c2_spec(bins=64)
    n = 50_000
    cols = synth.round_to_f32(synth.gen_c2(n=n, seed=49), spec)
    cols["dE"][31_337] = 0.5   # outside [-0.2, 0.2]
    ds = goo.Dataset.from_spec(ctx, spec, synth.round_to_f32(synth.gen_c2(n=n, seed=50), spec))
    model = goo.Model(ctx, spec)
    with pytest.raises(goo.GooError) as e:
        model.nll_grad_streamed(ds, _pinned(cols, spec), np.array(synth.param_values(spec)), n_chunks=4)
    assert e.value.code == goo.GOO_ERR_RANGE
    assert ds.n == 0
