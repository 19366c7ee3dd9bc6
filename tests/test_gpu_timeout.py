"""The timeout path of the bounded device waits, exercised without a GPU fault.

Kernels that stage input tiles in shared memory by bulk copies wait for each tile on an
mbarrier for a bounded time and report GOO_ERR_TIMEOUT when the wait runs out.  Two forms:
  * the wait limit shortened to one SM clock (goo_set_wait_limit): a wait whose copy has not
    landed gives up at once (in practice the copies land ahead of the waits); every block
    drains its own copies with the default limit before it exits, so each call either
    reports GOO_ERR_TIMEOUT or returns the exact result;
  * one tile's copies withheld (goo_debug_withhold_tile, a flag that nothing else sets): the
    waits for that tile run out after a short limit and the call must report
    GOO_ERR_TIMEOUT, while the block drains the copies it did issue.
Afterwards the next call with the default limit matches the oracle and the earlier result
bit for bit, so the context stays usable.
"""
import numpy as np
import pytest

import synth
from oracle import dalitz as od
from oracle import model as om

pytestmark = pytest.mark.gpu

SHORT_LIMIT = 200_000  # SM clocks, about 0.1 ms


@pytest.fixture(scope="module")
def goo():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1710_08826_gb300 import goo as g
    return g


@pytest.fixture(scope="module")
def ctx(goo):
    c = goo.Context(0)
    yield c
    c.withhold_tile(-1)
    c.set_wait_limit(0)


def _short_limit_calls(goo, ctx, evaluate, ref, rel=1e-12, tries=3):
    """`tries` calls with a one-clock wait limit: each is GOO_ERR_TIMEOUT or equals ref."""
    got = []
    ctx.set_wait_limit(1)
    try:
        for _ in range(tries):
            try:
                nll, g = evaluate()
            except goo.GooError as e:
                assert e.code == goo.GOO_ERR_TIMEOUT, e
                got.append("timeout")
                continue
            assert nll == pytest.approx(ref[0], rel=rel)
            np.testing.assert_allclose(g, ref[1], rtol=rel, atol=rel * np.abs(ref[1]).max())
            got.append("exact")
    finally:
        ctx.set_wait_limit(0)
    return got


def _withheld_tile_times_out(goo, ctx, evaluate, tile=1):
    """With the copies of the first block's tile `tile` withheld, the call reports GOO_ERR_TIMEOUT."""
    ctx.set_wait_limit(SHORT_LIMIT)
    ctx.withhold_tile(tile)
    try:
        with pytest.raises(goo.GooError) as e:
            evaluate()
        assert e.value.code == goo.GOO_ERR_TIMEOUT, e.value
    finally:
        ctx.withhold_tile(-1)
        ctx.set_wait_limit(0)


@pytest.mark.parametrize("jit", [True, False])
def test_c2_event_kernel(goo, ctx, jit):
    # 2M events: ~980 column tiles, several per block, so waits occur inside the tile loop
    spec = synth.c2_spec(bins=32)
    cols = synth.round_to_f32(synth.gen_c2(n=2_000_000, seed=41), spec)
    theta = np.array(synth.param_values(spec)) * 1.01
    ds = goo.Dataset.from_spec(ctx, spec, cols)
    model = goo.Model(ctx, spec)
    model.set_jit(jit)
    ref = model.nll_grad(ds, theta, "f32")
    _short_limit_calls(goo, ctx, lambda: model.nll_grad(ds, theta, "f32"), ref)
    _withheld_tile_times_out(goo, ctx, lambda: model.nll_grad(ds, theta, "f32"))
    # default limit again: the context is usable and the result is the oracle's
    nll, g = model.nll_grad(ds, theta, "f32")
    rnll, rg = om.TreeModel(spec).nll_grad(cols, theta)
    assert abs(nll - rnll) <= 1e-6 * abs(rnll)
    assert np.max(np.abs(g - rg)) <= 1e-4 * np.max(np.abs(rg))
    assert nll == ref[0] and np.array_equal(g, ref[1])


def test_c3_staged_kernel(goo, ctx):
    spec = synth.c3_spec(n_mc=50_000)
    kin = synth.DALITZ_MASSES
    cand = lambda n, s: synth.dalitz_candidates(n, s, kin["M"], kin["m1"], kin["m2"], kin["m3"])
    data = synth.round_to_f32(cand(400_000, 43), spec)
    mc = synth.round_to_f32(cand(50_000, 1710013), spec)
    ds = goo.Dataset.from_spec(ctx, spec, data)
    mcds = goo.Dataset.from_spec(ctx, spec, mc)
    model = goo.Model(ctx, spec, mc=mcds)
    theta = np.array(synth.param_values(spec))
    ref = model.nll_grad(ds, theta, "f32")
    _short_limit_calls(goo, ctx, lambda: model.nll_grad(ds, theta, "f32"), ref)
    _withheld_tile_times_out(goo, ctx, lambda: model.nll_grad(ds, theta, "f32"))
    nll, g = model.nll_grad(ds, theta, "f32")
    rnll, rg = od.DalitzModel(spec).nll_grad(data, mc, theta)
    assert abs(nll - rnll) <= 1e-6 * abs(rnll)
    assert nll == ref[0] and np.array_equal(g, ref[1])


def test_c4_staged_kernel(goo, ctx):
    from oracle import td4 as ot
    spec = synth.c4_spec(n_mc=20_000)
    kin = dict(synth.TD4_MASSES)
    tau, sig = synth.TD4_TIME["tau"], synth.TD4_TIME["sigma_t"]
    data = synth.gen_c4_candidates(200_000, 44, kin, 1.0 / tau)
    data["t"] = np.clip(synth.smear_times(data.pop("t_true"), sig, 45), *spec["observables"][5][1:])
    mc = synth.four_body_phase_space(20_000, 1710014, **synth.TD4_MASSES)
    mc["t"] = np.zeros(20_000)
    data, mc = synth.round_to_f32(data, spec), synth.round_to_f32(mc, spec)
    ds = goo.Dataset.from_spec(ctx, spec, data)
    mcds = goo.Dataset.from_spec(ctx, spec, mc)
    model = goo.Model(ctx, spec, mc=mcds)
    theta = np.array(synth.param_values(spec))
    ref = model.nll_grad(ds, theta, "f32")
    _short_limit_calls(goo, ctx, lambda: model.nll_grad(ds, theta, "f32"), ref)
    nll, g = model.nll_grad(ds, theta, "f32")
    m = ot.TD4Model(spec)
    rnll = m.nll(data, m.amplitudes(mc), theta)
    assert abs(nll - rnll) <= 1e-6 * abs(rnll)
    assert nll == ref[0] and np.array_equal(g, ref[1])


def test_batched_evaluation(goo, ctx):
    spec = synth.c3_spec(n_mc=50_000)
    kin = synth.DALITZ_MASSES
    cand = lambda n, s: synth.dalitz_candidates(n, s, kin["M"], kin["m1"], kin["m2"], kin["m3"])
    mc = synth.round_to_f32(cand(50_000, 1710013), spec)
    mcds = goo.Dataset.from_spec(ctx, spec, mc)
    model = goo.Model(ctx, spec, mc=mcds)
    theta = np.array(synth.param_values(spec))
    dss = [goo.Dataset.from_spec(ctx, spec, synth.round_to_f32(cand(n, 50 + i), spec))
           for i, n in enumerate([300_000, 70_001, 150_000])]
    thetas = np.array([theta] * len(dss))
    ref = goo.nll_grad_batch(model, dss, thetas)
    _short_limit_calls(goo, ctx, lambda: goo.nll_grad_batch(model, dss, thetas), ref)
    nll, g = goo.nll_grad_batch(model, dss, thetas)
    assert np.array_equal(nll, ref[0]) and np.array_equal(g, ref[1])


def test_limit_out_of_range_is_rejected(goo, ctx):
    with pytest.raises(goo.GooError) as e:
        ctx.set_wait_limit(1 << 32)
    assert e.value.code == goo.GOO_ERR_ARG
    with pytest.raises(goo.GooError) as e:
        ctx.withhold_tile(-2)
    assert e.value.code == goo.GOO_ERR_ARG
    with pytest.raises(goo.GooError) as e:
        ctx.set_wait_limit(-1)
    assert e.value.code == goo.GOO_ERR_ARG
