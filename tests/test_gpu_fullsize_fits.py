"""Fit-level gates at full size for the FP32 form of the amplitude models.

At a few million events the FP32 gradient's error, although far below 1e-4 of the gradient,
can be of the order of 0.01 standard deviations of a parameter, the accuracy the fits must
reach.  The FP32 fit therefore ends with Newton steps on FP64 gradients (goo_fit's
refinement).  These tests fit full-size samples drawn from each model twice -- FP64
throughout, and FP32 with the FP64 refinement -- and require every free parameter of the two
fits to agree within 0.01 of its FP64 error:
  * the time-dependent four-body model: 2,000,000 events, 3,000,000 MC points;
  * the time-dependent three-body model: 2,000,000 events, 1,000,000 MC points;
  * the three-body model with floating lineshapes (masses and widths free): 5,000,000
    events, 1,000,000 MC points.
The samples come from accept--reject on the oracle's rates (the four- and three-body
time-dependent models, in spawned worker processes) and from the device toy generator,
which its own tests pin to the oracle's density (the three-body model).
"""
import functools
import multiprocessing as mp
import os

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

WORKERS = max(1, min(16, os.cpu_count() or 1))


@pytest.fixture(scope="module")
def goo():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1710_08826_gb300 import goo as g
    return g


@pytest.fixture(scope="module")
def ctx(goo):
    return goo.Context(0)


def _compare(th32, err32, th64, err64, free, tol_sigma=0.01, tol_err=0.03):
    idx = np.flatnonzero(free)
    pulls = np.abs(th32[idx] - th64[idx]) / err64[idx]
    assert np.max(pulls) < tol_sigma, pulls
    np.testing.assert_allclose(err32[idx], err64[idx], rtol=tol_err)
    return float(np.max(pulls))


def _fit_pair(model, ds, start, free, steps):
    th64, err64, info64 = model.fit(ds, start, free, steps, precision="f64", gradient="adjoint")
    th32, err32, info32 = model.fit(ds, start, free, steps, precision="f32", gradient="adjoint", refine=True)
    assert info64["status"] == 0 and info32["status"] == 0, (info64, info32)
    thu, _, _ = model.fit(ds, start, free, steps, precision="f32", gradient="adjoint", refine=False)
    pull = _compare(th32, err32, th64, err64, free)
    idx = np.flatnonzero(free)
    unrefined = float(np.max(np.abs(thu[idx] - th64[idx]) / err64[idx]))
    print(f"refined FP32 fit: {pull:.2e} sigma from the FP64 fit; without the refinement {unrefined:.2e} sigma")
    # the FP32 form alone (its own Newton polish, no FP64 gradients) also lands within 0.01 sigma
    assert unrefined < 0.01, unrefined


def _td3_part(spec, theta, n, seed):
    import torch
    torch.set_num_threads(1)  # one thread per worker process: the pool has a worker per core
    from oracle import td3 as ot3
    k = synth.TD3_MASSES
    cand = functools.partial(synth.dalitz_candidates, M=k["M"], m1=k["m1"], m2=k["m2"], m3=k["m3"])
    return ot3.generate(spec, theta, n, seed, cand)


def test_td4_full_size_fit(goo, ctx):
    from oracle import td4 as ot
    spec = synth.c4_spec()
    theta = np.array(synth.param_values(spec))
    data = ot.generate(spec, theta, 2_000_000, 1710040, workers=WORKERS)
    mc = synth.four_body_phase_space(3_000_000, 1710014, **synth.TD4_MASSES)
    mc["t"] = np.zeros(3_000_000)
    data, mc = synth.round_to_f32(data, spec), synth.round_to_f32(mc, spec)
    m = ot.TD4Model(spec)
    free = np.ones(len(theta), bool)
    for i in (m.tp[0], m.tp[1], m.tp[3], m.re[0], m.im[0]):
        free[i] = False
    start = theta.copy()
    shift = [i for i in m.re + m.im if free[i]]
    start[shift] *= 1.03
    start[m.tp[2]] *= 1.01
    steps = np.array([p[3] if p[3] > 0 else 1.0 for p in spec["params"]])
    ds = goo.Dataset.from_spec(ctx, spec, data)
    mcds = goo.Dataset.from_spec(ctx, spec, mc)
    model = goo.Model(ctx, spec, mc=mcds)
    _fit_pair(model, ds, start, free, steps)


def test_td3_full_size_fit(goo, ctx):
    from oracle import td3 as ot3
    spec = synth.td3_spec()
    theta = np.array(synth.param_values(spec))
    n, parts = 2_000_000, WORKERS
    sizes = [n // parts + (1 if w < n % parts else 0) for w in range(parts)]
    with mp.get_context("spawn").Pool(parts) as pool:
        chunks = pool.starmap(_td3_part, [(spec, theta, sizes[w], 1710060 + 7 * w) for w in range(parts)])
    data = {k: np.concatenate([c[k] for c in chunks]) for k in ("s12", "s13", "t")}
    data["t"] = np.clip(data["t"], *spec["observables"][2][1:])
    k = synth.TD3_MASSES
    mc = synth.dalitz_candidates(1_000_000, 1710015, k["M"], k["m1"], k["m2"], k["m3"])
    mc["t"] = np.zeros(1_000_000)
    data, mc = synth.round_to_f32(data, spec), synth.round_to_f32(mc, spec)
    m = ot3.TD3Model(spec)
    free = np.array([not p[2] for p in spec["params"]])
    for i in (m.tp[0], m.tp[1], m.tp[3]):
        free[i] = False
    names = synth.param_names(spec)
    coef = np.array([nm.startswith(("re_", "im_")) for nm in names]) & free
    start = theta.copy()
    start[coef] *= 1.03
    steps = np.array([p[3] if p[3] > 0 else 1.0 for p in spec["params"]])
    ds = goo.Dataset.from_spec(ctx, spec, data)
    mcds = goo.Dataset.from_spec(ctx, spec, mc)
    model = goo.Model(ctx, spec, mc=mcds)
    _fit_pair(model, ds, start, free, steps)


def test_floating_lineshapes_full_size_fit(goo, ctx):
    spec = synth.c3_spec()
    kin = synth.DALITZ_MASSES
    mc = synth.round_to_f32(synth.dalitz_candidates(1_000_000, 1710013, kin["M"], kin["m1"], kin["m2"], kin["m3"]),
                            spec)
    mcds = goo.Dataset.from_spec(ctx, spec, mc)
    model = goo.Model(ctx, spec, mc=mcds)
    theta = np.array(synth.param_values(spec))
    a, b = goo.toy_generate(model, theta, None, 1710070, 5_000_000)
    ds = goo.Dataset.from_spec(ctx, spec, {"s12": a.astype(np.float64), "s13": b.astype(np.float64)})
    model.set_lineshapes("floating")
    names = synth.param_names(spec)
    free = np.array([not nm.endswith("_NR") for nm in names])
    start = theta.copy()
    for i, nm in enumerate(names):
        if nm.startswith("m0_"):
            start[i] += 0.002
        elif nm.startswith("w_"):
            start[i] *= 1.03
        elif nm.startswith(("re_", "im_")) and free[i]:
            start[i] *= 1.03
    steps = np.array([p[3] if p[3] > 0 else 1e-3 for p in spec["params"]])
    _fit_pair(model, ds, start, free, steps)
