"""GPU tests of the toy-MC server: device toy generation, batched NLL, continuous batching."""
import numpy as np
import pytest

import synth
from oracle import dalitz as od
from oracle import fit as ofit
from oracle import toys as otoys

pytestmark = pytest.mark.gpu

KIN = synth.DALITZ_MASSES


@pytest.fixture(scope="module")
def goo():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1710_08826_gb300 import goo as g
    return g


@pytest.fixture(scope="module")
def setup(goo):
    ctx = goo.Context(0)
    spec = synth.c3_spec(n_mc=200_000)
    mc = synth.round_to_f32(synth.dalitz_candidates(200_000, 1710013, KIN["M"], KIN["m1"], KIN["m2"], KIN["m3"]), spec)
    mcds = goo.Dataset.from_spec(ctx, spec, mc)
    model = goo.Model(ctx, spec, mc=mcds)
    theta = np.array(synth.param_values(spec))
    env = otoys.envelope(spec, theta)   # per-cell bounds of |S|^2, 48 x 48 cells
    return ctx, spec, mc, mcds, model, theta, env


def test_toy_generator_matches_oracle(goo, setup):
    ctx, spec, mc, mcds, model, theta, env = setup
    for seed, n in [(1710100, 700), (1710101, 1500), (1710777, 300)]:
        a, b = goo.toy_generate(model, theta, env, seed, n)
        ra, rb, _ = otoys.generate_toy(spec, theta, env, seed, n)
        np.testing.assert_array_equal(a, ra)
        np.testing.assert_array_equal(b, rb)


@pytest.mark.parametrize("grid", [(1, 1), (7, 13)])
def test_other_envelope_grids_match_oracle(goo, setup, grid):
    # one cell (the uniform box proposal with a single bound) and a non-square grid
    ctx, spec, mc, mcds, model, theta, env = setup
    e = otoys.envelope(spec, theta, *grid)
    a, b = goo.toy_generate(model, theta, e, 1710120, 900)
    ra, rb, _ = otoys.generate_toy(spec, theta, e, 1710120, 900)
    np.testing.assert_array_equal(a, ra)
    np.testing.assert_array_equal(b, rb)


def test_default_envelope_follows_the_same_density(goo, setup):
    # the library's own envelope (computed on the device at theta) gives other toys from the
    # same density: a two-sample chi2 of the Dalitz histograms against oracle-envelope toys
    ctx, spec, mc, mcds, model, theta, env = setup
    a0, b0 = goo.toy_generate(model, theta, None, 1710130, 200_000)
    a1, b1 = goo.toy_generate(model, theta, env, 1710131, 200_000)
    lo12, hi12, lo13, hi13 = otoys._box(KIN)
    h0 = np.histogram2d(a0, b0, 24, [[lo12, hi12], [lo13, hi13]])[0].ravel()
    h1 = np.histogram2d(a1, b1, 24, [[lo12, hi12], [lo13, hi13]])[0].ravel()
    k = (h0 + h1) > 20
    chi2 = np.sum((h0[k] - h1[k]) ** 2 / (h0[k] + h1[k]))
    assert chi2 / k.sum() < 1.3, (chi2, k.sum())


def test_envelope_arguments_are_checked(goo, setup):
    ctx, spec, mc, mcds, model, theta, env = setup
    n12, n13, bound = env
    with pytest.raises(ValueError):
        goo.toy_generate(model, theta, (n12, n13 + 1, bound), 1, 10)
    with pytest.raises(goo.GooError):
        goo.toy_generate(model, theta, (2, 2, np.zeros(4, np.float32)), 1, 10)
    with pytest.raises(goo.GooError):
        goo.toy_generate(model, theta, (1, 1, np.array([np.nan], np.float32)), 1, 10)


def test_toys_generated_together_equal_alone(goo, setup):
    ctx, spec, mc, mcds, model, theta, env = setup
    seeds = [1710150 + i for i in range(5)]
    sizes = [400, 3000, 17, 1200, 9000]
    together = goo.toys_generate(model, theta, env, seeds, sizes)
    for (a, b), sd, n in zip(together, seeds, sizes):
        a1, b1 = goo.toy_generate(model, theta, env, sd, n)
        np.testing.assert_array_equal(a, a1)
        np.testing.assert_array_equal(b, b1)
    ra, rb, _ = otoys.generate_toy(spec, theta, env, seeds[1], sizes[1])
    np.testing.assert_array_equal(together[1][0], ra)


def test_toys_follow_the_model(goo, setup):
    # the generated Dalitz distribution has the model's density: the NLL of the toy at the
    # generating point is lower than at a distorted point (by far more than statistics)
    ctx, spec, mc, mcds, model, theta, env = setup
    a, b = goo.toy_generate(model, theta, env, 1710200, 20_000)
    ds = goo.Dataset.from_spec(ctx, spec, {"s12": a.astype(np.float64), "s13": b.astype(np.float64)})
    th2 = theta.copy()
    names = synth.param_names(spec)
    th2[names.index("re_rho770_23")] *= 0.5
    assert model.nll(ds, theta, "f32") < model.nll(ds, th2, "f32") - 100


def _toy_ds(goo, ctx, spec, model, theta, env, seed, n):
    a, b = goo.toy_generate(model, theta, env, seed, n)
    return goo.Dataset.from_spec(ctx, spec, {"s12": a.astype(np.float64), "s13": b.astype(np.float64)})


def test_batch_matches_single_and_is_mix_independent(goo, setup):
    ctx, spec, mc, mcds, model, theta, env = setup
    sizes = [1000, 40_000, 17, 70_001]
    dss = [_toy_ds(goo, ctx, spec, model, theta, env, 1710300 + i, n) for i, n in enumerate(sizes)]
    rng = np.random.default_rng(5)
    names = synth.param_names(spec)
    coef = np.array([nm.startswith(("re_", "im_")) and not nm.endswith("NR") for nm in names])
    thetas = np.array([theta * np.where(coef, rng.uniform(0.9, 1.1, len(theta)), 1.0) for _ in sizes])
    nll, g = goo.nll_grad_batch(model, dss, thetas)
    for i, ds in enumerate(dss):
        n1, g1 = model.nll_grad(ds, thetas[i], "f32")
        assert abs(nll[i] - n1) <= 1e-6 * abs(n1) + 1e-6
        np.testing.assert_allclose(g[i][coef], g1[coef], rtol=1e-4, atol=1e-4 * np.abs(g1).max())
    # the same fit alone and in a different mix: bit-identical
    alone_n, alone_g = goo.nll_grad_batch(model, [dss[1]], thetas[1:2])
    mix_n, mix_g = goo.nll_grad_batch(model, [dss[3], dss[1], dss[0]], thetas[[3, 1, 0]])
    assert alone_n[0] == mix_n[1] and np.array_equal(alone_g[0], mix_g[1])


def _run(server, tickets, max_rounds=5000):
    for _ in range(max_rounds):
        q, a, d = server.step()
        if q == 0 and a == 0:
            break
    return {t: server.result(t) for t in tickets}


def test_server_fits_match_host_fitter_and_oracle(goo, setup):
    ctx, spec, mc, mcds, model, theta, env = setup
    names = synth.param_names(spec)
    free = np.array([not p[2] for p in spec["params"]])
    steps = np.array([p[3] if p[3] > 0 else 1.0 for p in spec["params"]])
    server = goo.Server(model, theta, envelope=env)
    toys = [(1710400 + i, n) for i, n in enumerate([3000, 800, 12_000, 5000, 1500, 30_000])]
    start = theta.copy()
    start[free] *= 1.05
    tickets = [server.submit(n, seed, start) for seed, n in toys]
    res = _run(server, tickets)
    for (seed, n), t in zip(toys, tickets):
        th, err, info = res[t]
        assert info["status"] == 0, info
        ds = _toy_ds(goo, ctx, spec, model, theta, env, seed, n)
        hth, herr, hinfo = model.fit(ds, start, free, steps, precision="f32")
        idx = np.flatnonzero(free)
        assert np.all(np.abs(th[idx] - hth[idx]) / herr[idx] < 0.01), (th[idx] - hth[idx]) / herr[idx]
        np.testing.assert_allclose(err[idx], herr[idx], rtol=0.03)
    # oracle fit of one toy (float32 events from the oracle's generator, float64 oracle)
    seed, n = toys[0]
    a, b, _ = otoys.generate_toy(spec, theta, env, seed, n)
    data = {"s12": np.asarray(a, np.float64), "s13": np.asarray(b, np.float64)}
    ref = od.DalitzModel(spec)
    rth, rerr, _, redm = ofit.fit(lambda t: ref.nll_grad(data, mc, t), start, free, steps)
    th = res[tickets[0]][0]
    idx = np.flatnonzero(free)
    assert np.all(np.abs(th[idx] - rth[idx]) / rerr[idx] < 0.01)
    assert names


def test_result_same_alone_and_in_mix(goo, setup):
    ctx, spec, mc, mcds, model, theta, env = setup
    start = theta.copy()
    free = np.array([not p[2] for p in spec["params"]])
    start[free] *= 0.95
    alone = goo.Server(model, theta, envelope=env)
    t = alone.submit(7000, 1710500, start)
    r_alone = _run(alone, [t])[t]
    mixed = goo.Server(model, theta, envelope=env, max_fits=3)
    tickets = [mixed.submit(n, s, start) for s, n in [(1710501, 20_000), (1710502, 900)]]
    tm = mixed.submit(7000, 1710500, start)
    tickets += [mixed.submit(n, s, start) for s, n in [(1710503, 4000), (1710504, 15_000)]]
    res = _run(mixed, tickets + [tm])
    assert np.array_equal(res[tm][0], r_alone[0]) and np.array_equal(res[tm][1], r_alone[1])
    assert res[tm][2]["iterations"] == r_alone[2]["iterations"]


def test_admission_respects_the_budget(goo, setup):
    ctx, spec, mc, mcds, model, theta, env = setup
    budget = 72 * 25_000 + 64 * 1024  # room for about one 20k-event toy at a time
    server = goo.Server(model, theta, envelope=env, budget_bytes=budget)
    tickets = [server.submit(n, 1710600 + i) for i, n in enumerate([20_000, 5000, 18_000, 9000])]
    peak_active = 0
    for _ in range(5000):
        q, a, d = server.step()
        peak_active = max(peak_active, a)
        assert server.stats()["arena_used"] <= budget
        if q == 0 and a == 0:
            break
    assert all(server.result(t) is not None for t in tickets)
    assert peak_active <= 2
    with pytest.raises(goo.GooError):
        server.submit(10_000_000, 1)


def _coefficient_objective(ref, spec, theta, data, G):
    """FP64 NLL and gradient over theta with the lineshapes fixed at theta: the amplitudes of
    the events and the MC Gram matrix G_kl = <A_k conj(A_l)> computed once by the oracle."""
    import torch
    with torch.no_grad():
        A = ref.amplitude_matrix(data, torch.as_tensor(theta))
    n = A.shape[0]

    def nll_grad(th):
        t = torch.tensor(np.asarray(th, np.float64), requires_grad=True)
        c = ref.coefficients(t)
        S = A @ c
        norm = (c.conj() @ (G.T @ c)).real  # mean over the MC sample of |sum_k c_k A_k|^2
        nll = -torch.log(S.real ** 2 + S.imag ** 2).sum() + n * torch.log(norm)
        (g,) = torch.autograd.grad(nll, t)
        return float(nll.detach()), g.numpy().copy()
    return nll_grad


def test_small_toys_converge_to_the_oracle_minimum(goo):
    # Toys of 1,000 to 2,700 events of the 4096-toy study (1M-point MC) on which the quasi-Newton
    # phase stopped where the likelihood is far from quadratic: its curvature estimate put the
    # EDM under the tolerance while the finite-difference Hessian gave 1.5 (toy 2007), or the
    # Hessian was indefinite (2327), or the Newton steps stalled at 1.3e-6 (2020).  The Newton
    # phase now hands such fits back to the quasi-Newton phase with that Hessian.  Served (FP32)
    # and host (FP64) fits must converge and agree with the oracle's minimum.
    ctx = goo.Context(0)
    spec = synth.c3_spec(n_mc=1_000_000)
    mc = synth.round_to_f32(synth.dalitz_candidates(1_000_000, 1710013, KIN["M"], KIN["m1"], KIN["m2"], KIN["m3"]),
                            spec)
    model = goo.Model(ctx, spec, mc=goo.Dataset.from_spec(ctx, spec, mc))
    theta = np.array(synth.param_values(spec))
    env = otoys.envelope(spec, theta)
    free = np.array([not p[2] for p in spec["params"]])
    steps = np.array([p[3] if p[3] > 0 else 1.0 for p in spec["params"]])
    idx = np.flatnonzero(free)
    sizes = synth.toy_sizes(4096)
    toys = [2007, 2020, 2327]
    server = goo.Server(model, theta, envelope=env)
    tickets = {i: server.submit(int(sizes[i]), 1710100 + i) for i in toys}
    res = _run(server, list(tickets.values()))
    ref = od.DalitzModel(spec)
    G = ref.gram(mc, theta)
    for i in toys:
        th, err, info = res[tickets[i]]
        assert info["status"] == 0, (i, info)
        a, b, _ = otoys.generate_toy(spec, theta, env, 1710100 + i, int(sizes[i]))
        data = {"s12": np.asarray(a, np.float64), "s13": np.asarray(b, np.float64)}
        rth, rerr, rnll, redm = ofit.fit(_coefficient_objective(ref, spec, theta, data, G), theta, free, steps)
        assert redm < 1e-8, (i, redm)
        assert np.all(np.abs(th[idx] - rth[idx]) / rerr[idx] < 0.01), (i, (th[idx] - rth[idx]) / rerr[idx])
        ds = goo.Dataset.from_spec(ctx, spec, data)
        hth, herr, hinfo = model.fit(ds, theta, free, steps, precision="f64", gradient="adjoint")
        assert hinfo["status"] == 0, (i, hinfo)
        assert np.all(np.abs(hth[idx] - rth[idx]) / rerr[idx] < 0.01), (i, (hth[idx] - rth[idx]) / rerr[idx])
        np.testing.assert_allclose(herr[idx], rerr[idx], rtol=0.03)
