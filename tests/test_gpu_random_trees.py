"""Property tests of the sum-of-products path: seeded random two-level models against the oracle.

Each case draws a model -- one to four products (or a single product, or a single leaf), each
of one to four leaves on distinct observables, leaves of every kind (Gaussian, exponential,
quadratic, Argus) in a random order, products in a random order, fractions, parameter values
and observable ranges -- and 1 to 64 events, and compares goo_nll_grad in both precisions with
the oracle's NLL and gradient.  Grid normalisation (24 bins per observable) where an Argus
leaf appears, else the analytic one.  Every fourth FP32 case runs the kernel specialised at
run time for the model's signature, the others the interpreter (NVRTC compiles take seconds).
"""
import numpy as np
import pytest

from oracle import model as om

N_CASES = 40


@pytest.fixture(scope="module")
def goo():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1710_08826_gb300 import goo as g
    return g


@pytest.fixture(scope="module")
def ctx(goo):
    return goo.Context(0)


def random_model(seed):
    """(spec, theta, columns) of a random two-level model and up to 64 events."""
    rng = np.random.default_rng(seed)
    n_obs = int(rng.integers(1, 5))
    obs = []
    for o in range(n_obs):
        lo = float(rng.uniform(0.5, 3.0))    # positive ranges: any leaf kind may sit on them
        obs.append((f"x{o}", lo, lo + float(rng.uniform(0.5, 4.0))))
    params = []

    def par(name, value):
        params.append((name, float(value), False, 0.01))
        return name

    def leaf(o, tag):
        name, lo, hi = obs[o]
        w = hi - lo
        kind = rng.choice(["gauss", "expo", "poly2", "argus"])
        if kind == "gauss":
            return ("gauss", name, par(f"mu_{tag}", rng.uniform(lo, hi)), par(f"sig_{tag}", rng.uniform(0.1, 0.8) * w))
        if kind == "expo":
            return ("expo", name, par(f"lam_{tag}", rng.uniform(-2.0, 2.0) / w))
        if kind == "poly2":
            # 1 + a1 x + a2 x^2 > 0 on [lo, hi]: small coefficients relative to the range
            s = max(abs(lo), abs(hi))
            return ("poly2", name, par(f"a1_{tag}", rng.uniform(-0.4, 0.4) / s),
                    par(f"a2_{tag}", rng.uniform(-0.2, 0.4) / s ** 2))
        # Argus: m > 0 below its endpoint
        return ("argus", name, par(f"m0_{tag}", hi + rng.uniform(0.05, 0.5) * w),
                par(f"c_{tag}", rng.uniform(-8.0, -0.5)), par(f"p_{tag}", rng.uniform(0.3, 1.2)))

    shape = rng.choice(["leaf", "prod", "add"], p=[0.1, 0.2, 0.7])
    if shape == "leaf":
        pdf = leaf(int(rng.integers(n_obs)), "0")
    else:
        K = 1 if shape == "prod" else int(rng.integers(2, 5))
        prods = []
        for k in range(K):
            m = int(rng.integers(1, n_obs + 1))
            cols = rng.permutation(n_obs)[:m]                # distinct observables, random order
            leaves = [leaf(int(o), f"{k}{j}") for j, o in enumerate(cols)]
            prods.append(("prod", leaves) if len(leaves) > 1 or rng.random() < 0.5 else leaves[0])
        if shape == "prod":
            pdf = prods[0] if prods[0][0] == "prod" else ("prod", [prods[0]])
        else:
            fr = rng.dirichlet(np.ones(K) * 2.0)[:-1] * 0.9
            pdf = ("add", [par(f"f{k}", fr[k]) for k in range(K - 1)], prods)
    argus = "'argus'" in repr(pdf)
    spec = dict(name=f"random_{seed}", observables=obs, params=params, pdf=pdf,
                norm=("grid", [24] * n_obs) if argus else ("analytic",))
    n = int(rng.integers(1, 65))
    cols = {o[0]: rng.uniform(o[1], o[2], n) for o in obs}
    theta = np.array([p[1] for p in params])
    return spec, theta, cols


def test_random_models_are_valid():
    # the generator's own invariants (checked on the CPU): distinct observables per product,
    # positive quadratics and Argus below its endpoint on every generated event
    for seed in range(N_CASES):
        spec, theta, cols = random_model(seed)
        ref = om.TreeModel(spec)
        dens = np.asarray(ref.density(cols, theta))
        assert np.all(np.isfinite(dens)) and np.all(dens > 0), seed


@pytest.mark.gpu
@pytest.mark.parametrize("seed", range(N_CASES))
@pytest.mark.parametrize("precision", ["f64", "f32"])
def test_random_model_matches_oracle(goo, ctx, seed, precision):
    import synth
    spec, theta, cols = random_model(seed)
    if precision == "f32":
        cols = synth.round_to_f32(cols, spec)
    ds = goo.Dataset.from_spec(ctx, spec, cols)
    model = goo.Model(ctx, spec)
    model.set_jit(precision == "f32" and seed % 4 == 0)
    nll, g = model.nll_grad(ds, theta, precision)
    rnll, rg = om.TreeModel(spec).nll_grad(cols, theta)
    # scale of the sums: a few events' log-densities may nearly cancel
    logf = np.log(np.asarray(om.TreeModel(spec).density(cols, theta)))
    scale = max(abs(rnll), float(np.sum(np.abs(logf))), 1.0)
    tol_nll, tol_g = (1e-9, 1e-6) if precision == "f64" else (1e-6, 1e-4)
    assert abs(nll - rnll) <= tol_nll * scale, (seed, nll, rnll)
    assert np.max(np.abs(g - rg)) <= tol_g * max(np.max(np.abs(rg)), 1.0), (seed, g, rg)
