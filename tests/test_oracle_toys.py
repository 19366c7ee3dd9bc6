"""Pins of the toy generator's oracle (oracle/toys.py): the cell choice has the envelope's
probabilities, the envelope bounds |S|^2, and accepted toys follow the model density."""
import numpy as np
import torch

import synth
from oracle import dalitz as od
from oracle import toys as ot

KIN = synth.DALITZ_MASSES


def _spec_theta():
    spec = synth.c3_spec(n_mc=1000)
    return spec, np.array(synth.param_values(spec))


def test_thresholds_partition_the_32_bit_range():
    bound = np.array([0.0, 3.0, 1.0, 0.0, 0.5, 2.5, 0.0], dtype=np.float32)
    thr = ot.thresholds(bound)
    assert thr[-1] == 1 << 32 and np.all(np.diff(thr.astype(np.int64)) >= 0)
    width = np.diff(np.concatenate([[0], thr.astype(np.int64)]))
    assert np.all(width[bound == 0] == 0)          # zero-bound cells are never chosen
    # widths are proportional to the bounds within one unit of 2^-32
    np.testing.assert_allclose(width / 2.0 ** 32, bound / bound.sum(), atol=2.0 ** -31)
    # the "first c with top < thr[c]" rule on uniform 32-bit words gives those frequencies
    top = np.random.default_rng(3).integers(0, 1 << 32, 400_000, dtype=np.uint64)
    cell = np.searchsorted(thr, top, side="right")
    counts = np.bincount(cell, minlength=bound.size)
    expect = 400_000 * bound / bound.sum()
    k = expect > 0
    assert np.all(counts[~k] == 0)
    chi2 = np.sum((counts[k] - expect[k]) ** 2 / expect[k])
    assert chi2 < 25, chi2   # 3 degrees of freedom


def _intensity(model, a, b, theta):
    A, B = torch.from_numpy(a), torch.from_numpy(b)
    ok = od.inside(A, B, model.kin)
    out = torch.zeros(A.numel(), dtype=torch.float64)
    th = torch.as_tensor(theta)
    with torch.no_grad():
        out[ok] = model.intensity(model.amplitude_matrix({"s12": A[ok], "s13": B[ok]}, th), th)
    return out.numpy(), ok.numpy()


def test_envelope_bounds_the_intensity():
    spec, theta = _spec_theta()
    model = od.DalitzModel(spec)
    lo12, hi12, lo13, hi13 = ot._box(KIN)
    rng = np.random.default_rng(11)
    for th in (theta, theta * np.where(np.arange(theta.size) % 4 >= 2, 1.15, 1.0)):
        n12, n13, bound = ot.envelope(spec, th)
        a, b = rng.uniform(lo12, hi12, 1_000_000), rng.uniform(lo13, hi13, 1_000_000)
        I, ok = _intensity(model, a, b, th)
        ci = np.minimum(((a - lo12) / ((hi12 - lo12) / n12)).astype(int), n12 - 1)
        cj = np.minimum(((b - lo13) / ((hi13 - lo13) / n13)).astype(int), n13 - 1)
        assert np.all(I[ok] <= bound.reshape(-1)[ci * n13 + cj][ok])


def test_accepted_toys_follow_the_model_density():
    # 20k accepted events against the intensity-weighted phase-space expectation in 8 x 8 bins
    spec, theta = _spec_theta()
    model = od.DalitzModel(spec)
    env = ot.envelope(spec, theta)
    a, b, idx = ot.generate_toy(spec, theta, env, 1710900, 20_000)
    assert a.size == 20_000 and np.all(np.diff(idx) > 0)
    I, ok = _intensity(model, a.astype(np.float64), b.astype(np.float64), theta)
    assert np.all(ok) and np.all(I > 0)
    lo12, hi12, lo13, hi13 = ot._box(KIN)
    rng = np.random.default_rng(12)
    ua, ub = rng.uniform(lo12, hi12, 2_000_000), rng.uniform(lo13, hi13, 2_000_000)
    w, _ = _intensity(model, ua, ub, theta)
    rng_ = [[lo12, hi12], [lo13, hi13]]
    expect = np.histogram2d(ua, ub, 8, rng_, weights=w)[0].ravel()
    expect *= a.size / expect.sum()
    counts = np.histogram2d(a, b, 8, rng_)[0].ravel()
    k = expect > 5
    assert counts[~k].sum() < 0.002 * a.size
    chi2 = np.sum((counts[k] - expect[k]) ** 2 / expect[k])
    assert chi2 / k.sum() < 1.6, (chi2, k.sum())


def test_a_misplaced_cell_grid_is_detected():
    # the same density test fails for toys whose cell rows are read in reverse s12 order, so it
    # has the power to see a wrong point placement
    spec, theta = _spec_theta()
    model = od.DalitzModel(spec)
    n12, n13, bound = ot.envelope(spec, theta, 24, 24)
    bt = bound.reshape(n12, n13)[::-1].copy()   # bounds of the reversed grid
    a, b, _ = ot.generate_toy(spec, theta, (n12, n13, bt), 1710901, 8000)
    lo12, hi12, lo13, hi13 = ot._box(KIN)
    rng = np.random.default_rng(13)
    ua, ub = rng.uniform(lo12, hi12, 1_000_000), rng.uniform(lo13, hi13, 1_000_000)
    w, _ = _intensity(model, ua, ub, theta)
    rng_ = [[lo12, hi12], [lo13, hi13]]
    expect = np.histogram2d(ua, ub, 8, rng_, weights=w)[0].ravel()
    expect *= a.size / expect.sum()
    counts = np.histogram2d(a, b, 8, rng_)[0].ravel()
    k = expect > 5
    chi2 = np.sum((counts[k] - expect[k]) ** 2 / expect[k])
    assert chi2 / k.sum() > 5, chi2
