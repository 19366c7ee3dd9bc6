"""Pins of the reference minimiser (oracle/fit.py): recovery of generated parameters."""
import numpy as np
import pytest

import synth
from oracle import fit as ofit
from oracle import model as om


def _fit_c1(cols):
    spec = synth.c1_spec()
    m = om.TreeModel(spec)
    truth = np.array(synth.param_values(spec))
    start = truth * 1.05
    steps = np.array([p[3] for p in spec["params"]])
    return ofit.fit(lambda t: m.nll_grad(cols, t), start, np.ones(4, bool), steps), truth


def test_c1_fit_recovers_truth_within_errors():
    (th, err, nll, edm), truth = _fit_c1(synth.gen_c1())
    pulls = (th - truth) / err
    assert np.all(np.abs(pulls) < 4.0), pulls
    assert edm < 1e-8
    assert np.all(err > 0) and err[0] < 0.02


def test_c1_pulls_over_toys():
    pulls = []
    for i in range(24):
        (th, err, _, _), truth = _fit_c1(synth.gen_c1(n=4000, seed=900 + i))
        pulls.append((th - truth) / err)
    pulls = np.array(pulls)
    # mean 0 and width 1 within generous statistical bounds for 24 toys
    assert np.all(np.abs(pulls.mean(axis=0)) < 0.8)
    assert np.all((pulls.std(axis=0) > 0.5) & (pulls.std(axis=0) < 1.6))
