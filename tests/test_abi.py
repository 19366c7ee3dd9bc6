"""The C-ABI library builds for sm_103a, loads without a GPU and exports every entry point that
include/goo.h declares; host-only calls (version, error text, the shard combiner) work on the
CPU."""
import ctypes
import math
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1710_08826_gb300 import buildlib
    path = buildlib.build()
    return ctypes.CDLL(path)


def declared_functions():
    text = open(os.path.join(ROOT, "include", "goo.h")).read()
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return sorted(set(re.findall(r"\b(goo_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for must in ("goo_init", "goo_dataset_upload", "goo_model_build", "goo_normalise", "goo_nll", "goo_nll_grad",
                 "goo_nll_partial", "goo_combine_partials", "goo_fit", "goo_server_create", "goo_nll_grad_batch",
                 "goo_nll_grad_static"):
        assert must in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_host_only_calls(lib):
    lib.goo_version.restype = ctypes.c_char_p
    assert lib.goo_version().decode()
    lib.goo_last_error.restype = ctypes.c_char_p
    # a NULL argument is rejected on the host with GOO_ERR_ARG and a message
    assert lib.goo_combine_partials(1, 0, None, None) == -1
    assert b"NULL" in lib.goo_last_error() or lib.goo_last_error()


def test_combine_partials_is_compensated_and_ordered():
    from paper_1710_08826_gb300 import goo
    P = 2
    rng = np.random.default_rng(5)
    # shard sums of very different magnitude: a naive left-to-right double sum loses bits
    parts = np.zeros((5, 3 + P))
    parts[:, 0] = [1e16, 1.0, -1e16, 3.0, 1e-3]
    parts[:, 2] = [10, 20, 30, 40, 50]
    parts[:, 3:] = rng.normal(size=(5, P))
    tot = goo.combine_partials(parts, P)
    assert tot[0] + tot[1] == pytest.approx(4.001, abs=1e-9)
    assert tot[2] == 150
    exact = [math.fsum(parts[:, 3 + j]) for j in range(P)]  # correctly rounded sums
    np.testing.assert_allclose(tot[3:], exact, rtol=4e-16, atol=0)


def test_faddeeva_approximation_against_scipy():
    from scipy.special import wofz
    from paper_1710_08826_gb300 import goo
    worst = {"f64": 0.0, "f32": 0.0}
    for re in (0.0, 1e-4, 3e-3, 0.05, 0.5, 2.0, 5.0):
        for im in np.concatenate([np.linspace(0, 10, 41), np.linspace(10, 200, 21)]):
            ref = wofz(re + 1j * im)
            for p in worst:
                worst[p] = max(worst[p], abs(goo.faddeeva(re + 1j * im, p) - ref) / abs(ref))
    assert worst["f64"] < 2e-14 and worst["f32"] < 2e-6, worst
