"""Host-side logic of the Python binding and of the server's finished-ticket call, without a
GPU: argument checks of goo_server_finished in the library, the binding's draining loop
(against a stand-in for the library call) and the model's argument buffer."""
import ctypes

import numpy as np
import pytest


@pytest.fixture(scope="module")
def goo():
    from paper_1710_08826_gb300 import buildlib
    buildlib.build()  # the binding loads the library at import
    from paper_1710_08826_gb300 import goo as g
    return g


def test_server_finished_rejects_bad_arguments(goo):
    n = ctypes.c_int(-5)
    buf = (ctypes.c_int64 * 4)()
    # NULL server, NULL count, negative capacity, NULL array with a positive capacity
    assert goo.lib.goo_server_finished(None, buf, 4, ctypes.byref(n)) == goo.GOO_ERR_ARG
    assert goo.lib.goo_server_finished(ctypes.c_void_p(8), buf, 4, None) == goo.GOO_ERR_ARG
    assert goo.lib.goo_server_finished(ctypes.c_void_p(8), buf, -1, ctypes.byref(n)) == goo.GOO_ERR_ARG
    assert goo.lib.goo_server_finished(ctypes.c_void_p(8), None, 4, ctypes.byref(n)) == goo.GOO_ERR_ARG
    assert n.value == -5  # nothing written on a refused call


def test_finished_drains_in_chunks(goo, monkeypatch):
    pending = list(range(101, 101 + 2500))
    calls = []

    def fake_finished(handle, tickets, cap, n):
        k = min(cap, len(pending))
        for i in range(k):
            tickets[i] = pending.pop(0)
        ctypes.cast(n, ctypes.POINTER(ctypes.c_int))[0] = k
        calls.append(k)
        return goo.GOO_OK

    monkeypatch.setattr(goo.lib, "goo_server_finished", fake_finished)
    server = object.__new__(goo.Server)
    server.handle = None
    got = server.finished(cap=1024)
    assert got == list(range(101, 101 + 2500))  # oldest first, each once
    assert calls == [1024, 1024, 452]           # a short chunk ends the loop
    assert server.finished(cap=1024) == [] and calls[-1] == 0


def test_finished_of_exactly_one_chunk_asks_again(goo, monkeypatch):
    pending = list(range(7, 7 + 16))
    calls = []

    def fake_finished(handle, tickets, cap, n):
        k = min(cap, len(pending))
        for i in range(k):
            tickets[i] = pending.pop(0)
        ctypes.cast(n, ctypes.POINTER(ctypes.c_int))[0] = k
        calls.append(k)
        return goo.GOO_OK

    monkeypatch.setattr(goo.lib, "goo_server_finished", fake_finished)
    server = object.__new__(goo.Server)
    server.handle = None
    assert server.finished(cap=16) == list(range(7, 23))
    assert calls == [16, 0]


def test_model_argument_buffer(goo):
    model = object.__new__(goo.Model)
    model.handle = None
    model.n_params = 3
    model._tb = np.zeros(3)
    model._tb_a = model._tb.ctypes.data
    theta = np.array([1.5, -2.0, 3.25])
    assert model._theta_addr(theta) == model._tb.ctypes.data
    np.testing.assert_array_equal(model._tb, theta)
    model._theta_addr([4, 5, 6])  # any sequence of the right length
    np.testing.assert_array_equal(model._tb, [4.0, 5.0, 6.0])
    with pytest.raises(ValueError):
        model._theta_addr([1.0, 2.0])
    with pytest.raises(ValueError):
        model._theta_addr(np.ones(4))
