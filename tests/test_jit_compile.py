"""The run-time specialised event kernel compiles for sm_103a on the CPU (goo_jit_check: the
library's own NVRTC path, without a GPU) for the leaf signatures the GPU tests use."""
import ctypes

import pytest

from paper_1710_08826_gb300 import buildlib

GAUSS, EXPO, POLY2, ARGUS = 1, 2, 3, 4


def sig(slots, L):
    """4 bits per slot k * L + l from a list of products (lists of opcodes)."""
    out = 0
    for k, leaves in enumerate(slots):
        for l, op in enumerate(leaves):
            out |= op << (4 * (k * L + l))
    return out


@pytest.fixture(scope="module")
def lib():
    lb = ctypes.CDLL(buildlib.build())
    lb.goo_jit_check.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong,
                                 ctypes.POINTER(ctypes.c_int64)]
    lb.goo_jit_check.restype = ctypes.c_int
    lb.goo_last_error.restype = ctypes.c_char_p
    return lb


@pytest.mark.parametrize("K,L,grad,slots", [
    (2, 3, 1, [[GAUSS, GAUSS, EXPO], [ARGUS, POLY2, EXPO]]),    # the 3-D model
    (2, 3, 0, [[GAUSS, GAUSS, EXPO], [ARGUS, POLY2, EXPO]]),
    (2, 3, 1, [[GAUSS], [EXPO]]),                               # the 1-D model: empty slots
    (4, 4, 0, [[GAUSS, EXPO], [ARGUS], [POLY2, POLY2, EXPO, GAUSS], [EXPO]]),
])
def test_specialised_kernel_compiles(lib, K, L, grad, slots):
    n = ctypes.c_int64(0)
    rc = lib.goo_jit_check(K, L, grad, sig(slots, L), ctypes.byref(n))
    assert rc == 0, lib.goo_last_error().decode()
    assert n.value > 0


def test_bad_shape_is_refused(lib):
    assert lib.goo_jit_check(5, 3, 1, 0x11, None) == -1
