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


def colmap(cols, L):
    """2 bits per slot k * L + l from a list of products (lists of observable indices)."""
    out = 0
    for k, leaves in enumerate(cols):
        for l, c in enumerate(leaves):
            out |= c << (2 * (k * L + l))
    return out


@pytest.fixture(scope="module")
def lib():
    lb = ctypes.CDLL(buildlib.build())
    lb.goo_jit_check.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_ulonglong, ctypes.c_ulonglong,
                                 ctypes.POINTER(ctypes.c_int64)]
    lb.goo_jit_check.restype = ctypes.c_int
    lb.goo_last_error.restype = ctypes.c_char_p
    return lb


@pytest.mark.parametrize("K,L,grad,slots,cols", [
    (2, 3, 1, [[GAUSS, GAUSS, EXPO], [ARGUS, POLY2, EXPO]], [[0, 1, 2], [0, 1, 2]]),    # the 3-D model
    (2, 3, 0, [[GAUSS, GAUSS, EXPO], [ARGUS, POLY2, EXPO]], [[0, 1, 2], [0, 1, 2]]),
    (2, 3, 1, [[GAUSS], [EXPO]], [[0], [0]]),                                           # the 1-D model
    (2, 3, 1, [[GAUSS, EXPO, POLY2], [EXPO, POLY2]], [[0, 0, 1], [0, 1]]),              # two leaves on one observable
    (4, 4, 0, [[GAUSS, EXPO], [ARGUS], [POLY2, POLY2, EXPO, GAUSS], [EXPO]], [[0, 1], [2], [3, 1, 0, 2], [3]]),
])
def test_specialised_kernel_compiles(lib, K, L, grad, slots, cols):
    n = ctypes.c_int64(0)
    rc = lib.goo_jit_check(K, L, grad, sig(slots, L), colmap(cols, L), ctypes.byref(n))
    assert rc == 0, lib.goo_last_error().decode()
    assert n.value > 0


def test_bad_shape_is_refused(lib):
    assert lib.goo_jit_check(5, 3, 1, 0x11, 0, None) == -1
