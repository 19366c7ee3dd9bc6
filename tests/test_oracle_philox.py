"""Pins of the oracle's Philox4x64-10 against numpy's independent Philox bit generator."""
import numpy as np
import pytest

from oracle import philox as op


@pytest.mark.parametrize("key", [0, 1, 12345, 2**64 - 1, 1710100 + (0x6F6F67 << 64), (7 << 64) + 3])
def test_blocks_match_numpy(key):
    bg = np.random.Philox(key=key, counter=0)
    raw = [int(v) for v in bg.random_raw(4 * 40)]
    k0, k1 = key & ((1 << 64) - 1), key >> 64
    for j in range(40):
        # numpy advances its 256-bit counter before producing a block: block j uses counter j+1
        assert list(op.philox4x64((j + 1, 0, 0, 0), (k0, k1))) == raw[4 * j:4 * j + 4]


def test_counter_carry_matches_numpy():
    # a counter whose low word wraps exercises the other counter words
    bg = np.random.Philox(key=99, counter=2**64 - 3)
    raw = [int(v) for v in bg.random_raw(16)]
    expect = []
    c = 2**64 - 3
    for _ in range(4):
        c += 1
        words = [(c >> (64 * i)) & ((1 << 64) - 1) for i in range(4)]
        expect += list(op.philox4x64(words, (99, 0)))
    assert expect == raw

