"""Philox4x64-10 counter-based random numbers (Salmon, Moraes, Dror, Shaw, SC'11).

One call maps a 256-bit counter (four 64-bit words) and a 128-bit key (two words) to four
64-bit outputs through ten rounds of: two 64x64->128-bit multiplications by the round
multipliers, an exchange/xor of the words with the key, and a key bump by the Weyl
constants.  Written here from that published definition in plain Python integers; pinned in
tests/test_oracle_philox.py against numpy's independent Philox bit generator.

The toy generator's streams: event candidate j of a toy with seed s uses
counter (j, 0, 0, 0) and key (s, 0x6f6f67); the first output picks an envelope cell and the
other three give the point in the cell and the acceptance uniform (oracle/toys.py).
"""
M0 = 0xD2E7470EE14C6C93
M1 = 0xCA5A826395121157
W0 = 0x9E3779B97F4A7C15
W1 = 0xBB67AE8584CAA73B
MASK = (1 << 64) - 1
TOY_KEY1 = 0x6F6F67


def _mulhilo(a, b):
    p = a * b
    return p >> 64, p & MASK


def philox4x64(counter, key, rounds=10):
    c0, c1, c2, c3 = (int(v) & MASK for v in counter)
    k0, k1 = (int(v) & MASK for v in key)
    for r in range(rounds):
        if r:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        hi0, lo0 = _mulhilo(M0, c0)
        hi1, lo1 = _mulhilo(M1, c2)
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
    return c0, c1, c2, c3

