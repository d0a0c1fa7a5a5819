"""Philox4x32-10 counter-based generator, written from its published definition.

Test infrastructure: only the tests, the smoke check and the benchmark's CPU
baseline may import this module; the CUDA path has its own implementation.

Reference: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random
numbers: as easy as 1, 2, 3", SC'11 (2011), Sec. 3 (the Philox S-P network):
a round maps (c0, c1, c2, c3) under key (k0, k1) to
    (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
with M0 = 0xD2511F53, M1 = 0xCD9E8D57, and the key is bumped by the Weyl
constants (0x9E3779B9, 0xBB67AE85) between rounds; Philox4x32-10 runs 10 rounds.

How the ILS solver maps draws onto the generator (the convention both sides
follow):
    key     = (seed & 0xffffffff, seed >> 32)
    counter = (t & 0xffffffff, t >> 32, k, chain)
for inner step ``t`` of outer iteration ``k`` of independent chain ``chain``.
One call yields two 53-bit uniforms in [0, 1): u0 from words (0, 1) and u1 from
words (2, 3), each as ((w_a >> 5) * 2**26 + (w_b >> 6)) / 2**53.
"""
from __future__ import annotations

MASK32 = 0xFFFFFFFF
M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85


def philox4x32_10(counter, key):
    """Return the four 32-bit output words for a 4-word counter and 2-word key."""
    c0, c1, c2, c3 = (int(v) & MASK32 for v in counter)
    k0, k1 = (int(v) & MASK32 for v in key)
    for rnd in range(10):
        if rnd > 0:
            k0 = (k0 + W0) & MASK32
            k1 = (k1 + W1) & MASK32
        prod0 = M0 * c0
        prod1 = M1 * c2
        hi0, lo0 = prod0 >> 32, prod0 & MASK32
        hi1, lo1 = prod1 >> 32, prod1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0), lo1, (hi0 ^ c3 ^ k1), lo0
    return c0, c1, c2, c3


def words_to_uniform(wa: int, wb: int) -> float:
    """53-bit uniform in [0, 1) from two 32-bit words (27 high bits of wa, 26 of wb)."""
    return ((wa >> 5) * 67108864 + (wb >> 6)) / 9007199254740992.0


def step_uniforms(seed: int, chain: int, k: int, t: int):
    """The two uniforms (u0, u1) drawn for inner step t of outer iteration k."""
    w = philox4x32_10((t & MASK32, (t >> 32) & MASK32, k & MASK32, chain & MASK32),
                      (seed & MASK32, (seed >> 32) & MASK32))
    return words_to_uniform(w[0], w[1]), words_to_uniform(w[2], w[3])
