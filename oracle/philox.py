"""Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11), written from its
published definition.  TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper's Monte Carlo sampling (Fig. "contraction", Steps 1-3) and its
random step lengths p in (0, 1) of the GO update draw random numbers; this
generator is the one both the oracle and the CUDA path implement, each from
the definition, so that draws match bit for bit.
"""

_M0 = 0xD2511F53
_M1 = 0xCD9E8D57
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = 0xFFFFFFFF


def philox4x32_10(ctr, key):
    """One block: 4 x 32-bit counter words, 2 x 32-bit key words -> 4 words.

    Each of the 10 rounds multiplies counter words 0 and 2 by the round
    multipliers (full 64-bit products), mixes the high halves with the other
    counter words and the round key, and the key is bumped by the Weyl
    constants between rounds."""
    c0, c1, c2, c3 = (int(x) & _MASK for x in ctr)
    k0, k1 = (int(x) & _MASK for x in key)
    for r in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> 32, p0 & _MASK
        hi1, lo1 = p1 >> 32, p1 & _MASK
        c0, c1, c2, c3 = hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0
        if r < 9:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
    return c0, c1, c2, c3


def uniform53(x0, x1):
    """u in [0, 1): the top 53 bits of the 64-bit word x1:x0, times 2^-53."""
    x = (int(x1) << 32) | int(x0)
    return float(x >> 11) * (2.0 ** -53)


def uniform_open53(x0, x1):
    """p in (0, 1) open: ((x >> 12) + 1/2) * 2^-52 of the 64-bit word x1:x0.
    (With 53 bits the largest value would round to 1.0.)"""
    x = (int(x1) << 32) | int(x0)
    return (float(x >> 12) + 0.5) * (2.0 ** -52)
