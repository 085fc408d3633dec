"""Philox4x32-10, the counter-based generator both sides draw from.

Published definition: J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11.  One round maps the
counter (c0, c1, c2, c3) with key (k0, k1) to
    (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0)),
with M0 = 0xD2511F53 and M1 = 0xCD9E8D57, and the key is bumped by the Weyl
constants (0x9E3779B9, 0xBB67AE85) between rounds; ten rounds.

The paper draws Monte Carlo samples (Sec. III) but names no generator; the
stream layout used here is this implementation's contract:
  key      = (seed mod 2^32, seed div 2^32)
  counter  = (walker, step mod 2^32, step div 2^32, 0)
  one call yields two proposals: words (0, 1) for the even one, (2, 3) for
  the odd one; the first word of a pair picks the bond, the second is the
  acceptance uniform.
"""

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Vectorised Philox4x32-10.  Arguments are integer arrays (or scalars)
    holding 32-bit values; returns four uint64 arrays holding 32-bit words."""
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in (c0, c1, c2, c3))
    k0 = int(k0) & 0xFFFFFFFF
    k1 = int(k1) & 0xFFFFFFFF
    for _ in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ np.uint64(k0), lo1, hi0 ^ c3 ^ np.uint64(k1), lo0)
        k0 = (k0 + _W0) & 0xFFFFFFFF
        k1 = (k1 + _W1) & 0xFFFFFFFF
    return c0, c1, c2, c3


def proposal_words(seed, step, walkers):
    """The four Philox words for call index `step` of every walker in `walkers`."""
    step = int(step)
    return philox4x32_10(walkers, step & 0xFFFFFFFF, step >> 32, 0,
                         seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF)


def bond_index(word, n_bonds):
    """Map a 32-bit word to a bond in [0, n_bonds): floor(word * n_bonds / 2^32)."""
    return ((np.asarray(word, dtype=np.uint64) * np.uint64(n_bonds)) >> np.uint64(32)).astype(np.int64)


def uniform(word):
    """Map a 32-bit word to the open interval (0, 1): ((word >> 9) + 1/2) / 2^23.

    Exact in float32 and float64, so both precisions see the same number."""
    return ((np.asarray(word, dtype=np.uint64) >> np.uint64(9)).astype(np.float64) + 0.5) * 2.0 ** -23
