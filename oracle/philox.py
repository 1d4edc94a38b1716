"""Philox4x32-10 counter-based generator (oracle side).

Test infrastructure only: this package is the plain CPU oracle. Only tests,
``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg may use it.

Written from the published definition of Philox (Salmon, Moraes, Dror, Shaw,
"Parallel random numbers: as easy as 1, 2, 3", SC'11): a 4 x 32-bit counter and
a 2 x 32-bit key; each of the 10 rounds multiplies two counter words by the
round constants, XORs the high halves with the other two words and the key,
and the key is bumped by the Weyl constants between rounds.

The method's random draws (fixed line, per-site uniforms, Metropolis uniform)
come from this generator with the counter layout below; the GPU side
implements the same definition independently.

Counter layout for one slice update:
  ctr0 = purpose << 24 | index       (index = r * Lc + x for site draws)
  ctr1 = slice | axis << 16
  ctr2 = step                        (sweep * 4 + colour, chosen by the caller)
  ctr3 = chain
  key  = (seed & 0xffffffff, seed >> 32)
A double uniform in [0, 1) takes the top 53 bits of (o0 << 32 | o1).
"""
from __future__ import annotations

M0 = 0xD2511F53
M1 = 0xCD9E8D57
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = 0xFFFFFFFF

PURPOSE_SITE = 0
PURPOSE_FIXED_ROW = 1
PURPOSE_FIXED_COL = 2
PURPOSE_MH = 3
PURPOSE_NET_SITE = 4
# proposals j >= 1 of one environment build (proposal 0 uses PURPOSE_SITE and PURPOSE_MH): the site
# draw of proposal j has index (j - 1) * (active sites) + site, its Metropolis draw index j - 1
PURPOSE_SITE_K = 5
PURPOSE_MH_K = 6


def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: returns four 32-bit outputs."""
    c0, c1, c2, c3 = (int(v) & MASK for v in ctr)
    k0, k1 = (int(v) & MASK for v in key)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + W0) & MASK
            k1 = (k1 + W1) & MASK
        p0 = M0 * c0
        p1 = M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK
        hi1, lo1 = p1 >> 32, p1 & MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK, lo1, (hi0 ^ c3 ^ k1) & MASK, lo0
    return c0, c1, c2, c3


def uniform(seed: int, purpose: int, index: int, slice_: int, axis: int, step: int, chain: int) -> float:
    """Uniform double in [0, 1) for one draw of the method."""
    ctr = ((purpose << 24) | index, slice_ | (axis << 16), step, chain)
    key = (seed & MASK, (seed >> 32) & MASK)
    o0, o1, _, _ = philox4x32_10(ctr, key)
    return (((o0 << 32) | o1) >> 11) * (1.0 / 9007199254740992.0)
