"""Philox4x32-10 counter-based generator, written from its published definition
(J. K. Salmon, M. A. Moraes, R. O. Dror, D. E. Shaw, "Parallel random numbers:
as easy as 1, 2, 3", SC11, 2011).

TEST INFRASTRUCTURE ONLY (part of the oracle).  The CUDA library carries its
own independent implementation of the same published generator; the two share
no code.  The initial conditions of the paper (section 7) draw Rayleigh moduli
and uniform phases per Fourier mode; both sides draw them from this generator,
keyed by the seed and counted by the mode's index, so that they can be
compared mode by mode.

One round maps (c0, c1, c2, c3) with key (k0, k1) to
    (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
with M0 = 0xD2511F53, M1 = 0xCD9E8D57; the key is bumped by the Weyl constants
W0 = 0x9E3779B9, W1 = 0xBB67AE85 between rounds; ten rounds.
"""
import numpy as np

M0 = np.uint64(0xD2511F53)
M1 = np.uint64(0xCD9E8D57)
W0 = 0x9E3779B9
W1 = 0xBB67AE85
MASK = np.uint64(0xFFFFFFFF)


def philox4x32_10(ctr, key):
    """ctr: uint32 array of shape (4, ...); key: (k0, k1) Python ints.
    Returns a uint32 array of shape (4, ...)."""
    c = [np.asarray(x, dtype=np.uint64) & MASK for x in ctr]
    k0, k1 = int(key[0]) & 0xFFFFFFFF, int(key[1]) & 0xFFFFFFFF
    for r in range(10):
        if r > 0:
            k0 = (k0 + W0) & 0xFFFFFFFF
            k1 = (k1 + W1) & 0xFFFFFFFF
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        hi0, lo0 = p0 >> np.uint64(32), p0 & MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & MASK
        c = [hi1 ^ c[1] ^ np.uint64(k0), lo1, hi0 ^ c[3] ^ np.uint64(k1), lo0]
    return np.stack([x.astype(np.uint32) for x in c])


def uniforms(lin, stream, draw, seed):
    """Four uniforms in (0, 1) per mode index `lin` (int64 array), as
    (x + 1/2) * 2^-32 of the four Philox outputs, with counter
    (lin_lo, lin_hi, stream, draw) and key (seed_lo, seed_hi)."""
    lin = np.asarray(lin, dtype=np.uint64)
    ctr = [lin & MASK, lin >> np.uint64(32),
           np.full(lin.shape, stream, dtype=np.uint64), np.full(lin.shape, draw, dtype=np.uint64)]
    out = philox4x32_10(ctr, (seed & 0xFFFFFFFF, (seed >> 32) & 0xFFFFFFFF))
    return (out.astype(np.float64) + 0.5) * 2.0 ** -32
