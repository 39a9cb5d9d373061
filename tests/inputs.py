"""Seeded synthetic inputs shared by the oracle-side and the GPU-side tests.

This module holds none of the method's arithmetic: it only draws arrays of
random numbers with numpy's PCG64 generator, shaped like the paper's lattice
fields (SoA, x fastest).  Random numbers that the method itself draws (the
Fourier-mode moduli and phases of the initial conditions) do not come from
here: each side implements Philox4x32-10 from its published definition.
"""
import numpy as np


def rng(seed):
    return np.random.default_rng(seed)


def smooth_field(N, seed, amp=1.0, kmax=None, mean=0.0):
    """A real periodic N^3 field: random Fourier amplitudes up to |n~| <= kmax
    (all modes when kmax is None), normalised to rms `amp`, plus `mean`."""
    r = rng(seed)
    f = r.standard_normal((N, N, N))
    if kmax is not None:
        F = np.fft.fftn(f)
        c = np.fft.fftfreq(N) * N
        nz, ny, nx = np.meshgrid(c, c, c, indexing="ij")
        F[np.sqrt(nx ** 2 + ny ** 2 + nz ** 2) > kmax] = 0
        f = np.fft.ifftn(F).real
    f = f - f.mean()
    s = np.sqrt((f ** 2).mean())
    return mean + amp * f / (s if s > 0 else 1.0)


def fields(Ns, N, seed, amp=1.0, kmax=None, means=None):
    means = means or [0.0] * Ns
    return np.stack([smooth_field(N, seed * 101 + i, amp, kmax, means[i]) for i in range(Ns)])


def angles(N, seed, scale=0.3):
    return rng(seed).uniform(-scale, scale, size=(3, N, N, N))
