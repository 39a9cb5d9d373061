"""Discrete Fourier transform convention and power spectra of the paper.

TEST INFRASTRUCTURE ONLY (part of the oracle).

Section 3.1 defines
    f(n~) = sum_n exp(+2 pi i n.n~/N) f(n),   f(n) = N^-3 sum_n~ exp(-2 pi i n~.n/N) f(n~),
with n~_i in (-N/2, N/2], k = k_IR n~, and the discrete power spectrum
    Delta_f(k) = k^3/(2 pi^2) (dx/N)^3 <|f(n~)|^2>_R(n~).
The shell average is read as the mean over the modes whose |n~| falls in
[b, b+1), with k_b = k_IR times the mean |n~| of the bin.
"""
import numpy as np


def mode_numbers(N):
    """Signed mode numbers n~ in (-N/2, N/2] for array index 0..N-1."""
    c = np.arange(N)
    return np.where(c <= N // 2, c, c - N)


def dft_forward(f):
    """The paper's forward transform, sum_n exp(+2 pi i n.n~/N) f(n)."""
    return np.fft.ifftn(f) * f.size


def dft_inverse(F):
    """The paper's inverse transform, N^-3 sum_n~ exp(-2 pi i n~.n/N) F(n~)."""
    return np.fft.fftn(F) / F.size


def isqrt_array(n2):
    """Exact integer square root (floor) of a non-negative integer array."""
    r = np.floor(np.sqrt(n2.astype(np.float64))).astype(np.int64)
    r = np.where((r + 1) * (r + 1) <= n2, r + 1, r)
    r = np.where(r * r > n2, r - 1, r)
    return r


def shell_bins(N):
    """Bin index floor(|n~|), |n~| and the bin count for an N^3 lattice."""
    m = mode_numbers(N)
    nz, ny, nx = np.meshgrid(m, m, m, indexing="ij")
    n2 = nx.astype(np.int64) ** 2 + ny.astype(np.int64) ** 2 + nz.astype(np.int64) ** 2
    b = isqrt_array(n2)
    return b, np.sqrt(n2.astype(np.float64)), int(b.max()) + 1


def spectrum(fields, dx, kIR):
    """Power spectrum of one real field (array N^3) or of a sum over real
    components (array (c, N, N, N); e.g. Re and Im of a complex field, or the
    components of a vector).  Returns (k_b, Delta_b, count_b) per shell."""
    f = np.asarray(fields, dtype=np.float64)
    if f.ndim == 3:
        f = f[None]
    N = f.shape[-1]
    P = np.zeros(f.shape[1:])
    for comp in f:
        P += np.abs(dft_forward(comp)) ** 2
    b, nabs, nb = shell_bins(N)
    cnt = np.bincount(b.ravel(), minlength=nb).astype(np.int64)
    sP = np.bincount(b.ravel(), weights=P.ravel(), minlength=nb)
    sn = np.bincount(b.ravel(), weights=nabs.ravel(), minlength=nb)
    k = kIR * sn / np.maximum(cnt, 1)
    Delta = k ** 3 / (2 * np.pi ** 2) * (dx / N) ** 3 * sP / np.maximum(cnt, 1)
    return k, Delta, cnt
