"""Pins of the oracle's scan observables (oracle/observe.py) against closed
forms: the equation of state of pure potential and pure kinetic energy
(section 4.4.1), the energy fraction of a single lattice mode (section 4.4),
and the k^3 spectrum of equal-power modes (section 3.1), a straight line that
the log-log interpolation must reproduce between the shells.
A wrong energy split, a dropped 1/3 in the pressure, a k_b taken as the
shell's lower edge, natural instead of decimal logarithms of Delta, or an
interpolation in linear k fails one of them."""
import math

import numpy as np

from oracle import ScalarLattice, ScalarModel
from oracle.observe import NK, log_spectrum_samples, observables
from oracle.spectra import dft_forward, dft_inverse


def _model(N, dx, q=3.0, lam=1.0):
    return ScalarModel(N=N, Ns=2, pexp=2, dx=dx, alpha=0.0, fmp2=0.0, lam=lam, q=q)


def _kj(kIR, kmax):
    return kIR * (kmax / kIR) ** ((np.arange(NK) + 0.5) / NK)


def _cos_mode(N, n, A):
    x = np.arange(N)
    z, y, xx = np.meshgrid(x, x, x, indexing="ij")
    return A * np.cos(2 * np.pi * (n[0] * xx + n[1] * y + n[2] * z) / N)


def _shell_stats(N, b):
    """Brute force over the mode numbers in (-N/2, N/2]: the count and the mean
    |n~| of the modes with b <= |n~| < b + 1."""
    r = [c if c <= N // 2 else c - N for c in range(N)]
    mags = [math.sqrt(a * a + c * c + d * d) for a in r for c in r for d in r]
    sel = [m for m in mags if b <= m < b + 1]
    return len(sel), sum(sel) / len(sel)


def test_pure_potential_and_pure_kinetic_equations_of_state():
    N, dx = 8, 0.5
    phi = np.zeros((2, N, N, N))
    phi[0] = 1.3  # homogeneous, at rest, chi = 0: rho = <V>, p = -<V>
    lat = ScalarLattice(_model(N, dx), phi, np.zeros_like(phi))
    o = observables(lat, kIR=2 * np.pi / (N * dx))
    assert o[0] == 0.0 and abs(o[1] + 1.0) < 1e-15
    pi = np.zeros((2, N, N, N))
    pi[0], pi[1] = 0.6, 0.8  # phi = chi = 0, homogeneous velocities: V = 0, p = rho
    lat = ScalarLattice(_model(N, dx), np.zeros_like(pi), pi)
    o = observables(lat, kIR=2 * np.pi / (N * dx))
    assert abs(o[1] - 1.0) < 1e-15
    assert abs(o[0] - 0.8 ** 2 / (0.6 ** 2 + 0.8 ** 2)) < 1e-15  # E_K[chi] / rho


def test_single_mode_energy_fraction_and_equation_of_state():
    """phi = phi0 at rest, chi = A cos(2 pi n.x/N): closed-form gradient and
    potential energies of one lattice mode."""
    N, dx, A, phi0, q, lam = 8, 0.7, 0.05, 1.2, 3.0, 1.0
    n = (1, 2, 0)
    kIR = 2 * np.pi / (N * dx)
    phi = np.stack([np.full((N, N, N), phi0), _cos_mode(N, n, A)])
    lat = ScalarLattice(_model(N, dx, q, lam), phi, np.zeros_like(phi))
    o = observables(lat, kIR)
    EG = sum(A * A * math.sin(math.pi * c / N) ** 2 for c in n) / dx ** 2  # sum_i <(D_i^+ chi)^2> / 2
    EV = 0.5 * lam * phi0 ** 2 + 0.5 * q * phi0 ** 2 * A * A / 2
    rho = EG + EV
    assert abs(o[0] - EG / rho) < 1e-13
    assert abs(o[1] - (-EG / 3 - EV) / rho) < 1e-13


def test_equal_power_modes_give_a_k_cubed_line():
    """chi whose Fourier modes all have one modulus c (random phases): every
    shell has Delta_b = norm c^2 k_b^3, a straight line in (ln k, log10 Delta),
    so the samples equal log10(norm c^2) + 3 log10 k_j between the first shell's
    momentum k_1 (its mean |n~|, counted by brute force) and k_max, and the first
    shell's value below k_1."""
    N, dx, c = 8, 0.6, 3.0
    kIR = 2 * np.pi / (N * dx)
    G = dft_forward(np.random.default_rng(4).standard_normal((N, N, N)))
    F = c * G / np.abs(G)
    F[0, 0, 0] = 0.0
    chi = dft_inverse(F)
    assert np.max(np.abs(chi.imag)) < 1e-12
    phi = np.stack([np.full((N, N, N), 1.0), chi.real])
    lat = ScalarLattice(_model(N, dx), phi, np.zeros_like(phi))
    kmax = 0.5 * N * kIR
    o = observables(lat, kIR, kmax)
    norm = (dx / N) ** 3 / (2 * np.pi ** 2)
    k1 = kIR * _shell_stats(N, 1)[1]
    for kj, v in zip(_kj(kIR, kmax), o[2:]):
        ref = math.log10(norm * c * c) + 3 * math.log10(max(kj, k1))
        assert abs(v - ref) < 1e-12, (kj, v, ref)


def test_zero_mode_and_empty_shells_are_skipped():
    """Shell 0 (k = 0) and a shell without power take no part: the samples
    follow the line through the two remaining shells."""
    k = np.array([0.0, 0.1, 0.2, 0.3])
    D = np.array([5.0, 1e-4, 0.0, 1e-2])
    v = log_spectrum_samples(k, D, kIR=0.1, kmax=0.3)
    kj = _kj(0.1, 0.3)
    ref = -4.0 + (np.log(kj) - math.log(0.1)) / math.log(3.0) * 2.0
    assert np.allclose(v, ref, rtol=0, atol=1e-12)


def test_default_upper_momentum_is_the_axis_nyquist_momentum():
    """Without kmax the 32 momenta end at the lattice's Nyquist momentum along an
    axis, pi/dx (beyond it the shells are incomplete corners of the cube): the
    default equals an explicit kmax = pi/dx, and with the equal-power k^3
    spectrum the last sample sits at that momentum's line value."""
    N, dx, c = 8, 0.6, 3.0
    kIR = 2 * np.pi / (N * dx)
    G = dft_forward(np.random.default_rng(5).standard_normal((N, N, N)))
    F = c * G / np.abs(G)
    F[0, 0, 0] = 0.0
    chi = dft_inverse(F).real
    phi = np.stack([np.full((N, N, N), 1.0), chi])
    lat = ScalarLattice(_model(N, dx), phi, np.zeros_like(phi))
    o_default = observables(lat, kIR)
    o_nyquist = observables(lat, kIR, math.pi / dx)
    assert np.allclose(o_default, o_nyquist, rtol=0, atol=1e-12)  # pi/dx = N k_IR/2 up to rounding
    norm = (dx / N) ** 3 / (2 * np.pi ** 2)
    k_last = _kj(kIR, math.pi / dx)[-1]
    assert abs(o_default[-1] - (math.log10(norm * c * c) + 3 * math.log10(k_last))) < 1e-12
