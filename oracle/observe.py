"""Scan observables of the two-field preheating model, composed from the
oracle's energies and spectra.

TEST INFRASTRUCTURE ONLY (part of the oracle).

The paper defines the quantities (section 4.4: volume-averaged energies and
the equation of state; section 3.1: the power spectrum); the selection of 34
numbers per lattice is a reading of a parameter-scan workload, not the paper's:
  - the daughter-field fraction eps_chi = (E_K[chi] + E_G[chi]) / rho, the
    kinetic plus gradient energy of chi over the total energy density
    rho = E_K + E_G + E_V (chi's potential energy is shared with phi through
    the interaction term, so it is not attributed to either field);
  - the equation of state w = p / rho with p = E_K - E_G/3 - E_V (section 4.4.1);
  - log10 of the chi power spectrum at 32 momenta spaced evenly in log k,
    k_j = k_IR (k_max/k_IR)^((j + 1/2)/32), j = 0..31, read off the shell
    spectrum (shells |n~| in [b, b+1), b >= 1, with non-zero power) by linear
    interpolation in (log k, log10 Delta), and held at the first or last
    shell's value outside the shells' range.
"""
import numpy as np

from .spectra import spectrum

OBS_SIZE = 34
NK = 32


def log_spectrum_samples(k, Delta, kIR, kmax):
    """log10 Delta at the NK momenta k_j from shell values (k_b, Delta_b):
    shell 0 (the zero mode) and shells without power are left out."""
    k = np.asarray(k, dtype=np.float64)
    Delta = np.asarray(Delta, dtype=np.float64)
    keep = (np.arange(k.size) >= 1) & (Delta > 0)
    lk = np.log(k[keep])
    lD = np.log10(Delta[keep])
    kj = np.exp(np.log(kIR) + (np.arange(NK) + 0.5) / NK * (np.log(kmax) - np.log(kIR)))
    if lk.size == 0:
        return np.full(NK, np.nan)
    return np.interp(np.log(kj), lk, lD)  # linear between shells, held constant outside


def observables(lattice, kIR, kmax=None):
    """The OBS_SIZE observables of a synchronized two-field ScalarLattice.
    kmax defaults to N k_IR / 2, the Nyquist momentum along an axis."""
    m = lattice.m
    if kmax is None or kmax <= 0:
        kmax = 0.5 * m.N * kIR
    E = lattice.energies()  # E_K[phi], E_K[chi], E_G[phi], E_G[chi], E_V terms
    EK, EG, EV = E[0] + E[1], E[2] + E[3], E[4] + E[5]
    rho = EK + EG + EV
    out = np.zeros(OBS_SIZE)
    out[0] = (E[1] + E[3]) / rho
    out[1] = (EK - EG / 3.0 - EV) / rho
    k, D, _ = spectrum(lattice.phi[1], m.dx, kIR)
    out[2:] = log_spectrum_samples(k, D, kIR, kmax)
    return out
