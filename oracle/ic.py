"""Initial conditions of section 7 in program units (FP64, numpy).

TEST INFRASTRUCTURE ONLY (part of the oracle).

Scalar singlets (section 7.1): each field is a homogeneous mode plus Gaussian
vacuum fluctuations with, per Fourier mode n~ of the paper's transform,
    |dphi(n~)|^2 = (w*/f*)^2 (N/dx)^3 / (2 a^2 w_k),   w_k = sqrt(k^2 + a^2 m^2),
    dphi(n~)  = (|l| e^{i th_l} + |r| e^{i th_r}) / sqrt(2),
    dphi'(n~) = a^{alpha-1} (i w_k/sqrt(2)) (|l| e^{i th_l} - |r| e^{i th_r}) - H dphi(n~),
with Rayleigh moduli |l|, |r| (mean square the variance above) and uniform
phases.  Readings where the paper is silent: the half-space of modes with
n~_x >= 0 is drawn and the rest follows from f(-n~) = f(n~)*; modes equal to
their own conjugate take sqrt(2) Re f; the zero mode carries no fluctuation;
a tachyonic m^2 < 0 enters w_k as |m^2|; H is the program Hubble rate of the
homogeneous mode alone, and b = a' then follows from the Hubble constraint of
the full lattice.

Charged scalar and U(1) field (section 7.2): the two real components of
phi = (phi_0 + i phi_1)/sqrt(2) are drawn as above but with |l_n| = |r_n| and
th_1r = th_0r + th_1l - th_0l, which makes the total charge vanish; the links
start at unity (A = 0) and the electric momenta solve the lattice Gauss law
sum_i D_i^- piA_i = (2e/kappa) Im[phi* pi] in Fourier space with the backward
lattice momentum.

Random draws: Philox4x32-10 with key = seed and counter (mode index in the
half layout [z][y][x <= N/2], stream, draw, ...) -- see philox.py.
"""
import numpy as np

from . import philox
from .core import potential_curvature, potential_terms
from .spectra import dft_forward, dft_inverse, mode_numbers


def _half_lin(N, iz, iy, ix):
    return (iz.astype(np.int64) * N + iy) * (N // 2 + 1) + ix


def _sign_class(c, N):
    """0 for components equal to their own negative mod N (0 and N/2), +1 for
    0 < c < N/2, -1 otherwise (c is a signed mode number)."""
    return np.where((c == 0) | (c == N // 2), 0, np.where(c > 0, 1, -1))


def mode_map(N):
    """For every full-lattice mode index (z, y, x): the half-layout index of
    the mode whose draws define it, whether it is the conjugate of that mode,
    and whether it is self-conjugate."""
    idx = np.arange(N)
    iz, iy, ix = np.meshgrid(idx, idx, idx, indexing="ij")
    m = mode_numbers(N)
    sz, sy, sx = _sign_class(m[iz], N), _sign_class(m[iy], N), _sign_class(m[ix], N)
    canon = (sx > 0) | ((sx == 0) & (sy > 0)) | ((sx == 0) & (sy == 0) & (sz > 0))
    selfc = (sx == 0) & (sy == 0) & (sz == 0)
    conj = ~(canon | selfc)
    niz, niy, nix = (-iz) % N, (-iy) % N, (-ix) % N
    sz_ = np.where(conj, niz, iz)
    sy_ = np.where(conj, niy, iy)
    sx_ = np.where(conj, nix, ix)
    lin = _half_lin(N, sz_, sy_, sx_)
    kabs = np.sqrt(m[iz].astype(np.float64) ** 2 + m[iy] ** 2 + m[ix] ** 2)
    zero = (m[iz] == 0) & (m[iy] == 0) & (m[ix] == 0)
    return lin, conj, selfc, zero, kabs


def _project(G, conj, selfc, zero):
    F = np.where(conj, np.conj(G), G)
    F = np.where(selfc, np.sqrt(2.0) * G.real + 0j, F)
    return np.where(zero, 0j, F)


def _omega(k, a, m2):
    m2 = abs(m2) if m2 < 0 else m2
    return np.sqrt(k * k + a * a * m2)


def scalar_ic(model, kIR, phibar, dphibar, seed, omega_over_fstar, a=1.0, fluct_scale=1.0, fluctuations=True):
    """Fields and momenta (Ns, N, N, N) plus b = a' for the scalar model.
    phibar, dphibar: homogeneous values and program-time derivatives."""
    N, Ns = model.N, model.Ns
    dx = 2.0 * np.pi / (kIR * N)
    alpha = model.alpha
    phibar = [float(x) for x in phibar[:Ns]]
    dphibar = [float(x) for x in dphibar[:Ns]]
    # program Hubble rate of the homogeneous mode: H^2 = a^{2 alpha}/3 (f*/m_p)^2 (K + V)
    v1, v2 = potential_terms(model, np.array(phibar[0]), np.array(phibar[1]) if Ns > 1 else None)
    EK0 = sum(d * d for d in dphibar) / (2.0 * a ** (2 * alpha))
    H = np.sqrt(max(a ** (2 * alpha) / 3.0 * model.fmp2 * (EK0 + float(v1) + float(v2)), 0.0))
    m2 = potential_curvature(model, phibar)
    phi = np.zeros((Ns, N, N, N))
    pi = np.zeros((Ns, N, N, N))
    for i in range(Ns):
        dphi = np.zeros((N, N, N))
        ddphi = np.zeros((N, N, N))
        if fluctuations:
            dphi, ddphi = _singlet_draw(N, alpha, kIR, m2[i], H, seed, i, omega_over_fstar, a, fluct_scale)
        phi[i] = phibar[i] + dphi
        pi[i] = a ** (3.0 - alpha) * (dphibar[i] + ddphi)
    return phi, pi, dx


def _charged_potential(model, mod2):
    """V, dV/dmod2 and d^2V/dmod2^2 of a gauge model's charged scalar at
    mod2 = |phi|^2: (lam/4)(mod2 - v2)^2 (sections 5, 6) or the monomial
    (lam/p)(2 mod2)^(p/2) of section 8 (2 mod2 is the squared canonical norm).
    Along a canonical real component chi the curvature is dV/dmod2 + chi^2 d^2V/dmod2^2."""
    lam = model.lam
    if getattr(model, "pot", 0) == 0:
        return 0.25 * lam * (mod2 - model.v2) ** 2, 0.5 * lam * (mod2 - model.v2), 0.5 * lam
    p, S = model.p, 2.0 * mod2
    d2 = 0.0 if p == 2 else lam * (p - 2) * S ** (p / 2 - 2)
    return lam / p * S ** (p / 2), lam * S ** (p / 2 - 1), d2


def u1_ic(model, kIR, phibar, dphibar, seed, omega_over_fstar, a=1.0, fluct_scale=1.0):
    """Complex scalar (2, N, N, N) as Re/Im planes, its momentum, links
    theta = 0 and Gauss-consistent electric momenta piA (3, N, N, N)."""
    N = model.N
    dx = 2.0 * np.pi / (kIR * N)
    alpha = model.alpha
    pb = [float(phibar[0]), float(phibar[1])]
    db = [float(dphibar[0]), float(dphibar[1])]
    s = 0.5 * (pb[0] ** 2 + pb[1] ** 2)
    Vbar, dv, d2 = _charged_potential(model, s)
    m2 = [dv + d2 * pb[n] ** 2 for n in range(2)]
    EK0 = 0.5 * (db[0] ** 2 + db[1] ** 2) / a ** (2 * alpha)
    H = np.sqrt(max(a ** (2 * alpha) / 3.0 * model.fmp2 * (EK0 + Vbar), 0.0))
    lin, conj, selfc, zero, nabs = mode_map(N)
    k = kIR * nabs
    u = philox.uniforms(lin, 0, 0, seed)
    v = philox.uniforms(lin, 0, 1, seed)
    th0l, th0r, th1l = 2 * np.pi * u[2], 2 * np.pi * u[3], 2 * np.pi * v[0]
    th1r = th0r + th1l - th0l
    comps, dcomps = [], []
    for n, (thl, thr) in enumerate([(th0l, th0r), (th1l, th1r)]):
        w = _omega(k, a, m2[n])
        with np.errstate(divide="ignore", invalid="ignore"):
            T = np.where(zero, 0.0, (omega_over_fstar ** 2) * (N / dx) ** 3 / (2 * a * a * w))
        T *= fluct_scale ** 2
        A = np.sqrt(-T * np.log(u[n]))
        el, er = np.exp(1j * thl), np.exp(1j * thr)
        G = A * (el + er) / np.sqrt(2.0)
        Gd = a ** (alpha - 1.0) * (1j * w / np.sqrt(2.0)) * A * (el - er) - H * G
        comps.append(pb[n] + dft_inverse(_project(G, conj, selfc, zero)).real)
        dcomps.append(db[n] + dft_inverse(_project(Gd, conj, selfc, zero)).real)
    phi = np.stack([comps[0], comps[1]]) / np.sqrt(2.0)
    pi = a ** (3.0 - alpha) * np.stack([dcomps[0], dcomps[1]]) / np.sqrt(2.0)
    # Gauss law in Fourier space: sum_i beta_i piA_i(n~) = R(n~), beta_i = (1 - e^{2 pi i n~_i/N})/dx
    rho = phi[0] * pi[1] - phi[1] * pi[0]
    R = dft_forward(2.0 * model.e / model.kappa * rho)
    m = mode_numbers(N)
    nz, ny, nx = np.meshgrid(m, m, m, indexing="ij")
    betas = [(1.0 - np.exp(2j * np.pi * c / N)) / dx for c in (nx, ny, nz)]
    den = sum(np.abs(bb) ** 2 for bb in betas)
    with np.errstate(divide="ignore", invalid="ignore"):
        piA = np.stack([dft_inverse(np.where(den > 0, np.conj(bb) * R / den, 0.0)).real for bb in betas])
    theta = np.zeros((3, N, N, N))
    return phi, pi, theta, piA, dx


def su2_ic(model, kIR, phibar, dphibar, seed, omega_over_fstar, a=1.0, fluct_scale=1.0):
    """Higgs doublet of the SU(2) sector with vacuum fluctuations and a
    Gauss-consistent start (section 7 for the doublet, section 6 for the Gauss law).

    phibar, dphibar: the four stored components (Re Phi_1, Im Phi_1, Re Phi_2,
    Im Phi_2) of the homogeneous doublet and their program-time derivatives,
    with zero homogeneous charge.  Each canonical real component
    sqrt(2) Phi_c fluctuates like a real scalar (the singlet draws of
    scalar_ic, Philox stream c) with the potential's curvature along that
    component (Higgs: m_c^2 = (lam/2)(|Phi|^2 - v2) + lam Phi_c^2).  The total colour charges Q^a = sum_n Im[Phi^dag sigma^a pi] are
    then removed by pi -> pi - sum_a (Q^a / sum_n |Phi|^2) i sigma^a Phi (since
    Im[Phi^dag sigma^a i sigma^b Phi] = delta_ab |Phi|^2), links start at unity and
    piB solves sum_i D_i^- piB_i^a = (g/kappa) Im[Phi^dag sigma^a pi] colour by colour
    in Fourier space.  Returns (phi (4,N,N,N), pi, u (3,4,N,N,N), piB (3,3,N,N,N), dx)."""
    phi, pi, dx = _doublet_draw(model, kIR, phibar, dphibar, seed, omega_over_fstar, a, fluct_scale)
    phi, pi, piB = _su2_gauss_start(model, phi, pi, dx)
    u = np.zeros((3, 4, model.N, model.N, model.N))
    u[:, 0] = 1.0
    return phi, pi, u, piB, dx


def _doublet_draw(model, kIR, phibar, dphibar, seed, omega_over_fstar, a, fluct_scale):
    """The doublet with the vacuum fluctuations of its four canonical
    components (Philox streams 0..3), before any charge is removed."""
    N = model.N
    dx = 2.0 * np.pi / (kIR * N)
    alpha = model.alpha
    pb = [float(x) for x in phibar[:4]]
    db = [float(x) for x in dphibar[:4]]
    s2 = sum(x * x for x in pb)
    Vbar, dv, d2 = _charged_potential(model, s2)
    m2 = [dv + d2 * 2.0 * pb[c] ** 2 for c in range(4)]  # canonical component sqrt(2) Phi_c
    EK0 = sum(d * d for d in db) / a ** (2 * alpha)
    H = np.sqrt(max(a ** (2 * alpha) / 3.0 * model.fmp2 * (EK0 + Vbar), 0.0))
    lin, conj, selfc, zero, nabs = mode_map(N)
    k = kIR * nabs
    phi = np.zeros((4, N, N, N))
    pi = np.zeros((4, N, N, N))
    for c in range(4):
        w = _omega(k, a, m2[c])
        with np.errstate(divide="ignore", invalid="ignore"):
            T = np.where(zero, 0.0, (omega_over_fstar ** 2) * (N / dx) ** 3 / (2 * a * a * w))
        T *= fluct_scale ** 2
        u = philox.uniforms(lin, c, 0, seed)
        L = np.sqrt(-T * np.log(u[0]))
        R = np.sqrt(-T * np.log(u[1]))
        el = np.exp(2j * np.pi * u[2])
        er = np.exp(2j * np.pi * u[3])
        G = (L * el + R * er) / np.sqrt(2.0)
        Gd = a ** (alpha - 1.0) * (1j * w / np.sqrt(2.0)) * (L * el - R * er) - H * G
        dphi = dft_inverse(_project(G, conj, selfc, zero)).real
        ddphi = dft_inverse(_project(Gd, conj, selfc, zero)).real
        phi[c] = pb[c] + dphi / np.sqrt(2.0)
        pi[c] = a ** (3.0 - alpha) * (db[c] + ddphi / np.sqrt(2.0))
    return phi, pi, dx


def _gauss_solve(N, dx, R):
    """piX_i(n~) = conj(beta_i) R(n~) / sum_j |beta_j|^2 with beta_i =
    (1 - e^{2 pi i n~_i/N})/dx, the solution of sum_i D_i^- piX_i = rho for
    R = DFT(rho) with R(0) = 0; returns the three components in position space."""
    m = mode_numbers(N)
    nz, ny, nx = np.meshgrid(m, m, m, indexing="ij")
    betas = [(1.0 - np.exp(2j * np.pi * cc / N)) / dx for cc in (nx, ny, nz)]
    den = sum(np.abs(bb) ** 2 for bb in betas)
    with np.errstate(divide="ignore", invalid="ignore"):
        return [dft_inverse(np.where(den > 0, np.conj(bb) * R / den, 0.0)).real for bb in betas]


def _su2_gauss_start(model, phi, pi, dx):
    """Removes the total colour charges and solves the SU(2) Gauss law with unit links."""
    N = model.N
    F1, F2 = phi[0] + 1j * phi[1], phi[2] + 1j * phi[3]
    P1, P2 = pi[0] + 1j * pi[1], pi[2] + 1j * pi[3]
    rho = _su2_charge(phi, pi)
    cq = rho.sum(axis=(1, 2, 3)) / (phi ** 2).sum()
    P1 = P1 - (cq[0] * 1j * F2 + cq[1] * F2 + cq[2] * 1j * F1)
    P2 = P2 - (cq[0] * 1j * F1 - cq[1] * F1 - cq[2] * 1j * F2)
    pi = np.stack([P1.real, P1.imag, P2.real, P2.imag])
    rho = _su2_charge(phi, pi)
    # Gauss law with unit links, colour by colour
    piB = np.zeros((3, 3, N, N, N))
    for ca in range(3):
        for i, sol in enumerate(_gauss_solve(N, dx, dft_forward(model.g / model.kappa * rho[ca]))):
            piB[i, ca] = sol
    return phi, pi, piB


def _singlet_draw(N, alpha, kIR, m2, H, seed, stream, omega_over_fstar, a, fluct_scale):
    """Vacuum fluctuations of a real scalar of curvature m2 (section 7): the
    Rayleigh moduli and uniform phases of the left- and right-moving waves of
    every mode drawn on Philox stream `stream`; returns the fluctuation of the
    field and of its program-time derivative in position space."""
    dx = 2.0 * np.pi / (kIR * N)
    lin, conj, selfc, zero, nabs = mode_map(N)
    k = kIR * nabs
    w = _omega(k, a, m2)
    with np.errstate(divide="ignore", invalid="ignore"):
        T = np.where(zero, 0.0, (omega_over_fstar ** 2) * (N / dx) ** 3 / (2 * a * a * w))
    T *= fluct_scale ** 2
    u = philox.uniforms(lin, stream, 0, seed)
    L = np.sqrt(-T * np.log(u[0]))
    R = np.sqrt(-T * np.log(u[1]))
    el = np.exp(2j * np.pi * u[2])
    er = np.exp(2j * np.pi * u[3])
    G = (L * el + R * er) / np.sqrt(2.0)
    Gd = a ** (alpha - 1.0) * (1j * w / np.sqrt(2.0)) * (L * el - R * er) - H * G
    return dft_inverse(_project(G, conj, selfc, zero)).real, dft_inverse(_project(Gd, conj, selfc, zero)).real


def su2u1_ic(model, kIR, phibar, dphibar, seed, omega_over_fstar, a=1.0, fluct_scale=1.0):
    """Initial conditions of the SU(2) x U(1) doublet with a singlet (sections 7
    and 8.3), with the charge constraints of section 7.2: every canonical
    component sqrt(2) Phi_c of the doublet gets left- and right-moving waves
    of one Rayleigh modulus (|l_c| = |r_c|) and phases with a common
    difference, th_c^r = th_0^r + th_c^l - th_0^l, so that the zero modes of the
    U(1) and the three SU(2) charges vanish mode by mode.  That cancellation
    needs one frequency for all four components: they are drawn with the mean
    of the four curvatures (each component's own when the homogeneous value is
    split evenly over the components).  Draws: moduli from Philox counter
    (mode, 0, 0), phases th_0^l, th_0^r, th_1^l, th_2^l from (mode, 0, 1) and th_3^l
    from (mode, 0, 2).  The singlet chi (model.chi) has zero homogeneous mode
    and velocity and the real-scalar fluctuations of curvature 2 q |Phi|^2
    (Philox stream 4).  Links start at unity and angles at zero; piB and piA
    solve the two Gauss laws in Fourier space.  Returns (phi, pi, u, piB,
    theta, piA, chi, pchi, dx)."""
    N = model.N
    dx = 2.0 * np.pi / (kIR * N)
    alpha = model.alpha
    pb = [float(x) for x in phibar[:4]]
    db = [float(x) for x in dphibar[:4]]
    s2 = sum(x * x for x in pb)
    Vbar, dv, d2 = _charged_potential(model, s2)
    m2 = float(np.mean([dv + d2 * 2.0 * pb[c] ** 2 for c in range(4)]))
    EK0 = sum(d * d for d in db) / a ** (2 * alpha)
    H = np.sqrt(max(a ** (2 * alpha) / 3.0 * model.fmp2 * (EK0 + Vbar), 0.0))
    lin, conj, selfc, zero, nabs = mode_map(N)
    k = kIR * nabs
    w = _omega(k, a, m2)
    with np.errstate(divide="ignore", invalid="ignore"):
        T = np.where(zero, 0.0, (omega_over_fstar ** 2) * (N / dx) ** 3 / (2 * a * a * w))
    T *= fluct_scale ** 2
    u = philox.uniforms(lin, 0, 0, seed)
    v = philox.uniforms(lin, 0, 1, seed)
    x = philox.uniforms(lin, 0, 2, seed)
    thl = [2 * np.pi * v[0], 2 * np.pi * v[2], 2 * np.pi * v[3], 2 * np.pi * x[0]]
    th0r = 2 * np.pi * v[1]
    phi = np.zeros((4, N, N, N))
    pi = np.zeros((4, N, N, N))
    for c in range(4):
        A = np.sqrt(-T * np.log(u[c]))
        el, er = np.exp(1j * thl[c]), np.exp(1j * (th0r + thl[c] - thl[0]))
        G = A * (el + er) / np.sqrt(2.0)
        Gd = a ** (alpha - 1.0) * (1j * w / np.sqrt(2.0)) * A * (el - er) - H * G
        phi[c] = pb[c] + dft_inverse(_project(G, conj, selfc, zero)).real / np.sqrt(2.0)
        pi[c] = a ** (3.0 - alpha) * (db[c] + dft_inverse(_project(Gd, conj, selfc, zero)).real / np.sqrt(2.0))
    chi = np.zeros((N, N, N))
    pchi = np.zeros((N, N, N))
    if model.chi:
        chi, dchi = _singlet_draw(N, alpha, kIR, 2.0 * model.q * s2, H, seed, 4, omega_over_fstar, a, fluct_scale)
        pchi = a ** (3.0 - alpha) * dchi
    rho = _su2_charge(phi, pi)
    piB = np.zeros((3, 3, N, N, N))
    for ca in range(3):
        for i, sol in enumerate(_gauss_solve(N, dx, dft_forward(model.g / model.kappa * rho[ca]))):
            piB[i, ca] = sol
    piA = np.zeros((3, N, N, N))
    if model.eA != 0.0:
        rho0 = phi[0] * pi[1] - phi[1] * pi[0] + phi[2] * pi[3] - phi[3] * pi[2]  # Im[Phi^dag pi]
        piA = np.stack(_gauss_solve(N, dx, dft_forward(2.0 * model.eA / model.kappa * rho0)))
    u = np.zeros((3, 4, N, N, N))
    u[:, 0] = 1.0
    return phi, pi, u, piB, np.zeros((3, N, N, N)), piA, chi, pchi, dx


def _su2_charge(phi, pi):
    """Im[Phi^dag sigma^a pi], a = 1..3, for doublets in the (Re, Im, Re, Im) layout."""
    x1, x2 = phi[0] + 1j * phi[1], phi[2] + 1j * phi[3]
    y1, y2 = pi[0] + 1j * pi[1], pi[2] + 1j * pi[3]
    return np.stack([np.imag(np.conj(x1) * y2 + np.conj(x2) * y1),
                     np.imag(np.conj(x1) * (-1j * y2) + np.conj(x2) * (1j * y1)),
                     np.imag(np.conj(x1) * y1 - np.conj(x2) * y2)])
