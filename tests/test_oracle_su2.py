"""Pins of the oracle's SU(2)-Higgs sector (section 6) against the mathematics:
forces as gradients of the paper's energy functional along the group
directions, exact unit norm of the drifted links, the discrete Gauss law to
round-off, gauge invariance of the evolution, and the convergence orders of
the velocity-Verlet compositions."""
import numpy as np
import pytest

from oracle import VV2, VV4, VV6, SU2Lattice, SU2Model
from oracle.spectra import dft_forward, dft_inverse, mode_numbers
from tests import inputs


def random_quaternions(shape, seed, spread):
    """Unit quaternions exp(i spread x.sigma/2) with x standard normal."""
    r = inputs.rng(seed)
    x = spread * r.standard_normal((3,) + shape)
    th = np.sqrt((x ** 2).sum(axis=0))
    s = np.where(th > 0, np.sin(0.5 * th) / np.where(th > 0, th, 1.0), 0.5)
    return np.concatenate([np.cos(0.5 * th)[None], s * x], axis=0)


def qmul(p, q):
    """Quaternion product (p0 + i p.s)(q0 + i q.s) = (p0 q0 - p.q) + i(p0 q + q0 p - p x q).s."""
    r0 = p[0] * q[0] - (p[1:] * q[1:]).sum(axis=0)
    cross = np.stack([p[2] * q[3] - p[3] * q[2], p[3] * q[1] - p[1] * q[3], p[1] * q[2] - p[2] * q[1]])
    return np.concatenate([r0[None], p[0] * q[1:] + q[0] * p[1:] - cross], axis=0)


def qconj(q):
    return np.concatenate([q[:1], -q[1:]], axis=0)


def umul(q, f):
    """U Phi for U = q0 + i q.sigma and Phi = (f0 + i f1, f2 + i f3)."""
    A, B = q[0] + 1j * q[3], q[2] + 1j * q[1]
    Cc, D = -q[2] + 1j * q[1], q[0] - 1j * q[3]
    p1, p2 = f[0] + 1j * f[1], f[2] + 1j * f[3]
    o1, o2 = A * p1 + B * p2, Cc * p1 + D * p2
    return np.stack([o1.real, o1.imag, o2.real, o2.imag])


def random_state(N, model, seed, spread=0.6, a=1.0):
    phi = inputs.fields(4, N, seed=seed, amp=0.5, kmax=N / 3, means=[0.6, 0.1, -0.2, 0.3])
    pi = inputs.fields(4, N, seed=seed + 1, amp=0.3, kmax=N / 3)
    u = np.stack([random_quaternions((N, N, N), seed + 2 + i, spread) for i in range(3)])
    piB = np.stack([inputs.fields(3, N, seed=seed + 10 + i, amp=0.3, kmax=N / 3) for i in range(3)])
    return SU2Lattice(model, phi, pi, u, piB, a=a)


def im_sigma(x, y):
    """Im[x^dag sigma^a y] for doublets in the (Re, Im, Re, Im) layout."""
    x1, x2 = x[0] + 1j * x[1], x[2] + 1j * x[3]
    y1, y2 = y[0] + 1j * y[1], y[2] + 1j * y[3]
    return np.stack([np.imag(np.conj(x1) * y2 + np.conj(x2) * y1),
                     np.imag(np.conj(x1) * (-1j * y2) + np.conj(x2) * (1j * y1)),
                     np.imag(np.conj(x1) * y1 - np.conj(x2) * y2)])


def gauss_state(N, model, seed):
    """Unit links, random doublet with the total charge of every colour removed
    (pi -> pi - sum_a c_a i sigma^a Phi), and piB from the linear Gauss law
    sum_i D_i^- piB_i^a = (g/kappa) Im[Phi^dag sigma^a pi] solved in Fourier space."""
    phi = inputs.fields(4, N, seed=seed, amp=0.5, kmax=N / 3, means=[0.7, 0.0, 0.2, -0.1])
    pi = inputs.fields(4, N, seed=seed + 1, amp=0.3, kmax=N / 3)
    rho = im_sigma(phi, pi)
    norm = (phi ** 2).sum()
    c = rho.sum(axis=(1, 2, 3)) / norm
    # Im[Phi^dag sigma^a (i sigma^b Phi)] = delta_ab |Phi|^2: subtracting c_b i sigma^b Phi removes the charge
    P1, P2 = pi[0] + 1j * pi[1], pi[2] + 1j * pi[3]
    F1, F2 = phi[0] + 1j * phi[1], phi[2] + 1j * phi[3]
    P1 = P1 - (c[0] * 1j * F2 + c[1] * F2 + c[2] * 1j * F1)
    P2 = P2 - (c[0] * 1j * F1 - c[1] * F1 - c[2] * 1j * F2)
    pi = np.stack([P1.real, P1.imag, P2.real, P2.imag])
    rho = im_sigma(phi, pi)
    assert np.max(np.abs(rho.sum(axis=(1, 2, 3)))) < 1e-10
    m = mode_numbers(N)
    nz, ny, nx = np.meshgrid(m, m, m, indexing="ij")
    betas = [(1.0 - np.exp(2j * np.pi * cc / N)) / model.dx for cc in (nx, ny, nz)]
    den = sum(np.abs(bb) ** 2 for bb in betas)
    piB = np.zeros((3, 3, N, N, N))
    for a in range(3):
        R = dft_forward(model.g / model.kappa * rho[a])
        with np.errstate(divide="ignore", invalid="ignore"):
            for i, bb in enumerate(betas):
                piB[i, a] = dft_inverse(np.where(den > 0, np.conj(bb) * R / den, 0.0)).real
    u = np.zeros((3, 4, N, N, N))
    u[:, 0] = 1.0
    return SU2Lattice(model, phi, pi, u, piB)


@pytest.mark.parametrize("a,alpha,pot", [(1.0, 0.0, 0), (1.4, 0.5, 0), (1.4, 0.5, 1)])
def test_su2_forces_are_minus_gradient_of_paper_energies(a, alpha, pot):
    """W = a^{3+alpha} N^3 (E_G^Phi + E_V + E_G^B) from the energies of section
    6.3.1: K_Phi = -dW/dPhi* = -(1/2) dW/d(component), and K_B,i^a =
    -(g dx/kappa) dW/d eps along U_i(n) -> exp(-i eps sigma^a/2) U_i(n).
    Both potentials: Higgs and the monomial inflaton (p = 4)."""
    N = 4
    m = SU2Model(N=N, dx=0.6, alpha=alpha, fmp2=0.3, lam=1.3, v2=0.7, g=0.9, kappa=1.6, pot=pot, p=4)
    lat = random_state(N, m, 5, a=a)
    Kp, KB = lat.kernels()
    scale = a ** (3 + alpha) * N ** 3

    def W():
        E = lat.energies()
        return scale * (E[1] + E[2] + E[4])

    h = 1e-6
    for (c, z, y, x) in [(0, 1, 2, 3), (3, 0, 0, 1), (2, 3, 1, 0)]:
        lat.phi[c, z, y, x] += h
        wp = W()
        lat.phi[c, z, y, x] -= 2 * h
        wm = W()
        lat.phi[c, z, y, x] += h
        d = (wp - wm) / (2 * h)
        assert abs(Kp[c, z, y, x] + 0.5 * d) < 1e-6 * (1 + abs(d)), (c, Kp[c, z, y, x], -0.5 * d)
    for (i, ca, z, y, x) in [(0, 0, 1, 2, 3), (1, 2, 0, 3, 1), (2, 1, 2, 0, 0), (2, 0, 3, 3, 2)]:
        q0 = lat.u[i, :, z, y, x].copy()
        vals = []
        for eps in (h, -h):
            e = np.zeros(4)
            e[0] = np.cos(0.5 * eps)
            e[1 + ca] = -np.sin(0.5 * eps)
            lat.u[i, :, z, y, x] = qmul(e[:, None], q0[:, None])[:, 0]
            vals.append(W())
        lat.u[i, :, z, y, x] = q0
        d = (vals[0] - vals[1]) / (2 * h)
        assert abs(KB[i, ca, z, y, x] + m.g * m.dx / m.kappa * d) < 1e-6 * (1 + abs(d)), (i, ca, KB[i, ca, z, y, x])


def test_su2_links_stay_unitary():
    """The link drift is the exact exponential exp(-i c piB.sigma/2) U, so the
    links stay unit quaternions to round-off over many steps."""
    N = 4
    m = SU2Model(N=N, dx=0.6, alpha=0.5, fmp2=0.0, lam=1.0, v2=1.0, g=1.2, kappa=0.8)
    lat = random_state(N, m, 11, a=1.3)
    lat.vv_steps(VV4, 0.05, 30)
    norms = (lat.u ** 2).sum(axis=1)
    assert np.max(np.abs(norms - 1.0)) < 1e-13


@pytest.mark.parametrize("integ,fmp2", [("vv2", 0.0), ("vv4", 0.6)])
def test_su2_gauss_law_holds_to_round_off(integ, fmp2):
    """From a Gauss-consistent start, kicks and exact drifts keep the discrete
    Gauss law of the gauge-invariant Hamiltonian, also while expanding."""
    N = 6
    m = SU2Model(N=N, dx=0.5, alpha=0.5, fmp2=fmp2, lam=1.0, v2=1.0, g=1.1, kappa=0.9)
    lat = gauss_state(N, m, 21)
    assert lat.gauss() < 1e-28
    if fmp2 > 0:
        lat.b = np.sqrt(fmp2 / 3.0 * lat.energies().sum())
    for _ in range(4):
        lat.vv_steps({"vv2": VV2, "vv4": VV4}[integ], 0.04, 5)
        assert lat.gauss() < 1e-26, lat.gauss()
    assert np.max(np.abs(lat.u[:, 1:])) > 1e-3  # the links moved off the identity


def test_su2_gauge_invariance_of_the_evolution():
    """Phi -> Omega Phi, pi -> Omega pi, U_i(n) -> Omega(n) U_i(n) Omega^dag(n+i),
    piB_i(n) -> Omega(n) piB_i(n) Omega^dag(n) commutes with the evolution
    (SU(2) toolkit, section 3.2.3)."""
    N = 4
    m = SU2Model(N=N, dx=0.6, alpha=0.0, fmp2=0.0, lam=1.0, v2=1.0, g=0.8, kappa=1.0)
    A = random_state(N, m, 31)
    Om = random_quaternions((N, N, N), 99, 2.0)

    def transform(lat):
        phi = umul(Om, lat.phi)
        pi = umul(Om, lat.pi)
        u = np.empty_like(lat.u)
        piB = np.empty_like(lat.piB)
        for i, ax in enumerate((2, 1, 0)):
            Om_p = np.roll(Om, -1, axis=ax + 1)
            u[i] = qmul(qmul(Om, lat.u[i]), qconj(Om_p))
            e = np.concatenate([np.zeros((1, N, N, N)), lat.piB[i]], axis=0)
            piB[i] = qmul(qmul(Om, e), qconj(Om))[1:]
        return SU2Lattice(m, phi, pi, u, piB)

    B = transform(A)
    assert np.allclose(A.energies(), B.energies(), rtol=1e-12, atol=1e-14)
    A.vv_steps(VV2, 0.05, 8)
    B.vv_steps(VV2, 0.05, 8)
    TA = transform(A)
    assert np.max(np.abs(TA.phi - B.phi)) < 1e-11
    assert np.max(np.abs(TA.pi - B.pi)) < 1e-11
    assert np.max(np.abs(TA.u - B.u)) < 1e-11
    assert np.max(np.abs(TA.piB - B.piB)) < 1e-11


@pytest.mark.parametrize("integ,order", [("vv2", 2), ("vv4", 4)])
def test_su2_vv_convergence_order(integ, order):
    N, T = 4, 0.4
    m = SU2Model(N=N, dx=0.7, alpha=0.0, fmp2=0.0, lam=1.0, v2=1.0, g=1.1, kappa=0.8)
    ref = random_state(N, m, 41)
    ref.vv_steps(VV6, T / 256, 256)
    errs = []
    for k in (8, 16):
        lat = random_state(N, m, 41)
        lat.vv_steps({"vv2": VV2, "vv4": VV4}[integ], T / k, k)
        errs.append(max(np.max(np.abs(lat.phi - ref.phi)), np.max(np.abs(lat.u - ref.u)),
                        np.max(np.abs(lat.pi - ref.pi)), np.max(np.abs(lat.piB - ref.piB))))
    slope = np.log2(errs[0] / errs[1])
    assert abs(slope - order) < 0.3, (errs, slope)


def test_su2_energy_conservation_static():
    """Static background: the total energy of VV4 stays constant to O(dt^4)."""
    N = 4
    m = SU2Model(N=N, dx=0.7, alpha=0.0, fmp2=0.0, lam=1.0, v2=1.0, g=1.0, kappa=1.0)
    drift = []
    for dt in (0.04, 0.02):
        lat = random_state(N, m, 51)
        E0 = lat.energies().sum()
        lat.vv_steps(VV4, dt, int(round(0.8 / dt)))
        drift.append(abs(lat.energies().sum() - E0) / E0)
    assert drift[1] < 1e-6 and np.log2(drift[0] / drift[1]) > 3.0, drift


def test_su2_vacuum_initial_conditions_satisfy_the_gauss_law():
    """The doublet's vacuum draw has no total colour charge after the projection,
    the electric momenta solve the Gauss law with unit links to round-off, the
    magnetic energy is exactly zero and each canonical component carries the
    variance of a real scalar of its curvature (Rayleigh draws, section 7)."""
    from oracle.ic import su2_ic
    N, dx = 16, 0.5
    m = SU2Model(N=N, dx=dx, alpha=0.0, fmp2=0.0, lam=1.0, v2=1.0, g=1.2, kappa=0.8)
    phi, pi, u, piB, _ = su2_ic(m, 2 * np.pi / (N * dx), [0.4, 0.0, 0.0, 0.3], [0.0, 0.0, 0.0, 0.0], seed=3,
                                omega_over_fstar=0.3)
    lat = SU2Lattice(m, phi, pi, u, piB)
    assert lat.gauss() < 1e-28
    assert lat.energies()[4] == 0.0 and lat.energies()[3] > 0.0
    assert abs(phi[0].mean() - 0.4) < 1e-12 and abs(phi[3].mean() - 0.3) < 1e-12
    # vacuum fluctuations: a nonzero, finite spread in every component
    assert np.all(phi.reshape(4, -1).std(axis=1) > 1e-4) and np.all(np.isfinite(pi))


def test_su2_vacuum_component_is_a_scaled_singlet_draw():
    """Component 0 of the doublet fluctuates exactly like the real scalar of
    the same curvature drawn on the same Philox stream, divided by sqrt(2)
    (canonical component sqrt(2) Phi_c)."""
    from oracle import ScalarModel
    from oracle.ic import scalar_ic, su2_ic
    N, dx, lam, v2 = 8, 0.6, 1.3, 0.5
    m = SU2Model(N=N, dx=dx, alpha=0.0, fmp2=0.0, lam=lam, v2=v2, g=1.0, kappa=1.0)
    kIR = 2 * np.pi / (N * dx)
    phi, pi, _, _, _ = su2_ic(m, kIR, [0.0, 0.0, 0.0, 0.0], [0.0] * 4, seed=11, omega_over_fstar=0.2)
    m2 = 0.5 * lam * (0.0 - v2)  # curvature of component 0 at Phi = 0 (tachyonic: |m^2| enters)
    sm = ScalarModel(N=N, Ns=1, pexp=2, dx=dx, alpha=0.0, fmp2=0.0, lam=m2)
    sphi, spi, _ = scalar_ic(sm, kIR, [0.0], [0.0], seed=11, omega_over_fstar=0.2)
    assert np.max(np.abs(phi[0] - sphi[0] / np.sqrt(2.0))) < 1e-15


def test_su2_magnetic_field_of_an_abelian_configuration():
    """Links exp(-i phi_i sigma^3/2) commute, so every plaquette is
    exp(-i Phi_jk sigma^3/2) with Phi_jk the summed angles: the SU(2) magnetic
    field of section 6.3 then has only a = 3, B_i^3 = 2 sin(Phi_jk/2)/(g dx^2)
    (the curl of A for small angles); its small-field <|B|^2> is 2 a^4 E_G^B/kappa."""
    from oracle.core import _u1_magnetic
    N, g, dx = 6, 1.3, 0.7
    m = SU2Model(N=N, dx=dx, alpha=0.0, fmp2=0.0, lam=1.0, v2=1.0, g=g, kappa=0.9)
    phi_ = inputs.angles(N, 61, scale=1.2)
    u = np.zeros((3, 4, N, N, N))
    u[:, 0] = np.cos(0.5 * phi_)
    u[:, 3] = -np.sin(0.5 * phi_)
    lat = SU2Lattice(m, np.zeros((4, N, N, N)), np.zeros((4, N, N, N)), u, np.zeros((3, 3, N, N, N)))
    B = lat.magnetic()
    assert np.max(np.abs(B[:, :2])) < 1e-14
    assert np.max(np.abs(B[:, 2] - _u1_magnetic(0.5 * phi_, 0.5 * g, dx, 0))) < 1e-12
    u[:, 0] = np.cos(0.005 * phi_)
    u[:, 3] = -np.sin(0.005 * phi_)
    small = SU2Lattice(m, np.zeros((4, N, N, N)), np.zeros((4, N, N, N)), u, np.zeros((3, 3, N, N, N)))
    B2 = (small.magnetic() ** 2).sum(axis=(0, 1)).mean()
    assert B2 == pytest.approx(2 * small.energies()[4] / m.kappa, rel=1e-3)
    # non-commuting small links (every colour): to first order in the angles
    # theta_i^a = -2 q_i^a = g dx A_i^a, B_i^a is the lattice curl of each colour's
    # angles over g dx^2 (written out here with rolls); the O(theta^2) rest is ~1%
    u = np.stack([random_quaternions((N, N, N), 71 + i, 0.01) for i in range(3)])
    mixed = SU2Lattice(m, np.zeros((4, N, N, N)), np.zeros((4, N, N, N)), u, np.zeros((3, 3, N, N, N)))
    B = mixed.magnetic()
    fwd = lambda f, d: np.roll(f, -1, axis=2 - d)  # f(n + d^), arrays indexed [z, y, x]
    for a in range(3):
        th = -2.0 * u[:, a + 1]
        for i in range(3):
            j, k = (i + 1) % 3, (i + 2) % 3
            curl = (th[j] + fwd(th[k], j) - fwd(th[j], k) - th[k]) / (g * dx * dx)
            assert np.max(np.abs(B[i, a] - curl)) < 0.05 * np.max(np.abs(curl)), (i, a)
    assert (B ** 2).sum(axis=(0, 1)).mean() == pytest.approx(2 * mixed.energies()[4] / m.kappa, rel=1e-3)


@pytest.mark.parametrize("alpha", [0.0, 1.0])
def test_one_colour_electric_field_expands_like_radiation(alpha):
    """Phi = 0, unit links and a uniform electric field of one colour (sigma_3)
    in every direction: the links stay commuting, the plaquettes unity, so piB is
    constant and its energy kappa piB^2/(2 a^4) is radiation.  The Friedmann
    equations (section 4.1) give a^n linear in t, a^n - a0^n = n a0^(n-1) b0 t with
    n = 2 - alpha, and the link U_i = exp(-i Phi_i sigma_3/2) turns at the rate
    g dx piB_i a^{alpha-1} (the drift of section 6.2), so
    Phi_i(t) = g dx piB_i (a - a0)/(a0^(n-1) b0)."""
    N = 4
    m = SU2Model(N=N, dx=0.7, alpha=alpha, fmp2=3.0, lam=1.0, v2=0.0, g=0.8, kappa=1.0, pot=1, p=4)
    z4 = np.zeros((4, N, N, N))
    u = np.zeros((3, 4, N, N, N))
    u[:, 0] = 1.0
    piB = np.zeros((3, 3, N, N, N))
    c = np.array([0.3, -0.2, 0.5])
    for i in range(3):
        piB[i, 2] = c[i]
    lat = SU2Lattice(m, z4, z4, u, piB, a=1.3)
    E = lat.energies()
    assert E[3] > 0 and np.all(E[[0, 1, 2, 4]] == 0), E
    a0 = lat.a
    b0 = np.sqrt(m.fmp2 / 3.0 * a0 ** (2 * (alpha + 1)) * E.sum())
    lat.b = b0
    dt, steps = 0.02, 100
    lat.vv_steps(VV4, dt, steps)
    n = 2.0 - alpha
    a_exact = (a0 ** n + n * a0 ** (n - 1) * b0 * dt * steps) ** (1.0 / n)
    assert abs(lat.a / a_exact - 1) < 1e-8, (lat.a, a_exact)
    Phi = 2 * np.arctan2(-lat.u[:, 3, 0, 0, 0], lat.u[:, 0, 0, 0, 0])
    Phi_exact = m.g * m.dx * c * (a_exact - a0) / (a0 ** (n - 1) * b0)
    assert np.allclose(Phi, Phi_exact, rtol=1e-8, atol=0), (Phi, Phi_exact)
