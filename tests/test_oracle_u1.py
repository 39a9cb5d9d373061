"""Pins of the oracle's compact U(1) sector (section 5.3) against the
mathematics: forces as gradients of the paper's energy functional, the Gauss
law to round-off, gauge invariance, energy conservation and B = 0 at start."""
import numpy as np
import pytest

from oracle import VV4, U1Lattice, U1Model
from oracle.ic import u1_ic
from tests import inputs


def _random_state(N, seed, model, a=1.0):
    phi = inputs.fields(2, N, seed=seed, amp=0.7, means=[0.5, -0.2])
    pi = inputs.fields(2, N, seed=seed + 1, amp=0.4)
    th = inputs.angles(N, seed + 2, scale=2.5)
    piA = inputs.fields(3, N, seed=seed + 3, amp=0.3)
    return U1Lattice(model, phi, pi, th, piA, a=a)


@pytest.mark.parametrize("a,alpha,pot,p,nc", [(1.0, 0.0, 0, 4, 0), (1.3, 0.5, 0, 4, 0), (1.3, 0.5, 1, 4, 0),
                                              (0.8, 1.0, 1, 6, 0), (1.3, 0.5, 0, 4, 1)])
def test_u1_forces_are_minus_gradient_of_paper_energies(a, alpha, pot, p, nc):
    """U = a^{3+alpha} N^3 (E_G^phi + E_V + E_G^A) from the energies of section
    5.4.1; then K_phi = -dU/dphi* = -(1/2)(dU/dRe + i dU/dIm) and
    K_A,i = -(e dx/kappa) dU/dtheta_i (theta_i = e dx A_i). Both potentials:
    Abelian-Higgs and the monomial inflaton; compact and (nc = 1) non-compact
    gauge kinetics (section 5.2)."""
    N = 5
    m = U1Model(N=N, dx=0.55, alpha=alpha, fmp2=0.7, lam=1.3, v2=0.8, e=0.9, kappa=1.7, pot=pot, p=p, noncompact=nc)
    lat = _random_state(N, 7, m, a=a)
    Kp, KA = lat.kernels()
    scale = a ** (3 + alpha) * N ** 3
    eps = 1e-6

    def U():
        E = lat.energies()
        return scale * (E[1] + E[2] + E[4])

    for (c, z, y, x) in [(0, 1, 2, 3), (1, 4, 0, 2), (0, 0, 4, 4)]:
        lat.phi[c, z, y, x] += eps
        up = U()
        lat.phi[c, z, y, x] -= 2 * eps
        um = U()
        lat.phi[c, z, y, x] += eps
        d = (up - um) / (2 * eps)
        assert abs(Kp[c, z, y, x] + 0.5 * d) < 1e-6 * (abs(d) + 1)
    for (i, z, y, x) in [(0, 1, 2, 3), (1, 4, 0, 2), (2, 0, 4, 4), (2, 3, 3, 1)]:
        lat.theta[i, z, y, x] += eps
        up = U()
        lat.theta[i, z, y, x] -= 2 * eps
        um = U()
        lat.theta[i, z, y, x] += eps
        d = (up - um) / (2 * eps)
        assert abs(KA[i, z, y, x] + m.e * m.dx / m.kappa * d) < 1e-6 * (abs(d) + 1)


def test_u1_drift_rates_match_kinetic_energies():
    """In a background with a fixed at a != 1 (f*/m_p = 0), one leapfrog step
    drifts phi by dt d(a^{3+alpha}N^3 E_K^phi)/dpi* and theta_i by
    (e dx/kappa) dt d(a^{3+alpha}N^3 E_K^A)/dpiA_i."""
    N, a, alpha, dt = 4, 1.6, 0.5, 0.01
    m = U1Model(N=N, dx=0.5, alpha=alpha, fmp2=0.0, lam=1.0, v2=1.0, e=1.1, kappa=0.6)
    lat = _random_state(N, 17, m, a=a)
    lat.EKm = (0.0, 0.0)
    phi0, th0 = lat.phi.copy(), lat.theta.copy()
    lat.lf_steps(dt, 1)
    # kinetic parts of a^{3+alpha} N^3 E: a^{alpha-3} sum |pi|^2 and a^{alpha-1} kappa sum piA^2 / 2
    dphi_rate = a ** (alpha - 3) * lat.pi           # d/dpi* of a^{alpha-3} |pi|^2
    dth_rate = m.e * m.dx / m.kappa * a ** (alpha - 1) * m.kappa * lat.piA
    assert np.allclose((lat.phi - phi0) / dt, dphi_rate, rtol=1e-12, atol=1e-12)
    assert np.allclose((lat.theta - th0) / dt, dth_rate, rtol=1e-12, atol=1e-12)
    assert lat.a == a


@pytest.mark.parametrize("fmp2,alpha,nc", [(0.0, 0.0, 0), (0.5, 0.5, 0), (0.5, 0.5, 1)])
def test_gauss_law_holds_to_round_off(fmp2, alpha, nc):
    """Starting from the Gauss-consistent initial condition of section 7.2, the
    compact (and the non-compact) leapfrog keeps the discrete Gauss law to
    machine precision."""
    N, dt = 8, 0.05
    m = U1Model(N=N, dx=0.5, alpha=alpha, fmp2=fmp2, lam=1.0, v2=1.0, e=1.0, kappa=1.0, noncompact=nc)
    kIR = 2 * np.pi / (N * 0.5)
    phi, pi, th, piA, dx = u1_ic(m, kIR, [0.0, 0.0], [0.0, 0.0], seed=5, omega_over_fstar=1.0)
    lat = U1Lattice(m, phi, pi, th, piA)
    assert lat.gauss() < 1e-14
    if fmp2 > 0:
        E = lat.energies()
        lat.b = np.sqrt(fmp2 / 3.0 * E.sum())
    lat.lf_prepare(dt)
    for _ in range(5):
        lat.lf_steps(dt, 10)
        assert lat.gauss() < 1e-13
    assert np.max(np.abs(lat.theta)) > 1e-3  # the links did move


def test_initial_magnetic_energy_is_exactly_zero():
    N = 8
    m = U1Model(N=N, dx=0.5, alpha=0.0, fmp2=0.0)
    phi, pi, th, piA, dx = u1_ic(m, 2 * np.pi / 4.0, [0.0, 0.0], [0.0, 0.0], seed=9, omega_over_fstar=1.0)
    E = U1Lattice(m, phi, pi, th, piA).energies()
    assert E[4] == 0.0 and E[3] > 0.0


def test_u1_energy_conservation_second_order():
    """Static background: with E_K averaged over the two half steps, the total
    energy of the compact leapfrog is conserved up to O(dt^2)."""
    N, T = 6, 1.0
    drift = []
    for dt in (0.04, 0.02):
        m = U1Model(N=N, dx=0.6, alpha=0.0, fmp2=0.0, lam=1.0, v2=1.0, e=1.3, kappa=0.8)
        lat = _random_state(N, 27, m)
        E0 = lat.energies().sum()
        lat.lf_prepare(dt)
        lat.lf_steps(dt, int(round(T / dt)))
        # after n steps the state is (phi_n, pi_{n-1/2}); a forward half kick
        # synchronizes the momenta with the fields
        E = lat.energies()
        Kp, KA = lat.kernels()
        pis = lat.pi + 0.5 * dt * Kp
        pas = lat.piA + 0.5 * dt * KA
        EKs = (pis ** 2).sum() / N ** 3 + m.kappa * (pas ** 2).sum() / (2 * N ** 3)
        drift.append(abs(EKs + E[1] + E[2] + E[4] - E0) / E0)
    slope = np.log2(drift[0] / drift[1])
    assert abs(slope - 2) < 0.3, (drift, slope)


@pytest.mark.parametrize("nc", [0, 1])
def test_gauge_invariance_of_the_evolution(nc):
    """phi -> e^{-i e alpha} phi, pi -> e^{-i e alpha} pi,
    theta_i -> theta_i - e (alpha(n+i) - alpha(n)) commutes with the leapfrog
    (U(1) toolkit, section 3.2.2), compact and non-compact."""
    N, dt = 6, 0.05
    m = U1Model(N=N, dx=0.6, alpha=0.0, fmp2=0.0, lam=1.0, v2=1.0, e=0.8, kappa=1.0, noncompact=nc)
    A = _random_state(N, 37, m)
    al = inputs.rng(99).uniform(-2, 2, size=(N, N, N))

    def transform(lat):
        ph = np.exp(-1j * m.e * al)
        c = (lat.phi[0] + 1j * lat.phi[1]) * ph
        p = (lat.pi[0] + 1j * lat.pi[1]) * ph
        th = lat.theta.copy()
        for i, ax in enumerate((2, 1, 0)):
            th[i] -= m.e * (np.roll(al, -1, axis=ax) - al)
        return U1Lattice(m, np.stack([c.real, c.imag]), np.stack([p.real, p.imag]), th, lat.piA)

    B = transform(A)
    assert np.allclose(A.energies(), B.energies(), rtol=1e-12)
    A.lf_prepare(dt)
    B.lf_prepare(dt)
    A.lf_steps(dt, 10)
    B.lf_steps(dt, 10)
    TA = transform(A)
    assert np.max(np.abs(TA.phi - B.phi)) < 1e-11
    assert np.max(np.abs(TA.pi - B.pi)) < 1e-11
    dth = np.angle(np.exp(1j * (TA.theta - B.theta)))
    assert np.max(np.abs(dth)) < 1e-11
    assert np.max(np.abs(TA.piA - B.piA)) < 1e-11


def _vv(name):
    from oracle import core
    return {"vv2": core.VV2, "vv4": core.VV4, "vv6": core.VV6}[name]


def test_u1_vv2_positions_equal_leapfrog_static():
    """Static background: VV2 (half kick, drift, half kick) composed over n
    steps is the staggered leapfrog started with a half kick, so fields and
    links agree to round-off and the leapfrog momenta, advanced half a step,
    are VV2's (section 5.3.1 vs 5.3.2)."""
    N, dt, n = 5, 0.03, 12
    m = U1Model(N=N, dx=0.6, alpha=0.0, fmp2=0.0, lam=1.0, v2=1.0, e=1.2, kappa=0.9)
    A = _random_state(N, 41, m)
    B = _random_state(N, 41, m)
    A.vv_steps(_vv("vv2"), dt, n)
    B.lf_prepare(dt)
    B.lf_steps(dt, n)
    assert np.max(np.abs(A.phi - B.phi)) < 1e-12
    assert np.max(np.abs(A.theta - B.theta)) < 1e-12
    Kp, KA = B.kernels()
    assert np.max(np.abs(A.pi - (B.pi + 0.5 * dt * Kp))) < 1e-12
    assert np.max(np.abs(A.piA - (B.piA + 0.5 * dt * KA))) < 1e-12


@pytest.mark.parametrize("integ", ["vv2", "vv4"])
def test_u1_vv_keeps_gauss_law(integ):
    """Kicks and drifts of the compact VVn each keep the discrete Gauss law, so
    the composed step does too, also in an expanding background."""
    N, dt = 8, 0.04
    m = U1Model(N=N, dx=0.5, alpha=0.5, fmp2=0.5, lam=1.0, v2=1.0, e=1.0, kappa=1.0)
    phi, pi, th, piA, _ = u1_ic(m, 2 * np.pi / (N * 0.5), [0.0, 0.0], [0.0, 0.0], seed=6, omega_over_fstar=1.0)
    lat = U1Lattice(m, phi, pi, th, piA)
    lat.b = np.sqrt(0.5 / 3.0 * lat.energies().sum())
    for _ in range(4):
        lat.vv_steps(_vv(integ), dt, 5)
        assert lat.gauss() < 1e-13
    assert lat.a > 1.0


@pytest.mark.parametrize("integ,order", [("vv2", 2), ("vv4", 4)])
def test_u1_vv_convergence_order(integ, order):
    """Global error after a fixed time against a VV6 solution at a small step:
    slope 2 for VV2 and 4 for VV4 (sections 4.3.2, 5.3.3)."""
    N, T = 4, 0.4
    m = U1Model(N=N, dx=0.7, alpha=0.0, fmp2=0.0, lam=1.0, v2=1.0, e=1.1, kappa=0.8)
    ref = _random_state(N, 53, m)
    ref.vv_steps(_vv("vv6"), T / 256, 256)
    errs = []
    for k in (8, 16):
        lat = _random_state(N, 53, m)
        lat.vv_steps(_vv(integ), T / k, k)
        errs.append(max(np.max(np.abs(lat.phi - ref.phi)), np.max(np.abs(lat.theta - ref.theta)),
                        np.max(np.abs(lat.pi - ref.pi)), np.max(np.abs(lat.piA - ref.piA))))
    slope = np.log2(errs[0] / errs[1])
    assert abs(slope - order) < 0.3, (errs, slope)


def test_u1_vv4_is_time_reversible_with_expansion():
    """The composed step is symmetric: n steps forward and n steps with -dt
    return the fields, links, momenta, a and b (expanding background)."""
    N, dt, n = 5, 0.02, 10
    m = U1Model(N=N, dx=0.6, alpha=0.5, fmp2=0.8, lam=1.0, v2=1.0, e=1.0, kappa=1.0)
    lat = _random_state(N, 61, m)
    lat.b = np.sqrt(0.8 / 3.0 * lat.energies().sum())
    s0 = (lat.phi.copy(), lat.pi.copy(), lat.theta.copy(), lat.piA.copy(), lat.a, lat.b)
    lat.vv_steps(_vv("vv4"), dt, n)
    assert lat.a > 1.0 + 1e-3
    lat.vv_steps(_vv("vv4"), -dt, n)
    for x, y in zip((lat.phi, lat.pi, lat.theta, lat.piA), s0[:4]):
        assert np.max(np.abs(x - y)) < 1e-11
    assert abs(lat.a - s0[4]) < 1e-13 and abs(lat.b - s0[5]) < 1e-12


@pytest.mark.parametrize("p", [2, 4])
def test_u1_monomial_homogeneous_oscillation_period(p):
    """A homogeneous real phi = chi/sqrt(2) in V = (lam/p)(2|phi|^2)^(p/2) with
    a = 1 fixed obeys chi'' = -lam chi^(p-1): for p = 2 a harmonic oscillation
    of period 2 pi/sqrt(lam); for p = 4 the quartic oscillator, whose period is
    4 sqrt(2) I/(chi0 sqrt(lam)) with I = int_0^1 du/sqrt(1 - u^4) =
    Gamma(1/4)^2/(4 sqrt(2 pi)). After one period the field is back at its
    start (the oracle's VV10 at a fine step)."""
    from math import gamma, pi, sqrt
    from oracle import VV10
    N, lam, chi0 = 4, 1.7, 1.3
    m = U1Model(N=N, dx=0.5, alpha=0.0, fmp2=0.0, lam=lam, e=0.8, kappa=1.0, pot=1, p=p)
    phi = np.zeros((2, N, N, N))
    phi[0] = chi0 / sqrt(2.0)
    lat = U1Lattice(m, phi, np.zeros_like(phi), np.zeros((3, N, N, N)), np.zeros((3, N, N, N)))
    if p == 2:
        T = 2 * pi / sqrt(lam)
    else:
        T = 4 * sqrt(2.0) * gamma(0.25) ** 2 / (4 * sqrt(2 * pi)) / (chi0 * sqrt(lam))
    n = 400
    lat.vv_steps(VV10, T / n, n // 2)
    assert abs(lat.phi[0, 0, 0, 0] * sqrt(2.0) + chi0) < 1e-10  # half a period: -chi0
    lat.vv_steps(VV10, T / n, n // 2)
    assert np.max(np.abs(lat.phi[0] * sqrt(2.0) - chi0)) < 1e-10
    assert np.max(np.abs(lat.phi[1])) == 0.0 and np.max(np.abs(lat.theta)) == 0.0


@pytest.mark.parametrize("pot,p", [(0, 4), (1, 2), (1, 4), (1, 6)])
def test_charged_potential_curvature_is_the_second_derivative(pot, p):
    """The curvature that sets the vacuum fluctuations (section 7) along a
    canonical component chi_0 of (chi_0, chi_1), mod2 = (chi_0^2 + chi_1^2)/2,
    against central second differences of V itself."""
    from oracle.ic import _charged_potential
    m = U1Model(N=4, dx=1.0, alpha=0.0, fmp2=0.0, lam=1.3, v2=0.7, pot=pot, p=p)
    chi1 = 0.4
    for chi0 in (0.3, 1.1, -0.8):
        h = 1e-4
        V = [_charged_potential(m, 0.5 * ((chi0 + d) ** 2 + chi1 ** 2))[0] for d in (-h, 0.0, h)]
        num = (V[0] - 2 * V[1] + V[2]) / (h * h)
        _, dv, d2 = _charged_potential(m, 0.5 * (chi0 ** 2 + chi1 ** 2))
        assert abs(dv + d2 * chi0 ** 2 - num) < 1e-6 * (1 + abs(num))
        if pot == 1 and p == 2:
            assert dv + d2 * chi0 ** 2 == pytest.approx(m.lam, rel=1e-15)  # plain mass term lam chi^2/2


@pytest.mark.parametrize("integ", ["vv2", "vv4"])
def test_noncompact_free_photon_is_the_exact_lattice_mode(integ):
    """Without charged matter (phi = pi = 0) the non-compact gauge field of
    section 5.2 is a free lattice photon: a transverse mode A_y(x) = cos(2 pi x/N)
    (so sum_i D_i^- A_i = 0) has omega^2 = k_L^2 = 4 sin^2(pi/N)/dx^2, and one VV2
    step maps (A, A') by the exact 2 x 2 matrix of that oscillator; VV4 is the
    Yoshida product of three such maps (static background, e = 1.3)."""
    N, dx, dt, n = 8, 0.7, 0.05, 40
    e, kappa = 1.3, 0.9
    m = U1Model(N=N, dx=dx, alpha=0.0, fmp2=0.0, lam=1.0, v2=0.0, e=e, kappa=kappa, noncompact=1)
    x = np.arange(N)
    prof = np.broadcast_to(np.cos(2 * np.pi * x / N)[None, None, :], (N, N, N))
    A0, V0 = 0.3, -0.2  # amplitude of A_y and of A_y' = piA_y (a = 1, alpha = 0)
    th = np.zeros((3, N, N, N))
    th[1] = e * dx * A0 * prof
    piA = np.zeros((3, N, N, N))
    piA[1] = V0 * prof
    zero = np.zeros((2, N, N, N))
    lat = U1Lattice(m, zero, zero, th, piA)
    w2 = 4 * np.sin(np.pi / N) ** 2 / dx ** 2

    def vv2_map(h):
        return np.array([[1 - h * h * w2 / 2, h], [-h * w2 * (1 - h * h * w2 / 4), 1 - h * h * w2 / 2]])

    w = _vv(integ)
    M = np.eye(2)
    for wp in w:
        M = vv2_map(wp * dt) @ M
    ref = np.linalg.matrix_power(M, n) @ np.array([A0, V0])
    lat.vv_steps(w, dt, n)
    got_A = lat.theta[1] / (e * dx)
    assert np.max(np.abs(got_A - ref[0] * prof)) < 1e-12
    assert np.max(np.abs(lat.piA[1] - ref[1] * prof)) < 1e-12
    assert np.max(np.abs(lat.theta[0])) == 0.0 and np.max(np.abs(lat.theta[2])) == 0.0


@pytest.mark.parametrize("nc,a,alpha", [(1, 1.0, 0.0), (1, 1.4, 0.5), (0, 1.2, 1.0)])
def test_u1_field_strengths_carry_the_gauge_energies(nc, a, alpha):
    """E_i = piA_i/a^{1-alpha} and B_i (section 5.4): <|E|^2> = 2 a^{2+2alpha} E_K^A/kappa
    exactly; non-compact <|B|^2> = 2 a^4 E_G^A/kappa exactly (E_G^A is half the
    squared lattice curl); compact, with small angles, the same to O(theta^2)."""
    N = 6
    m = U1Model(N=N, dx=0.6, alpha=alpha, fmp2=0.0, lam=1.0, v2=1.0, e=0.9, kappa=1.3, noncompact=nc)
    lat = _random_state(N, 19, m, a=a)
    if not nc:
        lat.theta *= 0.01
    E = lat.energies()
    assert (lat.electric() ** 2).sum(axis=0).mean() == pytest.approx(2 * a ** (2 + 2 * alpha) * E[3] / m.kappa,
                                                                     rel=1e-13)
    B2 = (lat.magnetic() ** 2).sum(axis=0).mean()
    assert B2 == pytest.approx(2 * a ** 4 * E[4] / m.kappa, rel=1e-13 if nc else 1e-3)



@pytest.mark.parametrize("alpha", [0.0, 1.0])
def test_homogeneous_electric_field_expands_like_radiation(alpha):
    """A uniform electric field with phi = 0 and unit links carries no charge
    and no plaquette, so piA stays constant and the energy is kappa piA^2/(2 a^4):
    radiation.  The Friedmann equations (section 4.1) then fix the expansion in
    closed form: with a' = b and b^2 = (f*/m_p)^2 a^{2(alpha+1)} rho / 3,
    a^2 = a0^2 + 2 a0 b0 t in cosmic time (alpha = 0) and a = a0 + b0 eta in
    conformal time (alpha = 1)."""
    N = 4
    m = U1Model(N=N, dx=0.7, alpha=alpha, fmp2=3.0, lam=1.0, e=0.5, kappa=1.0, pot=1, p=4)
    piA = np.stack([np.full((N, N, N), c) for c in (0.3, -0.2, 0.5)])
    z = np.zeros((2, N, N, N))
    lat = U1Lattice(m, z, z, np.zeros((3, N, N, N)), piA, a=1.3)
    E = lat.energies()
    assert E[3] > 0 and np.all(E[[0, 1, 2, 4]] == 0)
    a0 = lat.a
    b0 = np.sqrt(m.fmp2 / 3.0 * a0 ** (2 * (alpha + 1)) * E.sum())
    lat.b = b0
    dt, n = 0.02, 100
    lat.vv_steps(VV4, dt, n)
    t = dt * n
    a_exact = np.sqrt(a0 * a0 + 2 * a0 * b0 * t) if alpha == 0.0 else a0 + b0 * t
    assert abs(lat.a / a_exact - 1) < 1e-8, (lat.a, a_exact)  # VV4 at dt = 0.02: ~1e-10
    assert abs(lat.a / a0 - 1) > 0.2  # a grows by a sizeable factor
    assert np.max(np.abs(lat.piA - piA)) < 1e-15
    # theta_i' = e dx piA_i a^{alpha-1} (section 5.3): with a^n linear in t (n = 2 - alpha),
    # theta_i(t) - theta_i(0) = e dx piA_i (a - a0) / (a0^{n-1} b0)
    n_ = 2.0 - alpha
    th_exact = m.e * m.dx * piA[:, 0, 0, 0] * (a_exact - a0) / (a0 ** (n_ - 1) * b0)
    assert np.allclose(lat.theta[:, 0, 0, 0], th_exact, rtol=1e-8, atol=0), (lat.theta[:, 0, 0, 0], th_exact)
    assert np.ptp(lat.theta, axis=(1, 2, 3)).max() < 1e-14


def test_homogeneous_electric_field_leapfrog_converges_at_second_order():
    """The staggered leapfrog of section 5.3.1, started by its backward half
    kick, on the same radiation-dominated expansion (alpha = 0): a and the link
    angles at the integer steps approach the closed form as dt^2."""
    N = 4
    m = U1Model(N=N, dx=0.7, alpha=0.0, fmp2=3.0, lam=1.0, e=0.5, kappa=1.0, pot=1, p=4)
    piA = np.stack([np.full((N, N, N), c) for c in (0.3, -0.2, 0.5)])
    z = np.zeros((2, N, N, N))
    T, errs = 2.0, []
    for dt in (0.04, 0.02):
        lat = U1Lattice(m, z, z, np.zeros((3, N, N, N)), piA, a=1.3)
        a0 = lat.a
        b0 = np.sqrt(m.fmp2 / 3.0 * a0 ** 2 * lat.energies().sum())
        lat.b = b0
        lat.lf_prepare(dt)
        lat.lf_steps(dt, int(round(T / dt)))
        a_exact = np.sqrt(a0 * a0 + 2 * a0 * b0 * T)
        th_exact = m.e * m.dx * piA[:, 0, 0, 0] * (a_exact - a0) / (a0 * b0)
        errs.append(max(abs(lat.a / a_exact - 1), np.max(np.abs(lat.theta[:, 0, 0, 0] / th_exact - 1))))
    assert errs[1] < 1e-4, errs
    assert abs(np.log2(errs[0] / errs[1]) - 2) < 0.2, errs