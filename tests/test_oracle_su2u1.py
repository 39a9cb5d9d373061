"""Pins of the oracle's SU(2) x U(1) doublet with a singlet (the working example
of section 8.3) against the mathematics: every force is minus the gradient of
the lattice energy along its own direction (doublet components, singlet, U(1)
link angles, SU(2) group directions), the model reduces exactly to the
SU(2)-Higgs oracle without the U(1) sector and the singlet, both discrete Gauss
laws hold to round-off while expanding, the evolution commutes with U(1) and
SU(2) gauge transformations, and VV2/VV4 converge with their orders."""
import numpy as np
import pytest

from oracle import VV2, VV4, VV6, SU2Lattice, SU2U1Lattice, SU2U1Model
from oracle.spectra import dft_forward, dft_inverse, mode_numbers
from tests import inputs
from tests.test_oracle_su2 import qconj, qmul, random_quaternions, umul


def random_state(N, model, seed, spread=0.6, a=1.0):
    phi = inputs.fields(4, N, seed=seed, amp=0.5, kmax=N / 3, means=[0.6, 0.1, -0.2, 0.3])
    pi = inputs.fields(4, N, seed=seed + 1, amp=0.3, kmax=N / 3)
    u = np.stack([random_quaternions((N, N, N), seed + 2 + i, spread) for i in range(3)])
    piB = np.stack([inputs.fields(3, N, seed=seed + 10 + i, amp=0.3, kmax=N / 3) for i in range(3)])
    th = inputs.angles(N, seed + 20, scale=1.5)
    piA = inputs.fields(3, N, seed=seed + 21, amp=0.3, kmax=N / 3)
    chi = inputs.fields(1, N, seed=seed + 22, amp=0.5, kmax=N / 3, means=[0.2])[0]
    pchi = inputs.fields(1, N, seed=seed + 23, amp=0.3, kmax=N / 3)[0]
    return SU2U1Lattice(model, phi, pi, u, piB, th, piA, chi, pchi, a=a)


def _cplx(f):
    return f[0] + 1j * f[1], f[2] + 1j * f[3]


def _gen(b, F1, F2):
    """T_b Phi for T_0 = 1 (U(1)) and the Pauli matrices T_1..3."""
    return [(F1, F2), (F2, F1), (-1j * F2, 1j * F1), (F1, -F2)][b]


def charges(phi, pi):
    """Charge densities Im[Phi^dag T_b pi], b = 0 (U(1)), 1..3 (SU(2))."""
    F1, F2 = _cplx(phi)
    P1, P2 = _cplx(pi)
    out = []
    for b in range(4):
        G1, G2 = _gen(b, P1, P2)
        out.append(np.imag(np.conj(F1) * G1 + np.conj(F2) * G2))
    return np.stack(out)


def gauss_state(N, model, seed):
    """Unit links and zero angles, a random doublet whose four total charges are
    projected out (pi -> pi - sum_b c_b i T_b Phi with the 4 x 4 system
    M_ab = sum_n Re[Phi^dag T_a T_b Phi]), and electric momenta solving the two
    linear Gauss laws in Fourier space."""
    phi = inputs.fields(4, N, seed=seed, amp=0.5, kmax=N / 3, means=[0.7, 0.0, 0.2, -0.1])
    pi = inputs.fields(4, N, seed=seed + 1, amp=0.3, kmax=N / 3)
    F1, F2 = _cplx(phi)
    M = np.zeros((4, 4))
    for a in range(4):
        for b in range(4):
            G1, G2 = _gen(b, F1, F2)
            H1, H2 = _gen(a, G1, G2)
            M[a, b] = np.sum(np.real(np.conj(F1) * H1 + np.conj(F2) * H2))
    c = np.linalg.solve(M, charges(phi, pi).sum(axis=(1, 2, 3)))
    P1, P2 = _cplx(pi)
    for b in range(4):
        G1, G2 = _gen(b, F1, F2)
        P1, P2 = P1 - c[b] * 1j * G1, P2 - c[b] * 1j * G2
    pi = np.stack([P1.real, P1.imag, P2.real, P2.imag])
    rho = charges(phi, pi)
    assert np.max(np.abs(rho.sum(axis=(1, 2, 3)))) < 1e-10
    m = mode_numbers(N)
    nz, ny, nx = np.meshgrid(m, m, m, indexing="ij")
    betas = [(1.0 - np.exp(2j * np.pi * cc / N)) / model.dx for cc in (nx, ny, nz)]
    den = sum(np.abs(bb) ** 2 for bb in betas)

    def solve(R):
        with np.errstate(divide="ignore", invalid="ignore"):
            return [dft_inverse(np.where(den > 0, np.conj(bb) * R / den, 0.0)).real for bb in betas]

    piB = np.zeros((3, 3, N, N, N))
    for a in range(3):
        for i, sol in enumerate(solve(dft_forward(model.g / model.kappa * rho[1 + a]))):
            piB[i, a] = sol
    piA = np.stack(solve(dft_forward(2.0 * model.eA / model.kappa * rho[0])))
    u = np.zeros((3, 4, N, N, N))
    u[:, 0] = 1.0
    chi = inputs.fields(1, N, seed=seed + 5, amp=0.4, kmax=N / 3)[0]
    pchi = inputs.fields(1, N, seed=seed + 6, amp=0.2, kmax=N / 3)[0]
    return SU2U1Lattice(model, phi, pi, u, piB, np.zeros((3, N, N, N)), piA, chi, pchi)


@pytest.mark.parametrize("a,alpha,pot", [(1.0, 0.0, 0), (1.3, 1.0, 1)])
def test_su2u1_forces_are_minus_gradient_of_the_energy(a, alpha, pot):
    """W = a^{3+alpha} N^3 (E_G^Phi + E_V + E_G^B + E_G^A + E_G^chi): K_Phi =
    -(1/2) dW/d(component), K_chi = -dW/dchi, K_A,i = -(eA dx/kappa) dW/dtheta_i
    and K_B,i^a = -(g dx/kappa) dW/d eps along U_i -> exp(-i eps sigma^a/2) U_i."""
    N = 4
    m = SU2U1Model(N=N, dx=0.6, alpha=alpha, fmp2=0.3, lam=1.3, v2=0.7, g=0.9, kappa=1.6, pot=pot, p=4, eA=0.7,
                   q=1.4)
    lat = random_state(N, m, 5, a=a)
    Kp, KB, KA, Kc = lat.kernels()
    scale = a ** (3 + alpha) * N ** 3

    def W():
        E = lat.energies()
        return scale * (E[1] + E[2] + E[4] + E[6] + E[8])

    def dW(arr, idx, h=1e-6):
        arr[idx] += h
        wp = W()
        arr[idx] -= 2 * h
        wm = W()
        arr[idx] += h
        return (wp - wm) / (2 * h)

    for idx in [(0, 1, 2, 3), (3, 0, 0, 1), (2, 3, 1, 0)]:
        d = dW(lat.phi, idx)
        assert abs(Kp[idx] + 0.5 * d) < 1e-6 * (1 + abs(d)), ("phi", idx, Kp[idx], -0.5 * d)
    for idx in [(1, 2, 3), (0, 0, 0), (3, 1, 2)]:
        d = dW(lat.chi, idx)
        assert abs(Kc[idx] + d) < 1e-6 * (1 + abs(d)), ("chi", idx, Kc[idx], -d)
    for idx in [(0, 1, 2, 3), (1, 3, 0, 2), (2, 0, 3, 3)]:
        d = dW(lat.theta, idx)
        assert abs(KA[idx] + m.eA * m.dx / m.kappa * d) < 1e-6 * (1 + abs(d)), ("theta", idx, KA[idx])
    h = 1e-6
    for (i, ca, z, y, x) in [(0, 0, 1, 2, 3), (1, 2, 0, 3, 1), (2, 1, 2, 0, 0)]:
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
        assert abs(KB[i, ca, z, y, x] + m.g * m.dx / m.kappa * d) < 1e-6 * (1 + abs(d)), ("U", i, ca)


def test_su2u1_without_u1_and_singlet_is_the_su2_model():
    """eA = 0 and no singlet: kernels, energies and VV4 steps equal those of the
    SU(2)-Higgs oracle (the U(1) phase is 1 and the singlet absent)."""
    N = 4
    m = SU2U1Model(N=N, dx=0.6, alpha=0.5, fmp2=0.4, lam=1.2, v2=0.8, g=0.9, kappa=1.3, eA=0.0, q=0.0, chi=0)
    A = random_state(N, m, 9, a=1.2)
    B = SU2Lattice(m.su2(), A.phi, A.pi, A.u, A.piB, a=1.2)
    KpA, KBA, _, _ = A.kernels()
    KpB, KBB = B.kernels()
    assert np.max(np.abs(KpA - KpB)) < 1e-13 and np.max(np.abs(KBA - KBB)) < 1e-13
    EA, EB = A.energies(), B.energies()
    assert np.allclose(EA[:5], EB, rtol=1e-14, atol=0) and np.all(EA[5:] == 0.0)
    A.b = B.b = np.sqrt(0.4 / 3.0 * EB.sum())
    A.vv_steps(VV4, 0.03, 4)
    B.vv_steps(VV4, 0.03, 4)
    for x, y in [(A.phi, B.phi), (A.pi, B.pi), (A.u, B.u), (A.piB, B.piB)]:
        assert np.max(np.abs(x - y)) < 1e-13
    assert abs(A.a - B.a) < 1e-15 and abs(A.b - B.b) < 1e-14


@pytest.mark.parametrize("integ,fmp2", [("vv2", 0.0), ("vv4", 0.5)])
def test_su2u1_both_gauss_laws_hold_to_round_off(integ, fmp2):
    N = 6
    m = SU2U1Model(N=N, dx=0.5, alpha=1.0, fmp2=fmp2, lam=1.0, v2=1.0, g=1.1, kappa=0.9, pot=1, p=4, eA=0.8, q=1.5)
    lat = gauss_state(N, m, 21)
    g0 = lat.gauss()
    assert g0[0] < 1e-28 and g0[1] < 1e-28
    if fmp2 > 0:
        lat.b = np.sqrt(fmp2 / 3.0 * lat.energies().sum())
    for _ in range(4):
        lat.vv_steps({"vv2": VV2, "vv4": VV4}[integ], 0.04, 5)
        g = lat.gauss()
        assert g[0] < 1e-26 and g[1] < 1e-26, g
    assert np.max(np.abs(lat.u[:, 1:])) > 1e-3 and np.max(np.abs(lat.theta)) > 1e-4
    assert lat.energies()[6] > 0.0  # a magnetic U(1) field developed


def test_su2u1_gauge_invariance_of_the_evolution():
    """U(1): Phi -> e^{i beta} Phi, pi -> e^{i beta} pi, theta_i(n) -> theta_i(n) +
    beta(n+i) - beta(n); SU(2): Phi -> Omega Phi, U_i -> Omega(n) U_i Omega^dag(n+i),
    piB_i -> Omega piB_i Omega^dag.  Either commutes with the evolution."""
    N = 4
    m = SU2U1Model(N=N, dx=0.6, alpha=0.0, fmp2=0.0, lam=1.0, v2=1.0, g=0.8, kappa=1.0, eA=0.9, q=1.2)
    A = random_state(N, m, 31)
    beta = inputs.angles(N, 77, scale=3.0)[0]
    Om = random_quaternions((N, N, N), 99, 2.0)

    def phase(f, b):
        F1, F2 = _cplx(f)
        e = np.exp(1j * b)
        F1, F2 = e * F1, e * F2
        return np.stack([F1.real, F1.imag, F2.real, F2.imag])

    def transform(lat):
        phi = umul(Om, phase(lat.phi, beta))
        pi = umul(Om, phase(lat.pi, beta))
        u = np.empty_like(lat.u)
        piB = np.empty_like(lat.piB)
        th = np.empty_like(lat.theta)
        for i, ax in enumerate((2, 1, 0)):
            u[i] = qmul(qmul(Om, lat.u[i]), qconj(np.roll(Om, -1, axis=ax + 1)))
            e = np.concatenate([np.zeros((1, N, N, N)), lat.piB[i]], axis=0)
            piB[i] = qmul(qmul(Om, e), qconj(Om))[1:]
            th[i] = lat.theta[i] + np.roll(beta, -1, axis=ax) - beta
        return SU2U1Lattice(m, phi, pi, u, piB, th, lat.piA, lat.chi, lat.pchi)

    B = transform(A)
    assert np.allclose(A.energies(), B.energies(), rtol=1e-12, atol=1e-14)
    A.vv_steps(VV2, 0.05, 8)
    B.vv_steps(VV2, 0.05, 8)
    TA = transform(A)
    for x, y in [(TA.phi, B.phi), (TA.pi, B.pi), (TA.u, B.u), (TA.piB, B.piB), (TA.piA, B.piA), (TA.chi, B.chi)]:
        assert np.max(np.abs(x - y)) < 1e-11
    assert np.max(np.abs(np.angle(np.exp(1j * (TA.theta - B.theta))))) < 1e-11


@pytest.mark.parametrize("integ,order", [("vv2", 2), ("vv4", 4)])
def test_su2u1_vv_convergence_order(integ, order):
    N, T = 4, 0.4
    m = SU2U1Model(N=N, dx=0.7, alpha=0.0, fmp2=0.0, lam=1.0, v2=1.0, g=1.1, kappa=0.8, eA=0.7, q=1.3)
    ref = random_state(N, m, 41)
    ref.vv_steps(VV6, T / 256, 256)
    errs = []
    for k in (8, 16):
        lat = random_state(N, m, 41)
        lat.vv_steps({"vv2": VV2, "vv4": VV4}[integ], T / k, k)
        errs.append(max(np.max(np.abs(x - y)) for x, y in [(lat.phi, ref.phi), (lat.u, ref.u), (lat.piB, ref.piB),
                                                           (lat.theta, ref.theta), (lat.piA, ref.piA),
                                                           (lat.chi, ref.chi), (lat.pchi, ref.pchi)]))
    slope = np.log2(errs[0] / errs[1])
    assert abs(slope - order) < 0.3, (errs, slope)


def test_su2u1_energy_conservation_static():
    N = 4
    m = SU2U1Model(N=N, dx=0.7, alpha=0.0, fmp2=0.0, lam=1.0, v2=1.0, g=1.0, kappa=1.0, eA=0.8, q=1.1)
    drift = []
    for dt in (0.04, 0.02):
        lat = random_state(N, m, 51)
        E0 = lat.energies().sum()
        lat.vv_steps(VV4, dt, int(round(0.8 / dt)))
        drift.append(abs(lat.energies().sum() - E0) / E0)
    assert drift[1] < 1e-6 and np.log2(drift[0] / drift[1]) > 3.0, drift


def test_su2u1_vacuum_initial_conditions():
    """The constrained draws of section 7.2 (|l_c| = |r_c|, one l-r phase
    difference for all four components, one frequency) leave no total U(1)
    or SU(2) charge without any projection, for a homogeneous doublet split
    evenly over its components; both Gauss laws then hold at round-off with
    unit links and zero angles, the magnetic energies are exactly zero, and
    the singlet is the real-scalar draw of curvature 2 q |Phi|^2 on Philox
    stream 4 (the draw of scalar_ic, pinned by the shell statistics of the
    scalar initial conditions)."""
    from oracle.ic import _singlet_draw, su2u1_ic
    N, dx, omega = 16, 0.5, 0.3
    kIR = 2 * np.pi / (N * dx)
    c = 0.5 / np.sqrt(2.0)
    pb, db = [c] * 4, [-0.2 * c] * 4  # |Phi|^2 = 1/2 split evenly, radial velocity
    m = SU2U1Model(N=N, dx=dx, alpha=1.0, fmp2=0.4, lam=1.0, g=1.2, kappa=omega ** 2, pot=1, p=4, eA=0.9, q=1.0)
    phi, pi, u, piB, th, piA, chi, pchi, _ = su2u1_ic(m, kIR, pb, db, seed=3, omega_over_fstar=omega)
    Q = charges(phi, pi).sum(axis=(1, 2, 3))
    scale = np.sqrt((phi ** 2).sum() * (pi ** 2).sum())
    assert np.max(np.abs(Q)) < 1e-13 * scale, (Q, scale)
    lat = SU2U1Lattice(m, phi, pi, u, piB, th, piA, chi, pchi)
    g = lat.gauss()
    assert g[0] < 1e-26 and g[1] < 1e-26, g
    E = lat.energies()
    assert E[4] == 0.0 and E[6] == 0.0 and E[3] > 0 and E[5] > 0 and E[7] > 0 and E[8] > 0
    assert np.allclose(phi.mean(axis=(1, 2, 3)), pb, rtol=0, atol=1e-14)
    # unequal components: the common-frequency draws still cancel the charges
    phi2, pi2, *_ = su2u1_ic(m, kIR, [0.4, 0.0, 0.0, 0.3], [0.0] * 4, seed=5, omega_over_fstar=omega)
    Q2 = charges(phi2, pi2).sum(axis=(1, 2, 3))
    assert np.max(np.abs(Q2)) < 1e-13 * np.sqrt((phi2 ** 2).sum() * (pi2 ** 2).sum())
    # the singlet: zero mean, curvature 2 q |Phi|^2 = 1 on stream 4
    s2 = sum(x * x for x in pb)
    assert abs(2 * m.q * s2 - 1.0) < 1e-15
    H = np.sqrt(0.4 / 3.0 * (sum(d * d for d in db) + (2 * s2) ** 2 / 4))
    f, fd = _singlet_draw(N, 1.0, kIR, 2 * m.q * s2, H, 3, 4, omega, 1.0, 1.0)
    assert np.max(np.abs(f - chi)) == 0.0 and np.max(np.abs(fd - pchi)) < 1e-15
    assert abs(chi.mean()) < 1e-14 and chi.std() > 0.0



@pytest.mark.parametrize("sector,alpha", [("chi", 0.0), ("chi", 1.0), ("su2", 0.0), ("su2", 1.0), ("u1", 0.0)])
def test_homogeneous_fields_give_the_closed_form_expansion(sector, alpha):
    """With Phi = 0 and unit links, a uniform velocity of the singlet is pure
    kinetic energy (rho ~ a^-6, kination) and a uniform electric field of one
    colour (SU(2)) or of the U(1) is radiation (rho ~ a^-4).  The Friedmann
    equations (section 4.1; a' = b, b^2 = (f*/m_p)^2 a^{2(alpha+1)} rho / 3) make
    a^n grow linearly in program time, a^n - a0^n = n a0^(n-1) b0 t, with
    n = 3 - alpha for kination and n = 2 - alpha for radiation."""
    N = 4
    m = SU2U1Model(N=N, dx=0.7, alpha=alpha, fmp2=3.0, lam=1.0, v2=0.0, g=0.8, kappa=1.0, pot=1, p=4,
                   eA=0.5, q=1.5, chi=1)
    z4 = np.zeros((4, N, N, N))
    u = np.zeros((3, 4, N, N, N))
    u[:, 0] = 1.0
    piB = np.zeros((3, 3, N, N, N))
    piA = np.zeros((3, N, N, N))
    pchi = np.zeros((N, N, N))
    if sector == "chi":
        pchi[:] = 0.7
    elif sector == "su2":
        for i, c in enumerate((0.3, -0.2, 0.5)):
            piB[i, 2] = c  # one colour: the links stay commuting, the plaquettes unity
    else:
        for i, c in enumerate((0.3, -0.2, 0.5)):
            piA[i] = c
    lat = SU2U1Lattice(m, z4, z4, u, piB, None, piA, None, pchi, a=1.3)
    E = lat.energies()
    live = {"chi": [7], "su2": [3], "u1": [5]}[sector]
    assert np.all(E[live] > 0) and np.all(np.delete(E, live) == 0), E
    a0 = lat.a
    b0 = np.sqrt(m.fmp2 / 3.0 * a0 ** (2 * (alpha + 1)) * E.sum())
    lat.b = b0
    dt, steps = 0.02, 100
    lat.vv_steps(VV4, dt, steps)
    t = dt * steps
    n = (3.0 - alpha) if sector == "chi" else (2.0 - alpha)
    a_exact = (a0 ** n + n * a0 ** (n - 1) * b0 * t) ** (1.0 / n)
    assert abs(lat.a / a_exact - 1) < 1e-8, (lat.a, a_exact)  # VV4 at dt = 0.02: ~1e-10
    assert abs(lat.a / a0 - 1) > 0.1  # a grows by a sizeable factor
    # the drifts: chi' = pchi a^{alpha-3} and the link angles' rate a^{alpha-1}, integrated
    # over a^n linear in t: int a^-n dt = ln(a/a0)/(a0^(n-1) b0) (kination),
    # int a^(1-n) dt = (a - a0)/(a0^(n-1) b0) (radiation)
    if sector == "chi":
        chi_exact = 0.7 * np.log(a_exact / a0) / (a0 ** (n - 1) * b0)
        assert abs(lat.chi[0, 0, 0] / chi_exact - 1) < 1e-8, (lat.chi[0, 0, 0], chi_exact)
    elif sector == "su2":
        # U_i = exp(-i Phi_i sigma_3 / 2): q0 = cos(Phi/2), q3 = -sin(Phi/2)
        Phi = 2 * np.arctan2(-lat.u[:, 3, 0, 0, 0], lat.u[:, 0, 0, 0, 0])
        Phi_exact = m.g * m.dx * np.array([0.3, -0.2, 0.5]) * (a_exact - a0) / (a0 ** (n - 1) * b0)
        assert np.allclose(Phi, Phi_exact, rtol=1e-8, atol=0), (Phi, Phi_exact)
    else:
        th_exact = m.eA * m.dx * np.array([0.3, -0.2, 0.5]) * (a_exact - a0) / (a0 ** (n - 1) * b0)
        assert np.allclose(lat.theta[:, 0, 0, 0], th_exact, rtol=1e-8, atol=0), (lat.theta[:, 0, 0, 0], th_exact)

@pytest.mark.parametrize("a,alpha", [(1.0, 0.0), (1.4, 0.5), (0.8, 1.0)])
def test_electric_fields_carry_the_electric_energies(a, alpha):
    """E = pi_gauge/a^{1-alpha} for both gauge sectors (sections 5.4, 6.3):
    sum_i <|E_i|^2> = 2 a^{2+2 alpha} E_K/kappa exactly, for the U(1) field
    (E_K^A) and for the SU(2) field summed over colours (E_K^B); the same holds
    for the SU(2)-only model."""
    N = 6
    m = SU2U1Model(N=N, dx=0.6, alpha=alpha, fmp2=0.0, lam=1.0, v2=1.0, g=0.9, kappa=1.3, pot=0, eA=0.7, q=1.2,
                   chi=1)
    lat = random_state(N, m, 47, a=a)
    E = lat.energies()
    EA2 = (lat.electric(0) ** 2).sum(axis=0).mean()
    EB2 = (lat.electric(1) ** 2).sum(axis=(0, 1)).mean()
    assert EA2 == pytest.approx(2 * a ** (2 + 2 * alpha) * E[5] / m.kappa, rel=1e-13)
    assert EB2 == pytest.approx(2 * a ** (2 + 2 * alpha) * E[3] / m.kappa, rel=1e-13)
    s2 = SU2Lattice(m.su2(), lat.phi, lat.pi, lat.u, lat.piB, a=a)
    E2 = s2.energies()
    assert (s2.electric() ** 2).sum(axis=(0, 1)).mean() == pytest.approx(2 * a ** (2 + 2 * alpha) * E2[3] / m.kappa,
                                                                          rel=1e-13)
