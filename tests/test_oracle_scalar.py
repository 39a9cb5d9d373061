"""Pins of the oracle's scalar sector against what the paper and the mathematics fix.

Each test would fail on a plausible slip in the oracle: a wrong sign or scale of
the Laplacian, a dropped potential term, a wrong a-power in a kick, drift or
in K_a, wrong Yoshida weights, a broken half-kick order.
"""
import numpy as np
import pytest
from scipy.integrate import solve_ivp
from scipy.special import ellipj

import oracle
from oracle import ScalarLattice, ScalarModel
from oracle.spectra import dft_forward, dft_inverse, mode_numbers
from tests import inputs


def _vv_map(h, w2):
    """One velocity-Verlet step of x'' = -w2 x (kick h/2, drift h, kick h/2)."""
    c = 1.0 - 0.5 * h * h * w2
    return np.array([[c, h * np.ones_like(w2)], [-h * w2 * (1.0 - 0.25 * h * h * w2), c]])


def _apply(M, X, P):
    return M[0, 0] * X + M[0, 1] * P, M[1, 0] * X + M[1, 1] * P


@pytest.mark.parametrize("weights,tol", [(oracle.VV2, 1e-12), (oracle.VV4, 1e-12)])
def test_free_field_matches_exact_lattice_dispersion(weights, tol):
    """Free massive field, static background: every mode of the paper's DFT is
    an oscillator with w^2 = m^2 + sum_i 4 sin^2(pi n~_i/N)/dx^2 (section 3.2.1,
    forward/backward lattice momenta), and VVn is a product of 2x2 maps."""
    N, dx, m2, dt, steps = 8, 0.7, 0.5, 0.2, 10
    m = ScalarModel(N=N, Ns=1, pexp=2, dx=dx, alpha=0.0, fmp2=0.0, lam=m2)
    phi = inputs.fields(1, N, seed=3, amp=0.8)
    pi = inputs.fields(1, N, seed=4, amp=0.5)
    lat = ScalarLattice(m, phi, pi)
    lat.vv_steps(weights, dt, steps)
    k = mode_numbers(N)
    nz, ny, nx = np.meshgrid(k, k, k, indexing="ij")
    w2 = m2 + sum(4 * np.sin(np.pi * c / N) ** 2 for c in (nx, ny, nz)) / dx ** 2
    X, P = dft_forward(phi[0]), dft_forward(pi[0])
    for _ in range(steps):
        for w in weights:
            X, P = _apply(_vv_map(w * dt, w2), X, P)
    phi_x, pi_x = dft_inverse(X).real, dft_inverse(P).real
    assert np.max(np.abs(lat.phi[0] - phi_x)) < tol * np.max(np.abs(phi_x))
    assert np.max(np.abs(lat.pi[0] - pi_x)) < tol * np.max(np.abs(pi_x))
    assert lat.a == 1.0 and lat.b == 0.0


def test_summation_by_parts_links_laplacian_and_gradient_energy():
    """sum_n phi L[phi] = - sum_{n,k} (D_k^+ phi)^2 on a periodic lattice."""
    N, dx = 8, 0.3
    m = ScalarModel(N=N, Ns=1, pexp=2, dx=dx, alpha=0.0, fmp2=0.0, lam=0.0)
    phi = inputs.fields(1, N, seed=5)
    lat = ScalarLattice(m, phi, np.zeros_like(phi))
    K = lat.kernel()
    E = lat.energies()
    lhs = float(np.sum(phi[0] * K[0]))
    rhs = -2.0 * N ** 3 * E[2]
    assert abs(lhs - rhs) < 1e-12 * abs(rhs)


@pytest.mark.parametrize("a,alpha", [(1.0, 0.0), (1.37, 0.5), (2.1, 1.0)])
def test_kernels_are_minus_gradient_of_paper_energies(a, alpha):
    """With U = a^{3+alpha} N^3 (E_G + E_V) built from the energies of section
    4.4.1, the kick is K_i(n) = -dU/dphi_i(n) and the drift rate
    a^{-(3-alpha)} pi equals d(a^{3+alpha} N^3 E_K)/dpi (finite differences)."""
    N = 6
    m = ScalarModel(N=N, Ns=2, pexp=4, dx=0.45, alpha=alpha, fmp2=1.0, lam=0.8, q=3.0)
    phi = inputs.fields(2, N, seed=11, amp=0.4, means=[1.0, 0.1])
    pi = inputs.fields(2, N, seed=12, amp=0.6)
    lat = ScalarLattice(m, phi, pi, a=a)
    K = lat.kernel()
    scale = a ** (3 + alpha) * N ** 3
    eps = 1e-5
    for (i, z, y, x) in [(0, 1, 2, 3), (1, 4, 0, 5), (0, 5, 5, 0), (1, 2, 3, 1)]:
        g = []
        for s in (+1, -1):
            lat.phi[i, z, y, x] += s * eps
            E = lat.energies()
            g.append(scale * (E[2] + E[3] + E[4] + E[5]))
            lat.phi[i, z, y, x] -= s * eps
        dU = (g[0] - g[1]) / (2 * eps)
        assert abs(K[i, z, y, x] + dU) < 1e-7 * (abs(dU) + 1.0)
        h = []
        for s in (+1, -1):
            lat.pi[i, z, y, x] += s * eps
            E = lat.energies()
            h.append(scale * (E[0] + E[1]))
            lat.pi[i, z, y, x] -= s * eps
        dH = (h[0] - h[1]) / (2 * eps)
        assert abs(dH - a ** (alpha - 3) * pi[i, z, y, x]) < 1e-7 * (abs(dH) + 1.0)


def test_homogeneous_phi4_matches_jacobi_cn():
    """Static phi^4: phi'' = -phi^3 has phi(t) = phi0 cn(phi0 t | m = 1/2); VV4
    converges to it at fourth order and VV2 at second order."""
    N, phi0, T = 4, 1.3, 3.0
    m = ScalarModel(N=N, Ns=1, pexp=4, dx=1.0, alpha=0.0, fmp2=0.0, lam=1.0)
    exact = phi0 * ellipj(phi0 * T, 0.5)[1]
    errs = {}
    for name, w in (("vv2", oracle.VV2), ("vv4", oracle.VV4)):
        for dt in (0.02, 0.01):
            lat = ScalarLattice(m, np.full((1, N, N, N), phi0), np.zeros((1, N, N, N)))
            lat.vv_steps(w, dt, int(round(T / dt)))
            assert np.ptp(lat.phi) == 0.0
            errs[(name, dt)] = abs(lat.phi[0, 0, 0, 0] - exact)
    assert errs[("vv4", 0.01)] < 1e-8
    r2 = np.log2(errs[("vv2", 0.02)] / errs[("vv2", 0.01)])
    r4 = np.log2(errs[("vv4", 0.02)] / errs[("vv4", 0.01)])
    assert 1.9 < r2 < 2.1 and 3.8 < r4 < 4.2


def _frw_reference(pexp, lam, fmp2, alpha, phi0, T):
    """Textbook homogeneous FRW in cosmic time (phi'' + 3 H phi' + V' = 0,
    a''/a = -(f*/m_p)^2 (rho + 3p)/6, rho = K + V, p = K - V), re-parametrised by
    d eta = a^-alpha dt and integrated with DOP853 at rtol 1e-13."""
    def V(f):
        return lam / pexp * abs(f) ** pexp

    def dV(f):
        return lam * abs(f) ** (pexp - 2) * f

    def rhs(_, y):
        f, fd, a, ad = y
        rho = 0.5 * fd * fd + V(f)
        p = 0.5 * fd * fd - V(f)
        H = ad / a
        s = a ** alpha
        return [s * fd, s * (-3 * H * fd - dV(f)), s * ad, s * (-a * fmp2 * (rho + 3 * p) / 6.0)]

    ad0 = np.sqrt(fmp2 * V(phi0) / 3.0)
    sol = solve_ivp(rhs, (0, T), [phi0, 0.0, 1.0, ad0], method="DOP853", rtol=1e-13, atol=1e-15)
    f, fd, a, ad = sol.y[:, -1]
    return f, a, ad0


@pytest.mark.parametrize("pexp,alpha", [(2, 0.0), (4, 1.0), (4, 0.5)])
def test_expanding_homogeneous_mode_matches_ode(pexp, alpha):
    """The lattice homogeneous mode with self-consistent expansion follows the
    textbook Friedmann system, with O(dt^2) (VV2) and O(dt^4) (VV4) errors."""
    N, lam, fmp2, phi0, T = 2, 1.0, 1.5, 1.0, 4.0
    m = ScalarModel(N=N, Ns=1, pexp=pexp, dx=1.0, alpha=alpha, fmp2=fmp2, lam=lam)
    f_ref, a_ref, ad0 = _frw_reference(pexp, lam, fmp2, alpha, phi0, T)
    errs = {}
    for name, w in (("vv2", oracle.VV2), ("vv4", oracle.VV4)):
        for dt in (0.04, 0.02):
            lat = ScalarLattice(m, np.full((1, N, N, N), phi0), np.zeros((1, N, N, N)), a=1.0, b=ad0)
            lat.vv_steps(w, dt, int(round(T / dt)))
            errs[(name, dt)] = max(abs(lat.phi[0, 0, 0, 0] - f_ref), abs(lat.a - a_ref) / a_ref)
    assert errs[("vv4", 0.02)] < 1e-7
    r2 = np.log2(errs[("vv2", 0.04)] / errs[("vv2", 0.02)])
    r4 = np.log2(errs[("vv4", 0.04)] / errs[("vv4", 0.02)])
    assert 1.8 < r2 < 2.2 and 3.6 < r4 < 4.4


def _fluct_lattice(dt_unused=None, alpha=0.0, pexp=2, Ns=2, q=2.0, fmp2=1.0, N=8):
    m = ScalarModel(N=N, Ns=Ns, pexp=pexp, dx=0.6, alpha=alpha, fmp2=fmp2, lam=1.0, q=q)
    phi = inputs.fields(Ns, N, seed=21, amp=0.05, kmax=2.5, means=[1.0] + [0.0] * (Ns - 1))
    pi = inputs.fields(Ns, N, seed=22, amp=0.05, kmax=2.5)
    lat = ScalarLattice(m, phi, pi)
    lat.b = np.sqrt(lat.hubble_rhs())
    return m, phi, pi, lat


@pytest.mark.parametrize("weights,order", [(oracle.VV2, 2), (oracle.VV4, 4)])
def test_hubble_constraint_converges_at_integrator_order(weights, order):
    """Delta_e = |b^2 - rhs|/rhs at fixed time scales as dt^order (section
    4.3.2: VVn satisfies the Hubble constraint to O(dt^n))."""
    T = 2.0
    de = []
    for dt in (0.05, 0.025):
        m, phi, pi, lat = _fluct_lattice(alpha=0.0)
        lat.vv_steps(weights, dt, int(round(T / dt)))
        de.append(lat.hubble_violation())
    slope = np.log2(de[0] / de[1])
    assert abs(slope - order) < 0.25 * order / 2 + 0.2, (de, slope)


def test_vv_scheme_is_time_reversible():
    """n steps forward then n steps with -dt return the initial state (section 3.5)."""
    m, phi, pi, lat = _fluct_lattice(alpha=0.5, pexp=4)
    a0, b0 = lat.a, lat.b
    lat.vv_steps(oracle.VV4, 0.05, 20)
    assert np.max(np.abs(lat.phi - phi)) > 1e-3
    lat.vv_steps(oracle.VV4, -0.05, 20)
    assert np.max(np.abs(lat.phi - phi)) < 1e-12
    assert np.max(np.abs(lat.pi - pi)) < 1e-12
    assert abs(lat.a - a0) < 1e-13 and abs(lat.b - b0) < 1e-13


@pytest.mark.parametrize("weights,order", [(oracle.VV2, 2), (oracle.VV4, 4)])
def test_static_two_field_energy_conservation(weights, order):
    """Static background: the total energy of the coupled phi^2 chi^2 system is
    conserved up to O(dt^order); a dropped coupling term would break it."""
    T = 2.0
    drift = []
    for dt in (0.04, 0.02):
        m = ScalarModel(N=8, Ns=2, pexp=2, dx=0.6, alpha=0.0, fmp2=0.0, lam=1.0, q=8.0)
        phi = inputs.fields(2, 8, seed=31, amp=0.3, kmax=2.0, means=[1.0, 0.0])
        pi = inputs.fields(2, 8, seed=32, amp=0.3, kmax=2.0)
        lat = ScalarLattice(m, phi, pi)
        E0 = lat.energies().sum()
        lat.vv_steps(weights, dt, int(round(T / dt)))
        drift.append(abs(lat.energies().sum() - E0) / E0)
    slope = np.log2(drift[0] / drift[1])
    assert abs(slope - order) < 0.3, (drift, slope)


def test_staggered_leapfrog_equals_vv2_in_static_background():
    """In a static background scheme III is velocity-Verlet with momenta kept
    half a step behind: the field trajectories coincide to round-off."""
    m = ScalarModel(N=8, Ns=2, pexp=2, dx=0.6, alpha=0.0, fmp2=0.0, lam=1.0, q=4.0)
    phi = inputs.fields(2, 8, seed=41, amp=0.2, means=[1.0, 0.0])
    pi = inputs.fields(2, 8, seed=42, amp=0.2)
    vv = ScalarLattice(m, phi, pi)
    lf = ScalarLattice(m, phi, pi)
    lf.lf3_prepare(0.05)
    vv.vv_steps(oracle.VV2, 0.05, 30)
    lf.lf3_steps(0.05, 30)
    assert np.max(np.abs(vv.phi - lf.phi)) < 1e-12


def test_staggered_leapfrog_hubble_constraint_second_order():
    """Scheme III verifies its Hubble constraint
    b_{+1/2}^2 = (1/3)(f*/m_p)^2 a_{+1/2}^{2(alpha+1)} (E_K(+1/2) + <E_G> + <E_V>)
    to O(dt^2) (section 4.2.1)."""
    T = 2.0
    de = []
    for dt in (0.04, 0.02):
        m, phi, pi, lat = _fluct_lattice(alpha=1.0, pexp=4, Ns=1)
        lat.lf3_prepare(dt)
        n = int(round(T / dt))
        d = lat.lf3_steps(dt, n + 1, diag=True)
        EG_bar = 0.5 * (d[n - 1, 0] + d[n, 0])
        EV_bar = 0.5 * (d[n - 1, 1] + d[n, 1])
        EK, ah, bh = d[n - 1, 2], d[n - 1, 3], d[n - 1, 4]
        rhs = m.fmp2 / 3.0 * ah ** (2 * (m.alpha + 1)) * (EK + EG_bar + EV_bar)
        de.append(abs(bh * bh - rhs) / rhs)
    slope = np.log2(de[0] / de[1])
    assert 1.7 < slope < 2.3, (de, slope)



def test_staggered_leapfrog_start_stores_the_half_step_kinetic_energy():
    """The backward half kick that starts scheme III (section 4.2.1) leaves
    pi_{-1/2}, b_{-1/2} and E_K at -1/2, which the first step averages with
    E_K at +1/2.  That stored value is the kinetic energy <pi^2>/(2 a^6) of
    section 4.4.1 of the momenta pi_{-1/2} at the staggered scale factor
    a_{-1/2} = a - (dt/2) b_{-1/2}, evaluated here by the energy functional."""
    dt = 0.1
    m, phi, pi, lat = _fluct_lattice(alpha=0.5, pexp=4, Ns=2, fmp2=3.0)
    a0 = lat.a
    lat.lf3_prepare(dt)
    ahm = a0 - 0.5 * dt * lat.b
    assert abs(ahm - a0) > 1e-2 * a0  # expansion strong enough to tell a_{-1/2} from a
    E = ScalarLattice(m, lat.phi, lat.pi, a=ahm).energies()
    assert abs(lat.EKm - (E[0] + E[1])) <= 1e-13 * (E[0] + E[1]), (lat.EKm, E[0] + E[1])

def test_yoshida_weights():
    """Closed-form VV4 weights satisfy sum w = 1 and sum w^3 = 0 (fourth order);
    the tabulated VV6/8/10 weights sum to one."""
    w = np.array(oracle.VV4)
    assert abs(w.sum() - 1) < 1e-15 and abs((w ** 3).sum()) < 1e-14
    for ws in (oracle.VV6, oracle.VV8, oracle.VV10):
        assert abs(sum(ws) - 1.0) < 1e-14
    rows = [l.split() for l in open("tests/golden/yoshida_vv4_table.txt") if not l.startswith("#")]
    printed = {r[0]: float(r[1]) for r in rows}
    assert abs(printed["w1"] - w[0]) < 1e-15
    # the printed w2 is off by 2e-8: the closed form is used instead
    assert 1e-8 < abs(printed["w2"] - w[1]) < 1e-7


@pytest.mark.parametrize("weights,order", [(oracle.VV4, 4), (oracle.VV6, 6), (oracle.VV8, 8), (oracle.VV10, 10)])
def test_yoshida_compositions_reach_their_order(weights, order):
    """One step of the composed velocity-Verlet map of the harmonic oscillator
    x'' = -x differs from the exact rotation by O(h^(order+1)) (section 4.3.2):
    halving h divides the local error by 2^(order+1).  A mistyped, dropped or
    swapped weight of the appendix table lowers the order."""
    errs = []
    for h in (0.4, 0.2):
        M = np.eye(2)
        for w in weights:
            M = _vv_map(w * h, np.float64(1.0)) @ M
        exact = np.array([[np.cos(h), np.sin(h)], [-np.sin(h), np.cos(h)]])
        errs.append(np.max(np.abs(M - exact)))
    slope = np.log2(errs[0] / errs[1])
    assert abs(slope - (order + 1)) < 0.3, (errs, slope)


def test_fluid_background_massless_modes_match_closed_form():
    """Radiation fluid (w = 1/3) in conformal time (alpha = 1): p = 1 and
    a = a0 (1 + H0 eta) has a'' = 0, so for a free massless field u = a phi_k
    obeys u'' = -w^2 u with the lattice eigenvalue w^2 = sum_i 4 sin^2(pi n_i/N)/dx^2
    (section 3.2.1): u(eta) = u0 cos(w eta) + u0' sin(w eta)/w, and
    pi = a^2 phi' = a u' - a' u.  VV4 at a small step reaches it to O(dt^4)."""
    from oracle.core import Fluid
    N, dx, a0, H0, T = 8, 0.7, 1.3, 0.8, 1.0
    fl = Fluid(a0=a0, H0=H0, w=1.0 / 3.0, alpha=1.0)
    assert abs(fl.p - 1.0) < 1e-15
    m = ScalarModel(N=N, Ns=1, pexp=2, dx=dx, alpha=1.0, fmp2=0.0, lam=0.0)
    phi = inputs.fields(1, N, seed=5, amp=0.8, means=[0.3])
    pi = inputs.fields(1, N, seed=6, amp=0.5, means=[0.1])
    errs = []
    for dt in (0.01, 0.005):
        lat = ScalarLattice(m, phi, pi, a=a0)
        lat.t = 0.0
        lat.vv_steps_fluid(fl, oracle.VV4, dt, int(round(T / dt)))
        k = mode_numbers(N)
        nz, ny, nx = np.meshgrid(k, k, k, indexing="ij")
        w = np.sqrt(4 * (np.sin(np.pi * nx / N) ** 2 + np.sin(np.pi * ny / N) ** 2 + np.sin(np.pi * nz / N) ** 2)) / dx
        F0, P0 = dft_forward(phi[0]), dft_forward(pi[0])
        u0 = a0 * F0
        du0 = a0 * H0 * F0 + P0 / a0          # a' phi + a phi', phi' = pi / a^2
        ws = np.where(w > 0, w, 1.0)
        u = u0 * np.cos(w * T) + np.where(w > 0, du0 * np.sin(w * T) / ws, du0 * T)
        du = -u0 * w * np.sin(w * T) + du0 * np.cos(w * T)
        aT, bT = fl.a(T), fl.b(T)
        phi_ex = dft_inverse(u / aT).real
        pi_ex = dft_inverse(aT * du - bT * u).real
        errs.append(max(np.max(np.abs(lat.phi[0] - phi_ex)), np.max(np.abs(lat.pi[0] - pi_ex))))
        assert abs(lat.a - aT) < 1e-12 and abs(lat.t - T) < 1e-12
    assert errs[1] < 1e-6, errs
    assert 3.6 < np.log2(errs[0] / errs[1]) < 4.4, errs


def test_fluid_background_homogeneous_mode_matches_ode():
    """Matter fluid (w = 0), alpha = 0: a = a0 (1 + 3 H0 t/2)^(2/3).  The
    homogeneous phi^4 mode follows phi' = a^-3 pi, pi' = -a^3 lam phi^3
    (Hamiltonian form of section 4.2.3) integrated by DOP853."""
    from oracle.core import Fluid
    fl = Fluid(a0=1.0, H0=0.6, w=0.0, alpha=0.0)
    lam, phi0, T, N = 1.0, 1.0, 4.0, 2
    m = ScalarModel(N=N, Ns=1, pexp=4, dx=1.0, alpha=0.0, fmp2=0.0, lam=lam)

    def rhs(t, y):
        a = fl.a(t)
        return [y[1] / a ** 3, -a ** 3 * lam * y[0] ** 3]

    sol = solve_ivp(rhs, (0, T), [phi0, 0.0], method="DOP853", rtol=1e-13, atol=1e-15)
    lat = ScalarLattice(m, np.full((1, N, N, N), phi0), np.zeros((1, N, N, N)))
    lat.t = 0.0
    lat.vv_steps_fluid(fl, oracle.VV4, 0.01, 400)
    assert abs(lat.phi[0, 0, 0, 0] - sol.y[0, -1]) < 1e-8
    assert abs(lat.pi[0, 0, 0, 0] - sol.y[1, -1]) < 1e-8


def test_rk4_free_field_converges_to_exact_modes():
    """Static background: each lattice mode of a free massive field is an
    oscillator with w^2 = m^2 + sum_i 4 sin^2(pi n_i/N)/dx^2; the explicit RK4
    of section 4.3.1 reaches the exact solution with a global O(dt^4) error."""
    N, dx, m2, T = 8, 0.7, 0.5, 1.0
    m = ScalarModel(N=N, Ns=1, pexp=2, dx=dx, alpha=0.0, fmp2=0.0, lam=m2)
    phi = inputs.fields(1, N, seed=13, amp=0.8)
    pi = inputs.fields(1, N, seed=14, amp=0.5)
    k = mode_numbers(N)
    nz, ny, nx = np.meshgrid(k, k, k, indexing="ij")
    w = np.sqrt(m2 + 4 * (np.sin(np.pi * nx / N) ** 2 + np.sin(np.pi * ny / N) ** 2 + np.sin(np.pi * nz / N) ** 2) / dx ** 2)
    X0, P0 = dft_forward(phi[0]), dft_forward(pi[0])
    phi_ex = dft_inverse(X0 * np.cos(w * T) + P0 / w * np.sin(w * T)).real
    pi_ex = dft_inverse(-X0 * w * np.sin(w * T) + P0 * np.cos(w * T)).real
    errs = []
    for dt in (0.02, 0.01):
        lat = ScalarLattice(m, phi, pi)
        lat.rk4_steps(dt, int(round(T / dt)))
        errs.append(max(np.max(np.abs(lat.phi[0] - phi_ex)), np.max(np.abs(lat.pi[0] - pi_ex))))
    assert errs[1] < 1e-6, errs
    assert 3.7 < np.log2(errs[0] / errs[1]) < 4.3, errs


@pytest.mark.parametrize("pexp,alpha", [(2, 0.0), (4, 1.0)])
def test_rk4_expanding_homogeneous_mode_matches_ode(pexp, alpha):
    """RK4 with self-consistent expansion against the textbook Friedmann
    system (DOP853): error O(dt^4) in phi and a."""
    N, lam, fmp2, phi0, T = 2, 1.0, 1.5, 1.0, 4.0
    m = ScalarModel(N=N, Ns=1, pexp=pexp, dx=1.0, alpha=alpha, fmp2=fmp2, lam=lam)
    f_ref, a_ref, ad0 = _frw_reference(pexp, lam, fmp2, alpha, phi0, T)
    errs = []
    for dt in (0.04, 0.02):
        lat = ScalarLattice(m, np.full((1, N, N, N), phi0), np.zeros((1, N, N, N)), a=1.0, b=ad0)
        lat.rk4_steps(dt, int(round(T / dt)))
        errs.append(max(abs(lat.phi[0, 0, 0, 0] - f_ref), abs(lat.a - a_ref) / a_ref))
    assert errs[1] < 1e-7, errs
    assert 3.6 < np.log2(errs[0] / errs[1]) < 4.4, errs



def test_rk4_and_vv6_agree_on_an_expanding_inhomogeneous_lattice():
    """Gradients and expansion together: RK4 (section 4.3.1, velocity form with
    its own right-hand side) and VV6 (section 4.3.2, Hamiltonian momenta), each
    pinned to exact solutions above, solve the same equations of motion, so on
    a fluctuating two-field lattice on which a grows by 60% they agree to their
    discretisation errors (~6e-10 of the fluctuations), far below the effect of a
    wrong power of a in any term."""
    T = 1.0
    m, phi, pi, lat_rk = _fluct_lattice(alpha=0.0, pexp=4, Ns=2, fmp2=3.0)
    lat_vv = ScalarLattice(m, phi, pi, a=lat_rk.a, b=lat_rk.b)
    lat_rk.rk4_steps(0.005, int(round(T / 0.005)))
    lat_vv.vv_steps(oracle.VV6, 0.02, int(round(T / 0.02)))
    assert lat_vv.a > 1.5
    scale = np.max(np.abs(lat_vv.phi - lat_vv.phi.mean(axis=(1, 2, 3), keepdims=True)))
    assert np.max(np.abs(lat_rk.phi - lat_vv.phi)) < 1e-8 * scale
    assert abs(lat_rk.a / lat_vv.a - 1) < 1e-10


def _printed_tableaux():
    """The paper's printed Gauss-Legendre tableaux (tests/golden), evaluated
    with sqrt and the four operations only."""
    import ast
    import math
    import os
    import re

    allowed = (ast.Expression, ast.BinOp, ast.UnaryOp, ast.Add, ast.Sub, ast.Mult, ast.Div, ast.USub, ast.Call,
               ast.Name, ast.Load, ast.Constant)

    def ev(expr, env):
        tree = ast.parse(expr, mode="eval")
        assert all(isinstance(n, allowed) for n in ast.walk(tree)), expr
        return eval(compile(tree, "<tableau>", "eval"), {"__builtins__": {}}, dict(env, sqrt=math.sqrt))

    path = os.path.join(os.path.dirname(__file__), "golden", "gauss_legendre_tableaux.txt")
    tabs, s, env = {}, None, {}
    for line in open(path):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        m = re.match(r"\[s=(\d)\]", line)
        if m:
            s, env = int(m.group(1)), {}
            tabs[s] = {"A": [], "c": None}
        elif line.startswith("def "):
            name, expr = line[4:].split("=", 1)
            env[name.strip()] = ev(expr.strip(), env)
        elif line.startswith("row "):
            tabs[s]["A"].append([ev(e.strip(), env) for e in line[4:].split(";")])
        elif line.startswith("c "):
            tabs[s]["c"] = [ev(e.strip(), env) for e in line[2:].split(";")]
    return {k: (np.array(v["A"]), np.array(v["c"])) for k, v in tabs.items()}


def _collocation_ok(A, c):
    """Order conditions of the s-stage Gauss method: B(2s) sum_j c_j tau_j^(k-1) = 1/k
    (k <= 2s) and C(s) sum_j A_ij tau_j^(k-1) = tau_i^k / k (k <= s), tau_i = row sums."""
    s = len(c)
    tau = A.sum(axis=1)
    ok = all(abs((c * tau ** (k - 1)).sum() - 1.0 / k) < 1e-13 for k in range(1, 2 * s + 1))
    return ok and all(np.max(np.abs(A @ tau ** (k - 1) - tau ** k / k)) < 1e-13 for k in range(1, s + 1))


def test_gauss_legendre_tableaux_from_definition_match_printed_tables():
    """The tableaux computed from the collocation definition equal the printed
    ones for s = 2, 3, 4 and satisfy the order conditions for s = 2..5; the
    printed s = 5 table violates them (misprints), so the definition is used."""
    from oracle.core import gl_tableau
    printed = _printed_tableaux()
    for s in (2, 3, 4):
        A, c = gl_tableau(s)
        assert np.max(np.abs(A - printed[s][0])) < 1e-14 and np.max(np.abs(c - printed[s][1])) < 1e-14, s
    for s in (2, 3, 4, 5):
        assert _collocation_ok(*gl_tableau(s)), s
    assert not _collocation_ok(*printed[5])
    assert np.max(np.abs(gl_tableau(5)[1] - printed[5][1])) < 1e-14  # the printed weights are right


@pytest.mark.parametrize("s,order", [(2, 4), (3, 6)])
def test_gauss_legendre_free_field_converges_to_exact_modes(s, order):
    """Static background: the s-stage Gauss-Legendre method reaches the exact
    lattice modes with a global error O(dt^(2s))."""
    N, dx, m2, T = 8, 0.7, 0.5, 1.0
    m = ScalarModel(N=N, Ns=1, pexp=2, dx=dx, alpha=0.0, fmp2=0.0, lam=m2)
    phi = inputs.fields(1, N, seed=13, amp=0.8)
    pi = inputs.fields(1, N, seed=14, amp=0.5)
    k = mode_numbers(N)
    nz, ny, nx = np.meshgrid(k, k, k, indexing="ij")
    w = np.sqrt(m2 + 4 * (np.sin(np.pi * nx / N) ** 2 + np.sin(np.pi * ny / N) ** 2 + np.sin(np.pi * nz / N) ** 2) / dx ** 2)
    X0, P0 = dft_forward(phi[0]), dft_forward(pi[0])
    phi_ex = dft_inverse(X0 * np.cos(w * T) + P0 / w * np.sin(w * T)).real
    errs = []
    for dt in (0.1, 0.05):
        lat = ScalarLattice(m, phi, pi)
        lat.gl_steps(s, dt, int(round(T / dt)))
        errs.append(np.max(np.abs(lat.phi[0] - phi_ex)))
    assert abs(np.log2(errs[0] / errs[1]) - order) < 0.4, errs


@pytest.mark.parametrize("s,dts,bound", [(2, (0.08, 0.04), 1e-7), (3, (0.4, 0.2), 2e-8)])
def test_gauss_legendre_expanding_homogeneous_mode_matches_ode(s, dts, bound):
    """s-stage Gauss-Legendre with self-consistent expansion against the
    Friedmann system (DOP853): global order 2s (s = 3 has unequal weights c_m,
    so every stage's derivative of a and b must enter with its own weight)."""
    N, lam, fmp2, phi0, T = 2, 1.0, 1.5, 1.0, 4.0
    m = ScalarModel(N=N, Ns=1, pexp=4, dx=1.0, alpha=1.0, fmp2=fmp2, lam=lam)
    f_ref, a_ref, ad0 = _frw_reference(4, lam, fmp2, 1.0, phi0, T)
    errs = []
    for dt in dts:
        lat = ScalarLattice(m, np.full((1, N, N, N), phi0), np.zeros((1, N, N, N)), a=1.0, b=ad0)
        lat.gl_steps(s, dt, int(round(T / dt)))
        errs.append(max(abs(lat.phi[0, 0, 0, 0] - f_ref), abs(lat.a - a_ref) / a_ref))
    assert errs[1] < bound, errs
    assert abs(np.log2(errs[0] / errs[1]) - 2 * s) < 0.4, errs


def _mathieu_reference(k2, qs, phi0, T):
    """chi'' + (k^2 + q* phi0^2 cos^2 t) chi = 0 from chi = 1, chi' = 0 (DOP853),
    and the Floquet multiplier of largest modulus from the monodromy matrix over
    the period pi of cos^2 t."""
    from scipy.integrate import solve_ivp

    def f(t, y):
        w2 = k2 + qs * phi0 * phi0 * np.cos(t) ** 2
        return [y[1], -w2 * y[0], y[3], -w2 * y[2]]

    sol = solve_ivp(f, [0.0, T], [1.0, 0.0, 0.0, 1.0], rtol=1e-12, atol=1e-14, method="DOP853", dense_output=True)
    one = solve_ivp(f, [0.0, np.pi], [1.0, 0.0, 0.0, 1.0], rtol=1e-12, atol=1e-14, method="DOP853")
    M = np.array([[one.y[0, -1], one.y[2, -1]], [one.y[1, -1], one.y[3, -1]]])
    return sol, np.max(np.abs(np.linalg.eigvals(M)))


def test_parametric_resonance_matches_mathieu_floquet():
    """Linear regime of phi^2 chi^2 preheating in a static background (section
    8.1): with phi = phi0 cos t (free, m = 1) and a tiny chi in one lattice mode,
    that mode obeys the Mathieu equation chi'' + (k_L^2 + q* phi0^2 cos^2 t) chi = 0
    with the lattice momentum k_L^2 = 4 sin^2(pi/N)/dx^2.  q* = 10, k_L = 0.5 lies
    in the first instability band (Floquet exponent ~0.24): the oracle's VV4 run
    follows the ODE solution over eight periods, and its growth per period at the
    end is the Floquet multiplier of the monodromy matrix."""
    N, qs, phi0, dt = 8, 10.0, 1.0, 0.01
    dx = 2.0 * np.sin(np.pi / N) / 0.5
    k2 = (2.0 * np.sin(np.pi / N) / dx) ** 2
    m = ScalarModel(N=N, Ns=2, pexp=2, dx=dx, alpha=0.0, fmp2=0.0, lam=1.0, q=qs)
    x = np.arange(N)
    mode = np.broadcast_to(np.cos(2 * np.pi * x / N)[None, None, :], (N, N, N))
    eps = 1e-9
    phi = np.stack([np.full((N, N, N), phi0), eps * mode])
    lat = ScalarLattice(m, phi, np.zeros_like(phi))
    sol, lam_max = _mathieu_reference(k2, qs, phi0, 8 * np.pi)
    amps = []
    steps_per_period = int(round(np.pi / dt))
    dtp = np.pi / steps_per_period
    for n in range(8):
        lat.vv_steps(oracle.VV4, dtp, steps_per_period)
        c = (lat.phi[1] * mode).sum() / (mode * mode).sum() / eps
        amps.append(c)
        ref = sol.sol((n + 1) * np.pi)[0]
        assert abs(c - ref) < 1e-5 * max(1.0, abs(ref)), (n, c, ref)  # VV4 error at dt = pi/314, amplified e^{6}
    assert abs(lat.phi[0].mean() - phi0 * np.cos(8 * np.pi)) < 1e-9
    growth = abs(amps[-1] / amps[-2])
    assert abs(growth - lam_max) < 0.02 * lam_max, (growth, lam_max)
    assert np.log(lam_max) / np.pi > 0.2  # a genuine instability band
