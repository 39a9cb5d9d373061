"""ctypes front of the oracle's C core, plus the integrator weights.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).
"""
import ctypes as C
from dataclasses import dataclass

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(_build.build())
        d = C.POINTER(C.c_double)
        vp = C.c_void_p
        for name, args, res in [
            ("orc_scalar_kernel", [vp, d, C.c_double, d], None),
            ("orc_scalar_energies", [vp, d, d, C.c_double, d], None),
            ("orc_scalar_Ka", [vp, C.c_double, d], C.c_double),
            ("orc_scalar_hubble_rhs", [vp, C.c_double, d], C.c_double),
            ("orc_scalar_vv_step", [vp, C.c_int, d, C.c_double, d, d, d, d], None),
            ("orc_scalar_lf3_prepare", [vp, C.c_double, d, d, C.c_double, d, d], None),
            ("orc_scalar_lf3_step", [vp, C.c_double, d, d, d, d, d, d], None),
            ("orc_u1_kernels", [vp, d, d, C.c_double, d, d], None),
            ("orc_u1_energies", [vp, d, d, d, d, C.c_double, d], None),
            ("orc_u1_Ka", [vp, C.c_double, d], C.c_double),
            ("orc_u1_gauss", [vp, d, d, d, d, d, d], None),
            ("orc_u1_lf_prepare", [vp, C.c_double, d, d, d, d, C.c_double, d, d, d], None),
            ("orc_u1_lf_step", [vp, C.c_double, d, d, d, d, d, d, d, d], None),
            ("orc_u1_vv_step", [vp, C.c_int, d, C.c_double, d, d, d, d, d, d], None),
            ("orc_scalar_vv_step_fluid", [vp, vp, C.c_int, d, C.c_double, d, d, d], None),
            ("orc_scalar_rk4_step", [vp, C.c_double, d, d, d, d], None),
            ("orc_scalar_gl_step", [vp, C.c_int, d, d, C.c_double, C.c_double, C.c_int, d, d, d, d], C.c_int),
            ("orc_su2_kernels", [vp, d, d, C.c_double, d, d], None),
            ("orc_su2_energies", [vp, d, d, d, d, C.c_double, d], None),
            ("orc_su2_Ka", [vp, C.c_double, d], C.c_double),
            ("orc_su2_gauss", [vp, d, d, d, d, d], None),
            ("orc_su2_vv_step", [vp, C.c_int, d, C.c_double, d, d, d, d, d, d], None),
            ("orc_su2u1_kernels", [vp, d, d, d, d, C.c_double, d, d, d, d], None),
            ("orc_su2u1_energies", [vp, d, d, d, d, d, d, d, d, C.c_double, d], None),
            ("orc_su2u1_Ka", [vp, C.c_double, d], C.c_double),
            ("orc_su2u1_gauss", [vp, d, d, d, d, d, d], None),
            ("orc_su2u1_vv_step", [vp, C.c_int, d, C.c_double, d, d, d, d, d, d, d, d, d, d], None),
            ("orc_set_threads", [C.c_int], None),
            ("orc_max_threads", [], C.c_int),
        ]:
            f = getattr(_lib, name)
            f.argtypes = args
            f.restype = res
    return _lib


def _p(x):
    assert x.dtype == np.float64 and x.flags.c_contiguous
    return x.ctypes.data_as(C.POINTER(C.c_double))


class _ScalarModelC(C.Structure):
    _fields_ = [("N", C.c_int64), ("Ns", C.c_int32), ("pexp", C.c_int32), ("dx", C.c_double),
                ("alpha", C.c_double), ("fmp2", C.c_double), ("lam", C.c_double), ("q", C.c_double)]


class _U1ModelC(C.Structure):
    _fields_ = [("N", C.c_int64), ("dx", C.c_double), ("alpha", C.c_double), ("fmp2", C.c_double),
                ("lam", C.c_double), ("v2", C.c_double), ("e", C.c_double), ("kappa", C.c_double),
                ("pot", C.c_int32), ("p", C.c_int32), ("noncompact", C.c_int32), ("pad", C.c_int32)]


# --- Yoshida weights (section 3.4.1 and the appendix table of VVn weights) ---
# VV4 is written in closed form, w1 = w3 = 1/(2 - 2^(1/3)), w2 = -2^(1/3)/(2 - 2^(1/3)),
# because the printed w2 of the table makes the three weights sum to 1 - 2e-8.
_C3 = 2.0 ** (1.0 / 3.0)
VV2 = (1.0,)
VV4 = (1.0 / (2.0 - _C3), -_C3 / (2.0 - _C3), 1.0 / (2.0 - _C3))
_VV6_HALF = (0.78451361047755726382, 0.23557321335935813368, -1.1776799841788710069, 1.3151863206839112189)
_VV8_HALF = (0.74167036435061295345, -0.40910082580003159400, 0.19075471029623837995, -0.57386247111608226666,
             0.29906418130365592384, 0.33462491824529818378, 0.31529309239676659663, -0.79688793935291635402)
_VV10_HALF = (-0.48159895600253002870, 0.0036303931544595926879, 0.50180317558723140279, 0.28298402624506254868,
              0.80702967895372223806, -0.026090580538592205447, -0.87286590146318071547, -0.52373568062510581643,
              0.44521844299952789252, 0.18612289547097907887, 0.23137327866438360633, -0.52191036590418628905,
              0.74866113714499296793, 0.066736511890604057532, -0.80360324375670830316, 0.91249037635867994571)


def _sym(half):
    return tuple(half) + tuple(reversed(half[:-1]))


VV6 = _sym(_VV6_HALF)
VV8 = _sym(_VV8_HALF)
VV10 = _sym(_VV10_HALF)


@dataclass
class ScalarModel:
    """Program-unit scalar model of sections 4 and 8.1:
    V = (lam/p)|phi|^p + (q/2) phi^2 chi^2, Ns = 1 or 2 fields."""
    N: int
    Ns: int
    pexp: int
    dx: float
    alpha: float
    fmp2: float
    lam: float = 1.0
    q: float = 0.0

    def c(self):
        return _ScalarModelC(self.N, self.Ns, self.pexp, self.dx, self.alpha, self.fmp2, self.lam, self.q)


def gl_tableau(s):
    """Butcher tableau (A, c) of the s-stage Gauss-Legendre method from its
    definition (section 3.4.2): collocation at the roots tau_i of the shifted
    Legendre polynomial P_s(2 tau - 1), A_ij = int_0^{tau_i} l_j, c_j = int_0^1 l_j
    with l_j the Lagrange basis on the nodes."""
    x, _ = np.polynomial.legendre.leggauss(s)
    tau = (x + 1.0) / 2.0
    A = np.zeros((s, s))
    c = np.zeros(s)
    for j in range(s):
        lj = np.poly1d([1.0])
        for k in range(s):
            if k != j:
                lj = lj * np.poly1d([1.0, -tau[k]]) / (tau[j] - tau[k])
        P = lj.integ()
        c[j] = P(1.0) - P(0.0)
        for i in range(s):
            A[i, j] = P(tau[i]) - P(0.0)
    return A, c


class _FluidC(C.Structure):
    _fields_ = [("a0", C.c_double), ("H0", C.c_double), ("p", C.c_double)]


@dataclass
class Fluid:
    """Scale factor sourced by an external fluid of equation of state w
    (section 4.1): a(eta) = a0 (1 + H0 eta / p)^p, p = 2/(3(1 + w) - 2 alpha)."""
    a0: float
    H0: float
    w: float
    alpha: float

    @property
    def p(self):
        return 2.0 / (3.0 * (1.0 + self.w) - 2.0 * self.alpha)

    def a(self, t):
        return self.a0 * (1.0 + self.H0 * t / self.p) ** self.p

    def b(self, t):
        return self.a0 * self.H0 * (1.0 + self.H0 * t / self.p) ** (self.p - 1.0)


@dataclass
class U1Model:
    """Program-unit charged scalar of section 5 with V = (lam/4)(|phi|^2 - v2)^2
    (Abelian-Higgs, pot = 0) or the monomial inflaton V = (lam/p)(2|phi|^2)^(p/2)
    of section 8 (pot = 1); gauge coupling e, kappa = (omega*/f*)^2; the compact
    (section 5.3) or, with noncompact = 1, the non-compact (section 5.2) gauge
    kinetics."""
    N: int
    dx: float
    alpha: float
    fmp2: float
    lam: float = 1.0
    v2: float = 1.0
    e: float = 1.0
    kappa: float = 1.0
    pot: int = 0
    p: int = 4
    noncompact: int = 0

    def c(self):
        return _U1ModelC(self.N, self.dx, self.alpha, self.fmp2, self.lam, self.v2, self.e, self.kappa, self.pot,
                         self.p, self.noncompact, 0)


def potential_terms(m, phi, chi=None):
    """V_1 = (lam/p)|phi|^p, V_2 = (q/2) phi^2 chi^2 (numpy, elementwise)."""
    v1 = m.lam / m.pexp * np.abs(phi) ** m.pexp
    v2 = 0.5 * m.q * phi ** 2 * chi ** 2 if (m.Ns > 1 and chi is not None) else 0.0 * phi
    return v1, v2


def potential_curvature(m, phibar):
    """d^2V/dphi_i^2 at homogeneous values phibar (section 8.1)."""
    f0 = phibar[0]
    f1 = phibar[1] if m.Ns > 1 else 0.0
    out = [(m.pexp - 1) * m.lam * abs(f0) ** (m.pexp - 2) + (m.q * f1 * f1 if m.Ns > 1 else 0.0)]
    if m.Ns > 1:
        out.append(m.q * f0 * f0)
    return out


class ScalarLattice:
    """Scalar lattice state (phi, pi: float64 arrays of shape (Ns, N, N, N)),
    with a and b = a' in program units."""

    def __init__(self, model, phi, pi, a=1.0, b=0.0):
        self.m = model
        self._mc = model.c()
        self.phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(model.Ns, model.N, model.N, model.N).copy()
        self.pi = np.ascontiguousarray(pi, dtype=np.float64).reshape(model.Ns, model.N, model.N, model.N).copy()
        self.a = float(a)
        self.b = float(b)
        self.EKm = None  # E_K at the previous half step (leapfrog only)

    def _mp(self):
        return C.byref(self._mc)

    def kernel(self, a=None):
        K = np.zeros_like(self.phi)
        lib().orc_scalar_kernel(self._mp(), _p(self.phi), self.a if a is None else a, _p(K))
        return K

    def energies(self):
        out = np.zeros(6)
        lib().orc_scalar_energies(self._mp(), _p(self.phi), _p(self.pi), self.a, _p(out))
        return out

    def Ka(self, E=None):
        E = self.energies() if E is None else np.ascontiguousarray(E, dtype=np.float64)
        return lib().orc_scalar_Ka(self._mp(), self.a, _p(E))

    def hubble_rhs(self, E=None):
        E = self.energies() if E is None else np.ascontiguousarray(E, dtype=np.float64)
        return lib().orc_scalar_hubble_rhs(self._mp(), self.a, _p(E))

    def vv_steps(self, weights, dt, n=1):
        w = np.ascontiguousarray(weights, dtype=np.float64)
        a = C.c_double(self.a)
        b = C.c_double(self.b)
        for _ in range(n):
            lib().orc_scalar_vv_step(self._mp(), len(w), _p(w), dt, _p(self.phi), _p(self.pi), C.byref(a), C.byref(b))
        self.a, self.b = a.value, b.value

    def vv_steps_fluid(self, fluid, weights, dt, n=1):
        """VVn with the scale factor of an external fluid (section 4.1):
        fluid = Fluid(a0, H0, w, alpha); self.t is the program time."""
        w = np.ascontiguousarray(weights, dtype=np.float64)
        f = _FluidC(fluid.a0, fluid.H0, fluid.p)
        t = C.c_double(getattr(self, "t", 0.0))
        for _ in range(n):
            lib().orc_scalar_vv_step_fluid(self._mp(), C.byref(f), len(w), _p(w), dt, _p(self.phi), _p(self.pi),
                                           C.byref(t))
        self.t = t.value
        self.a = fluid.a(self.t)
        self.b = fluid.b(self.t)

    def rk4_steps(self, dt, n=1):
        """Explicit RK4 of section 4.3.1.  The scheme integrates the velocities
        v = phi'; self.pi (Hamiltonian momenta a^{3-alpha} phi') is converted
        to v before and back after the steps."""
        v = np.ascontiguousarray(self.pi / self.a ** (3.0 - self.m.alpha))
        a, b = C.c_double(self.a), C.c_double(self.b)
        for _ in range(n):
            lib().orc_scalar_rk4_step(self._mp(), dt, _p(self.phi), _p(v), C.byref(a), C.byref(b))
        self.a, self.b = a.value, b.value
        self.pi = v * self.a ** (3.0 - self.m.alpha)

    def gl_steps(self, s, dt, n=1, tol=1e-14, maxit=60):
        """Gauss-Legendre implicit RK with s stages (order 2s; sections 3.4.2, 4.3.3,
        Scheme II).  Returns the fixed-point sweeps of the last step."""
        A, c = gl_tableau(s)
        A = np.ascontiguousarray(A)
        c = np.ascontiguousarray(c)
        a, b = C.c_double(self.a), C.c_double(self.b)
        it = 0
        for _ in range(n):
            it = lib().orc_scalar_gl_step(self._mp(), s, _p(A), _p(c), dt, tol, maxit, _p(self.phi), _p(self.pi),
                                          C.byref(a), C.byref(b))
        self.a, self.b = a.value, b.value
        return it

    def lf3_prepare(self, dt):
        b = C.c_double(self.b)
        ekm = C.c_double(0.0)
        lib().orc_scalar_lf3_prepare(self._mp(), dt, _p(self.phi), _p(self.pi), self.a, C.byref(b), C.byref(ekm))
        self.b, self.EKm = b.value, ekm.value

    def lf3_steps(self, dt, n=1, diag=False):
        a, b, ekm = C.c_double(self.a), C.c_double(self.b), C.c_double(self.EKm)
        rows = []
        d = np.zeros(5)
        for _ in range(n):
            lib().orc_scalar_lf3_step(self._mp(), dt, _p(self.phi), _p(self.pi), C.byref(a), C.byref(b),
                                      C.byref(ekm), _p(d))
            if diag:
                rows.append(d.copy())
        self.a, self.b, self.EKm = a.value, b.value, ekm.value
        return np.array(rows) if diag else None

    def hubble_violation(self):
        """Delta_e = |b^2 - rhs| / rhs of the Hubble constraint (synchronized state)."""
        rhs = self.hubble_rhs()
        return abs(self.b ** 2 - rhs) / rhs


class U1Lattice:
    """Compact U(1) state: phi, pi of shape (2, N, N, N) (real and imaginary
    planes of the complex field), theta, piA of shape (3, N, N, N)."""

    def __init__(self, model, phi, pi, theta, piA, a=1.0, b=0.0):
        self.m = model
        self._mc = model.c()
        N = model.N
        self.phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(2, N, N, N).copy()
        self.pi = np.ascontiguousarray(pi, dtype=np.float64).reshape(2, N, N, N).copy()
        self.theta = np.ascontiguousarray(theta, dtype=np.float64).reshape(3, N, N, N).copy()
        self.piA = np.ascontiguousarray(piA, dtype=np.float64).reshape(3, N, N, N).copy()
        self.a, self.b = float(a), float(b)
        self.EKm = None

    def _mp(self):
        return C.byref(self._mc)

    def kernels(self):
        Kp = np.zeros_like(self.phi)
        KA = np.zeros_like(self.theta)
        lib().orc_u1_kernels(self._mp(), _p(self.phi), _p(self.theta), self.a, _p(Kp), _p(KA))
        return Kp, KA

    def energies(self):
        out = np.zeros(5)
        lib().orc_u1_energies(self._mp(), _p(self.phi), _p(self.pi), _p(self.theta), _p(self.piA), self.a, _p(out))
        return out

    def gauss(self, return_fields=False):
        N = self.m.N
        lhs = np.zeros((N, N, N))
        rhs = np.zeros((N, N, N))
        out = np.zeros(3)
        lib().orc_u1_gauss(self._mp(), _p(self.phi), _p(self.pi), _p(self.piA), _p(lhs), _p(rhs), _p(out))
        dg = np.sqrt(out[0]) / np.sqrt(out[1] + out[2]) if out[1] + out[2] > 0 else np.sqrt(out[0])
        return (dg, lhs, rhs) if return_fields else dg

    def lf_prepare(self, dt):
        b, ek, eka = C.c_double(self.b), C.c_double(0), C.c_double(0)
        lib().orc_u1_lf_prepare(self._mp(), dt, _p(self.phi), _p(self.pi), _p(self.theta), _p(self.piA), self.a,
                                C.byref(b), C.byref(ek), C.byref(eka))
        self.b, self.EKm = b.value, (ek.value, eka.value)

    def electric(self):
        """E_i = piA_i / a^{1-alpha} (section 5.4), shape (3, N, N, N)."""
        return self.piA / self.a ** (1.0 - self.m.alpha)

    def magnetic(self):
        """B_i with (i, j, k) cyclic (section 5.4): sin(theta_jk)/(e dx^2) in the
        compact formulation (-Im V_jk/(e dx^2), V_jk = exp(-i theta_jk)), the
        lattice curl theta_jk/(e dx^2) = eps_ijk D_j^+ A_k in the non-compact one."""
        return _u1_magnetic(self.theta, self.m.e, self.m.dx, self.m.noncompact)

    def vv_steps(self, weights, dt, n=1):
        """Compact velocity-Verlet VVn (sections 5.3.2, 5.3.3) on synchronized data."""
        w = np.ascontiguousarray(weights, dtype=np.float64)
        a, b = C.c_double(self.a), C.c_double(self.b)
        for _ in range(n):
            lib().orc_u1_vv_step(self._mp(), len(w), _p(w), dt, _p(self.phi), _p(self.pi), _p(self.theta),
                                 _p(self.piA), C.byref(a), C.byref(b))
        self.a, self.b = a.value, b.value

    def lf_steps(self, dt, n=1):
        a, b = C.c_double(self.a), C.c_double(self.b)
        ek, eka = C.c_double(self.EKm[0]), C.c_double(self.EKm[1])
        for _ in range(n):
            lib().orc_u1_lf_step(self._mp(), dt, _p(self.phi), _p(self.pi), _p(self.theta), _p(self.piA),
                                 C.byref(a), C.byref(b), C.byref(ek), C.byref(eka))
        self.a, self.b, self.EKm = a.value, b.value, (ek.value, eka.value)


class _SU2ModelC(C.Structure):
    _fields_ = [("N", C.c_int64), ("dx", C.c_double), ("alpha", C.c_double), ("fmp2", C.c_double),
                ("lam", C.c_double), ("v2", C.c_double), ("g", C.c_double), ("kappa", C.c_double),
                ("pot", C.c_int32), ("p", C.c_int32)]


@dataclass
class SU2Model:
    """Program-unit SU(2)-Higgs model of section 6: V = (lam/4)(|Phi|^2 - v2)^2
    (pot = 0) or the monomial inflaton (lam/p)(2|Phi|^2)^(p/2) of section 8
    (pot = 1); gauge coupling g = g_B Q_B, kappa = (omega*/f*)^2."""
    N: int
    dx: float
    alpha: float
    fmp2: float
    lam: float = 1.0
    v2: float = 1.0
    g: float = 1.0
    kappa: float = 1.0
    pot: int = 0
    p: int = 4

    def c(self):
        return _SU2ModelC(self.N, self.dx, self.alpha, self.fmp2, self.lam, self.v2, self.g, self.kappa, self.pot,
                          self.p)


class SU2Lattice:
    """SU(2) state: phi, pi of shape (4, N, N, N) (Re/Im of the two doublet
    components), links u of shape (3, 4, N, N, N) (unit quaternions
    q0 + i q.sigma), piB of shape (3, 3, N, N, N)."""

    def __init__(self, model, phi, pi, u, piB, a=1.0, b=0.0):
        N = model.N
        self.m = model
        self.phi = np.ascontiguousarray(phi, dtype=np.float64).reshape(4, N, N, N).copy()
        self.pi = np.ascontiguousarray(pi, dtype=np.float64).reshape(4, N, N, N).copy()
        self.u = np.ascontiguousarray(u, dtype=np.float64).reshape(3, 4, N, N, N).copy()
        self.piB = np.ascontiguousarray(piB, dtype=np.float64).reshape(3, 3, N, N, N).copy()
        self.a, self.b = a, b

    def _mp(self):
        self._mc = self.m.c()
        return C.byref(self._mc)

    def kernels(self):
        Kp = np.zeros_like(self.phi)
        KB = np.zeros_like(self.piB)
        lib().orc_su2_kernels(self._mp(), _p(self.phi), _p(self.u), self.a, _p(Kp), _p(KB))
        return Kp, KB

    def energies(self):
        out = np.zeros(5)
        lib().orc_su2_energies(self._mp(), _p(self.phi), _p(self.pi), _p(self.u), _p(self.piB), self.a, _p(out))
        return out

    def Ka(self):
        E = np.ascontiguousarray(self.energies())
        return lib().orc_su2_Ka(self._mp(), self.a, _p(E))

    def gauss(self):
        out = np.zeros(3)
        lib().orc_su2_gauss(self._mp(), _p(self.phi), _p(self.pi), _p(self.u), _p(self.piB), _p(out))
        return out[0] / max(out[1] + out[2], 1e-300)

    def electric(self):
        """E_i^a = piB_i^a / a^{1-alpha} (section 6.3), shape (3, 3, N, N, N)."""
        return self.piB / self.a ** (1.0 - self.m.alpha)

    def magnetic(self):
        """B_i^a = (eps_ijk/(2 g dx^2)) Tr[(i sigma^a/2)(U_jk - U_kj)] (section 6.3),
        i.e. -2 q_a[U_jk]/(g dx^2) for (i, j, k) cyclic, shape (3, 3, N, N, N)."""
        return _su2_magnetic(self.u, self.m.g, self.m.dx)

    def vv_steps(self, weights, dt, n=1):
        """SU(2) velocity-Verlet VVn (sections 6.2.2, 6.2.3) on synchronized data."""
        w = np.ascontiguousarray(weights, dtype=np.float64)
        a, b = C.c_double(self.a), C.c_double(self.b)
        for _ in range(n):
            lib().orc_su2_vv_step(self._mp(), len(w), _p(w), dt, _p(self.phi), _p(self.pi), _p(self.u),
                                  _p(self.piB), C.byref(a), C.byref(b))
        self.a, self.b = a.value, b.value


class _SU2U1ModelC(C.Structure):
    _fields_ = [("N", C.c_int64), ("dx", C.c_double), ("alpha", C.c_double), ("fmp2", C.c_double),
                ("lam", C.c_double), ("v2", C.c_double), ("g", C.c_double), ("kappa", C.c_double),
                ("pot", C.c_int32), ("p", C.c_int32), ("eA", C.c_double), ("q", C.c_double),
                ("chi", C.c_int32), ("pad", C.c_int32)]


@dataclass
class SU2U1Model:
    """Program-unit doublet of the working example of section 8.3: SU(2)
    coupling g = g_B Q_B, U(1) coupling eA = g_A Q_A (0: no U(1) sector), a
    real singlet chi (chi = 1) with V_int = q |Phi|^2 chi^2, and the Higgs
    (pot = 0) or monomial (pot = 1) potential of the doublet."""
    N: int
    dx: float
    alpha: float
    fmp2: float
    lam: float = 1.0
    v2: float = 1.0
    g: float = 1.0
    kappa: float = 1.0
    pot: int = 0
    p: int = 4
    eA: float = 1.0
    q: float = 0.0
    chi: int = 1

    def c(self):
        return _SU2U1ModelC(self.N, self.dx, self.alpha, self.fmp2, self.lam, self.v2, self.g, self.kappa, self.pot,
                            self.p, self.eA, self.q, self.chi, 0)

    def su2(self):
        return SU2Model(N=self.N, dx=self.dx, alpha=self.alpha, fmp2=self.fmp2, lam=self.lam, v2=self.v2, g=self.g,
                        kappa=self.kappa, pot=self.pot, p=self.p)


class SU2U1Lattice:
    """SU(2) x U(1) + chi state: the SU(2) arrays of SU2Lattice plus link
    angles theta and electric momenta piA of shape (3, N, N, N) and the singlet
    chi, pchi of shape (N, N, N)."""

    def __init__(self, model, phi, pi, u, piB, theta=None, piA=None, chi=None, pchi=None, a=1.0, b=0.0):
        N = model.N
        self.m = model
        arr = lambda x, shape: (np.zeros(shape) if x is None else
                                np.ascontiguousarray(x, dtype=np.float64).reshape(shape).copy())
        self.phi = arr(phi, (4, N, N, N))
        self.pi = arr(pi, (4, N, N, N))
        self.u = arr(u, (3, 4, N, N, N))
        self.piB = arr(piB, (3, 3, N, N, N))
        self.theta = arr(theta, (3, N, N, N))
        self.piA = arr(piA, (3, N, N, N))
        self.chi = arr(chi, (N, N, N))
        self.pchi = arr(pchi, (N, N, N))
        self.a, self.b = a, b

    def _mp(self):
        self._mc = self.m.c()
        return C.byref(self._mc)

    def kernels(self):
        Kp, KB = np.zeros_like(self.phi), np.zeros_like(self.piB)
        KA, Kc = np.zeros_like(self.piA), np.zeros_like(self.chi)
        lib().orc_su2u1_kernels(self._mp(), _p(self.phi), _p(self.u), _p(self.theta), _p(self.chi), self.a, _p(Kp),
                                _p(KB), _p(KA), _p(Kc))
        return Kp, KB, KA, Kc

    def energies(self):
        """E_K^Phi, E_G^Phi, E_V, E_K^B, E_G^B, E_K^A, E_G^A, E_K^chi, E_G^chi."""
        out = np.zeros(9)
        lib().orc_su2u1_energies(self._mp(), _p(self.phi), _p(self.pi), _p(self.u), _p(self.piB), _p(self.theta),
                                 _p(self.piA), _p(self.chi), _p(self.pchi), self.a, _p(out))
        return out

    def Ka(self):
        E = np.ascontiguousarray(self.energies())
        return lib().orc_su2u1_Ka(self._mp(), self.a, _p(E))

    def gauss(self):
        """(SU(2), U(1)) Gauss residuals <G^2>/(<lhs^2> + <rhs^2>)."""
        out = np.zeros(6)
        lib().orc_su2u1_gauss(self._mp(), _p(self.phi), _p(self.pi), _p(self.u), _p(self.piB), _p(self.piA), _p(out))
        return out[0] / max(out[1] + out[2], 1e-300), out[3] / max(out[4] + out[5], 1e-300)

    def electric(self, sector):
        """E of the U(1) (sector 0) or SU(2) (sector 1) field."""
        return (self.piA if sector == 0 else self.piB) / self.a ** (1.0 - self.m.alpha)

    def magnetic(self, sector):
        return _u1_magnetic(self.theta, self.m.eA, self.m.dx, 0) if sector == 0 else _su2_magnetic(self.u, self.m.g,
                                                                                                      self.m.dx)

    def vv_steps(self, weights, dt, n=1):
        w = np.ascontiguousarray(weights, dtype=np.float64)
        a, b = C.c_double(self.a), C.c_double(self.b)
        for _ in range(n):
            lib().orc_su2u1_vv_step(self._mp(), len(w), _p(w), dt, _p(self.phi), _p(self.pi), _p(self.u),
                                    _p(self.piB), _p(self.theta), _p(self.piA), _p(self.chi), _p(self.pchi),
                                    C.byref(a), C.byref(b))
        self.a, self.b = a.value, b.value


def _shift(a, d):
    """a(n + d^) on the periodic lattice, arrays indexed [z, y, x], d = 0, 1, 2 for x, y, z."""
    return np.roll(a, -1, axis=a.ndim - 1 - d)


def _u1_magnetic(theta, e, dx, noncompact):
    out = np.zeros_like(theta)
    for i in range(3):
        j, k = (i + 1) % 3, (i + 2) % 3
        t = theta[j] + _shift(theta[k], j) - _shift(theta[j], k) - theta[k]
        out[i] = (t if noncompact else np.sin(t)) / (e * dx * dx)
    return out


def _qmul(p, q):
    r0 = p[0] * q[0] - p[1] * q[1] - p[2] * q[2] - p[3] * q[3]
    r1 = p[0] * q[1] + q[0] * p[1] - (p[2] * q[3] - p[3] * q[2])
    r2 = p[0] * q[2] + q[0] * p[2] - (p[3] * q[1] - p[1] * q[3])
    r3 = p[0] * q[3] + q[0] * p[3] - (p[1] * q[2] - p[2] * q[1])
    return np.stack([r0, r1, r2, r3])


def _su2_magnetic(u, g, dx):
    conj = np.array([1.0, -1.0, -1.0, -1.0])[:, None, None, None]
    out = np.zeros((3, 3) + u.shape[2:])
    for i in range(3):
        j, k = (i + 1) % 3, (i + 2) % 3
        P = _qmul(_qmul(_qmul(u[j], _shift(u[k], j)), conj * _shift(u[j], k)), conj * u[k])
        out[i] = -2.0 * P[1:] / (g * dx * dx)
    return out
