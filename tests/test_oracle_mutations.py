"""The oracle's pins catch plausible mistakes in the oracle.

Each case plants one mistake in a scratch copy of oracle/: a wrong neighbour,
a flipped sign, a dropped conjugate, a wrong power of the scale factor, a
wrong constant.  It then runs the pin files that cover that part in a
subprocess and requires at least one pin to fail: a real test failure, not a
build or collection error.  An unmutated copy must pass the same files, so a
failure is the mistake's doing.

The cases cover:
  - the scalar sector of section 4: the Laplacian, the section-8.1 potential,
    the Hamiltonian energies, the scale-factor kernel, the drifts and kicks of
    velocity-Verlet and of leapfrog scheme III, the Yoshida weights, the
    prescribed fluid background, RK4 and the Gauss-Legendre stages;
  - the U(1) sector of section 5: forces, currents, parallel transport, the
    gauge energies and their weight in the Friedmann kernel, the Gauss law;
  - the SU(2) toolkit of section 3.2.3 and the sector of section 6: quaternion
    algebra, the doublet action of a link, the Pauli projections, the adjoint
    transport of the Gauss law, the exact link drift;
  - the SU(2) x U(1) + chi working example of section 8.3: the combined hop,
    the U(1) current, the singlet's kernel and energies, both Gauss laws;
  - the spectra of section 3.1 and the vacuum initial conditions of section 7
    (mode variances, the Hubble term, the charge constraints, the Gauss solve);
  - the counter-based generator, the surrogate MLP and the scan observables.

Only oracle/ is touched, and only in a temporary directory; no GPU is used.
"""
import os
import shutil
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

# (name, oracle file, original text, planted text, pin files)
CASES = [
    ("laplacian-wrong-neighbour", "lattice_oracle.c",
     "f[site(N, x, y, wrap(z + 1, N))] + f[site(N, x, y, wrap(z - 1, N))] -",
     "f[site(N, x, y, wrap(z + 1, N))] + f[site(N, x, y, wrap(z + 1, N))] -", ["test_oracle_scalar.py"]),
    ("laplacian-diagonal", "lattice_oracle.c", "6.0 * f[n]) * idx2;", "4.0 * f[n]) * idx2;",
     ["test_oracle_scalar.py"]),
    ("interaction-force-sign", "lattice_oracle.c", "*dchi = m->q * phi * phi * chi;",
     "*dchi = -m->q * phi * phi * chi;", ["test_oracle_scalar.py"]),
    ("interaction-energy-factor", "lattice_oracle.c", "? 0.5 * m->q * phi * phi * chi * chi : 0.0;",
     "? m->q * phi * phi * chi * chi : 0.0;", ["test_oracle_scalar.py"]),
    ("kinetic-energy-a-power", "lattice_oracle.c", "out[i] = sk[i] / V / (2.0 * a6);",
     "out[i] = sk[i] / V / (2.0 * a2);", ["test_oracle_scalar.py"]),
    ("friedmann-kernel-coefficient", "lattice_oracle.c", "           ((m->alpha - 2.0) * EK + m->alpha * EG",
     "           ((m->alpha - 1.0) * EK + m->alpha * EG", ["test_oracle_scalar.py"]),
    ("kernel-gradient-a-power", "lattice_oracle.c",
     "const double a1 = pow(a, 1.0 + m->alpha), a3 = pow(a, 3.0 + m->alpha);\n",
     "const double a1 = pow(a, 2.0 + m->alpha), a3 = pow(a, 3.0 + m->alpha);\n", ["test_oracle_scalar.py"]),
    ("drift-a-power", "lattice_oracle.c", "drift(m, phi, pi, h * pow(ah, -(3.0 - m->alpha)));",
     "drift(m, phi, pi, h * pow(ah, -(1.0 - m->alpha)));", ["test_oracle_scalar.py"]),
    ("scale-factor-half-step", "lattice_oracle.c",
     "        *a = ah + 0.5 * h * bh;\n        kick(m, phi, pi, *a, 0.5 * h, K);\n        orc_scalar_energies(",
     "        *a = ah + h * bh;\n        kick(m, phi, pi, *a, 0.5 * h, K);\n        orc_scalar_energies(",
     ["test_oracle_scalar.py"]),
    ("u1-magnetic-force-sign", "lattice_oracle.c", "return m->noncompact ? t : sin(t); }",
     "return m->noncompact ? t : -sin(t); }", ["test_oracle_u1.py"]),
    ("u1-current-sign", "lattice_oracle.c", "const double cur = pr[n] * ui - pim[n] * ur;",
     "const double cur = pim[n] * ur - pr[n] * ui;", ["test_oracle_u1.py"]),
    ("u1-backward-link-conjugate", "lattice_oracle.c", "const double wr = cos(tm) * pr[nm] - sin(tm) * pim[nm];",
     "const double wr = cos(tm) * pr[nm] + sin(tm) * pim[nm];", ["test_oracle_u1.py"]),
    ("su2-quaternion-conjugate", "lattice_oracle.c", "r[0] = q[0]; r[1] = -q[1]; r[2] = -q[2]; r[3] = -q[3];",
     "r[0] = q[0]; r[1] = q[1]; r[2] = -q[2]; r[3] = -q[3];", ["test_oracle_su2.py"]),
    ("su2-product-cross-term", "lattice_oracle.c",
     "const double r1 = p[0] * q[1] + q[0] * p[1] - (p[2] * q[3] - p[3] * q[2]);",
     "const double r1 = p[0] * q[1] + q[0] * p[1] + (p[2] * q[3] - p[3] * q[2]);", ["test_oracle_su2.py"]),
    ("spectrum-power-of-k", "spectra.py", "Delta = k ** 3 / (2 * np.pi ** 2)", "Delta = k ** 2 / (2 * np.pi ** 2)",
     ["test_oracle_ic.py", "test_oracle_observe.py"]),
    ("ic-self-conjugate-amplitude", "ic.py", "F = np.where(selfc, np.sqrt(2.0) * G.real + 0j, F)",
     "F = np.where(selfc, G.real + 0j, F)", ["test_oracle_ic.py"]),
    ("philox-weyl-constant", "philox.py", "\nW0 = 0x9E3779B9\n", "\nW0 = 0x9E3779B8\n", ["test_oracle_ic.py"]),
    ("gelu-derivative", "mlp.py", "x * np.exp(-0.5 * x * x) / np.sqrt(2.0 * np.pi)",
     "x * np.exp(-x * x) / np.sqrt(2.0 * np.pi)", ["test_oracle_mlp.py"]),
    ("w-pressure", "observe.py", "out[1] = (EK - EG / 3.0 - EV) / rho", "out[1] = (EK - EG - EV) / rho",
     ["test_oracle_observe.py"]),
    ("lf3-drift-scale-factor", "lattice_oracle.c",
     "const double ah = 0.5 * (*a + an);\n    drift(m, phi, pi, dt * pow(ah",
     "const double ah = *a;\n    drift(m, phi, pi, dt * pow(ah", ["test_oracle_scalar.py"]),
    ("lf3-prepare-kinetic-a", "lattice_oracle.c",
     "*EKm = S / V / (2.0 * pow(ahm, 6.0));",
     "*EKm = S / V / (2.0 * pow(a, 6.0));", ["test_oracle_scalar.py"]),
    ("u1-electric-energy-factor", "lattice_oracle.c",
     "out[3] = m->kappa * ska / V / (2.0 * a4);\n    out[4] = m->kappa * sga",
     "out[3] = m->kappa * ska / V / a4;\n    out[4] = m->kappa * sga", ["test_oracle_u1.py"]),
    ("u1-magnetic-energy-a-power", "lattice_oracle.c",
     "out[4] = m->kappa * sga / V / (a4 * m->e * m->e * dx4);",
     "out[4] = m->kappa * sga / V / (a2 * m->e * m->e * dx4);", ["test_oracle_u1.py"]),
    ("u1-Ka-gauge-weight", "lattice_oracle.c",
     "(m->alpha + 1.0) * EV + (m->alpha - 1.0) * (EKA + EGA));",
     "(m->alpha + 1.0) * EV + (m->alpha - 2.0) * (EKA + EGA));", ["test_oracle_u1.py"]),
    ("u1-gauss-charge-factor", "lattice_oracle.c",
     "const double r = 2.0 * m->e / m->kappa * rho;",
     "const double r = m->e / m->kappa * rho;", ["test_oracle_u1.py", "test_oracle_ic.py"]),
    ("u1-lf-link-drift-a-power", "lattice_oracle.c",
     "const double cth = m->e * m->dx * dt * pow(ah, -(1.0 - m->alpha));",
     "const double cth = m->e * m->dx * dt * pow(ah, -(3.0 - m->alpha));", ["test_oracle_u1.py"]),
    ("u1-vv-scalar-drift-weight", "lattice_oracle.c",
     "const double cphi = h * pow(ah, -(3.0 - m->alpha));\n        const double cth = m->e",
     "const double cphi = dt * pow(ah, -(3.0 - m->alpha));\n        const double cth = m->e", ["test_oracle_u1.py"]),
    ("fluid-drift-midpoint", "lattice_oracle.c",
     "drift(m, phi, pi, h * pow(0.5 * (a + an), -(3.0 - m->alpha)));",
     "drift(m, phi, pi, h * pow(a, -(3.0 - m->alpha)));", ["test_oracle_scalar.py"]),
    ("fluid-exponent-alpha", "core.py",
     "return 2.0 / (3.0 * (1.0 + self.w) - 2.0 * self.alpha)",
     "return 2.0 / (3.0 * (1.0 + self.w) - self.alpha)", ["test_oracle_scalar.py"]),
    ("rk4-weights", "lattice_oracle.c",
     "w[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0}",
     "w[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 6.0, 1.0 / 3.0}", ["test_oracle_scalar.py"]),
    ("rk4-friction", "lattice_oracle.c",
     "c2 = (3.0 - m->alpha) * b / a",
     "c2 = (2.0 - m->alpha) * b / a", ["test_oracle_scalar.py"]),
    ("rk4-stage-node", "lattice_oracle.c",
     "c[4] = {0.0, 0.5, 0.5, 1.0}",
     "c[4] = {0.0, 0.5, 1.0, 1.0}", ["test_oracle_scalar.py"]),
    ("su2-gauss-transport-direction", "lattice_oracle.c",
     "qmul(qc, e, t);\n                    qmul(t, q, tr);",
     "qmul(q, e, t);\n                    qmul(t, qc, tr);", ["test_oracle_su2.py"]),
    ("su2-magnetic-energy-factor", "lattice_oracle.c",
     "out[4] = 2.0 * m->kappa * sgb / V / (a4 * dx4 * m->g * m->g);\n}",
     "out[4] = m->kappa * sgb / V / (a4 * dx4 * m->g * m->g);\n}", ["test_oracle_su2.py"]),
    ("su2-drift-half-angle", "lattice_oracle.c",
     "const double s = th > 0 ? sin(0.5 * th) / th : 0.5;",
     "const double s = th > 0 ? sin(th) / th : 0.5;", ["test_oracle_su2.py"]),
    ("su2-umul-entry", "lattice_oracle.c",
     "cr = -q[2], ci = q[1], dr = q[0]",
     "cr = -q[2], ci = -q[1], dr = q[0]", ["test_oracle_su2.py"]),
    ("su2-im-sigma2-sign", "lattice_oracle.c",
     "z[0] = y[3]; z[1] = -y[2]; z[2] = -y[1]; z[3] = y[0];",
     "z[0] = -y[3]; z[1] = y[2]; z[2] = y[1]; z[3] = -y[0];", ["test_oracle_su2.py"]),
    ("su2-current-coefficient", "lattice_oracle.c",
     "const double cJ = m->g / (m->kappa * m->dx), cM = 2.0 / (m->g * m->dx * m->dx * m->dx);\n#pragma omp parallel for schedule(static)\n    for (int64_t z = 0; z < N; ++z)\n        for (int64_t y = 0; y < N; ++y)\n            for (int64_t x = 0; x < N; ++x) {\n                const int64_t n = site(N, x, y, z);\n                double f[4], lap[4] = {0, 0, 0, 0};",
     "const double cJ = 2.0 * m->g / (m->kappa * m->dx), cM = 2.0 / (m->g * m->dx * m->dx * m->dx);\n#pragma omp parallel for schedule(static)\n    for (int64_t z = 0; z < N; ++z)\n        for (int64_t y = 0; y < N; ++y)\n            for (int64_t x = 0; x < N; ++x) {\n                const int64_t n = site(N, x, y, z);\n                double f[4], lap[4] = {0, 0, 0, 0};", ["test_oracle_su2.py"]),
    ("su2u1-whop-phase-sign", "lattice_oracle.c",
     "o[0] = c * u[0] + s * u[1];\n    o[1] = c * u[1] - s * u[0];\n    o[2] = c * u[2] + s * u[3];\n    o[3] = c * u[3] - s * u[2];",
     "o[0] = c * u[0] - s * u[1];\n    o[1] = c * u[1] + s * u[0];\n    o[2] = c * u[2] - s * u[3];\n    o[3] = c * u[3] + s * u[2];", ["test_oracle_su2u1.py"]),
    ("su2u1-KA-current-factor", "lattice_oracle.c",
     "KA[(int64_t)i * V + n] = A1 * 2.0 * m->eA / (m->kappa * m->dx) * im_dot(f, t)",
     "KA[(int64_t)i * V + n] = A1 * m->eA / (m->kappa * m->dx) * im_dot(f, t)", ["test_oracle_su2u1.py"]),
    ("su2u1-chi-kernel-factor", "lattice_oracle.c",
     "Kc[n] = -A3 * 2.0 * m->q * mod2 * chi[n]",
     "Kc[n] = -A3 * m->q * mod2 * chi[n]", ["test_oracle_su2u1.py"]),
    ("su2u1-Ka-drops-chi-kinetic", "lattice_oracle.c",
     "((m->alpha - 2.0) * (E[0] + E[7]) + m->alpha * (E[1] + E[8])",
     "((m->alpha - 2.0) * E[0] + m->alpha * (E[1] + E[8])", ["test_oracle_su2u1.py"]),
    ("su2u1-u1-gauss-charge", "lattice_oracle.c",
     "const double r = 2.0 * m->eA / m->kappa * im_dot(f, p);",
     "const double r = m->eA / m->kappa * im_dot(f, p);", ["test_oracle_su2u1.py"]),
    ("su2u1-chi-gradient-energy-factor", "lattice_oracle.c",
     "out[8] = sgc / V / dx2 / (2.0 * a2);",
     "out[8] = sgc / V / dx2 / a2;", ["test_oracle_su2u1.py"]),
    ("gl-stage-matrix-transposed", "lattice_oracle.c",
     "x += dt * A[l * s + mm] * Dold[(int64_t)(2 * mm) * M + n];\n                    y += dt * A[l * s + mm]",
     "x += dt * A[mm * s + l] * Dold[(int64_t)(2 * mm) * M + n];\n                    y += dt * A[mm * s + l]", ["test_oracle_scalar.py"]),
    ("gl-tableau-transposed", "core.py",
     "A[i, j] = P(tau[i]) - P(0.0)",
     "A[j, i] = P(tau[i]) - P(0.0)", ["test_oracle_scalar.py"]),
    ("vv8-weight-digit-slip", "core.py",
     "-0.40910082580003159400",
     "-0.40910028580003159400", ["test_oracle_scalar.py", "test_oracle_u1.py"]),
    ("vv4-closed-form", "core.py",
     "VV4 = (1.0 / (2.0 - _C3), -_C3 / (2.0 - _C3), 1.0 / (2.0 - _C3))",
     "VV4 = (1.0 / (2.0 - _C3), _C3 / (2.0 - _C3), 1.0 / (2.0 - _C3))", ["test_oracle_scalar.py"]),
    ("spectrum-volume-factor", "spectra.py",
     "(dx / N) ** 3 * sP",
     "(dx / N) ** 2 * sP", ["test_oracle_ic.py", "test_oracle_observe.py"]),
    ("spectrum-bins-rounded", "spectra.py",
     "    b = isqrt_array(n2)\n",
     "    b = np.rint(np.sqrt(n2)).astype(np.int64)\n", ["test_oracle_ic.py", "test_oracle_observe.py"]),
    ("observe-eps-chi-takes-interaction", "observe.py",
     "out[0] = (E[1] + E[3]) / rho",
     "out[0] = (E[1] + E[3] + E[5]) / rho", ["test_oracle_observe.py"]),
    ("observe-momentum-offset", "observe.py",
     "(np.arange(NK) + 0.5) / NK",
     "np.arange(NK) / NK", ["test_oracle_observe.py"]),
    ("mlp-bias-grad-mean", "mlp.py",
     "gb[l] = dZ.sum(axis=0)",
     "gb[l] = dZ.mean(axis=0)", ["test_oracle_mlp.py"]),
    ("mlp-loss-normalisation", "mlp.py",
     "dZ = 2.0 * (Y - T) / (B * n_out)",
     "dZ = 2.0 * (Y - T) / B", ["test_oracle_mlp.py"]),
    ("mlp-activation-derivative-argument", "mlp.py",
     "dZ = dH * gelu_prime(Z[l - 1])",
     "dZ = dH * gelu_prime(H[l])", ["test_oracle_mlp.py"]),
    ("mlp-flatten-order", "mlp.py",
     "np.concatenate([W.ravel(), b.ravel()])",
     "np.concatenate([b.ravel(), W.ravel()])", ["test_oracle_mlp.py"]),
    ("ic-charge-cancelling-phase", "ic.py",
     "th1r = th0r + th1l - th0l",
     "th1r = th0r - th1l + th0l", ["test_oracle_ic.py", "test_oracle_u1.py"]),
    ("ic-gauss-forward-difference", "ic.py",
     "    betas = [(1.0 - np.exp(2j * np.pi * c / N)) / dx for c in (nx, ny, nz)]",
     "    betas = [(1.0 - np.exp(-2j * np.pi * c / N)) / dx for c in (nx, ny, nz)]", ["test_oracle_ic.py", "test_oracle_u1.py"]),
    ("ic-singlet-hubble-sign", "ic.py",
     "(L * el - R * er) - H * G\n    return",
     "(L * el - R * er) + H * G\n    return", ["test_oracle_ic.py"]),
    ("ic-frequency-mass-a", "ic.py",
     "return np.sqrt(k * k + a * a * m2)",
     "return np.sqrt(k * k + m2)", ["test_oracle_ic.py"]),
    ("ic-rayleigh-mean-square", "ic.py",
     "\n    L = np.sqrt(-T * np.log(u[0]))\n",
     "\n    L = np.sqrt(-2.0 * T * np.log(u[0]))\n", ["test_oracle_ic.py"]),
    ("ic-su2-charge-removal-sign", "ic.py",
     "P1 = P1 - (cq[0] * 1j * F2",
     "P1 = P1 + (cq[0] * 1j * F2", ["test_oracle_ic.py", "test_oracle_su2.py"]),
    ("ic-momentum-a-power", "ic.py",
     "        pi[i] = a ** (3.0 - alpha) * (dphibar[i] + ddphi)",
     "        pi[i] = a ** (2.0 - alpha) * (dphibar[i] + ddphi)", ["test_oracle_ic.py", "test_oracle_scalar.py"]),
    ("su2u1-ic-phase-constraint", "ic.py",
     "er = np.exp(1j * thl[c]), np.exp(1j * (th0r + thl[c] - thl[0]))",
     "er = np.exp(1j * thl[c]), np.exp(1j * (th0r - thl[c] + thl[0]))", ["test_oracle_su2u1.py", "test_oracle_ic.py"]),
    ("su2-ic-charge-normalisation", "ic.py",
     "cq = rho.sum(axis=(1, 2, 3)) / (phi ** 2).sum()",
     "cq = rho.sum(axis=(1, 2, 3)) / (phi ** 2).mean()", ["test_oracle_su2.py", "test_oracle_ic.py"]),
    ("su2-charge-sigma2-sign", "ic.py",
     "np.imag(np.conj(x1) * (-1j * y2) + np.conj(x2) * (1j * y1))",
     "np.imag(np.conj(x1) * (1j * y2) + np.conj(x2) * (-1j * y1))", ["test_oracle_su2.py", "test_oracle_su2u1.py", "test_oracle_ic.py"]),
    ("gauss-solve-conjugate", "ic.py",
     "return [dft_inverse(np.where(den > 0, np.conj(bb) * R / den, 0.0)).real for bb in betas]",
     "return [dft_inverse(np.where(den > 0, bb * R / den, 0.0)).real for bb in betas]", ["test_oracle_su2.py", "test_oracle_su2u1.py", "test_oracle_ic.py"]),
    ("u1-magnetic-field-orientation", "core.py",
     "t = theta[j] + _shift(theta[k], j) - _shift(theta[j], k) - theta[k]",
     "t = theta[j] + _shift(theta[k], k) - _shift(theta[j], j) - theta[k]", ["test_oracle_u1.py", "test_oracle_su2u1.py"]),
    ("observe-interpolation-in-k", "observe.py",
     "return np.interp(np.log(kj), lk, lD)",
     "return np.interp(kj, np.exp(lk), lD)", ["test_oracle_observe.py"]),
    ("mode-map-axis-modes", "ic.py",
     "canon = (sx > 0) | ((sx == 0) & (sy > 0)) | ((sx == 0) & (sy == 0) & (sz > 0))",
     "canon = (sx > 0) | ((sx == 0) & (sy > 0))", ["test_oracle_ic.py"]),
    ("gelu-erf-argument", "mlp.py",
     "return 0.5 * x * (1.0 + erf(x / np.sqrt(2.0)))",
     "return 0.5 * x * (1.0 + erf(x / 2.0))", ["test_oracle_mlp.py"]),
    ("potential-curvature-factor", "core.py",
     "out = [(m.pexp - 1) * m.lam * abs(f0) ** (m.pexp - 2)",
     "out = [m.pexp * m.lam * abs(f0) ** (m.pexp - 2)", ["test_oracle_ic.py"]),
    ("gradient-energy-factor", "lattice_oracle.c",
     "out[2 + i] = sg[i] / V / (2.0 * a2);",
     "out[2 + i] = sg[i] / V / a2;", ["test_oracle_scalar.py"]),
    ("hubble-rhs-a-power", "lattice_oracle.c",
     "return m->fmp2 / 3.0 * pow(a, 2.0 * (m->alpha + 1.0)) * (EK + EG + EV);",
     "return m->fmp2 / 3.0 * pow(a, 2.0 * m->alpha + 1.0) * (EK + EG + EV);", ["test_oracle_scalar.py"]),
    ("potential-normalisation", "lattice_oracle.c",
     "*v1 = m->lam / m->pexp * ipow(fabs(phi), m->pexp);",
     "*v1 = m->lam * ipow(fabs(phi), m->pexp);", ["test_oracle_scalar.py"]),
    ("potential-gradient-power", "lattice_oracle.c",
     "*dphi = m->lam * ipow(fabs(phi), m->pexp - 2) * phi;",
     "*dphi = m->lam * ipow(fabs(phi), m->pexp - 1) * phi;", ["test_oracle_scalar.py"]),
    ("gauge-higgs-derivative", "lattice_oracle.c",
     "*dv = 0.5 * lam * (mod2 - v2);",
     "*dv = lam * (mod2 - v2);", ["test_oracle_u1.py", "test_oracle_su2.py"]),
    ("gauge-monomial-derivative", "lattice_oracle.c",
     "*dv = lam * pow(s, 0.5 * p - 1.0);",
     "*dv = 0.5 * lam * pow(s, 0.5 * p - 1.0);", ["test_oracle_u1.py", "test_oracle_su2.py"]),
    ("su2u1-vv-closing-b-half-kick", "lattice_oracle.c",
     "        *b += 0.5 * h * orc_su2u1_Ka(m, *a, E);\n    }",
     "        *b += h * orc_su2u1_Ka(m, *a, E);\n    }", ["test_oracle_su2u1.py"]),
    ("su2u1-vv-chi-drift-power", "lattice_oracle.c",
     "for (int64_t n = 0; n < V; ++n) chi[n] += cphi * pchi[n];",
     "for (int64_t n = 0; n < V; ++n) chi[n] += h * pchi[n];", ["test_oracle_su2u1.py"]),
    ("su2u1-vv-u1-link-drift-power", "lattice_oracle.c",
     "const double cth = m->eA * m->dx * h * pow(ah, -(1.0 - m->alpha));",
     "const double cth = m->eA * m->dx * h * pow(ah, -(3.0 - m->alpha));", ["test_oracle_su2u1.py"]),
    ("su2-vv-link-drift-coupling", "lattice_oracle.c",
     "su2_drift(m, phi, pi, u, piB, h * pow(ah, -(3.0 - m->alpha)), m->g * m->dx * h * pow(ah, -(1.0 - m->alpha)));",
     "su2_drift(m, phi, pi, u, piB, h * pow(ah, -(3.0 - m->alpha)), m->dx * h * pow(ah, -(1.0 - m->alpha)));", ["test_oracle_su2.py"]),
    ("u1-lf-prepare-electric-kinetic-power", "lattice_oracle.c",
     "*EKm_A = m->kappa * sa / V / (2.0 * pow(ahm, 4.0));",
     "*EKm_A = m->kappa * sa / V / (2.0 * pow(ahm, 6.0));", ["test_oracle_u1.py"]),
    ("u1-lf-prepare-b-half-kick", "lattice_oracle.c",
     "    *b -= 0.5 * dt * orc_u1_Ka(m, a, E);",
     "    *b -= dt * orc_u1_Ka(m, a, E);", ["test_oracle_u1.py"]),
    ("rk4-scale-factor-stage", "lattice_oracle.c",
     "const double an = *a + c[p] * dt * bp, bn = *b + c[p] * dt * ka;",
     "const double an = *a + c[p] * dt * *b, bn = *b + c[p] * dt * ka;", ["test_oracle_scalar.py"]),
    ("rk4-kinetic-energy-power", "lattice_oracle.c",
     "const double EK = sk / V / (2.0 * pow(a, 2.0 * m->alpha))",
     "const double EK = sk / V / (2.0 * pow(a, 2.0 * m->alpha + 2.0))", ["test_oracle_scalar.py"]),
    ("gl-scale-factor-weights", "lattice_oracle.c",
     "        da += dt * c[mm] * Daold[mm];",
     "        da += dt * c[0] * Daold[mm];", ["test_oracle_scalar.py"]),
    ("gl-drift-power", "lattice_oracle.c",
     "const double cdr = pow(al, -(3.0 - m->alpha));",
     "const double cdr = pow(al, -(2.0 - m->alpha));", ["test_oracle_scalar.py"]),
    ("fluid-scale-factor-power", "lattice_oracle.c",
     "static double fluid_a(const orc_fluid* f, double t) { return f->a0 * pow(1.0 + f->H0 * t / f->p, f->p); }",
     "static double fluid_a(const orc_fluid* f, double t) { return f->a0 * pow(1.0 + f->H0 * t, f->p); }", ["test_oracle_scalar.py"]),
    ("vv-scalar-first-half-kick", "lattice_oracle.c",
     "        kick(m, phi, pi, *a, 0.5 * h, K);\n        const double ah = *a + 0.5 * h * bh;",
     "        kick(m, phi, pi, *a, h, K);\n        const double ah = *a + 0.5 * h * bh;", ["test_oracle_scalar.py"]),
    ("u1-noncompact-magnetic-energy", "lattice_oracle.c",
     "return m->noncompact ? 0.5 * t * t : 1.0 - cos(t); }",
     "return m->noncompact ? t * t : 1.0 - cos(t); }", ["test_oracle_u1.py"]),
    ("su2-plaquette-order", "lattice_oracle.c",
     "    qmul(Ui, Uj_i, t1);\n    qmul(t1, c1, t2);\n    qmul(t2, c2, P);",
     "    qmul(Uj_i, Ui, t1);\n    qmul(t1, c1, t2);\n    qmul(t2, c2, P);", ["test_oracle_su2.py"]),
    ("su2-staple-conjugation", "lattice_oracle.c",
     "                        qmul(Ujc, P2, s1);\n                        qmul(s1, Uj, Q);\n                        for (int c = 0; c < 3; ++c) mag[c] += P1[c + 1] - Q[c + 1];\n                    }\n                    for (int c = 0; c < 3; ++c) KB[((int64_t)i * 3 + c) * V + n] = A1 * cJ * js[c] + Am * cM * mag[c];\n                }\n                const double mod2 = f[0] * f[0] + f[1] * f[1] + f[2] * f[2] + f[3] * f[3];\n                double dv;\n                gauge_potential(m->pot, m->p, m->lam, m->v2, mod2, &dv);\n                for (int c = 0; c < 4; ++c) Kp[(int64_t)c * V + n] = -A3 * dv * f[c] + A1 * lap[c] * idx2;",
     "                        qmul(Uj, P2, s1);\n                        qmul(s1, Ujc, Q);\n                        for (int c = 0; c < 3; ++c) mag[c] += P1[c + 1] - Q[c + 1];\n                    }\n                    for (int c = 0; c < 3; ++c) KB[((int64_t)i * 3 + c) * V + n] = A1 * cJ * js[c] + Am * cM * mag[c];\n                }\n                const double mod2 = f[0] * f[0] + f[1] * f[1] + f[2] * f[2] + f[3] * f[3];\n                double dv;\n                gauge_potential(m->pot, m->p, m->lam, m->v2, mod2, &dv);\n                for (int c = 0; c < 4; ++c) Kp[(int64_t)c * V + n] = -A3 * dv * f[c] + A1 * lap[c] * idx2;", ["test_oracle_su2.py"]),
    ("u1-kernel-magnetic-a-power", "lattice_oracle.c",
     "a1 * (2.0 * m->e / dx) / m->kappa * cur + am / (m->e * dx * dx * dx) * mag;",
     "a1 * (2.0 * m->e / dx) / m->kappa * cur + a1 / (m->e * dx * dx * dx) * mag;", ["test_oracle_u1.py"]),
    ("u1-kernel-current-a-power", "lattice_oracle.c",
     "a1 * (2.0 * m->e / dx) / m->kappa * cur + am / (m->e * dx * dx * dx) * mag;",
     "am * (2.0 * m->e / dx) / m->kappa * cur + am / (m->e * dx * dx * dx) * mag;", ["test_oracle_u1.py"]),
    ("u1-kernel-magnetic-coupling", "lattice_oracle.c",
     "a1 * (2.0 * m->e / dx) / m->kappa * cur + am / (m->e * dx * dx * dx) * mag;",
     "a1 * (2.0 * m->e / dx) / m->kappa * cur + am / (m->e * m->e * dx * dx * dx) * mag;", ["test_oracle_u1.py"]),
    ("u1-vv-closing-b-half-kick", "lattice_oracle.c",
     "        orc_u1_energies(m, phi, pi, th, piA, *a, E);\n        *b = bh + 0.5 * h * orc_u1_Ka(m, *a, E);",
     "        *b = bh + 0.5 * h * orc_u1_Ka(m, *a, E);\n        orc_u1_energies(m, phi, pi, th, piA, *a, E);", ["test_oracle_u1.py"]),
    ("u1-vv-link-drift-a-power", "lattice_oracle.c",
     "const double cth = m->e * m->dx * h * pow(ah, -(1.0 - m->alpha));",
     "const double cth = m->e * m->dx * h * pow(ah, -(3.0 - m->alpha));", ["test_oracle_u1.py"]),
    ("su2-kernel-magnetic-a-power", "lattice_oracle.c",
     "                    for (int c = 0; c < 3; ++c) KB[((int64_t)i * 3 + c) * V + n] = A1 * cJ * js[c] + Am * cM * mag[c];\n                }\n                const double mod2 = f[0] * f[0] + f[1] * f[1] + f[2] * f[2] + f[3] * f[3];\n                double dv;\n                gauge_potential(m->pot, m->p, m->lam, m->v2, mod2, &dv);\n                for (int c = 0; c < 4; ++c) Kp[(int64_t)c * V + n] = -A3 * dv * f[c] + A1 * lap[c] * idx2;",
     "                    for (int c = 0; c < 3; ++c) KB[((int64_t)i * 3 + c) * V + n] = A1 * cJ * js[c] + A1 * cM * mag[c];\n                }\n                const double mod2 = f[0] * f[0] + f[1] * f[1] + f[2] * f[2] + f[3] * f[3];\n                double dv;\n                gauge_potential(m->pot, m->p, m->lam, m->v2, mod2, &dv);\n                for (int c = 0; c < 4; ++c) Kp[(int64_t)c * V + n] = -A3 * dv * f[c] + A1 * lap[c] * idx2;", ["test_oracle_su2.py"]),
    ("su2u1-KA-magnetic-coupling", "lattice_oracle.c",
     "Am / (m->eA * m->dx * m->dx * m->dx) * magA;",
     "Am / (m->eA * m->eA * m->dx * m->dx * m->dx) * magA;", ["test_oracle_su2u1.py"]),
    ("su2u1-backward-hop-phase", "lattice_oracle.c",
     "whop(qmc, -tm, fm, tb);",
     "whop(qmc, tm, fm, tb);", ["test_oracle_su2u1.py"]),
    ("su2u1-u1-magnetic-energy-coupling", "lattice_oracle.c",
     "out[6] = u1 ? m->kappa * sga / V / (a4 * dx4 * m->eA * m->eA) : 0.0;",
     "out[6] = u1 ? m->kappa * sga / V / (a4 * dx4 * m->eA) : 0.0;", ["test_oracle_su2u1.py"]),
    ("rk4-potential-a-power", "lattice_oracle.c",
     "c3 = pow(a, 2.0 * m->alpha);",
     "c3 = pow(a, 2.0 + 2.0 * m->alpha);", ["test_oracle_scalar.py"]),
    ("rk4-gradient-a-power", "lattice_oracle.c",
     "const double c1 = pow(a, -2.0 * (1.0 - m->alpha))",
     "const double c1 = pow(a, -(1.0 - m->alpha))", ["test_oracle_scalar.py"]),
    ("fluid-closing-kick-a", "lattice_oracle.c",
     "        kick(m, phi, pi, an, 0.5 * h, K);\n        *t += h;",
     "        kick(m, phi, pi, a, 0.5 * h, K);\n        *t += h;", ["test_oracle_scalar.py"]),
    ("u1-ic-canonical-normalisation", "ic.py",
     "    phi = np.stack([comps[0], comps[1]]) / np.sqrt(2.0)",
     "    phi = np.stack([comps[0], comps[1]])", ["test_oracle_ic.py", "test_oracle_u1.py"]),
    ("su2-ic-curvature-canonical-factor", "ic.py",
     "    m2 = [dv + d2 * 2.0 * pb[c] ** 2 for c in range(4)]  # canonical component sqrt(2) Phi_c",
     "    m2 = [dv + d2 * pb[c] ** 2 for c in range(4)]  # canonical component sqrt(2) Phi_c", ["test_oracle_ic.py", "test_oracle_su2.py"]),
    ("dft-normalisation", "spectra.py",
     "return np.fft.ifftn(f) * f.size",
     "return np.fft.ifftn(f)", ["test_oracle_ic.py", "test_oracle_observe.py", "test_oracle_scalar.py"]),
    ("observe-spectrum-of-phi", "observe.py",
     "k, D, _ = spectrum(lattice.phi[1], m.dx, kIR)",
     "k, D, _ = spectrum(lattice.phi[0], m.dx, kIR)", ["test_oracle_observe.py"]),
    ("lf3-b-uses-average-kinetic", "lattice_oracle.c",
     "        const double EKbar = 0.5 * (EKm + EKp);",
     "        const double EKbar = EKp;", ["test_oracle_scalar.py"]),
    ("u1-electric-field-a-power", "core.py",
     "        return self.piA / self.a ** (1.0 - self.m.alpha)",
     "        return self.piA / self.a ** (3.0 - self.m.alpha)", ["test_oracle_u1.py"]),
    ("su2u1-electric-field-a-power", "core.py",
     "return (self.piA if sector == 0 else self.piB) / self.a ** (1.0 - self.m.alpha)",
     "return (self.piA if sector == 0 else self.piB) / self.a ** (2.0 - self.m.alpha)", ["test_oracle_su2u1.py"]),
    ("u1-magnetic-field-scale", "core.py",
     "out[i] = (t if noncompact else np.sin(t)) / (e * dx * dx)",
     "out[i] = (t if noncompact else np.sin(t)) / (e * dx)", ["test_oracle_u1.py", "test_oracle_su2u1.py"]),
    ("su2-electric-field-a-power", "core.py",
     "        return self.piB / self.a ** (1.0 - self.m.alpha)",
     "        return self.piB / self.a ** (2.0 - self.m.alpha)", ["test_oracle_su2.py", "test_oracle_su2u1.py"]),
    ("su2-magnetic-field-scale", "core.py",
     "out[i] = -2.0 * P[1:] / (g * dx * dx)",
     "out[i] = -1.0 * P[1:] / (g * dx * dx)", ["test_oracle_su2.py", "test_oracle_su2u1.py"]),
    ("philox-rounds", "philox.py",
     "    for r in range(10):",
     "    for r in range(9):", ["test_oracle_ic.py"]),
    ("gl-convergence-test", "lattice_oracle.c",
     "if (dd <= tol * tol * nn) break;",
     "if (dd <= tol * nn) break;", ["test_oracle_scalar.py"]),
    ("lf3-b-kernel-at-half-step", "lattice_oracle.c",
     "        const double bn = bm + dt * Ka_scalar(m, a, EKbar, EG, EV);",
     "        const double bn = bm + dt * Ka_scalar(m, ah, EKbar, EG, EV);", ["test_oracle_scalar.py"]),
    ("u1-gradient-energy-half", "lattice_oracle.c",
     "    out[1] = sg / V / a2;\n    out[2] = sv / V;\n    out[3] = m->kappa * ska",
     "    out[1] = sg / V / (2.0 * a2);\n    out[2] = sv / V;\n    out[3] = m->kappa * ska", ["test_oracle_u1.py"]),
    ("su2-gradient-energy-half", "lattice_oracle.c",
     "    out[1] = sg / V / (m->dx * m->dx) / a2;",
     "    out[1] = sg / V / (m->dx * m->dx) / (2.0 * a2);", ["test_oracle_su2.py"]),
    ("su2u1-gradient-energy-half", "lattice_oracle.c",
     "    out[1] = sg / V / dx2 / a2;",
     "    out[1] = sg / V / dx2 / (2.0 * a2);", ["test_oracle_su2u1.py"]),
    ("su2-gauss-charge-factor", "lattice_oracle.c",
     "const double r = m->g / m->kappa * rho[c];",
     "const double r = 2.0 * m->g / m->kappa * rho[c];", ["test_oracle_su2.py", "test_oracle_ic.py"]),
    ("su2-kinetic-energy-half", "lattice_oracle.c",
     "    out[0] = sk / V / a6;\n    out[1] = sg / V / (m->dx * m->dx) / a2;",
     "    out[0] = sk / V / (2.0 * a6);\n    out[1] = sg / V / (m->dx * m->dx) / a2;", ["test_oracle_su2.py"]),
    ("su2u1-interaction-energy-factor", "lattice_oracle.c",
     "sv += m->q * mod2 * chi[n] * chi[n];",
     "sv += 0.5 * m->q * mod2 * chi[n] * chi[n];", ["test_oracle_su2u1.py"]),
    ("u1-higgs-potential-factor", "lattice_oracle.c",
     "return 0.25 * lam * (mod2 - v2) * (mod2 - v2);",
     "return 0.5 * lam * (mod2 - v2) * (mod2 - v2);", ["test_oracle_u1.py", "test_oracle_su2.py"]),
    ("su2u1-ic-singlet-curvature", "ic.py",
     "chi, dchi = _singlet_draw(N, alpha, kIR, 2.0 * model.q * s2,",
     "chi, dchi = _singlet_draw(N, alpha, kIR, model.q * s2,", ["test_oracle_su2u1.py", "test_oracle_ic.py"]),
    ("u1-ic-homogeneous-kinetic-energy", "ic.py",
     "    EK0 = 0.5 * (db[0] ** 2 + db[1] ** 2) / a ** (2 * alpha)",
     "    EK0 = (db[0] ** 2 + db[1] ** 2) / a ** (2 * alpha)", ["test_oracle_ic.py", "test_oracle_u1.py"]),
    ("su2-ic-homogeneous-kinetic-energy", "ic.py",
     "    EK0 = sum(d * d for d in db) / a ** (2 * alpha)\n    H = np.sqrt(max(a ** (2 * alpha) / 3.0 * model.fmp2 * (EK0 + Vbar), 0.0))\n    lin, conj, selfc, zero, nabs = mode_map(N)\n    k = kIR * nabs\n    phi = np.zeros((4, N, N, N))",
     "    EK0 = 0.5 * sum(d * d for d in db) / a ** (2 * alpha)\n    H = np.sqrt(max(a ** (2 * alpha) / 3.0 * model.fmp2 * (EK0 + Vbar), 0.0))\n    lin, conj, selfc, zero, nabs = mode_map(N)\n    k = kIR * nabs\n    phi = np.zeros((4, N, N, N))", ["test_oracle_ic.py", "test_oracle_su2.py"]),
    ("scalar-curvature-interaction-term", "core.py",
     "(m.q * f1 * f1 if m.Ns > 1 else 0.0)]",
     "(2.0 * m.q * f1 * f1 if m.Ns > 1 else 0.0)]", ["test_oracle_ic.py", "test_oracle_scalar.py"]),
    ("spectrum-drops-last-shell", "spectra.py",
     "return b, np.sqrt(n2.astype(np.float64)), int(b.max()) + 1",
     "return b, np.sqrt(n2.astype(np.float64)), int(b.max())", ["test_oracle_ic.py", "test_oracle_observe.py"]),
    ("observe-default-kmax", "observe.py",
     "        kmax = 0.5 * m.N * kIR",
     "        kmax = m.N * kIR", ["test_oracle_observe.py"]),
    ("su2-drift-rotation-direction", "lattice_oracle.c",
     "for (int c = 0; c < 3; ++c) ex[c + 1] = -s * e[c];",
     "for (int c = 0; c < 3; ++c) ex[c + 1] = s * e[c];", ["test_oracle_su2.py", "test_oracle_su2u1.py"]),
    ("su2-im-sigma1-swap", "lattice_oracle.c",
     "z[0] = y[2]; z[1] = y[3]; z[2] = y[0]; z[3] = y[1];",
     "z[0] = y[2]; z[1] = -y[3]; z[2] = y[0]; z[3] = -y[1];", ["test_oracle_su2.py", "test_oracle_su2u1.py"]),
    ("su2-im-sigma3-sign", "lattice_oracle.c",
     "z[0] = y[0]; z[1] = y[1]; z[2] = -y[2]; z[3] = -y[3];",
     "z[0] = y[0]; z[1] = y[1]; z[2] = y[2]; z[3] = y[3];", ["test_oracle_su2.py", "test_oracle_su2u1.py"]),
    ("su2-umul-diagonal-phase", "lattice_oracle.c",
     "const double ar = q[0], ai = q[3], br = q[2]",
     "const double ar = q[0], ai = -q[3], br = q[2]", ["test_oracle_su2.py", "test_oracle_su2u1.py"]),
    ("su2-magnetic-plaquette-helper-conjugate", "core.py",
     "conj = np.array([1.0, -1.0, -1.0, -1.0])[:, None, None, None]",
     "conj = np.array([1.0, 1.0, -1.0, -1.0])[:, None, None, None]", ["test_oracle_su2.py", "test_oracle_su2u1.py"]),
    ("su2-gauss-divergence-sign", "lattice_oracle.c",
     "div[c] += (piB[((int64_t)i * 3 + c) * V + n] - tr[c + 1]) / m->dx;",
     "div[c] += (piB[((int64_t)i * 3 + c) * V + n] + tr[c + 1]) / m->dx;", ["test_oracle_su2.py", "test_oracle_su2u1.py", "test_oracle_ic.py"]),
]

PIN_FILES = sorted({p for case in CASES for p in case[4]})


def _scratch_copy(dst):
    """oracle/ and the CPU pin files (with what they import) under dst."""
    shutil.copytree(os.path.join(ROOT, "oracle"), os.path.join(dst, "oracle"),
                    ignore=shutil.ignore_patterns("_build", "__pycache__"))
    os.makedirs(os.path.join(dst, "tests"))
    shutil.copytree(os.path.join(ROOT, "tests", "golden"), os.path.join(dst, "tests", "golden"))
    for f in ["__init__.py", "inputs.py"] + PIN_FILES:
        shutil.copy(os.path.join(ROOT, "tests", f), os.path.join(dst, "tests", f))
    # the pin files need no GPU check: a conftest without the torch import
    with open(os.path.join(dst, "tests", "conftest.py"), "w") as fh:
        fh.write("def pytest_configure(config):\n"
                 "    config.addinivalue_line('markers', 'gpu: needs a CUDA GPU')\n")


def _run_pins(dst, pins):
    env = dict(os.environ, PYTHONPATH=dst, OMP_NUM_THREADS="2", PYTHONDONTWRITEBYTECODE="1")
    r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider"] +
                       ["tests/" + p for p in pins], cwd=dst, env=env, capture_output=True, text=True,
                       timeout=600)
    lines = r.stdout.strip().splitlines()
    return r.returncode, (lines[-1] if lines else r.stderr[-400:])


def _one(tmp, case):
    name, fname, old, new, pins = case
    dst = os.path.join(tmp, name)
    _scratch_copy(dst)
    path = os.path.join(dst, "oracle", fname)
    with open(path) as fh:
        src = fh.read()
    if src.count(old) != 1:
        return name, (None, "the original text occurs %d times in %s" % (src.count(old), fname))
    with open(path, "w") as fh:
        fh.write(src.replace(old, new))
    # the mutant must still build, so that a pin fails on its arithmetic, not on gcc
    b = subprocess.run([sys.executable, "-c", "from oracle import build; build.build(force=True)"], cwd=dst,
                       env=dict(os.environ, PYTHONPATH=dst), capture_output=True, text=True, timeout=300)
    if b.returncode != 0:
        return name, (None, "the mutant does not build: " + b.stderr[-300:])
    return name, _run_pins(dst, pins)


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    """Run the unmutated copy and every mutant, a few at a time."""
    tmp = str(tmp_path_factory.mktemp("oracle_mutants"))
    base = os.path.join(tmp, "unmutated")
    _scratch_copy(base)
    clean = _run_pins(base, PIN_FILES)
    with ThreadPoolExecutor(max_workers=max(2, min(6, (os.cpu_count() or 2) - 1))) as pool:
        res = dict(pool.map(lambda c: _one(tmp, c), CASES))
    return clean, res


def test_unmutated_copy_passes_the_pins(outcomes):
    rc, summary = outcomes[0]
    assert rc == 0 and "passed" in summary and "failed" not in summary, summary


@pytest.mark.parametrize("name", [c[0] for c in CASES])
def test_planted_mistake_fails_a_pin(outcomes, name):
    clean_rc, _ = outcomes[0]
    assert clean_rc == 0
    rc, summary = outcomes[1][name]
    assert rc is not None, summary
    # exit status 1 with "failed" and no "error": a pin failed, the copy built and collected
    assert rc == 1 and "failed" in summary and "error" not in summary, summary
