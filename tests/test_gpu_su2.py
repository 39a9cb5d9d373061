"""Parity of the CUDA SU(2)-Higgs path (through the C ABI) with the FP64
oracle, and the discrete Gauss law to round-off (section 6)."""
import math

import numpy as np
import pytest

import oracle
import paper_2006_15122_gb300 as cl
from oracle import SU2Model
from tests.test_oracle_su2 import gauss_state, random_state

pytestmark = pytest.mark.gpu


def rel(x, y):
    return float(np.max(np.abs(x - y)) / max(np.max(np.abs(y)), 1e-300))


def gpu_su2(m, integ, prec, fmp=0.0):
    model = cl.make_model(kind=cl.CL_MODEL_SU2, alpha=m.alpha, fstar_over_mp=fmp, omega_over_fstar=math.sqrt(m.kappa),
                          lam=m.lam, vev2=m.v2, gauge_e=m.g, potential=m.pot, pexp=m.p)
    kIR = 2 * math.pi / (m.N * m.dx)
    return cl.Lattice(model, cl.make_grid(m.N, kIR, 0.04, integ, prec), cl.make_init(phi0=(0.5, 0.0, 0.0, 0.0), spectrum=0))


def load(lat, ref):
    for c in range(4):
        lat.set_field(cl.FIELD(c), ref.phi[c])
        lat.set_field(cl.MOMENTUM(c), ref.pi[c])
    for i in range(3):
        for c in range(4):
            lat.set_field(cl.SU2_LINK(i, c), ref.u[i, c])
        for a in range(3):
            lat.set_field(cl.SU2_EMOMENTUM(i, a), ref.piB[i, a])
    lat.set_background(ref.a, ref.b, 0.0)


def fetch(lat, N):
    phi = np.stack([lat.get_field(cl.FIELD(c)) for c in range(4)])
    pi = np.stack([lat.get_field(cl.MOMENTUM(c)) for c in range(4)])
    u = np.stack([np.stack([lat.get_field(cl.SU2_LINK(i, c)) for c in range(4)]) for i in range(3)])
    piB = np.stack([np.stack([lat.get_field(cl.SU2_EMOMENTUM(i, a)) for a in range(3)]) for i in range(3)])
    return phi, pi, u, piB


@pytest.mark.parametrize("integ,fmp,alpha,pot", [("vv2", 0.0, 0.0, 0), ("vv4", 0.7, 0.5, 0), ("vv4", 0.7, 1.0, 1)])
def test_su2_fp64_velocity_verlet_matches_oracle(integ, fmp, alpha, pot):
    """Higgs potential and (pot = 1) the monomial inflaton (lam/4)(2|Phi|^2)^2."""
    N, dt = 8, 0.04
    m = SU2Model(N=N, dx=0.6, alpha=alpha, fmp2=fmp * fmp, lam=1.2, v2=0.8, g=0.9, kappa=1.21, pot=pot, p=4)
    ref = random_state(N, m, 7)
    if fmp > 0:
        ref.b = math.sqrt(fmp * fmp / 3.0 * ref.energies().sum())
    lat = gpu_su2(m, integ, cl.CL_FP64, fmp)
    load(lat, ref)
    lat.evolve(3)
    lat.evolve(4)
    ref.vv_steps({"vv2": oracle.VV2, "vv4": oracle.VV4}[integ], dt, 7)
    phi, pi, u, piB = fetch(lat, N)
    assert rel(phi, ref.phi) < 1e-12
    assert rel(pi, ref.pi) < 1e-12
    assert np.max(np.abs(u - ref.u)) < 1e-12
    assert rel(piB, ref.piB) < 1e-12
    mm = lat.measure_means()
    assert abs(mm["a"] - ref.a) < 1e-13 and abs(mm["b"] - ref.b) < 1e-12 * (1 + abs(ref.b))
    E = ref.energies()
    got = [mm["EK"][0], mm["EG"][0], mm["EV"][0], mm["EK"][1], mm["EG"][1]]
    assert np.allclose(got, E, rtol=1e-11, atol=1e-14), (got, E)
    lat.close()


@pytest.mark.parametrize("N,prec,tol", [(40, cl.CL_FP64, 1e-12), (24, cl.CL_FP32, 1e-6), (64, cl.CL_FP32, 1e-6)])
def test_su2_many_tiles_match_oracle(N, prec, tol):
    """Lattices of several x-y tiles of the kick (8 x 8 sites in FP64 and when 32
    does not divide N, 32 x 8 in FP32 otherwise), with each block's run of planes
    crossing from one tile to the next: three expanding VV2 steps against the
    oracle."""
    dt, fmp = 0.04, 0.7
    m = SU2Model(N=N, dx=0.6, alpha=0.5, fmp2=fmp * fmp, lam=1.2, v2=0.8, g=0.9, kappa=1.21, pot=0, p=4)
    ref = random_state(N, m, 11)
    ref.b = math.sqrt(fmp * fmp / 3.0 * ref.energies().sum())
    lat = gpu_su2(m, "vv2", prec, fmp)
    load(lat, ref)
    lat.evolve(3)
    ref.vv_steps(oracle.VV2, dt, 3)
    phi, pi, u, piB = fetch(lat, N)
    errs = (rel(phi, ref.phi), rel(pi, ref.pi), float(np.max(np.abs(u - ref.u))), rel(piB, ref.piB))
    assert max(errs) < tol, errs
    mm = lat.measure_means()
    E = ref.energies()
    got = [mm["EK"][0], mm["EG"][0], mm["EV"][0], mm["EK"][1], mm["EG"][1]]
    assert np.allclose(got, E, rtol=10 * tol, atol=1e-14), (got, E)
    lat.close()


def test_su2_fp32_100_steps_match_oracle_pointwise():
    """FP32 over the first 100 steps (the pointwise bound 1e-5): a charge-free
    doublet with unit links and Gauss-law electric momenta on 64^3 (32 x 8 kick
    tiles), expanding VV2, against the FP64 oracle."""
    N, dt, fmp = 64, 0.04, 0.7
    m = SU2Model(N=N, dx=0.6, alpha=0.5, fmp2=fmp * fmp, lam=1.2, v2=0.8, g=0.9, kappa=1.21, pot=0, p=4)
    ref = gauss_state(N, m, 11)
    ref.b = math.sqrt(fmp * fmp / 3.0 * ref.energies().sum())
    lat = gpu_su2(m, "vv2", cl.CL_FP32, fmp)
    load(lat, ref)
    lat.evolve(40)
    lat.evolve(60)
    ref.vv_steps(oracle.VV2, dt, 100)
    phi, pi, u, piB = fetch(lat, N)
    errs = (rel(phi, ref.phi), rel(pi, ref.pi), float(np.max(np.abs(u - ref.u))), rel(piB, ref.piB))
    assert max(errs) < 1e-5, errs
    lat.close()


def test_su2_leapfrog_equals_velocity_verlet_positions_static():
    """Static background: the staggered leapfrog started by a half kick moves
    fields and links exactly as VV2 does (oracle VV2 as reference)."""
    N, dt, n = 8, 0.04, 9
    m = SU2Model(N=N, dx=0.6, alpha=0.0, fmp2=0.0, lam=1.0, v2=1.0, g=1.1, kappa=0.9)
    ref = random_state(N, m, 17)
    lat = gpu_su2(m, "lf", cl.CL_FP64)
    load(lat, ref)
    lat.evolve(n)
    ref.vv_steps(oracle.VV2, dt, n)
    phi, _, u, _ = fetch(lat, N)
    assert rel(phi, ref.phi) < 1e-12
    assert np.max(np.abs(u - ref.u)) < 1e-12
    lat.close()


@pytest.mark.parametrize("prec,tol", [(cl.CL_FP64, 1e-13), (cl.CL_FP32, 1e-5)])
def test_su2_gauss_law_is_preserved(prec, tol):
    N = 16
    m = SU2Model(N=N, dx=0.5, alpha=0.5, fmp2=0.36, lam=1.0, v2=1.0, g=1.1, kappa=0.9)
    ref = gauss_state(N, m, 23)
    ref.b = math.sqrt(0.36 / 3.0 * ref.energies().sum())
    lat = gpu_su2(m, "vv4", prec, 0.6)
    load(lat, ref)
    g = [lat.measure_means()["gauss_violation"]]
    for _ in range(4):
        lat.evolve(10)
        g.append(lat.measure_means()["gauss_violation"])
    assert max(g) < tol, g
    u = np.stack([lat.get_field(cl.SU2_LINK(i, c)) for i in range(3) for c in range(1, 4)])
    assert np.max(np.abs(u)) > 1e-3  # the links moved off the identity
    lat.close()


def test_su2_homogeneous_start_and_refusals():
    m = SU2Model(N=16, dx=0.5, alpha=0.0, fmp2=0.0)
    lat = gpu_su2(m, "vv2", cl.CL_FP64)
    assert np.all(lat.get_field(cl.FIELD(0)) == 0.5) and np.all(lat.get_field(cl.SU2_LINK(1, 0)) == 1.0)
    mm = lat.measure_means()
    assert mm["gauss_violation"] == 0.0 and mm["EG"][1] == 0.0
    lat.evolve(5)
    assert np.allclose(lat.get_field(cl.FIELD(0)), lat.get_field(cl.FIELD(0)).mean(), rtol=0, atol=1e-14)
    lat.close()
    model = cl.make_model(kind=cl.CL_MODEL_SU2, gauge_e=1.0)
    with pytest.raises(cl.LatticeError):  # a uniform charge violates the Gauss law
        cl.Lattice(model, cl.make_grid(16, 0.5, 0.04, "vv2", cl.CL_FP64),
                   cl.make_init(phi0=(1.0, 0.0, 0.0, 0.0), dphi0=(0.0, 0.0, 0.0, 1.0), spectrum=0))


@pytest.mark.parametrize("prec,pot", [(cl.CL_FP64, 0), (cl.CL_FP32, 0), (cl.CL_FP64, 1)])
def test_su2_vacuum_initial_conditions_match_oracle(prec, pot):
    """lattice_init with vacuum fluctuations: the doublet, its momenta (with
    the colour charges projected out) and the Gauss-consistent electric momenta
    against the oracle's SU(2) initial conditions; Gauss law at round-off."""
    from oracle.ic import su2_ic
    N, dx, omega = 16, 0.5, 0.3
    m = SU2Model(N=N, dx=dx, alpha=0.0, fmp2=0.0, lam=1.0, v2=1.0, g=1.2, kappa=omega * omega, pot=pot, p=4)
    kIR = 2 * math.pi / (N * dx)
    model = cl.make_model(kind=cl.CL_MODEL_SU2, omega_over_fstar=omega, lam=1.0, vev2=1.0, gauge_e=1.2,
                          potential=pot, pexp=4)
    lat = cl.Lattice(model, cl.make_grid(N, kIR, 0.04, "vv2", prec),
                     cl.make_init(phi0=(0.4, 0.0, 0.0, 0.3), seed=5, spectrum=1))
    phi, pi, u, piB, _ = su2_ic(m, kIR, [0.4, 0.0, 0.0, 0.3], [0.0] * 4, seed=5, omega_over_fstar=omega)
    gphi, gpi, gu, gpiB = fetch(lat, N)
    tol = 1e-12 if prec == cl.CL_FP64 else 2e-6
    assert rel(gphi, phi) < tol and rel(gpi, pi) < tol, (rel(gphi, phi), rel(gpi, pi))
    assert rel(gpiB, piB) < 10 * tol, rel(gpiB, piB)
    assert np.all(gu[:, 0] == 1.0) and np.all(gu[:, 1:] == 0.0)
    mm = lat.measure_means()
    assert mm["gauss_violation"] < (1e-13 if prec == cl.CL_FP64 else 1e-5)
    assert mm["EG"][1] == 0.0
    lat.evolve(10)
    assert lat.measure_means()["gauss_violation"] < (1e-13 if prec == cl.CL_FP64 else 1e-5)
    lat.close()
