"""Parity of the CUDA compact-U(1) path (through the C ABI) with the FP64
oracle, and the Gauss law to round-off (section 5.3)."""
import math

import numpy as np
import pytest

import paper_2006_15122_gb300 as cl
from oracle import U1Lattice, U1Model
from oracle.ic import u1_ic
from tests import inputs

pytestmark = pytest.mark.gpu


def rel(x, y):
    return float(np.max(np.abs(x - y)) / max(np.max(np.abs(y)), 1e-300))


def angle_err(a, b):
    return float(np.max(np.abs(np.angle(np.exp(1j * (a - b))))))


def gpu_u1(N, kIR, dt, prec, fmp=0.0, alpha=0.0, e=1.0, lam=1.0, v2=1.0, omega=1.0, spectrum=0, seed=0,
           phi0=(0.0, 0.0), integ="lf", pot=0, p=4, dphi0=(0.0, 0.0), nc=0):
    m = cl.make_model(kind=cl.CL_MODEL_U1, alpha=alpha, fstar_over_mp=fmp, omega_over_fstar=omega, lam=lam,
                      vev2=v2, gauge_e=e, potential=pot, pexp=p, noncompact=nc)
    g = cl.make_grid(N, kIR, dt, integ, prec)
    return cl.Lattice(m, g, cl.make_init(phi0=phi0, dphi0=dphi0, seed=seed, spectrum=spectrum))


def get_all(lat):
    phi = np.stack([lat.get_field(cl.FIELD(i)) for i in range(2)])
    pi = np.stack([lat.get_field(cl.MOMENTUM(i)) for i in range(2)])
    th = np.stack([lat.get_field(cl.LINK(i)) for i in range(3)])
    pa = np.stack([lat.get_field(cl.EMOMENTUM(i)) for i in range(3)])
    return phi, pi, th, pa


@pytest.mark.parametrize("fmp,alpha", [(0.0, 0.0), (0.8, 0.5)])
def test_u1_fp64_leapfrog_matches_oracle(fmp, alpha):
    N, kIR, dt = 16, 2 * math.pi / (16 * 0.5), 0.05
    lat = gpu_u1(N, kIR, dt, cl.CL_FP64, fmp=fmp, alpha=alpha, e=0.9, lam=1.2, v2=0.7, omega=1.1)
    om = U1Model(N=N, dx=0.5, alpha=alpha, fmp2=fmp * fmp, lam=1.2, v2=0.7, e=0.9, kappa=1.21)
    phi = inputs.fields(2, N, seed=3, amp=0.6, kmax=4, means=[0.4, -0.1])
    pi = inputs.fields(2, N, seed=4, amp=0.3, kmax=4)
    th = inputs.angles(N, 5, scale=0.4)
    pa = inputs.fields(3, N, seed=6, amp=0.2, kmax=4)
    ref = U1Lattice(om, phi, pi, th, pa)
    ref.b = math.sqrt(fmp * fmp / 3 * ref.energies().sum()) if fmp > 0 else 0.0
    for i in range(2):
        lat.set_field(cl.FIELD(i), phi[i])
        lat.set_field(cl.MOMENTUM(i), pi[i])
    for i in range(3):
        lat.set_field(cl.LINK(i), th[i])
        lat.set_field(cl.EMOMENTUM(i), pa[i])
    lat.set_background(1.0, ref.b, 0.0)
    ref.lf_prepare(dt)
    lat.evolve(3)
    lat.evolve(4)
    ref.lf_steps(dt, 7)
    gphi, gpi, gth, gpa = get_all(lat)
    assert rel(gphi, ref.phi) < 1e-12
    assert rel(gpi, ref.pi) < 1e-12
    assert angle_err(gth, ref.theta) < 1e-12
    assert rel(gpa, ref.piA) < 1e-12
    mm = lat.measure_means()
    assert abs(mm["a"] - ref.a) < 1e-13 and abs(mm["b"] - ref.b) < 1e-12 + 1e-12 * abs(ref.b)
    lat.close()


@pytest.mark.parametrize("N,prec,tol,nc", [(40, cl.CL_FP64, 1e-12, 0), (40, cl.CL_FP64, 1e-12, 1),
                                           (24, cl.CL_FP32, 2e-6, 0), (64, cl.CL_FP32, 2e-6, 0)])
def test_u1_many_tiles_match_oracle(N, prec, tol, nc):
    """Lattices of several x-y tiles of the pass (8 x 8 sites in FP64 and when 32
    does not divide N, 32 x 8 in FP32 otherwise), with each block's run of planes
    crossing from one tile to the next: expanding leapfrog steps against the
    oracle, compact and (FP64) non-compact."""
    fmp, alpha, dx = 0.8, 0.5, 0.5
    kIR, dt = 2 * math.pi / (N * dx), 0.05
    lat = gpu_u1(N, kIR, dt, prec, fmp=fmp, alpha=alpha, e=0.9, lam=1.2, v2=0.7, omega=1.1, nc=nc)
    om = U1Model(N=N, dx=dx, alpha=alpha, fmp2=fmp * fmp, lam=1.2, v2=0.7, e=0.9, kappa=1.21, noncompact=nc)
    phi = inputs.fields(2, N, seed=13, amp=0.6, kmax=4, means=[0.4, -0.1])
    pi = inputs.fields(2, N, seed=14, amp=0.3, kmax=4)
    th = inputs.angles(N, 15, scale=0.4)
    pa = inputs.fields(3, N, seed=16, amp=0.2, kmax=4)
    ref = U1Lattice(om, phi, pi, th, pa)
    ref.b = math.sqrt(fmp * fmp / 3 * ref.energies().sum())
    for i in range(2):
        lat.set_field(cl.FIELD(i), phi[i])
        lat.set_field(cl.MOMENTUM(i), pi[i])
    for i in range(3):
        lat.set_field(cl.LINK(i), th[i])
        lat.set_field(cl.EMOMENTUM(i), pa[i])
    lat.set_background(1.0, ref.b, 0.0)
    ref.lf_prepare(dt)
    lat.evolve(3)
    ref.lf_steps(dt, 3)
    gphi, gpi, gth, gpa = get_all(lat)
    errs = (rel(gphi, ref.phi), rel(gpi, ref.pi), angle_err(gth, ref.theta) if not nc else rel(gth, ref.theta),
            rel(gpa, ref.piA))
    assert max(errs) < tol, errs
    lat.close()


def test_u1_initial_conditions_match_oracle():
    N, dx = 16, 0.5
    kIR = 2 * math.pi / (N * dx)
    lat = gpu_u1(N, kIR, 0.05, cl.CL_FP64, spectrum=1, seed=31)
    om = U1Model(N=N, dx=dx, alpha=0.0, fmp2=0.0, lam=1.0, v2=1.0, e=1.0, kappa=1.0)
    phi, pi, th, pa, _ = u1_ic(om, kIR, [0.0, 0.0], [0.0, 0.0], seed=31, omega_over_fstar=1.0)
    gphi, gpi, gth, gpa = get_all(lat)
    assert rel(gphi, phi) < 1e-12 and rel(gpi, pi) < 1e-12 and rel(gpa, pa) < 1e-11
    assert np.all(gth == 0.0)
    mm = lat.measure_means()
    assert mm["gauss_violation"] < 1e-13
    assert mm["EG"][1] == 0.0  # magnetic energy exactly zero with unit links
    lat.close()


@pytest.mark.parametrize("prec,tol", [(cl.CL_FP64, 1e-13), (cl.CL_FP32, 1e-5)])
def test_u1_gauss_law_is_preserved(prec, tol):
    """The abelian-Higgs configuration (lam = e = v = 1, dx = 0.5, dt = 0.1 dx):
    the Gauss constraint stays at round-off and does not drift."""
    N, dx = 32, 0.5
    lat = gpu_u1(N, 2 * math.pi / (N * dx), 0.05, prec, spectrum=1, seed=7)
    g = []
    for _ in range(5):
        lat.evolve(20)
        g.append(lat.measure_means()["gauss_violation"])
    assert max(g) < tol, g
    mm = lat.measure_means()
    assert mm["EG"][1] > 0.0  # magnetic field has developed
    lat.close()


@pytest.mark.parametrize("integ,fmp,alpha", [("vv2", 0.0, 0.0), ("vv4", 0.8, 0.5), ("vv6", 0.5, 0.0),
                                            ("vv8", 0.8, 0.5), ("vv10", 0.5, 1.0)])
def test_u1_fp64_velocity_verlet_matches_oracle(integ, fmp, alpha):
    """Compact VV2/VVn (sections 5.3.2, 5.3.3): merged-kick passes on the GPU
    against the unmerged oracle step, 7 steps in two evolve calls."""
    import oracle
    N, kIR, dt = 16, 2 * math.pi / (16 * 0.5), 0.04
    lat = gpu_u1(N, kIR, dt, cl.CL_FP64, fmp=fmp, alpha=alpha, e=0.9, lam=1.2, v2=0.7, omega=1.1, integ=integ)
    om = U1Model(N=N, dx=0.5, alpha=alpha, fmp2=fmp * fmp, lam=1.2, v2=0.7, e=0.9, kappa=1.21)
    phi = inputs.fields(2, N, seed=13, amp=0.6, kmax=4, means=[0.4, -0.1])
    pi = inputs.fields(2, N, seed=14, amp=0.3, kmax=4)
    th = inputs.angles(N, 15, scale=0.4)
    pa = inputs.fields(3, N, seed=16, amp=0.2, kmax=4)
    ref = U1Lattice(om, phi, pi, th, pa)
    ref.b = math.sqrt(fmp * fmp / 3 * ref.energies().sum()) if fmp > 0 else 0.0
    for i in range(2):
        lat.set_field(cl.FIELD(i), phi[i])
        lat.set_field(cl.MOMENTUM(i), pi[i])
    for i in range(3):
        lat.set_field(cl.LINK(i), th[i])
        lat.set_field(cl.EMOMENTUM(i), pa[i])
    lat.set_background(1.0, ref.b, 0.0)
    lat.evolve(3)
    lat.evolve(4)
    ref.vv_steps({"vv2": oracle.VV2, "vv4": oracle.VV4, "vv6": oracle.VV6, "vv8": oracle.VV8,
                  "vv10": oracle.VV10}[integ], dt, 7)
    gphi, gpi, gth, gpa = get_all(lat)
    assert rel(gphi, ref.phi) < 1e-12
    assert rel(gpi, ref.pi) < 1e-12
    assert angle_err(gth, ref.theta) < 1e-12
    assert rel(gpa, ref.piA) < 1e-12
    mm = lat.measure_means()
    assert abs(mm["a"] - ref.a) < 1e-13 and abs(mm["b"] - ref.b) < 1e-12 + 1e-12 * abs(ref.b)
    assert abs(mm["t"] - 7 * dt) < 1e-12
    E = ref.energies()
    assert abs(mm["EK"][0] - E[0]) < 1e-11 * E.sum() and abs(mm["EK"][1] - E[3]) < 1e-11 * E.sum()
    lat.close()


@pytest.mark.parametrize("prec,tol", [(cl.CL_FP64, 1e-13), (cl.CL_FP32, 1e-5)])
def test_u1_velocity_verlet_keeps_gauss_law(prec, tol):
    N, dx = 32, 0.5
    lat = gpu_u1(N, 2 * math.pi / (N * dx), 0.05, prec, spectrum=1, seed=8, integ="vv4")
    g = []
    for _ in range(4):
        lat.evolve(10)
        g.append(lat.measure_means()["gauss_violation"])
    assert max(g) < tol, g
    assert lat.measure_means()["EG"][1] > 0.0
    lat.close()


@pytest.mark.parametrize("integ,fmp,alpha,p", [("vv4", 0.8, 1.0, 4), ("vv2", 0.5, 0.0, 6), ("lf", 0.0, 0.0, 2)])
def test_u1_monomial_inflaton_matches_oracle(integ, fmp, alpha, p):
    """Charged inflaton V = (lam/p)(2|phi|^2)^(p/2) (section 8) with expansion:
    fields, links, momenta, background and E_V against the oracle."""
    import oracle
    N, dx, dt = 16, 0.5, 0.04
    kIR = 2 * math.pi / (N * dx)
    lat = gpu_u1(N, kIR, dt, cl.CL_FP64, fmp=fmp, alpha=alpha, e=0.9, lam=1.2, omega=1.1, integ=integ, pot=1, p=p,
                 phi0=(0.9, 0.0))
    om = U1Model(N=N, dx=dx, alpha=alpha, fmp2=fmp * fmp, lam=1.2, e=0.9, kappa=1.21, pot=1, p=p)
    phi = inputs.fields(2, N, seed=23, amp=0.6, kmax=4, means=[0.6, -0.2])
    pi = inputs.fields(2, N, seed=24, amp=0.3, kmax=4)
    th = inputs.angles(N, 25, scale=0.4)
    pa = inputs.fields(3, N, seed=26, amp=0.2, kmax=4)
    ref = U1Lattice(om, phi, pi, th, pa)
    ref.b = math.sqrt(fmp * fmp / 3 * ref.energies().sum()) if fmp > 0 else 0.0
    for i in range(2):
        lat.set_field(cl.FIELD(i), phi[i])
        lat.set_field(cl.MOMENTUM(i), pi[i])
    for i in range(3):
        lat.set_field(cl.LINK(i), th[i])
        lat.set_field(cl.EMOMENTUM(i), pa[i])
    lat.set_background(1.0, ref.b, 0.0)
    E0 = ref.energies()
    assert lat.measure_means()["EV"][0] == pytest.approx(E0[2], rel=1e-13)
    if integ == "lf":
        ref.lf_prepare(dt)
        lat.evolve(7)
        ref.lf_steps(dt, 7)
    else:
        lat.evolve(7)
        ref.vv_steps({"vv2": oracle.VV2, "vv4": oracle.VV4}[integ], dt, 7)
    gphi, gpi, gth, gpa = get_all(lat)
    assert rel(gphi, ref.phi) < 1e-12
    assert rel(gpi, ref.pi) < 1e-12
    assert angle_err(gth, ref.theta) < 1e-12
    assert rel(gpa, ref.piA) < 1e-12
    mm = lat.measure_means()
    assert abs(mm["a"] - ref.a) < 1e-13 and abs(mm["b"] - ref.b) < 1e-12 + 1e-12 * abs(ref.b)
    if integ != "lf":
        assert mm["EV"][0] == pytest.approx(ref.energies()[2], rel=1e-11)
    lat.close()


@pytest.mark.parametrize("p", [2, 4])
def test_u1_monomial_initial_conditions_match_oracle(p):
    """Vacuum fluctuations about a homogeneous inflaton phi0 = (1.3, 0.4)/sqrt(2)
    with the monomial potential's curvature along each component and the
    Hubble rate of its energy (section 7), fp64 against the oracle."""
    N, dx = 16, 0.5
    kIR = 2 * math.pi / (N * dx)
    lat = gpu_u1(N, kIR, 0.02, cl.CL_FP64, fmp=0.7, alpha=1.0, e=0.8, lam=1.1, spectrum=1, seed=41, pot=1, p=p,
                 phi0=(1.3, 0.4), dphi0=(-0.26, -0.08), omega=0.6)
    om = U1Model(N=N, dx=dx, alpha=1.0, fmp2=0.49, lam=1.1, e=0.8, kappa=0.36, pot=1, p=p)
    phi, pi, th, pa, _ = u1_ic(om, kIR, [1.3, 0.4], [-0.26, -0.08], seed=41, omega_over_fstar=0.6)
    gphi, gpi, gth, gpa = get_all(lat)
    assert rel(gphi, phi) < 1e-12 and rel(gpi, pi) < 1e-12 and rel(gpa, pa) < 1e-11
    assert np.all(gth == 0.0)
    lat.close()


@pytest.mark.parametrize("integ,fmp,alpha", [("lf", 0.0, 0.0), ("vv2", 0.8, 0.5), ("vv4", 0.5, 1.0)])
def test_u1_noncompact_matches_oracle(integ, fmp, alpha):
    """Non-compact gauge kinetics (section 5.2): fields, unwrapped angles and
    momenta against the oracle after 7 steps, FP64, with expansion; large
    angles (|theta| up to 2.5) so that the compact and non-compact forms differ."""
    import oracle
    N, kIR, dt = 16, 2 * math.pi / (16 * 0.5), 0.04
    lat = gpu_u1(N, kIR, dt, cl.CL_FP64, fmp=fmp, alpha=alpha, e=0.9, lam=1.2, v2=0.7, omega=1.1, integ=integ, nc=1)
    om = U1Model(N=N, dx=0.5, alpha=alpha, fmp2=fmp * fmp, lam=1.2, v2=0.7, e=0.9, kappa=1.21, noncompact=1)
    phi = inputs.fields(2, N, seed=33, amp=0.6, kmax=4, means=[0.4, -0.1])
    pi = inputs.fields(2, N, seed=34, amp=0.3, kmax=4)
    th = inputs.angles(N, 35, scale=2.5)
    pa = inputs.fields(3, N, seed=36, amp=0.2, kmax=4)
    ref = U1Lattice(om, phi, pi, th, pa)
    ref.b = math.sqrt(fmp * fmp / 3 * ref.energies().sum()) if fmp > 0 else 0.0
    for i in range(2):
        lat.set_field(cl.FIELD(i), phi[i])
        lat.set_field(cl.MOMENTUM(i), pi[i])
    for i in range(3):
        lat.set_field(cl.LINK(i), th[i])
        lat.set_field(cl.EMOMENTUM(i), pa[i])
    lat.set_background(1.0, ref.b, 0.0)
    assert lat.measure_means()["EG"][1] == pytest.approx(ref.energies()[4], rel=1e-12)
    if integ == "lf":
        ref.lf_prepare(dt)
        lat.evolve(7)
        ref.lf_steps(dt, 7)
    else:
        lat.evolve(7)
        ref.vv_steps({"vv2": oracle.VV2, "vv4": oracle.VV4}[integ], dt, 7)
    gphi, gpi, gth, gpa = get_all(lat)
    assert rel(gphi, ref.phi) < 1e-12 and rel(gpi, ref.pi) < 1e-12
    assert np.max(np.abs(gth - ref.theta)) < 1e-12  # unwrapped: equal as numbers, not just as phases
    assert rel(gpa, ref.piA) < 1e-12
    mm = lat.measure_means()
    assert abs(mm["a"] - ref.a) < 1e-13 and abs(mm["b"] - ref.b) < 1e-12 + 1e-12 * abs(ref.b)
    lat.close()


@pytest.mark.parametrize("prec,tol", [(cl.CL_FP64, 1e-13), (cl.CL_FP32, 1e-5)])
def test_u1_noncompact_keeps_gauss_law(prec, tol):
    N, dx = 32, 0.5
    lat = gpu_u1(N, 2 * math.pi / (N * dx), 0.05, prec, spectrum=1, seed=8, integ="vv4", nc=1)
    g = []
    for _ in range(4):
        lat.evolve(10)
        g.append(lat.measure_means()["gauss_violation"])
    assert max(g) < tol, g
    assert lat.measure_means()["EG"][1] > 0.0
    lat.close()


@pytest.mark.parametrize("nc", [0, 1])
def test_u1_gauge_field_spectra_match_oracle(nc):
    """Electric and magnetic spectra of the U(1) field (section 5.4) against the
    oracle's fields E_i = piA_i/a^{1-alpha} and B_i of the same (expanded) state."""
    from oracle.spectra import spectrum
    N, dx = 16, 0.5
    kIR = 2 * math.pi / (N * dx)
    lat = gpu_u1(N, kIR, 0.04, cl.CL_FP64, fmp=0.6, alpha=0.5, e=0.9, omega=1.1, integ="vv2", nc=nc, spectrum=1, seed=4)
    lat.evolve(20)
    mm = lat.measure_means()
    gphi, gpi, gth, gpa = get_all(lat)
    om = U1Model(N=N, dx=dx, alpha=0.5, fmp2=0.36, lam=1.0, v2=1.0, e=0.9, kappa=1.21, noncompact=nc)
    ref = U1Lattice(om, gphi, gpi, gth, gpa, a=mm["a"])
    for what, fld in ((0, ref.electric()), (1, ref.magnetic())):
        k, D, c = lat.gauge_spectrum(0, what)
        rk, rD, rc = spectrum(fld, dx, kIR)
        assert np.array_equal(c, rc) and np.allclose(k, rk, rtol=1e-14)
        assert np.max(np.abs(D - rD)) < 1e-10 * np.max(rD), (what, np.max(np.abs(D - rD)), np.max(rD))
    with pytest.raises(cl.LatticeError):
        lat.gauge_spectrum(1, 0)  # no SU(2) sector here
    lat.close()
