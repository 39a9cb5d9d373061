"""Parity of the CUDA SU(2) x U(1) + chi path (the working example of section
8.3, through the C ABI) with the FP64 oracle: fields, links, momenta, the
background and the per-sector energies, both Gauss laws to round-off, and the
constrained vacuum initial conditions."""
import math

import numpy as np
import pytest

import oracle
import paper_2006_15122_gb300 as cl
from oracle import SU2U1Lattice, SU2U1Model
from tests.test_oracle_su2u1 import gauss_state, random_state

pytestmark = pytest.mark.gpu


def rel(x, y):
    return float(np.max(np.abs(x - y)) / max(np.max(np.abs(y)), 1e-300))


def angle_err(a, b):
    return float(np.max(np.abs(np.angle(np.exp(1j * (a - b))))))


def gpu_lattice(m, integ, prec, fmp=0.0, init=None):
    model = cl.make_model(kind=cl.CL_MODEL_SU2, n_fields=2 if m.chi else 1, alpha=m.alpha, fstar_over_mp=fmp,
                          omega_over_fstar=math.sqrt(m.kappa), lam=m.lam, vev2=m.v2, gauge_e=m.g, q=m.q,
                          potential=m.pot, pexp=m.p, gauge_e_u1=m.eA)
    kIR = 2 * math.pi / (m.N * m.dx)
    if init is None:
        init = cl.make_init(phi0=(0.5, 0.0, 0.0, 0.0), spectrum=0)
    return cl.Lattice(model, cl.make_grid(m.N, kIR, 0.04, integ, prec), init)


def load(lat, ref):
    for c in range(4):
        lat.set_field(cl.FIELD(c), ref.phi[c])
        lat.set_field(cl.MOMENTUM(c), ref.pi[c])
    for i in range(3):
        for c in range(4):
            lat.set_field(cl.SU2_LINK(i, c), ref.u[i, c])
        for a in range(3):
            lat.set_field(cl.SU2_EMOMENTUM(i, a), ref.piB[i, a])
        if ref.m.eA > 0:
            lat.set_field(cl.LINK(i), ref.theta[i])
            lat.set_field(cl.EMOMENTUM(i), ref.piA[i])
    if ref.m.chi:
        lat.set_field(cl.SINGLET, ref.chi)
        lat.set_field(cl.SINGLET_MOMENTUM, ref.pchi)
    lat.set_background(ref.a, ref.b, 0.0)


def fetch(lat, m):
    N = m.N
    g = lat.get_field
    out = {
        "phi": np.stack([g(cl.FIELD(c)) for c in range(4)]),
        "pi": np.stack([g(cl.MOMENTUM(c)) for c in range(4)]),
        "u": np.stack([np.stack([g(cl.SU2_LINK(i, c)) for c in range(4)]) for i in range(3)]),
        "piB": np.stack([np.stack([g(cl.SU2_EMOMENTUM(i, a)) for a in range(3)]) for i in range(3)]),
        "theta": np.zeros((3, N, N, N)), "piA": np.zeros((3, N, N, N)),
        "chi": np.zeros((N, N, N)), "pchi": np.zeros((N, N, N)),
    }
    if m.eA > 0:
        out["theta"] = np.stack([g(cl.LINK(i)) for i in range(3)])
        out["piA"] = np.stack([g(cl.EMOMENTUM(i)) for i in range(3)])
    if m.chi:
        out["chi"] = g(cl.SINGLET)
        out["pchi"] = g(cl.SINGLET_MOMENTUM)
    return out


def check_state(got, ref, tol):
    keys = ["phi", "pi", "piB"] + (["piA"] if ref.m.eA > 0 else []) + (["chi", "pchi"] if ref.m.chi else [])
    for k in keys:
        assert rel(got[k], getattr(ref, k)) < tol, (k, rel(got[k], getattr(ref, k)))
    assert np.max(np.abs(got["u"] - ref.u)) < tol
    if ref.m.eA > 0:
        assert angle_err(got["theta"], ref.theta) < tol


@pytest.mark.parametrize("integ,fmp,alpha,pot,eA,chi", [("vv2", 0.0, 0.0, 0, 0.7, 1), ("vv4", 0.7, 1.0, 1, 0.7, 1),
                                                        ("vv4", 0.5, 0.5, 0, 0.0, 1), ("vv2", 0.5, 0.5, 1, 0.6, 0)])
def test_su2u1_fp64_velocity_verlet_matches_oracle(integ, fmp, alpha, pot, eA, chi):
    """7 steps in two evolve calls, FP64, against the oracle's unmerged VVn;
    with and without the U(1) sector and the singlet."""
    N, dt = 8, 0.04
    m = SU2U1Model(N=N, dx=0.6, alpha=alpha, fmp2=fmp * fmp, lam=1.2, v2=0.8, g=0.9, kappa=1.21, pot=pot, p=4, eA=eA,
                   q=1.3, chi=chi)
    ref = random_state(N, m, 7)
    if fmp > 0:
        ref.b = math.sqrt(fmp * fmp / 3.0 * ref.energies().sum())
    lat = gpu_lattice(m, integ, cl.CL_FP64, fmp)
    load(lat, ref)
    E0 = ref.energies()
    mm = lat.measure_means()
    got0 = [mm["EK"][0], mm["EG"][0], mm["EV"][0], mm["EK"][1], mm["EG"][1], mm["EK"][2], mm["EG"][2], mm["EK"][3],
            mm["EG"][3]]
    assert np.allclose(got0, E0, rtol=1e-12, atol=1e-15), (got0, E0)
    lat.evolve(3)
    lat.evolve(4)
    ref.vv_steps({"vv2": oracle.VV2, "vv4": oracle.VV4}[integ], dt, 7)
    check_state(fetch(lat, m), ref, 1e-12)
    mm = lat.measure_means()
    assert abs(mm["a"] - ref.a) < 1e-13 and abs(mm["b"] - ref.b) < 1e-12 * (1 + abs(ref.b))
    E = ref.energies()
    got = [mm["EK"][0], mm["EG"][0], mm["EV"][0], mm["EK"][1], mm["EG"][1], mm["EK"][2], mm["EG"][2], mm["EK"][3],
           mm["EG"][3]]
    assert np.allclose(got, E, rtol=1e-11, atol=1e-14), (got, E)
    lat.close()


@pytest.mark.parametrize("N,prec,tol", [(40, cl.CL_FP64, 1e-12), (24, cl.CL_FP32, 1e-6), (64, cl.CL_FP32, 1e-6)])
def test_su2u1_many_tiles_match_oracle(N, prec, tol):
    """Several x-y tiles of the kick, block runs of planes crossing tiles: three
    expanding VV2 steps with the U(1) sector and the singlet against the oracle."""
    dt, fmp = 0.04, 0.7
    m = SU2U1Model(N=N, dx=0.6, alpha=1.0, fmp2=fmp * fmp, lam=1.2, v2=0.8, g=0.9, kappa=1.21, pot=1, p=4, eA=0.7,
                   q=1.3, chi=1)
    ref = random_state(N, m, 13)
    ref.b = math.sqrt(fmp * fmp / 3.0 * ref.energies().sum())
    lat = gpu_lattice(m, "vv2", prec, fmp)
    load(lat, ref)
    lat.evolve(3)
    ref.vv_steps(oracle.VV2, dt, 3)
    check_state(fetch(lat, m), ref, tol)
    mm = lat.measure_means()
    E = ref.energies()
    got = [mm["EK"][0], mm["EG"][0], mm["EV"][0], mm["EK"][1], mm["EG"][1], mm["EK"][2], mm["EG"][2], mm["EK"][3],
           mm["EG"][3]]
    assert np.allclose(got, E, rtol=10 * tol, atol=1e-14), (got, E)
    lat.close()


def test_su2u1_fp32_100_steps_match_oracle_pointwise():
    """FP32 over the first 100 steps (the pointwise bound 1e-5): the charge-free
    doublet with the U(1) sector and the singlet, unit links and Gauss-law
    electric momenta, on 64^3, expanding VV2, against the FP64 oracle."""
    N, dt, fmp = 64, 0.04, 0.7
    m = SU2U1Model(N=N, dx=0.6, alpha=1.0, fmp2=fmp * fmp, lam=1.2, v2=0.8, g=0.9, kappa=1.21, pot=1, p=4, eA=0.7,
                   q=1.3, chi=1)
    ref = gauss_state(N, m, 13)
    ref.b = math.sqrt(fmp * fmp / 3.0 * ref.energies().sum())
    lat = gpu_lattice(m, "vv2", cl.CL_FP32, fmp)
    load(lat, ref)
    lat.evolve(40)
    lat.evolve(60)
    ref.vv_steps(oracle.VV2, dt, 100)
    check_state(fetch(lat, m), ref, 1e-5)
    lat.close()


def test_su2u1_leapfrog_equals_velocity_verlet_positions_static():
    N, dt, n = 8, 0.04, 9
    m = SU2U1Model(N=N, dx=0.6, alpha=0.0, fmp2=0.0, lam=1.0, v2=1.0, g=1.1, kappa=0.9, eA=0.8, q=1.2)
    ref = random_state(N, m, 17)
    lat = gpu_lattice(m, "lf", cl.CL_FP64)
    load(lat, ref)
    lat.evolve(n)
    ref.vv_steps(oracle.VV2, dt, n)
    got = fetch(lat, m)
    assert rel(got["phi"], ref.phi) < 1e-12 and rel(got["chi"], ref.chi) < 1e-12
    assert np.max(np.abs(got["u"] - ref.u)) < 1e-12 and angle_err(got["theta"], ref.theta) < 1e-12
    lat.close()


@pytest.mark.parametrize("prec,tol", [(cl.CL_FP64, 1e-13), (cl.CL_FP32, 1e-5)])
def test_su2u1_both_gauss_laws_are_preserved(prec, tol):
    N = 16
    m = SU2U1Model(N=N, dx=0.5, alpha=1.0, fmp2=0.36, lam=1.0, v2=1.0, g=1.1, kappa=0.9, pot=1, p=4, eA=0.8, q=1.5)
    ref = gauss_state(N, m, 23)
    ref.b = math.sqrt(0.36 / 3.0 * ref.energies().sum())
    lat = gpu_lattice(m, "vv4", prec, 0.6)
    load(lat, ref)
    g = [lat.measure_means()["gauss_violation"]]
    for _ in range(4):
        lat.evolve(10)
        g.append(lat.measure_means()["gauss_violation"])
    assert max(g) < tol, g
    # each law separately, by the oracle's residuals on the evolved GPU state
    got = fetch(lat, m)
    probe = SU2U1Lattice(m, got["phi"], got["pi"], got["u"], got["piB"], got["theta"], got["piA"], got["chi"],
                         got["pchi"])
    gs = probe.gauss()
    assert math.sqrt(gs[0]) < tol and math.sqrt(gs[1]) < tol, gs
    assert np.max(np.abs(got["theta"])) > 1e-4 and np.max(np.abs(got["u"][:, 1:])) > 1e-3
    lat.close()


@pytest.mark.parametrize("prec", [cl.CL_FP64, cl.CL_FP32])
def test_su2u1_vacuum_initial_conditions_match_oracle(prec):
    """The constrained doublet draws, the singlet and both Gauss-law solves
    against the oracle's initial conditions; the charges vanish without a
    projection, so both Gauss laws hold at round-off from the start."""
    from oracle.ic import su2u1_ic
    N, dx, omega = 16, 0.5, 0.3
    c = 0.5 / math.sqrt(2.0)
    pb, db = [c] * 4, [-0.2 * c] * 4
    m = SU2U1Model(N=N, dx=dx, alpha=1.0, fmp2=0.4, lam=1.0, g=1.2, kappa=omega ** 2, pot=1, p=4, eA=0.9, q=1.0)
    kIR = 2 * math.pi / (N * dx)
    lat = gpu_lattice(m, "vv2", prec, math.sqrt(0.4), cl.make_init(phi0=pb, dphi0=db, seed=5, spectrum=1))
    phi, pi, u, piB, th, piA, chi, pchi, _ = su2u1_ic(m, kIR, pb, db, seed=5, omega_over_fstar=omega)
    got = fetch(lat, m)
    tol = 1e-12 if prec == cl.CL_FP64 else 2e-6
    assert rel(got["phi"], phi) < tol and rel(got["pi"], pi) < tol
    assert rel(got["chi"], chi) < tol and rel(got["pchi"], pchi) < tol
    assert rel(got["piB"], piB) < 10 * tol and rel(got["piA"], piA) < 10 * tol
    assert np.all(got["u"][:, 0] == 1.0) and np.all(got["u"][:, 1:] == 0.0) and np.all(got["theta"] == 0.0)
    mm = lat.measure_means()
    assert mm["gauss_violation"] < (1e-13 if prec == cl.CL_FP64 else 1e-5)
    assert mm["EG"][1] == 0.0 and mm["EG"][2] == 0.0 and mm["EK"][2] > 0 and mm["EK"][3] > 0
    lat.evolve(10)
    assert lat.measure_means()["gauss_violation"] < (1e-13 if prec == cl.CL_FP64 else 1e-5)
    k, D, cnt = lat.spectrum(1)  # the singlet's spectrum
    assert np.all(np.isfinite(D)) and D[1:].max() > 0 and cnt.sum() == N ** 3
    lat.close()


def test_su2u1_refusals():
    base = dict(kind=cl.CL_MODEL_SU2, gauge_e=1.0, gauge_e_u1=0.5)
    g = cl.make_grid(16, 0.5, 0.04, "vv2", cl.CL_FP64)
    with pytest.raises(cl.LatticeError):  # a uniform U(1) charge violates its Gauss law
        cl.Lattice(cl.make_model(**base), g, cl.make_init(phi0=(1.0, 0.0, 0.0, 0.0), dphi0=(0.0, 0.3, 0.0, 0.0),
                                                           spectrum=0))
    with pytest.raises(cl.LatticeError):
        cl.Lattice(cl.make_model(**dict(base, n_fields=3)), g, cl.make_init(spectrum=0))
    with pytest.raises(cl.LatticeError):
        cl.Lattice(cl.make_model(**dict(base, gauge_e_u1=-1.0)), g, cl.make_init(spectrum=0))


def test_su2u1_gauge_field_spectra_match_oracle():
    """Electric and magnetic spectra of both gauge sectors (sections 5.4, 6.3)
    against the oracle's fields of the same evolved state."""
    from oracle.spectra import spectrum
    N = 8
    m = SU2U1Model(N=N, dx=0.6, alpha=1.0, fmp2=0.49, lam=1.2, v2=0.8, g=0.9, kappa=1.21, pot=1, p=4, eA=0.7, q=1.3)
    ref = random_state(N, m, 7)
    ref.b = math.sqrt(0.49 / 3.0 * ref.energies().sum())
    lat = gpu_lattice(m, "vv4", cl.CL_FP64, 0.7)
    load(lat, ref)
    lat.evolve(5)
    got = fetch(lat, m)
    mm = lat.measure_means()
    probe = SU2U1Lattice(m, got["phi"], got["pi"], got["u"], got["piB"], got["theta"], got["piA"], got["chi"],
                         got["pchi"], a=mm["a"])
    kIR = 2 * math.pi / (N * m.dx)
    for sector in (0, 1):
        for what in (0, 1):
            fld = probe.electric(sector) if what == 0 else probe.magnetic(sector)
            fld = fld.reshape((-1,) + fld.shape[-3:])
            k, D, c = lat.gauge_spectrum(sector, what)
            rk, rD, rc = spectrum(fld, m.dx, kIR)
            assert np.array_equal(c, rc)
            assert np.max(np.abs(D - rD)) < 1e-10 * np.max(rD), (sector, what)
    lat.close()


@pytest.mark.parametrize("prec", [cl.CL_FP32, cl.CL_FP64])
def test_su2u1_checkpoint_continuation_is_bitwise(prec):
    """lattice_save / lattice_restore carry all 37 arrays and the background:
    evolving on from a restored checkpoint repeats the run bit for bit."""
    import os
    import tempfile
    N = 8
    m = SU2U1Model(N=N, dx=0.6, alpha=1.0, fmp2=0.49, lam=1.2, v2=0.8, g=0.9, kappa=1.21, pot=1, p=4, eA=0.7, q=1.3)
    ref = random_state(N, m, 9)
    ref.b = math.sqrt(0.49 / 3.0 * ref.energies().sum())
    lat = gpu_lattice(m, "vv4", prec, 0.7)
    load(lat, ref)
    lat.evolve(3)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        lat.save(path)
        lat.evolve(4)
        a, ma = fetch(lat, m), lat.measure_means()
        lat.restore(path)
        lat.evolve(4)
        b, mb = fetch(lat, m), lat.measure_means()
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert ma["a"] == mb["a"] and ma["b"] == mb["b"]
    # the Gauss residual sums with FP64 atomics: equal up to their order
    assert ma["gauss_violation"] == pytest.approx(mb["gauss_violation"], rel=1e-12)
    lat.close()
