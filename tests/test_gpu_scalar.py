"""Parity of the CUDA scalar path (through the C ABI) with the FP64 oracle.

FP64 runs must match the oracle to 1e-12 relative per step; FP32 runs to
1e-5 relative pointwise on the fluctuation arrays for the first 100 steps
and to 1e-3 on spectra and volume averages (max-norm relative error per
array, ||x - y||_inf / ||y||_inf)."""
import math
import os
import tempfile

import numpy as np
import pytest

import oracle
import paper_2006_15122_gb300 as cl
from oracle import ScalarLattice, ScalarModel
from oracle.ic import scalar_ic
from oracle.spectra import spectrum as oracle_spectrum
from tests import inputs

pytestmark = pytest.mark.gpu

WEIGHTS = {"vv2": oracle.VV2, "vv4": oracle.VV4, "vv6": oracle.VV6, "vv8": oracle.VV8, "vv10": oracle.VV10}


def rel(x, y):
    return float(np.max(np.abs(x - y)) / max(np.max(np.abs(y)), 1e-300))


def make_pair(N, Ns, pexp, alpha, fmp, lam, q, integ, prec, kIR=0.5, dt=0.01, seed=1, amp=0.2, means=None,
              a=1.0, b=None, omega=1.0):
    """A GPU lattice and an oracle lattice holding the same random state."""
    dx = 2 * math.pi / (kIR * N)
    m = cl.make_model(n_fields=Ns, pexp=pexp, alpha=alpha, fstar_over_mp=fmp, lam=lam, q=q, omega_over_fstar=omega)
    g = cl.make_grid(N, kIR, dt, integ, prec)
    lat = cl.Lattice(m, g, cl.make_init(phi0=means or [0.0] * Ns, spectrum=0))
    om = ScalarModel(N=N, Ns=Ns, pexp=pexp, dx=dx, alpha=alpha, fmp2=fmp * fmp, lam=lam, q=q)
    phi = inputs.fields(Ns, N, seed=seed, amp=amp, kmax=N / 4, means=means)
    pi = inputs.fields(Ns, N, seed=seed + 7, amp=amp)
    ref = ScalarLattice(om, phi, pi, a=a)
    ref.b = np.sqrt(ref.hubble_rhs()) if (b is None and fmp > 0) else (b or 0.0)
    for i in range(Ns):
        lat.set_field(cl.FIELD(i), phi[i])
        lat.set_field(cl.MOMENTUM(i), pi[i])
    lat.set_background(a, ref.b, 0.0)
    return lat, ref


def fields_of(lat, Ns):
    return (np.stack([lat.get_field(cl.FIELD(i)) for i in range(Ns)]),
            np.stack([lat.get_field(cl.MOMENTUM(i)) for i in range(Ns)]))


@pytest.mark.parametrize("N,Ns,pexp,alpha,integ", [
    (24, 1, 4, 1.0, "vv2"), (40, 2, 2, 0.0, "vv4"), (64, 2, 4, 0.5, "vv4"), (32, 1, 6, 1.5, "vv6"),
    (32, 2, 2, 0.5, "vv8"), (40, 2, 4, 1.0, "vv10")])
def test_fp64_single_step_matches_oracle(N, Ns, pexp, alpha, integ):
    lat, ref = make_pair(N, Ns, pexp, alpha, fmp=1.2, lam=1.0, q=3.0, integ=integ, prec=cl.CL_FP64,
                         means=[0.9, 0.1][:Ns])
    lat.evolve(1)
    ref.vv_steps(WEIGHTS[integ], 0.01, 1)
    phi, pi = fields_of(lat, Ns)
    for i in range(Ns):
        assert rel(phi[i], ref.phi[i]) < 1e-12
        assert rel(pi[i], ref.pi[i]) < 1e-12
    mm = lat.measure_means()
    assert abs(mm["a"] - ref.a) < 1e-14 * ref.a and abs(mm["b"] - ref.b) < 1e-12 * abs(ref.b)
    lat.close()


@pytest.mark.parametrize("integ", ["vv8", "vv10"])
def test_fp64_vv8_vv10_several_steps_match_oracle(integ):
    """The VV8 and VV10 weights of the library (appendix table) against the
    oracle's own copy: 5 expanding steps of the two-field model in two calls."""
    lat, ref = make_pair(32, 2, 2, 0.0, fmp=1.0, lam=1.0, q=5.0, integ=integ, prec=cl.CL_FP64, means=[1.0, 0.0])
    lat.evolve(2)
    lat.evolve(3)
    ref.vv_steps(WEIGHTS[integ], 0.01, 5)
    phi, pi = fields_of(lat, 2)
    for i in range(2):
        assert rel(phi[i], ref.phi[i]) < 1e-12
        assert rel(pi[i], ref.pi[i]) < 1e-12
    mm = lat.measure_means()
    assert abs(mm["a"] - ref.a) < 1e-14 * ref.a and abs(mm["b"] - ref.b) < 1e-12 * abs(ref.b)
    lat.close()


@pytest.mark.parametrize("integ", ["vv4", "lf"])
def test_fp64_long_call_crosses_graph_pieces(integ):
    """One evolve call of 150 steps runs as three recorded graphs (64 + 64 + 22
    steps) that continue one pass sequence: it must equal the oracle's 150 steps
    (velocity-Verlet: 3 x 150 + 1 passes; leapfrog: one closing drift)."""
    N, dt, steps = 16, 0.01, 150
    lat, ref = make_pair(N, 2, 2, 0.0, fmp=1.0, lam=1.0, q=5.0, integ=integ, prec=cl.CL_FP64, means=[1.0, 0.0])
    lat.evolve(steps)
    if integ == "lf":
        ref.lf3_prepare(dt)
        ref.lf3_steps(dt, steps)
    else:
        ref.vv_steps(oracle.VV4, dt, steps)
    phi, pi = fields_of(lat, 2)
    for i in range(2):
        assert rel(phi[i], ref.phi[i]) < 1e-11
        assert rel(pi[i], ref.pi[i]) < 1e-11
    mm = lat.measure_means()
    assert abs(mm["a"] - ref.a) < 1e-13 * ref.a and abs(mm["t"] - steps * dt) < 1e-12
    lat.close()


def test_fp64_many_steps_vv4_and_means():
    lat, ref = make_pair(48, 2, 2, 0.0, fmp=1.0, lam=1.0, q=5.0, integ="vv4", prec=cl.CL_FP64, means=[1.0, 0.0])
    for _ in range(3):
        lat.evolve(7)
        ref.vv_steps(oracle.VV4, 0.01, 7)
    phi, pi = fields_of(lat, 2)
    assert rel(phi, ref.phi) < 1e-11 and rel(pi, ref.pi) < 1e-11
    mm = lat.measure_means()
    E = ref.energies()
    assert np.allclose(mm["EK"][:2], E[0:2], rtol=1e-11) and np.allclose(mm["EG"][:2], E[2:4], rtol=1e-11)
    assert np.allclose(mm["EV"][:2], E[4:6], rtol=1e-11)
    assert abs(mm["mean"][0] - ref.phi[0].mean()) < 1e-12
    assert abs(mm["var"][1] - ref.phi[1].var()) < 1e-11 * ref.phi[1].var()
    assert abs(mm["hubble_violation"] - ref.hubble_violation()) < 1e-9
    assert mm["step"] == 21 and abs(mm["t"] - 0.21) < 1e-12
    lat.close()


def test_fp64_leapfrog_matches_oracle():
    lat, ref = make_pair(32, 2, 2, 0.5, fmp=1.0, lam=1.0, q=2.0, integ="lf", prec=cl.CL_FP64, means=[1.0, 0.0])
    ref.lf3_prepare(0.01)
    lat.evolve(5)
    lat.evolve(6)
    ref.lf3_steps(0.01, 11)
    phi, pi = fields_of(lat, 2)
    assert rel(phi, ref.phi) < 1e-12 and rel(pi, ref.pi) < 1e-12
    mm = lat.measure_means()
    assert abs(mm["a"] - ref.a) < 1e-13 and abs(mm["b"] - ref.b) < 1e-12 * abs(ref.b)
    assert abs(mm["EK"][0] - ref.EKm) < 1e-12 * ref.EKm
    lat.close()


@pytest.mark.parametrize("N,prec", [(32, cl.CL_FP64), (48, cl.CL_FP32)])
def test_initial_conditions_match_oracle(N, prec):
    """Same seed, same Philox draws: the device ICs equal the oracle's (FP64
    to 1e-12; FP32 to its rounding), and b comes from the Hubble constraint."""
    kIR, omega, fmp = 0.5, 0.05, 1.0
    dx = 2 * math.pi / (kIR * N)
    m = cl.make_model(n_fields=2, pexp=2, lam=1.0, q=2.0, omega_over_fstar=omega, fstar_over_mp=fmp)
    lat = cl.Lattice(m, cl.make_grid(N, kIR, 0.01, "vv2", prec), cl.make_init(phi0=(1.0, 0.0), dphi0=(-0.1, 0.0), seed=77))
    om = ScalarModel(N=N, Ns=2, pexp=2, dx=dx, alpha=0.0, fmp2=fmp * fmp, lam=1.0, q=2.0)
    phi, pi, _ = scalar_ic(om, kIR, [1.0, 0.0], [-0.1, 0.0], seed=77, omega_over_fstar=omega)
    gphi, gpi = fields_of(lat, 2)
    tol = 1e-12 if prec == cl.CL_FP64 else 1e-6
    for i in range(2):
        assert rel(gphi[i] - gphi[i].mean(), phi[i] - phi[i].mean()) < tol
        assert rel(gpi[i], pi[i]) < tol
    ref = ScalarLattice(om, phi, pi)
    mm = lat.measure_means()
    # the device evaluates the Hubble constraint on its stored (FP32-rounded) fluctuations
    assert abs(mm["b"] - np.sqrt(ref.hubble_rhs())) < (1e-12 if prec == cl.CL_FP64 else 1e-7) * mm["b"]
    lat.close()


def test_fp32_pointwise_parity_100_steps():
    """Two-field preheating-like state (mean 1 plus 1e-3 fluctuations), FP32
    fluctuation arrays with FP64 means: 100 VV4 steps within 1e-5 relative."""
    N = 32
    lat, ref = make_pair(N, 2, 2, 0.0, fmp=1.4, lam=1.0, q=400.0, integ="vv4", prec=cl.CL_FP32, kIR=0.5, dt=0.005,
                         amp=1e-3, means=[1.0, 0.0])
    lat.evolve(100)
    ref.vv_steps(oracle.VV4, 0.005, 100)
    phi, pi = fields_of(lat, 2)
    for i in range(2):
        d_gpu = phi[i] - phi[i].mean()
        d_ref = ref.phi[i] - ref.phi[i].mean()
        assert rel(d_gpu, d_ref) < 1e-5, (i, rel(d_gpu, d_ref))
        assert rel(pi[i] - pi[i].mean(), ref.pi[i] - ref.pi[i].mean()) < 1e-5
    mm = lat.measure_means()
    E = ref.energies()
    assert abs(mm["a"] - ref.a) < 1e-9
    assert np.allclose(mm["EK"][:2], E[0:2], rtol=1e-5) and np.allclose(mm["EG"][:2], E[2:4], rtol=1e-5)
    lat.close()


@pytest.mark.parametrize("N,steps", [(128, 100), (256, 40)])
def test_fp32_production_tile_matches_oracle(N, steps):
    """Two-field lattices on the compiled-in x-y tiles of the FP32 pass: 32 x 8
    threads of 4 sites at 128^3 (after the small-lattice halving of the rows)
    and 32 x 16 at 256^3 (the tile of the 1024^3 workload), a 5-stage ring,
    several tiles in every direction: expanding VV4 steps in two calls against
    the oracle within the FP32 pointwise bound."""
    lat, ref = make_pair(N, 2, 2, 0.0, fmp=1.4, lam=1.0, q=400.0, integ="vv4", prec=cl.CL_FP32, kIR=0.5, dt=0.005,
                         seed=21, amp=1e-3, means=[1.0, 0.0])
    lat.evolve(30)
    lat.evolve(steps - 30)
    ref.vv_steps(oracle.VV4, 0.005, steps)
    phi, pi = fields_of(lat, 2)
    for i in range(2):
        assert rel(phi[i] - phi[i].mean(), ref.phi[i] - ref.phi[i].mean()) < 1e-5
        assert rel(pi[i] - pi[i].mean(), ref.pi[i] - ref.pi[i].mean()) < 1e-5
    mm = lat.measure_means()
    E = ref.energies()
    assert abs(mm["a"] - ref.a) < 1e-9  # a follows the FP32 energies through K_a
    assert np.allclose(mm["EK"][:2], E[0:2], rtol=1e-5) and np.allclose(mm["EG"][:2], E[2:4], rtol=1e-5)
    lat.close()


def test_spectrum_matches_oracle():
    N, kIR = 32, 0.4
    lat, ref = make_pair(N, 2, 2, 0.0, fmp=0.0, lam=1.0, q=1.0, integ="vv2", prec=cl.CL_FP64, kIR=kIR)
    dx = 2 * math.pi / (kIR * N)
    for f in range(2):
        for what, arr in ((0, ref.phi[f]), (1, ref.pi[f])):
            k, D, c = lat.spectrum(f, what)
            k0, D0, c0 = oracle_spectrum(arr, dx, kIR)
            assert np.array_equal(c, c0)
            assert np.allclose(k, k0, rtol=1e-13)
            # modes beyond the band limit of the input hold only rounding noise
            assert np.allclose(D, D0, rtol=1e-10, atol=1e-10 * D0.max())
    lat.close()


def test_checkpoint_continuation_is_bitwise():
    lat, _ = make_pair(32, 2, 2, 0.0, fmp=1.0, lam=1.0, q=2.0, integ="vv4", prec=cl.CL_FP32, means=[1.0, 0.0])
    lat.evolve(3)
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "ck.bin")
        lat.save(path)
        lat.evolve(4)
        a = fields_of(lat, 2)
        ma = lat.measure_means()
        lat.restore(path)
        lat.evolve(4)
        b = fields_of(lat, 2)
        mb = lat.measure_means()
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        assert ma["a"] == mb["a"] and ma["b"] == mb["b"]
        with open(path, "r+b") as fp:
            fp.seek(-5, 2)
            fp.write(b"\x00\x01\x02\x03\x04")
        with pytest.raises(cl.LatticeError) as e:
            lat.restore(path)
        assert e.value.status == cl.CL_ERR_IO
    lat.close()


def test_nonfinite_state_is_reported():
    lat, _ = make_pair(16, 1, 2, 0.0, fmp=0.0, lam=1.0, q=0.0, integ="vv2", prec=cl.CL_FP32)
    bad = np.zeros((16, 16, 16))
    bad[3, 4, 5] = np.nan
    lat.set_field(cl.MOMENTUM(0), bad)
    lat.evolve(2)
    with pytest.raises(cl.LatticeError) as e:
        lat.measure_means()
    assert e.value.status == cl.CL_ERR_NONFINITE
    lat.close()


@pytest.mark.parametrize("integ,w,alpha", [("vv4", 1.0 / 3.0, 1.0), ("vv2", 0.0, 0.0)])
def test_fluid_background_matches_oracle(integ, w, alpha):
    """Prescribed expansion of an external fluid (section 4.1): the GPU passes
    against the oracle's VVn with a(t) = a0 (1 + H0 t/p)^p, 9 steps in two calls."""
    from oracle.core import Fluid
    N, kIR, dt, H0, a0 = 24, 0.6, 0.01, 0.7, 1.2
    model = cl.make_model(n_fields=2, pexp=2, alpha=alpha, lam=1.0, q=30.0, omega_over_fstar=0.05,
                          background=cl.CL_BG_FLUID, fluid_w=w, hubble0=H0)
    lat = cl.Lattice(model, cl.make_grid(N, kIR, dt, integ, cl.CL_FP64), cl.make_init(phi0=(1.0, 0.0), a0=a0))
    om = ScalarModel(N=N, Ns=2, pexp=2, dx=2 * math.pi / (kIR * N), alpha=alpha, fmp2=0.0, lam=1.0, q=30.0)
    phi = inputs.fields(2, N, seed=71, amp=0.05, kmax=4, means=[1.0, 0.0])
    pi = inputs.fields(2, N, seed=72, amp=0.05, kmax=4)
    for f in range(2):
        lat.set_field(cl.FIELD(f), phi[f])
        lat.set_field(cl.MOMENTUM(f), pi[f])
    lat.set_background(0.0, 0.0, 0.0)
    fl = Fluid(a0=a0, H0=H0, w=w, alpha=alpha)
    ref = ScalarLattice(om, phi, pi, a=a0)
    ref.t = 0.0
    lat.evolve(4)
    lat.evolve(5)
    ref.vv_steps_fluid(fl, {"vv2": oracle.VV2, "vv4": oracle.VV4}[integ], dt, 9)
    gphi = np.stack([lat.get_field(cl.FIELD(f)) for f in range(2)])
    gpi = np.stack([lat.get_field(cl.MOMENTUM(f)) for f in range(2)])
    assert rel(gphi - gphi.mean(axis=(1, 2, 3), keepdims=True), ref.phi - ref.phi.mean(axis=(1, 2, 3), keepdims=True)) < 1e-11
    assert rel(gpi, ref.pi) < 1e-11
    mm = lat.measure_means()
    assert abs(mm["a"] - fl.a(9 * dt)) < 1e-13 and abs(mm["b"] - fl.b(9 * dt)) < 1e-13
    assert abs(mm["t"] - 9 * dt) < 1e-13 and mm["hubble_violation"] == 0.0
    lat.close()


def test_fluid_background_rejects_leapfrog_and_bad_w():
    for integ, w in (("lf", 0.0), ("vv2", -2.0)):
        model = cl.make_model(n_fields=1, pexp=2, background=cl.CL_BG_FLUID, fluid_w=w, hubble0=0.5)
        with pytest.raises(cl.LatticeError):
            cl.Lattice(model, cl.make_grid(16, 0.5, 0.01, integ, cl.CL_FP64), cl.make_init())


@pytest.mark.parametrize("N,alpha,pexp", [(24, 0.0, 2), (16, 1.0, 4)])
def test_rk4_matches_oracle(N, alpha, pexp):
    """Explicit RK4 of section 4.3.1 on the GPU (four stage passes per step,
    full fields in FP64) against the oracle's RK4, 5 steps in two calls, with
    self-consistent expansion."""
    kIR, dt, fmp = 0.6, 0.01, 0.9
    model = cl.make_model(n_fields=2, pexp=pexp, alpha=alpha, lam=1.0, q=20.0, omega_over_fstar=0.05,
                          fstar_over_mp=fmp)
    lat = cl.Lattice(model, cl.make_grid(N, kIR, dt, "rk4", cl.CL_FP64), cl.make_init(phi0=(1.0, 0.0)))
    om = ScalarModel(N=N, Ns=2, pexp=pexp, dx=2 * math.pi / (kIR * N), alpha=alpha, fmp2=fmp * fmp, lam=1.0, q=20.0)
    phi = inputs.fields(2, N, seed=81, amp=0.05, kmax=4, means=[1.0, 0.0])
    pi = inputs.fields(2, N, seed=82, amp=0.05, kmax=4)
    for f in range(2):
        lat.set_field(cl.FIELD(f), phi[f])
        lat.set_field(cl.MOMENTUM(f), pi[f])
    ref = ScalarLattice(om, phi, pi)
    ref.b = math.sqrt(ref.hubble_rhs())
    lat.set_background(1.0, ref.b, 0.0)
    lat.evolve(2)
    lat.evolve(3)
    ref.rk4_steps(dt, 5)
    gphi = np.stack([lat.get_field(cl.FIELD(f)) for f in range(2)])
    gpi = np.stack([lat.get_field(cl.MOMENTUM(f)) for f in range(2)])
    assert rel(gphi, ref.phi) < 1e-12
    assert rel(gpi, ref.pi) < 1e-12
    mm = lat.measure_means()
    assert abs(mm["a"] - ref.a) < 1e-13 and abs(mm["b"] - ref.b) < 1e-12 * abs(ref.b) + 1e-14
    assert abs(mm["t"] - 5 * dt) < 1e-13
    lat.close()


def test_rk4_hubble_constraint_order_four():
    """The Hubble constraint of RK4 converges at fourth order in dt."""
    vals = []
    for dt in (0.02, 0.01):
        model = cl.make_model(n_fields=1, pexp=4, alpha=1.0, lam=1.0, omega_over_fstar=0.01, fstar_over_mp=1.0)
        lat = cl.Lattice(model, cl.make_grid(16, 0.5, dt, "rk4", cl.CL_FP64), cl.make_init(phi0=(1.0,), seed=3,
                                                                                      fluct_scale=100.0))
        lat.evolve(int(round(2.0 / dt)))
        vals.append(lat.measure_means()["hubble_violation"])
        lat.close()
    assert 3.5 < math.log2(vals[0] / vals[1]) < 4.5, vals


def test_rk4_rejects_fp32_and_fluid():
    with pytest.raises(cl.LatticeError):
        cl.Lattice(cl.make_model(n_fields=1), cl.make_grid(16, 0.5, 0.01, "rk4", cl.CL_FP32), cl.make_init())
    with pytest.raises(cl.LatticeError):
        cl.Lattice(cl.make_model(n_fields=1, background=cl.CL_BG_FLUID, hubble0=0.5),
                   cl.make_grid(16, 0.5, 0.01, "rk4", cl.CL_FP64), cl.make_init())


@pytest.mark.parametrize("s,N", [(2, 16), (3, 24), (5, 8)])
def test_gauss_legendre_matches_oracle(s, N):
    """Implicit Gauss-Legendre (sections 3.4.2, 4.3.3) on the GPU: fixed-point
    stage sweeps with a device-side convergence flag, against the oracle's
    Gauss-Legendre step, 3 steps in two calls, self-consistent expansion."""
    kIR, dt, fmp = 0.6, 0.02, 0.9
    model = cl.make_model(n_fields=2, pexp=2, alpha=0.0, lam=1.0, q=20.0, omega_over_fstar=0.05, fstar_over_mp=fmp)
    lat = cl.Lattice(model, cl.make_grid(N, kIR, dt, "gl%d" % s, cl.CL_FP64), cl.make_init(phi0=(1.0, 0.0)))
    om = ScalarModel(N=N, Ns=2, pexp=2, dx=2 * math.pi / (kIR * N), alpha=0.0, fmp2=fmp * fmp, lam=1.0, q=20.0)
    phi = inputs.fields(2, N, seed=91, amp=0.05, kmax=N / 4, means=[1.0, 0.0])
    pi = inputs.fields(2, N, seed=92, amp=0.05, kmax=N / 4)
    for f in range(2):
        lat.set_field(cl.FIELD(f), phi[f])
        lat.set_field(cl.MOMENTUM(f), pi[f])
    ref = ScalarLattice(om, phi, pi)
    ref.b = math.sqrt(ref.hubble_rhs())
    lat.set_background(1.0, ref.b, 0.0)
    lat.evolve(1)
    lat.evolve(2)
    ref.gl_steps(s, dt, 3)
    gphi = np.stack([lat.get_field(cl.FIELD(f)) for f in range(2)])
    gpi = np.stack([lat.get_field(cl.MOMENTUM(f)) for f in range(2)])
    assert rel(gphi, ref.phi) < 1e-12
    assert rel(gpi, ref.pi) < 1e-12
    mm = lat.measure_means()
    assert abs(mm["a"] - ref.a) < 1e-13 and abs(mm["b"] - ref.b) < 1e-12 * abs(ref.b)
    assert abs(mm["t"] - 3 * dt) < 1e-13
    lat.close()


def test_gauss_legendre_reports_stage_equations_that_do_not_converge():
    """A time step beyond the bound that keeps the stage sweeps contracting
    (forced past the init check): the step is not applied, the lattice stops and
    the next synchronizing call reports CL_ERR_TIMEOUT instead of a silent result."""
    N, kIR, dt = 16, 0.5, 0.8  # omega_max dt ~ 3.6, sweep growth ~ 1.4 per sweep on GL2
    model = cl.make_model(n_fields=1, pexp=2, alpha=0.0, lam=1.0, omega_over_fstar=0.05, fstar_over_mp=0.0)
    lat = cl.Lattice(model, cl.make_grid(N, kIR, dt, "gl2", cl.CL_FP64, force_dt=True), cl.make_init(phi0=(1.0,)))
    phi = inputs.fields(1, N, seed=93, amp=0.05, means=[1.0])
    lat.set_field(cl.FIELD(0), phi[0])
    lat.set_background(1.0, 0.0, 0.0)
    lat.evolve(2)
    with pytest.raises(cl.LatticeError) as e:
        lat.measure_means()
    assert e.value.status == cl.CL_ERR_TIMEOUT and "did not converge" in str(e.value)
    assert np.max(np.abs(lat.get_field(cl.FIELD(0)) - phi[0])) < 1e-14  # nothing applied
    lat.close()


@pytest.mark.parametrize("prec,tol", [(cl.CL_FP64, 1e-5), (cl.CL_FP32, 2e-3)])
def test_parametric_resonance_matches_mathieu_floquet(prec, tol):
    """The GPU lattice in the linear regime of phi^2 chi^2 preheating (static
    background, q* = 10, one chi mode at k_L = 0.5): its amplitude follows the
    Mathieu equation chi'' + (k_L^2 + q* cos^2 t) chi = 0 over eight periods
    and grows per period by the Floquet multiplier of the monodromy matrix
    (the mean/fluctuation split carries phi = cos t exactly in FP64)."""
    from tests.test_oracle_scalar import _mathieu_reference
    N, qs = 8, 10.0
    dx = 2.0 * math.sin(math.pi / N) / 0.5
    kIR = 2 * math.pi / (N * dx)
    k2 = (2.0 * math.sin(math.pi / N) / dx) ** 2
    steps = int(round(math.pi / 0.01))
    dt = math.pi / steps
    m = cl.make_model(n_fields=2, pexp=2, lam=1.0, q=qs, omega_over_fstar=1.0)
    lat = cl.Lattice(m, cl.make_grid(N, kIR, dt, "vv4", prec), cl.make_init(phi0=(1.0, 0.0), spectrum=0))
    x = np.arange(N)
    mode = np.ascontiguousarray(np.broadcast_to(np.cos(2 * np.pi * x / N)[None, None, :], (N, N, N)))
    eps = 1e-6
    lat.set_field(cl.FIELD(1), eps * mode)
    sol, lam_max = _mathieu_reference(k2, qs, 1.0, 8 * np.pi)
    amps = []
    for n in range(8):
        lat.evolve(steps)
        c = (lat.get_field(cl.FIELD(1)) * mode).sum() / (mode * mode).sum() / eps
        amps.append(c)
        ref = sol.sol((n + 1) * np.pi)[0]
        assert abs(c - ref) < tol * max(1.0, abs(ref)), (n, c, ref)
    assert abs(amps[-1] / amps[-2] - lam_max) < 0.02 * lam_max
    lat.close()


@pytest.mark.parametrize("prec", [cl.CL_FP32, cl.CL_FP64])
def test_stored_representation_round_trip_is_exact(prec):
    """lattice_get_stored / lattice_set_stored: mean + array is exactly the full
    field of lattice_get_field, a lattice loaded from the stored arrays (host
    buffers) holds the same fields bit for bit, and it evolves like the original
    (to the rounding of the handle's precision: the pending mean shifts are folded
    into the arrays)."""
    N, kIR, dt = 32, 0.5, 0.005
    model = cl.make_model(n_fields=2, pexp=2, lam=1.0, q=200.0, omega_over_fstar=0.05, fstar_over_mp=1.0)
    grid = cl.make_grid(N, kIR, dt, "vv4", prec)
    a = cl.Lattice(model, grid, cl.make_init(phi0=(1.0, 0.0), seed=41))
    b = cl.Lattice(model, grid, cl.make_init(phi0=(0.3, 0.0), seed=2))
    a.evolve(7)
    which = [cl.FIELD(0), cl.FIELD(1), cl.MOMENTUM(0), cl.MOMENTUM(1)]
    for w in which:
        arr, mean = a.get_stored(w)
        full = a.get_field(w)
        assert arr.dtype == (np.float32 if prec == cl.CL_FP32 else np.float64)
        assert np.array_equal(mean + arr.astype(np.float64), full), w
        b.set_stored(w, arr, mean)
        assert np.array_equal(b.get_field(w), full), w
    mm = a.measure_means()
    b.set_background(mm["a"], mm["b"], mm["t"])
    a.evolve(5)
    b.evolve(5)
    tol = 1e-5 if prec == cl.CL_FP32 else 1e-12
    for w in which:
        x, y = b.get_field(w), a.get_field(w)
        assert rel(x - x.mean(), y - y.mean()) < tol, w
    with pytest.raises(ValueError):
        b.set_stored(cl.FIELD(0), np.zeros(N ** 3, dtype=np.float16), 0.0)
    a.close()
    b.close()
