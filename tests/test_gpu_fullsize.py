"""Parity at the full sizes of the workloads, in the launch configurations
that bench.py times:

- the 1024^3 two-field lattice (FP32 fluctuations, VV4, the bench's tile and
  grid): with chi = 0 and a static background every Fourier mode of phi is an
  exact lattice oscillator, so sampled sites are checked one by one against the
  closed form (the product of the VV2 maps of section 4.3.2);
- the 32^3 FP64 phi^4 leapfrog with self-consistent expansion, 2000 steps,
  against the oracle;
- the 128^3 two-field preheating lattice (q* = 4e4, VV4, FP32 fluctuations)
  over 2000 steps against the oracle from one shared vacuum start: pointwise
  within 1e-5 for the first 100 steps, then spectra and volume averages within
  1e-3;
- the 128^3 compact U(1) leapfrog in FP32 against the oracle: pointwise within
  1e-5 for 100 steps, spectra within 1e-3 while the trajectories stay inside
  their Lyapunov horizon, volume averages within 1e-3 and the Gauss law of the
  GPU state, evaluated by the oracle, at FP32 round-off over 1000 steps."""
import math

import numpy as np
import pytest

import oracle
import paper_2006_15122_gb300 as cl
from oracle import ScalarLattice, ScalarModel, U1Lattice, U1Model
from oracle.spectra import spectrum as oracle_spectrum

pytestmark = pytest.mark.gpu


def _vv_product(weights, h, w2, steps):
    M = np.eye(2)
    for wp in weights:
        k = wp * h
        c = 1.0 - 0.5 * k * k * w2
        M = np.array([[c, k], [-k * w2 * (1.0 - 0.25 * k * k * w2), c]]) @ M
    return np.linalg.matrix_power(M, steps)


def test_1024_cubed_vv4_fp32_plane_wave_matches_closed_form():
    torch = pytest.importorskip("torch")
    import bench

    N, steps, eps = 1024, 100, 1e-3
    nvec = (3, 5, 7)
    model = cl.make_model(n_fields=2, pexp=2, alpha=0.0, fstar_over_mp=0.0, omega_over_fstar=bench.OMEGA_FSTAR,
                          lam=1.0, q=bench.QSTAR)
    lat = cl.Lattice(model, cl.make_grid(N, bench.KIR, bench.DT, "vv4", cl.CL_FP32),
                     cl.make_init(phi0=(1.0, 0.0), spectrum=0))
    dx = 2 * math.pi / (bench.KIR * N)
    x = torch.arange(N, device="cuda", dtype=torch.float64)
    ang = 2 * math.pi / N
    phase = (ang * nvec[2] * x).view(N, 1, 1) + (ang * nvec[1] * x).view(1, N, 1) + (ang * nvec[0] * x).view(1, 1, N)
    field = 1.0 + eps * torch.cos(phase)
    lat.set_field(cl.FIELD(0), field)
    del field
    lat.evolve(steps)
    got = torch.empty((N, N, N), device="cuda", dtype=torch.float64)
    lat.get_field(cl.FIELD(0), got)
    # closed form: the mean (k = 0, w^2 = lam) and the plane wave (w^2 = lam + k_L^2), both from (1, 0)
    w2k = 1.0 + sum(4 * math.sin(math.pi * c / N) ** 2 for c in nvec) / dx ** 2
    X0 = _vv_product(oracle.VV4, bench.DT, 1.0, steps)[0, 0]
    Xk = _vv_product(oracle.VV4, bench.DT, w2k, steps)[0, 0]
    rng = np.random.default_rng(11)
    idx = torch.as_tensor(rng.integers(0, N, size=(3, 4096)), device="cuda")
    sample = got[idx[0], idx[1], idx[2]]
    ph = phase[idx[0], idx[1], idx[2]]
    ref = X0 + eps * Xk * torch.cos(ph)
    err = (sample - ref).abs().max().item()
    # the FP32 pointwise bound: max-norm error over the fluctuation's own amplitude eps |Xk|
    assert err < 1e-5 * eps * abs(Xk), (err / (eps * abs(Xk)), X0, Xk)
    mm = lat.measure_means()
    assert abs(mm["mean"][0] - X0) < 1e-12 and mm["a"] == 1.0
    lat.get_field(cl.FIELD(1), got)
    assert got.abs().max().item() == 0.0  # chi = 0 is exact: its force is q phi^2 chi
    lat.close()


def test_32_cubed_phi4_fp64_leapfrog_2000_steps_matches_oracle():
    """The phi^4 workload at its full size and length: 32^3, k_IR = 0.5,
    dt = 0.01, scheme III with self-consistent expansion (alpha = 1, f*/m_p = 1,
    omega*/f* = 1e-2), vacuum start (section 7), against the oracle."""
    from oracle.ic import scalar_ic
    N, kIR, dt, steps = 32, 0.5, 0.01, 2000
    dx = 2 * math.pi / (kIR * N)
    model = cl.make_model(n_fields=1, pexp=4, alpha=1.0, fstar_over_mp=1.0, omega_over_fstar=1e-2, lam=1.0)
    lat = cl.Lattice(model, cl.make_grid(N, kIR, dt, "lf", cl.CL_FP64), cl.make_init(phi0=(1.0,), seed=0))
    om = ScalarModel(N=N, Ns=1, pexp=4, dx=dx, alpha=1.0, fmp2=1.0, lam=1.0)
    phi, pi, _ = scalar_ic(om, kIR, [1.0], [0.0], seed=0, omega_over_fstar=1e-2)
    ref = ScalarLattice(om, phi, pi)
    ref.b = math.sqrt(1.0 / 3.0 * ref.energies().sum())
    assert np.max(np.abs(lat.get_field(cl.FIELD(0)) - phi[0])) < 1e-13
    ref.lf3_prepare(dt)
    ref.lf3_steps(dt, steps)
    lat.evolve(steps)
    g = lat.get_field(cl.FIELD(0))
    dphi = ref.phi[0] - ref.phi[0].mean()
    assert abs(g.mean() - ref.phi[0].mean()) < 1e-9
    assert np.max(np.abs((g - g.mean()) - dphi)) < 1e-6 * np.max(np.abs(dphi))
    mm = lat.measure_means()
    assert abs(mm["a"] - ref.a) < 1e-10 * ref.a
    assert mm["hubble_violation"] < 1e-4
    lat.close()


def test_128_cubed_u1_fp32_leapfrog_keeps_gauss_law():
    N, dx = 128, 0.5
    model = cl.make_model(kind=cl.CL_MODEL_U1, lam=1.0, vev2=1.0, gauge_e=1.0, omega_over_fstar=1.0)
    lat = cl.Lattice(model, cl.make_grid(N, 2 * math.pi / (N * dx), 0.1 * dx, "lf", cl.CL_FP32),
                     cl.make_init(seed=7))
    g = []
    for _ in range(4):
        lat.evolve(100)
        g.append(lat.measure_means()["gauss_violation"])
    assert max(g) < 1e-5, g
    mm = lat.measure_means()
    assert mm["EG"][1] > 0 and np.isfinite(mm["rho"])
    lat.close()


def test_128_cubed_two_field_vv2_vv4_hubble_constraint():
    """The q = 1e4 preheating lattice (128^3, k_IR = 0.1, dt = 0.005, FP32
    fluctuations, f*/m_p = 1.396, omega*/f* = 5.13e-6) over 2000 steps: the Hubble
    constraint stays satisfied, and VV4 keeps it better than VV2 (section 4.3.2)."""
    de = {}
    for integ in ("vv2", "vv4"):
        model = cl.make_model(n_fields=2, pexp=2, alpha=0.0, fstar_over_mp=1.396, omega_over_fstar=5.13e-6, lam=1.0,
                              q=4.0e4)
        lat = cl.Lattice(model, cl.make_grid(128, 0.1, 0.005, integ, cl.CL_FP32), cl.make_init(phi0=(1.0, 0.0), seed=0))
        lat.evolve(2000)
        mm = lat.measure_means()
        de[integ] = mm["hubble_violation"]
        assert np.isfinite(mm["rho"]) and mm["a"] > 1.0
        lat.close()
    assert de["vv2"] < 1e-3 and de["vv4"] < de["vv2"], de


def _rel(x, y):
    return float(np.max(np.abs(x - y)) / max(np.max(np.abs(y)), 1e-300))


def _spectrum_err(got, ref):
    """Largest relative difference over the shells b >= 1 where the oracle has power."""
    (k, D, c), (k2, D2, c2) = got, ref
    assert np.array_equal(c, c2) and np.allclose(k, k2, rtol=1e-12)
    m = (np.arange(D2.size) >= 1) & (D2 > 0)
    return float(np.max(np.abs(D[m] - D2[m]) / D2[m]))


def test_128_cubed_two_field_vv4_fp32_matches_oracle_over_2000_steps():
    """The q = 1e4 preheating workload at its size and length (128^3,
    k_IR = 0.1, dt = 0.005, q* = 4e4, f*/m_p = 1.396, omega*/f* = 5.13e-6, VV4,
    FP32 fluctuations with FP64 means, 2000 steps) from the vacuum start the
    oracle draws with the same Philox key."""
    from oracle.ic import scalar_ic
    N, kIR, dt, q, fmp, om_ = 128, 0.1, 0.005, 4.0e4, 1.396, 5.13e-6
    dx = 2 * math.pi / (kIR * N)
    model = cl.make_model(n_fields=2, pexp=2, alpha=0.0, fstar_over_mp=fmp, omega_over_fstar=om_, lam=1.0, q=q)
    lat = cl.Lattice(model, cl.make_grid(N, kIR, dt, "vv4", cl.CL_FP32), cl.make_init(phi0=(1.0, 0.0), seed=3))
    om = ScalarModel(N=N, Ns=2, pexp=2, dx=dx, alpha=0.0, fmp2=fmp * fmp, lam=1.0, q=q)
    phi, pi, _ = scalar_ic(om, kIR, [1.0, 0.0], [0.0, 0.0], seed=3, omega_over_fstar=om_)
    ref = ScalarLattice(om, phi, pi)
    ref.b = math.sqrt(ref.hubble_rhs())
    lat.evolve(100)
    ref.vv_steps(oracle.VV4, dt, 100)
    for f in range(2):
        g, p = lat.get_field(cl.FIELD(f)), lat.get_field(cl.MOMENTUM(f))
        assert _rel(g - g.mean(), ref.phi[f] - ref.phi[f].mean()) < 1e-5, f
        assert _rel(p - p.mean(), ref.pi[f] - ref.pi[f].mean()) < 1e-5, f
    lat.evolve(1900)
    ref.vv_steps(oracle.VV4, dt, 1900)
    mm = lat.measure_means()
    E = ref.energies()
    assert abs(mm["a"] - ref.a) < 1e-3 * ref.a and abs(mm["b"] - ref.b) < 1e-3 * abs(ref.b)
    assert abs(mm["mean"][0] - ref.phi[0].mean()) < 1e-3 * abs(ref.phi[0].mean())
    assert abs(mm["mean"][1] - ref.phi[1].mean()) < 1e-3 * ref.phi[1].std()  # <chi> ~ 0: against its rms
    for f in range(2):
        assert abs(mm["var"][f] - ref.phi[f].var()) < 1e-3 * ref.phi[f].var(), f
        assert abs(mm["EK"][f] - E[f]) < 1e-3 * E[f] and abs(mm["EG"][f] - E[2 + f]) < 1e-3 * E[2 + f], f
        assert abs(mm["EV"][f] - E[4 + f]) < 1e-3 * abs(E[4 + f]), f
        for what, arr in ((0, ref.phi[f]), (1, ref.pi[f])):
            err = _spectrum_err(lat.spectrum(f, what), oracle_spectrum(arr, dx, kIR))
            assert err < 1e-3, (f, what, err)
    lat.close()


def test_128_cubed_u1_fp32_leapfrog_matches_oracle():
    """The abelian-Higgs workload (128^3, dx = 0.5, dt = 0.1 dx, lam = e = v = 1,
    symmetric-phase vacuum start, compact leapfrog, FP32) against the oracle from
    the same start.  The tachyonic roll-off is chaotic: an FP32 trajectory leaves
    the FP64 one at a Lyapunov rate of about 0.2 per unit time, so spectra are
    compared at step 500 and volume averages at step 1000, where the pointwise
    difference has grown to O(1e-1) but the averages still agree."""
    from oracle.ic import u1_ic
    N, dx, dt = 128, 0.5, 0.05
    kIR = 2 * math.pi / (N * dx)
    model = cl.make_model(kind=cl.CL_MODEL_U1, lam=1.0, vev2=1.0, gauge_e=1.0, omega_over_fstar=1.0)
    lat = cl.Lattice(model, cl.make_grid(N, kIR, dt, "lf", cl.CL_FP32), cl.make_init(seed=7))
    om = U1Model(N=N, dx=dx, alpha=0.0, fmp2=0.0, lam=1.0, v2=1.0, e=1.0, kappa=1.0)
    phi, pi, th, pa, _ = u1_ic(om, kIR, [0.0, 0.0], [0.0, 0.0], seed=7, omega_over_fstar=1.0)
    ref = U1Lattice(om, phi, pi, th, pa)
    ref.lf_prepare(dt)

    def state():
        return (np.stack([lat.get_field(cl.FIELD(i)) for i in range(2)]),
                np.stack([lat.get_field(cl.MOMENTUM(i)) for i in range(2)]),
                np.stack([lat.get_field(cl.LINK(i)) for i in range(3)]),
                np.stack([lat.get_field(cl.EMOMENTUM(i)) for i in range(3)]))

    lat.evolve(100)
    ref.lf_steps(dt, 100)
    gphi, gpi, gth, gpa = state()
    assert _rel(gphi, ref.phi) < 1e-5 and _rel(gpi, ref.pi) < 1e-5 and _rel(gpa, ref.piA) < 1e-5
    dth = np.abs(np.angle(np.exp(1j * (gth - ref.theta))))
    assert dth.max() < 1e-5 * np.abs(ref.theta).max()
    lat.evolve(400)
    ref.lf_steps(dt, 400)
    assert _spectrum_err(lat.spectrum(0, 0), oracle_spectrum(ref.phi, dx, kIR)) < 1e-3
    assert _spectrum_err(lat.gauge_spectrum(0, 0), oracle_spectrum(ref.electric(), dx, kIR)) < 1e-3
    assert _spectrum_err(lat.gauge_spectrum(0, 1), oracle_spectrum(ref.magnetic(), dx, kIR)) < 1e-3
    lat.evolve(500)
    ref.lf_steps(dt, 500)
    mm = lat.measure_means()
    E = ref.energies()  # E_K^phi, E_G^phi, E_V, E_K^A, E_G^A
    got = [mm["EK"][0], mm["EG"][0], mm["EV"][0], mm["EK"][1], mm["EG"][1]]
    assert np.allclose(got, E, rtol=1e-3, atol=0.0), (got, E)
    for i in range(2):
        assert abs(mm["mean2"][i] - (ref.phi[i] ** 2).mean()) < 1e-3 * (ref.phi[i] ** 2).mean()
    gphi, gpi, gth, gpa = state()
    gauss_of_gpu_state = U1Lattice(om, gphi, gpi, gth, gpa).gauss()
    assert gauss_of_gpu_state < 1e-5 and mm["gauss_violation"] < 1e-5, (gauss_of_gpu_state, mm["gauss_violation"])
    lat.close()


def test_1024_cubed_fp32_reductions_match_fp64_sums_of_the_same_arrays():
    """The throughput workload (1024^3, q* = 4e5, k_IR = 0.1, dt = 0.002, VV4,
    FP32 fluctuations) from its vacuum start: the energies and variances that the
    FP32 pass reduces (thread runs of at most 32 sites, folded per warp into FP64,
    compensated FP64 sums across the grid) against FP64 sums of the same arrays.
    The fluctuation-only quantities (variances, gradient energies) carry the
    whole FP32 reduction error; the bound 1e-6 is 17 FP32 ulps."""
    torch = pytest.importorskip("torch")
    import bench

    N = 1024
    model = cl.make_model(n_fields=2, pexp=2, alpha=0.0, fstar_over_mp=bench.FSTAR_MP,
                          omega_over_fstar=bench.OMEGA_FSTAR, lam=1.0, q=bench.QSTAR)
    lat = cl.Lattice(model, cl.make_grid(N, bench.KIR, bench.DT, "vv4", cl.CL_FP32),
                     cl.make_init(phi0=(1.0, 0.0), seed=0))
    lat.evolve(3)
    mm = lat.measure_means()
    a = mm["a"]
    dx = 2 * math.pi / (bench.KIR * N)
    f = [torch.empty((N, N, N), device="cuda", dtype=torch.float64) for _ in range(2)]
    for i in range(2):
        lat.get_field(cl.FIELD(i), f[i])
    for i in range(2):
        mean = f[i].mean()
        var = ((f[i] - mean) ** 2).mean().item()
        eg = sum(((torch.roll(f[i], -1, d) - f[i]) ** 2).mean().item() for d in range(3)) / (2 * a * a * dx * dx)
        assert abs(mm["var"][i] - var) < 1e-6 * var, (i, (mm["var"][i] - var) / var)
        assert abs(mm["EG"][i] - eg) < 1e-6 * eg, (i, (mm["EG"][i] - eg) / eg)
    ev1 = (0.5 * bench.QSTAR * (f[0] * f[1]) ** 2).mean().item()
    assert abs(mm["EV"][1] - ev1) < 1e-6 * ev1, (mm["EV"][1] - ev1) / ev1
    del f
    p = torch.empty((N, N, N), device="cuda", dtype=torch.float64)
    for i in range(2):
        lat.get_field(cl.MOMENTUM(i), p)
        ek = (p ** 2).mean().item() / (2 * a ** 6)
        dvar = ((p - p.mean()) ** 2).mean().item()
        # E_K of chi is all fluctuation; that of phi is dominated by the FP64 mean
        assert abs(mm["EK"][i] - ek) < 1e-6 * ek, (i, (mm["EK"][i] - ek) / ek, dvar)
    del p
    lat.close()
    torch.cuda.empty_cache()
