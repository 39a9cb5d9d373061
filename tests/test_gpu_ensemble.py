"""Batched ensembles: every member of a mixed-size ensemble, advanced by the
multi-lattice persistent pass, matches the FP64 oracle run of the same model,
seed and size; the observations agree with the members' own measurements."""
import math

import numpy as np
import pytest

import oracle
import paper_2006_15122_gb300 as cl
from oracle import ScalarLattice, ScalarModel
from oracle.ic import scalar_ic

pytestmark = pytest.mark.gpu


def rel(x, y):
    return float(np.max(np.abs(x - y)) / max(np.max(np.abs(y)), 1e-300))


def make(Ns, qs, prec, kIR=0.5, dt=0.005, integ="vv4", omega=0.05, fmp=1.0):
    model = cl.make_model(n_fields=2, pexp=2, lam=1.0, q=0.0, omega_over_fstar=omega, fstar_over_mp=fmp)
    seeds = [101 + i for i in range(len(Ns))]
    ens = cl.Ensemble(model, qs, Ns, seeds, cl.make_grid(32, kIR, dt, integ, prec), cl.make_init(phi0=(1.0, 0.0)))
    return ens, seeds


def test_ensemble_members_match_oracle_fp64():
    Ns, qs, kIR, dt, omega, fmp = [32, 64, 32], [50.0, 200.0, 800.0], 0.5, 0.005, 0.05, 1.0
    ens, seeds = make(Ns, qs, cl.CL_FP64, kIR, dt, "vv4", omega, fmp)
    ens.evolve(2)
    ens.evolve(2)
    for i, (N, q, seed) in enumerate(zip(Ns, qs, seeds)):
        om = ScalarModel(N=N, Ns=2, pexp=2, dx=2 * math.pi / (kIR * N), alpha=0.0, fmp2=fmp * fmp, lam=1.0, q=q)
        phi, pi, _ = scalar_ic(om, kIR, [1.0, 0.0], [0.0, 0.0], seed=seed, omega_over_fstar=omega)
        ref = ScalarLattice(om, phi, pi)
        ref.b = math.sqrt(ref.hubble_rhs())
        ref.vv_steps(oracle.VV4, dt, 4)
        m = ens.member(i)
        gphi = np.stack([m.get_field(cl.FIELD(f)) for f in range(2)])
        gpi = np.stack([m.get_field(cl.MOMENTUM(f)) for f in range(2)])
        assert rel(gphi, ref.phi) < 1e-11, (i, rel(gphi, ref.phi))
        assert rel(gpi, ref.pi) < 1e-11, (i, rel(gpi, ref.pi))
        mm = m.measure_means()
        assert abs(mm["a"] - ref.a) < 1e-13 and abs(mm["b"] - ref.b) < 1e-11 * ref.b
    ens.close()


def test_ensemble_matches_single_lattices_fp32():
    Ns, qs = [32, 64, 96, 32], [100.0, 400.0, 1600.0, 25.0]
    ens, seeds = make(Ns, qs, cl.CL_FP32)
    ens.evolve(10)
    model = cl.make_model(n_fields=2, pexp=2, lam=1.0, omega_over_fstar=0.05, fstar_over_mp=1.0)
    for i in (1, 2):
        model.q = qs[i]
        lat = cl.Lattice(model, cl.make_grid(Ns[i], 0.5, 0.005, "vv4", cl.CL_FP32), cl.make_init(phi0=(1.0, 0.0), seed=seeds[i]))
        lat.evolve(10)
        a = lat.get_field(cl.FIELD(1))
        b = ens.member(i).get_field(cl.FIELD(1))
        assert rel(b - b.mean(), a - a.mean()) < 1e-5
        lat.close()
    ens.close()


@pytest.mark.parametrize("kmax_arg", [0.0, 5.0])
def test_ensemble_observations_agree_with_members(kmax_arg):
    """ensemble_observe against each member's own measurements; the spectrum
    momenta span [kIR, kmax], kmax = N_min kIR / 2 by default or as given."""
    Ns, qs, kIR = [32, 64, 96], [300.0, 3000.0, 30.0], 0.5
    ens, _ = make(Ns, qs, cl.CL_FP32, kIR=kIR, dt=0.004)
    ens.evolve(25)
    obs, t = ens.observe(kmax_arg)
    assert obs.shape == (3, cl.CL_OBS_SIZE) and np.all(np.isfinite(obs))
    assert abs(t - 25 * 0.004) < 1e-9
    kmax = kmax_arg if kmax_arg > 0 else 0.5 * min(Ns) * kIR
    for i in range(3):
        m = ens.member(i)
        mm = m.measure_means()
        eps = (mm["EK"][1] + mm["EG"][1]) / mm["rho"]
        assert abs(obs[i, 0] - eps) < 1e-6 * max(eps, 1e-30) + 1e-12
        assert abs(obs[i, 1] - mm["w"]) < 1e-6
        k, D, c = m.spectrum(1, 0)
        sel = (c > 0) & (D > 0) & (k > 0)
        lk, lD = np.log(k[sel]), np.log10(D[sel])
        kj = np.log(kIR) + (np.arange(32) + 0.5) / 32 * (np.log(kmax) - np.log(kIR))
        ref = np.interp(kj, lk, lD)
        assert np.allclose(obs[i, 2:], ref, atol=1e-4), (obs[i, 2:], ref)
    ens.close()


def _oracle_run(N, q, seed, kIR, dt, steps, omega=0.05, fmp=1.0):
    om = ScalarModel(N=N, Ns=2, pexp=2, dx=2 * math.pi / (kIR * N), alpha=0.0, fmp2=fmp * fmp, lam=1.0, q=q)
    phi, pi, _ = scalar_ic(om, kIR, [1.0, 0.0], [0.0, 0.0], seed=seed, omega_over_fstar=omega)
    ref = ScalarLattice(om, phi, pi)
    ref.b = math.sqrt(ref.hubble_rhs())
    ref.vv_steps(oracle.VV4, dt, steps)
    return ref


def _check_obs(got, want):
    """FP32 outputs: eps_chi and w to their rounding, log10 Delta to 1e-5."""
    assert abs(got[0] - want[0]) < 1e-6 * abs(want[0]) + 1e-12, (got[0], want[0])
    assert abs(got[1] - want[1]) < 1e-6, (got[1], want[1])
    assert np.allclose(got[2:], want[2:], rtol=0, atol=1e-5), (got[2:], want[2:])


@pytest.mark.parametrize("kmax", [0.0, 3.1])
def test_lattice_observe_matches_oracle_composition(kmax):
    """lattice_observe of an FP64 lattice against the oracle's composition of
    the same observables (oracle/observe.py) from the oracle's own run."""
    from oracle.observe import observables
    N, q, seed, kIR, dt, steps = 48, 2500.0, 17, 0.5, 0.004, 30
    model = cl.make_model(n_fields=2, pexp=2, lam=1.0, q=q, omega_over_fstar=0.05, fstar_over_mp=1.0)
    lat = cl.Lattice(model, cl.make_grid(N, kIR, dt, "vv4", cl.CL_FP64), cl.make_init(phi0=(1.0, 0.0), seed=seed))
    lat.evolve(steps)
    obs, t = lat.observe(kmax)
    ref = _oracle_run(N, q, seed, kIR, dt, steps)
    _check_obs(obs, observables(ref, kIR, kmax if kmax > 0 else None))
    assert abs(t - steps * dt) < 1e-12
    lat.close()


def test_ensemble_observations_match_oracle_composition():
    """ensemble_observe of a mixed-size FP64 ensemble: every member's 34 numbers
    against the oracle composition of its own oracle run, with the spectrum
    momenta up to the smallest member's axis Nyquist momentum."""
    from oracle.observe import observables
    Ns, qs, kIR, dt, steps = [32, 64, 32], [80.0, 900.0, 4000.0], 0.5, 0.004, 12
    ens, seeds = make(Ns, qs, cl.CL_FP64, kIR=kIR, dt=dt)
    ens.evolve(steps)
    obs, _ = ens.observe()
    kmax = 0.5 * min(Ns) * kIR
    for i, (N, q, seed) in enumerate(zip(Ns, qs, seeds)):
        _check_obs(obs[i], observables(_oracle_run(N, q, seed, kIR, dt, steps), kIR, kmax))
    ens.close()
