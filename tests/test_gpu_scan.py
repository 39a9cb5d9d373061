"""Batched parameter scans: the tile autotuner leaves the physics unchanged,
batched and one-at-a-time runs give the same observations, and the surrogate
fitted to an ensemble answers held-out couplings within the seed scatter at a
small fraction of the cost of running their lattices."""
import time

import numpy as np
import pytest

import paper_2006_15122_gb300 as cl
from paper_2006_15122_gb300 import scan

pytestmark = pytest.mark.gpu


def rel(x, y):
    return float(np.max(np.abs(x - y)) / max(np.max(np.abs(y)), 1e-300))


def fp64_ensemble(Ns, qs):
    spec = scan.ScanSpec(fstar_over_mp=1.0, omega_over_fstar=0.05, kIR=0.5, dt=0.005, precision=cl.CL_FP64,
                         sizes=tuple(Ns))
    return cl.Ensemble(spec.model(), qs, Ns, [11 + i for i in range(len(Ns))], spec.grid(min(Ns)), spec.init())


def test_autotune_preserves_state_and_results():
    Ns, qs = [32, 64, 32], [50.0, 200.0, 800.0]
    a, b = fp64_ensemble(Ns, qs), fp64_ensemble(Ns, qs)
    a.evolve(3)
    b.evolve(3)
    before = [a.member(i).measure_means() for i in range(3)]
    f0 = a.member(1).get_field(cl.FIELD(1))
    tried = a.autotune()
    assert len(tried) >= 4 and all(ms > 0 for _, ms in tried)
    assert a.tile() in [t for t, _ in tried]
    assert np.array_equal(a.member(1).get_field(cl.FIELD(1)), f0)
    for i in range(3):
        m = a.member(i).measure_means()
        assert m["a"] == before[i]["a"] and m["b"] == before[i]["b"] and m["t"] == before[i]["t"]
    a.evolve(4)
    b.evolve(4)
    for i in range(3):
        for w in (cl.FIELD(0), cl.FIELD(1), cl.MOMENTUM(1)):
            x, y = a.member(i).get_field(w), b.member(i).get_field(w)
            assert rel(x, y) < 1e-12, (i, w, rel(x, y))
    a.close()
    b.close()


@pytest.mark.parametrize("tile", [(8, 16, 16, 4), (16, 8, 32, 6), (8, 8, 8, 5)])
def test_explicit_tiles_give_the_same_fields(tile):
    Ns, qs = [32, 64], [100.0, 400.0]
    a, b = fp64_ensemble(Ns, qs), fp64_ensemble(Ns, qs)
    a.set_tile(tile)
    assert a.tile() == tile
    a.evolve(5)
    b.evolve(5)
    for i in range(2):
        assert rel(a.member(i).get_field(cl.FIELD(1)), b.member(i).get_field(cl.FIELD(1))) < 1e-12
    a.close()
    b.close()


@pytest.mark.parametrize("tile", [(3, 32, 32, 5), (8, 32, 32, 3), (8, 32, 48, 5), (16, 32, 32, 5), (8, 6, 32, 5)])
def test_inadmissible_tiles_are_rejected(tile):
    ens = fp64_ensemble([32, 64], [100.0, 400.0])
    t0 = ens.tile()
    with pytest.raises(cl.LatticeError):
        ens.set_tile(tile)
    assert ens.tile() == t0
    ens.close()


def test_batched_and_plain_observations_agree():
    spec = scan.ScanSpec(sizes=(32, 64), steps_per_slice=8, n_slices=4)
    qs = np.array([300.0, 3000.0, 3e4])
    Ns, seeds = [32, 64, 32], [5, 6, 7]
    obs, times, info = scan.ensemble_observations(spec, qs, Ns, seeds)
    assert np.allclose(times, spec.times(), rtol=1e-12)
    for i in range(3):
        p, t = scan.plain_observations(spec, qs[i], Ns[i], seeds[i])
        assert np.allclose(t, times, rtol=1e-12)
        assert np.all(np.isfinite(p))
        assert np.allclose(obs[i, :, :2], p[:, :2], rtol=1e-4, atol=1e-7), (obs[i, :, :2], p[:, :2])
        assert np.allclose(obs[i, :, 2:], p[:, 2:], atol=1e-4)


def test_surrogate_answers_held_out_couplings():
    """What the trained network gains over the method without it: each
    held-out coupling costs the lattice a full run, the network one batched
    query, at an error within the scatter between seeds."""
    spec = scan.ScanSpec(sizes=(32,), steps_per_slice=16, n_slices=16, kIR=0.2)
    n = 96
    qs = scan.log_uniform_q(n, 1e2, 1e4, seed=1234)
    obs, times, _ = scan.ensemble_observations(spec, qs, [32] * n, list(range(n)))
    X, Y = scan.training_pairs(qs, times, obs)
    net, hist, _ = scan.fit_surrogate(X, Y, epochs=150, batch=256, lr=2e-3)
    assert np.all(np.isfinite(hist)) and hist[-1] < 0.2 * hist[0]
    qh = scan.log_uniform_q(8, 1.5e2, 8e3, seed=99)
    R = 2
    ref, _, _ = scan.ensemble_observations(spec, np.repeat(qh, R), [32] * (8 * R), list(range(1000, 1000 + 8 * R)))
    ref = ref.reshape(8, R, spec.n_slices, -1)
    # one plain run for the cost of the method without the network
    t0 = time.perf_counter()
    scan.plain_observations(spec, qh[0], 32, 1000)
    t_plain = time.perf_counter() - t0
    Xq = np.stack([np.repeat(np.log10(qh), spec.n_slices), np.tile(times, 8)], axis=1)
    net.predict(Xq)
    t0 = time.perf_counter()
    pred = net.predict(Xq).reshape(8, spec.n_slices, -1)
    t_query = (time.perf_counter() - t0) / 8
    s = scan.score(pred, ref)
    assert s["w_abs"]["p95"] < 0.02, s["w_abs"]
    assert s["eps_chi_abs"]["p95"] < 0.02, s["eps_chi_abs"]
    assert s["spectrum_rel"]["median"] < max(0.02, 1.5 * s["floor"]["spectrum_rel"]["median"]), s
    assert t_query * 50 < t_plain, (t_query, t_plain)
    net.close()


def test_queries_outside_the_trained_range_or_in_disagreement_fall_back_to_the_lattice():
    """answer_queries: a coupling outside the trained q range is answered by a
    lattice run of the fallback size and seed (batched with the other fallbacks),
    identical to a one-member ensemble of that lattice; inside the range, where
    the two networks agree, the answer is their mean prediction."""
    spec = scan.ScanSpec(sizes=(32,), steps_per_slice=8, n_slices=8, kIR=0.2, dt=0.005)
    n = 48
    qs = scan.log_uniform_q(n, 1e2, 1e3, seed=7)
    obs, times, _ = scan.ensemble_observations(spec, qs, [32] * n, list(range(n)))
    X, Y = scan.training_pairs(qs, times, obs)
    nets = [scan.fit_surrogate(X, Y, epochs=60, batch=128, seed=k)[0] for k in range(2)]
    qh = np.array([300.0, 2e3])  # the second lies outside [min qs, max qs] (and is VV4-stable at this dt)
    ans, fb, est, t_q, t_fb = scan.answer_queries(nets, qh, times, (qs.min(), qs.max()), spec, tol=0.02,
                                                  seeds=[11, 12], size=32)
    assert ans.shape == (2, spec.n_slices, cl.CL_OBS_SIZE) and est.shape == (2, spec.n_slices)
    assert fb[1] and t_fb > 0
    direct, _, _ = scan.ensemble_observations(spec, qh[1:], [32], [12], autotune=False)
    assert np.array_equal(ans[1], direct[0])
    plain, _ = scan.plain_observations(spec, qh[1], 32, 12)  # the single-lattice path: FP32 round-off apart
    assert np.allclose(ans[1], plain, rtol=1e-3, atol=1e-5)
    if not fb[0]:
        Xq = np.stack([np.repeat(np.log10(qh[:1]), spec.n_slices), times], axis=1).astype(np.float32)
        mean = 0.5 * (nets[0].predict(Xq) + nets[1].predict(Xq))
        assert np.allclose(ans[0], mean, rtol=1e-6, atol=1e-6)
    for net in nets:
        net.close()
