"""Host-side logic of the parameter scan (no GPU): the two-network error
estimate and the scoring against fresh runs."""
import numpy as np

from paper_2006_15122_gb300 import scan


def test_disagreement_is_the_larger_absolute_gap_of_eps_and_w():
    pa = np.zeros((2, 3, 34), dtype=np.float32)
    pb = np.zeros_like(pa)
    pb[0, 1, 0] = 0.03   # eps_chi
    pb[1, 2, 1] = -0.01  # w
    pb[1, 0, 5] = 2.0    # a spectrum bin: not part of the estimate
    est = scan.disagreement(pa, pb)
    assert est.shape == (2, 3)
    assert np.isclose(est[0, 1], 0.03) and np.isclose(est[1, 2], 0.01) and est[1, 0] == 0.0


def test_score_reports_errors_floor_and_reference_standard_error():
    rng = np.random.default_rng(3)
    ref = rng.normal(0.0, 0.01, size=(4, 4, 5, 34))
    pred = ref.mean(axis=1)
    s = scan.score(pred, ref)
    assert s["eps_chi_abs"]["max"] < 1e-12 and s["w_abs"]["within_2pct"] == 1.0
    se = s["reference_stderr"]["w_abs"]["median"]
    assert 0.001 < se < 0.01  # std 0.01 over sqrt(4) seeds, about 0.005 * sqrt(3/4)
    assert s["floor"]["w_abs"]["median"] > se


class _Net:
    """A stand-in network: a fixed function of (log10 q, t), plus an offset."""

    def __init__(self, offset):
        self.offset = offset

    def predict(self, X):
        X = np.asarray(X, dtype=np.float64)
        out = np.zeros((len(X), 34), dtype=np.float32)
        out[:, 0] = 0.1 * X[:, 0] + self.offset
        out[:, 1] = 0.01 * X[:, 1]
        return out


def test_answer_queries_routes_fallbacks_to_one_batched_ensemble(monkeypatch):
    """Queries outside the trained range, or where the two networks disagree on
    too many slices, are answered by one batched ensemble of fallback runs (the
    fallback size, their own seeds, in query order); the others by the networks'
    mean."""
    calls = []

    def fake_ensemble(spec, qs, Ns, seeds, autotune=True, stream=None):
        calls.append((list(qs), list(Ns), list(seeds), autotune))
        obs = np.zeros((len(qs), spec.n_slices, 34), dtype=np.float32)
        obs[:, :, 0] = np.asarray(seeds, dtype=np.float32)[:, None]  # marks which run answered
        return obs, spec.times(), {}

    monkeypatch.setattr(scan, "ensemble_observations", fake_ensemble)
    spec = scan.ScanSpec(sizes=(32, 64, 96), steps_per_slice=2, n_slices=5)
    times = spec.times()
    qs = np.array([200.0, 5.0, 300.0, 1e6])
    nets = [_Net(0.0), _Net(0.0)]
    ans, fb, est, tq, tf = scan.answer_queries(nets, qs, times, (100.0, 1e4), spec, seeds=[11, 12, 13, 14])
    assert list(fb) == [False, True, False, True]  # out of range: q = 5 and q = 1e6
    assert calls == [([5.0, 1e6], [64, 64], [12, 14], False)]  # one ensemble, middle size, no tuning
    assert np.all(ans[1, :, 0] == 12) and np.all(ans[3, :, 0] == 14)
    assert np.allclose(ans[0, :, 0], 0.1 * np.log10(200.0)) and np.allclose(ans[2, :, 1], 0.01 * times)
    # inside the range but the networks disagree by 0.05 on eps_chi at every slice: fallback
    calls.clear()
    ans, fb, est, tq, tf = scan.answer_queries([_Net(0.0), _Net(0.05)], qs[:1], times, (100.0, 1e4), spec,
                                               seeds=[21])
    assert list(fb) == [True] and np.allclose(est, 0.05) and calls[0][2] == [21]
    # nothing falls back: no ensemble at all
    calls.clear()
    scan.answer_queries(nets, qs[[0, 2]], times, (100.0, 1e4), spec)
    assert calls == []
