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
