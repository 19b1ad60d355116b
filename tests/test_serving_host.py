"""Host-side pieces of the serving driver (no GPU)."""
import numpy as np

from paper_2004_06352_gb300 import serving


def test_poisson_arrivals_rate_and_order():
    t = serving.poisson_arrivals(20000, 250.0, seed=1)
    assert np.all(np.diff(t) > 0)
    assert abs(20000 / t[-1] - 250.0) / 250.0 < 0.03


def test_mixed_requests_shape():
    r = serving.mixed_requests(5000, seed=2, n_models=8)
    maps = [x for x in r if x[0] == "map"]
    chi2 = [x for x in r if x[0] == "chi2"]
    assert abs(len(maps) / len(r) - 0.6) < 0.03
    assert set(x[2] for x in maps) == set(serving.MAP_SIDES)
    P = np.array([x[2] for x in chi2])
    assert P.min() >= 16 and P.max() <= 4096
    # log-uniform: median near sqrt(16 * 4096) = 256
    assert 200 < np.median(P) < 330
    assert set(x[1] for x in r) == set(range(8))


def test_percentiles():
    p = serving.percentiles(np.arange(1, 101))
    assert abs(p["p50_ms"] - 50.5) < 1e-9 and abs(p["p99_ms"] - 99.01) < 1e-9
    assert serving.percentiles([])["p50_ms"] is None
