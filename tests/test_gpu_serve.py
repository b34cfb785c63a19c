"""Serving on the device: requests of different sizes, cross sections and
step counts arrive while others run; each result (per-cell T^00, T^0x,
counts) is bit-identical to the same request run alone."""
import numpy as np
import pytest

from paper_1208_0961_gb300 import cuba
from paper_1208_0961_gb300 import serve as S

pytestmark = pytest.mark.gpu


def test_served_results_equal_results_alone():
    reqs = S.poisson_stream(n_requests=10, rate_hz=200.0, seed=3, n_min=5e3, n_max=6e4, steps_min=3,
                            steps_max=25, sigma_mb_max=50.0)
    be = S.CudaBackend(budget_bytes=64 << 20, max_sims=6)
    try:
        served = S.Server(be, quantum=4).run(reqs, keep_observables=True)
    finally:
        be.close()
    assert served["served"] == 10 and served["rejected"] == 0
    alone = S.run_alone(lambda r: S.CudaBackend(budget_bytes=64 << 20, max_sims=1), reqs, keep_observables=True)
    a = {r.rid: r.observables for r in alone["results"]}
    for r in served["results"]:
        for x, y in zip(r.observables, a[r.rid]):
            assert np.array_equal(x, y), "request %d differs" % r.rid
    assert served["p99_s"] is not None and served["p50_s"] <= served["p99_s"]
