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
    be = S.CudaBackend(budget_bytes=256 << 20, max_sims=6)
    try:
        served = S.Server(be, quantum=4).run(reqs, keep_observables=True)
    finally:
        be.close()
    assert served["served"] == 10 and served["rejected"] == 0
    alone = S.run_alone(lambda r: S.CudaBackend.for_request(r), reqs, keep_observables=True)
    a = {r.rid: r.observables for r in alone["results"]}
    for r in served["results"]:
        for x, y in zip(r.observables, a[r.rid]):
            assert np.array_equal(x, y), "request %d differs" % r.rid
    assert served["p99_s"] is not None and served["p50_s"] <= served["p99_s"]


def test_served_requests_match_the_oracle():
    """FP64 requests served in one batch: each request's observables equal
    the oracle's run of the same request (its Philox-sampled initial state,
    its steps): counts exactly, T^00 and T^0x to 1e-9 of the largest T^00."""
    from oracle import oracle as O
    reqs = S.poisson_stream(n_requests=6, rate_hz=500.0, seed=5, n_min=3e3, n_max=2e4, steps_min=2,
                            steps_max=6, sigma_mb_max=60.0)
    be = S.CudaBackend(budget_bytes=256 << 20, precision=cuba.CUBA_FP64, max_sims=6)
    try:
        served = S.Server(be, quantum=2).run(reqs, keep_observables=True)
    finally:
        be.close()
    assert served["served"] == 6
    by_id = {r.rid: r for r in reqs}
    for res in served["results"]:
        r = by_id[res.rid]
        op = O.make_params(L=r.L, n=r.n_cells, dt=r.dt, sigma_fm2=r.sigma_fm2, n_test=r.n_test, seed=r.seed)
        st = O.init_thermal(op, r.n, r.regions)
        st, _, _, _ = O.sort(op, st)
        for k in range(r.steps):
            st, _ = O.step(op, k, st, trace=False)
        _, _, _, cs = O.sort(op, st)
        oT00, oT0x, ocnt = O.observables(op, st, cs)
        T00, T0x, cnt = res.observables
        assert np.array_equal(cnt, ocnt), "request %d: counts differ" % r.rid
        scale = max(np.abs(oT00).max(), 1e-300)
        assert np.max(np.abs(T00 - oT00)) <= 1e-9 * scale, "request %d: T00" % r.rid
        assert np.max(np.abs(T0x - oT0x)) <= 1e-9 * scale, "request %d: T0x" % r.rid
