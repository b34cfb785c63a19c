"""Autotuner of the collision-step launch shape: it times every candidate
threshold on a saved copy of the state and leaves the simulation exactly as
it found it; the results of stepping do not depend on the threshold."""
import numpy as np
import pytest

from paper_1208_0961_gb300 import cuba
from paper_1208_0961_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _sim(L, cells, n, seed):
    regs = [((0.0, 0.0, 0.0), L, 0.4)]
    p = cuba.make_params(L=L, n_cells=cells, dt=0.05, sigma_fm2=5e-4, n_test=2.0, precision=cuba.CUBA_FP32,
                         seed=seed)
    sim = cuba.Sim(p, n)
    sim.init_thermal(n, regs)
    return sim


def test_autotune_leaves_state_and_results_unchanged():
    L, cells, n = (1.6, 1.6, 1.6), (16, 16, 16), 100000
    a = _sim(L, cells, n, 5)
    b = _sim(L, cells, n, 5)
    try:
        a.step(2)
        b.step(2)
        before = a.get_state()
        stats_before = a.stats()
        chosen, ms = cuba.cuba_autotune(a.h, 2)
        assert chosen in cuba.TUNE_CANDIDATES
        assert all(v > 0 for v in ms.values())
        assert cuba.cuba_get_small_max(a.h) == chosen
        assert np.array_equal(a.get_state(), before)
        assert a.stats() == stats_before
        assert cuba.cuba_get_step(a.h) == 2
        a.step(3)
        cuba.cuba_set_small_max(b.h, 0 if chosen else 32)
        b.step(3)
        assert np.array_equal(a.get_state(), b.get_state())
        assert a.stats() == b.stats()
    finally:
        a.close()
        b.close()
