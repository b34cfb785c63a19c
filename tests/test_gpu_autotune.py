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


@pytest.mark.parametrize("small_blocks,tile_blocks", [(1, 2), (1, 4), (2, 2), (2, 8)])
def test_launch_shapes_give_identical_steps(small_blocks, tile_blocks):
    """Every blocks-per-iteration shape of the two pair kernels steps a
    mixed-occupancy state (small cells and 32-row items) to the same bits."""
    L, cells, n = (1.6, 1.6, 0.8), (16, 16, 4), 60000   # about 60 particles per cell
    a = _sim(L, cells, n, 9)
    b = _sim(L, cells, n, 9)
    try:
        cuba.cuba_set_launch_shape(a.h, 48, 2, 4)
        cuba.cuba_set_launch_shape(b.h, 48, small_blocks, tile_blocks)
        assert cuba.cuba_get_launch_shape(b.h) == {"small_max": 48, "small_blocks": small_blocks,
                                                   "tile_blocks": tile_blocks}
        a.step(3)
        b.step(3)
        assert np.array_equal(a.get_state(), b.get_state())
        assert a.stats() == b.stats()
    finally:
        a.close()
        b.close()


def test_autotune_shape_leaves_state_unchanged():
    L, cells, n = (1.6, 1.6, 1.6), (16, 16, 16), 100000
    a = _sim(L, cells, n, 6)
    try:
        a.step(1)
        before = a.get_state()
        shape, ms = cuba.cuba_autotune_shape(a.h, 2)
        assert shape["small_max"] in cuba.TUNE_CANDIDATES
        assert shape["small_blocks"] in (1, 2) and shape["tile_blocks"] in (2, 4, 8)
        assert len(ms) == 13 and all(v > 0 for v in ms.values())
        assert cuba.cuba_get_launch_shape(a.h) == shape
        assert np.array_equal(a.get_state(), before)
        assert cuba.cuba_get_step(a.h) == 1
    finally:
        a.close()
    c = _sim(L, cells, 10, 1)
    try:
        with pytest.raises(cuba.CubaError):
            cuba.cuba_set_launch_shape(c.h, 32, 3, 4)
        with pytest.raises(cuba.CubaError):
            cuba.cuba_set_launch_shape(c.h, 32, 2, 6)
    finally:
        c.close()
