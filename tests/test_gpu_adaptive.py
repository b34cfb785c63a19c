"""GPU parity of the adaptive time step (kappa > 0) against the oracle: the
step's dt bit-exact (the same rule on the same cell counts), then the step as
for a fixed dt (keys, permutation, positions, accepted and executed pairs,
momenta); the dt sequence and the simulated time over several steps, through
single launches and through the captured graph; a batch mixing adaptive and
fixed members (each identical alone and in the mix)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1208_0961_gb300 import cuba
from paper_1208_0961_gb300 import workloads as W

from test_gpu_parity import _one_step_compare, _pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("skip", [False, True])
def test_adaptive_single_step(fp32, skip):
    cfg = W.riemann_1d(20000, 100, 0.05, 10.0)
    st0 = W.thermal_state(20000, cfg["regions"], seed=1)
    na, ne = _one_step_compare(cfg["L"], cfg["n_cells"], 0.09, cfg["sigma_fm2"], cfg["n_test"], fp32, 0, st0,
                               skip=skip, kappa=0.05)
    assert na > 100


def test_adaptive_3d_small_cells():
    L = (1.6, 1.6, 1.6)
    regs = [((0.0, 0.0, 0.0), L, 0.4)]
    st0 = W.thermal_state(81920, regs, seed=8)
    _one_step_compare(L, (16, 16, 16), 0.09, 5e-4, 2.0, True, 31, st0, step_index=2, small_max=64, kappa=0.2)


def test_adaptive_dt_sequence_and_time():
    cfg = W.riemann_1d(30000, 100, 0.05, 30.0)
    st0 = W.thermal_state(30000, cfg["regions"], seed=3)
    p, op = _pair(cfg["L"], cfg["n_cells"], 0.09, cfg["sigma_fm2"], cfg["n_test"], False, 7, kappa=0.1)
    a = cuba.Sim(p, 30000)
    b = cuba.Sim(p, 30000)
    try:
        a.set_state(st0)
        b.set_state(st0)
        t = 0.0
        dts = []
        for k in range(6):
            g = a.get_state()
            _, _, _, cs = O.sort(op, g)
            want = O.adaptive_dt(op, int(np.diff(cs).max()))
            a.step(1)
            t_gpu, dt_gpu = a.time()
            assert dt_gpu == want, k
            t += want
            assert t_gpu == t, k
            dts.append(dt_gpu)
        assert len(set(dts)) > 1 and max(dts) < 0.09
        b.step(6)                      # one captured graph, six replays
        assert b.time() == a.time()
        assert np.array_equal(b.get_state(), a.get_state())
    finally:
        a.close()
        b.close()


def test_adaptive_and_fixed_members_in_one_batch():
    prec = cuba.CUBA_FP32
    members = []
    for k, (n, cells, sigma, kappa) in enumerate([(20000, 100, 10.0, 0.1), (15000, 60, 30.0, 0.0),
                                                  (9000, 300, 3.0, 0.2)]):
        cfg = W.riemann_1d(n, cells, 0.9 * 10.0 / cells, sigma)
        p = cuba.make_params(L=cfg["L"], n_cells=cfg["n_cells"], dt=cfg["dt"], sigma_fm2=cfg["sigma_fm2"],
                             n_test=cfg["n_test"], precision=prec, seed=60 + k, kappa=kappa)
        st = W.thermal_state(n, cfg["regions"], seed=70 + k).astype(np.float32)
        members.append((p, st))
    alone = []
    for p, st in members:
        sim = cuba.Sim(p, st.shape[1])
        try:
            sim.set_state(st)
            sim.step(4)
            alone.append((sim.get_state(), sim.time()))
        finally:
            sim.close()
    b = cuba.Batch(cuba.make_batch_config(prec, max_sims=4, max_particles=60000, max_cells=600))
    try:
        ids = [b.add_state(p, st) for p, st in members]
        b.step(4)
        for (ref, tm), i in zip(alone, ids):
            assert np.array_equal(b.get_state(i), ref)
            assert b.get_time(i) == tm
    finally:
        b.close()
