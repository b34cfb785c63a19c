"""GPU parity of massive particles and of the screened angular distribution
against the oracle: one step from the same state (keys, permutation,
positions bit-exact, accepted and executed pairs identical, momenta within
1e-12 / 1e-5 of the pair energy), both acceptance modes and both cell paths;
Juttner sampling (positions exact, momenta 1e-13); observables and totals with
E = sqrt(|p|^2 + m^2); energy conserved over many steps."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1208_0961_gb300 import cuba
from paper_1208_0961_gb300 import workloads as W

from test_gpu_parity import _one_step_compare, _pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("mass,mu,skip", [(0.5, 0.0, False), (0.0, 0.3, False), (0.4, 0.2, True)])
def test_massive_screened_single_step(fp32, mass, mu, skip):
    cfg = W.riemann_1d(20000, 100, 0.05, 10.0)
    st0 = W.thermal_state(20000, cfg["regions"], seed=1)
    na, ne = _one_step_compare(cfg["L"], cfg["n_cells"], cfg["dt"], cfg["sigma_fm2"], cfg["n_test"], fp32, 0, st0,
                               skip=skip, mass=mass, mu=mu)
    assert na > 500 and ne > 200


@pytest.mark.parametrize("small_max", [0, 64])
def test_massive_small_cells(small_max):
    L = (1.6, 1.6, 1.6)
    regs = [((0.0, 0.0, 0.0), L, 0.4)]
    st0 = W.thermal_state(81920, regs, seed=8)
    _one_step_compare(L, (16, 16, 16), 0.05, 5e-4, 2.0, True, 31, st0, step_index=2, small_max=small_max,
                      mass=0.3, mu=0.5)


def test_juttner_sampling_observables_and_totals():
    m = 0.6
    cfg = W.riemann_1d(30000, 100, 0.05, 10.0)
    p, op = _pair(cfg["L"], cfg["n_cells"], cfg["dt"], cfg["sigma_fm2"], cfg["n_test"], False, 99, mass=m)
    sim = cuba.Sim(p, 30000)
    try:
        sim.init_thermal(30000, cfg["regions"])
        g = sim.get_state()
        T00, T0x, cnt = sim.observables()
        tot, n = sim.totals()
    finally:
        sim.close()
    o = O.init_thermal(op, 30000, cfg["regions"])
    o, _, _, cs = O.sort(op, o)
    assert np.array_equal(g[:3], o[:3])
    E = np.sqrt((o[3:] ** 2).sum(axis=0) + m * m)
    assert np.max(np.abs(g[3:] - o[3:]).max(axis=0) / E) < 1e-13
    oT00, oT0x, ocnt = O.observables(op, g, cs)
    assert np.array_equal(cnt, ocnt)
    assert np.max(np.abs(T00 - oT00)) <= 1e-12 * np.max(oT00)
    ot = O.totals(g, m)
    assert abs(tot[0] - ot[0]) <= 1e-12 * ot[0] and n == 30000


def test_massive_screened_energy_conservation():
    cfg = W.riemann_1d(20000, 100, 0.05, 10.0)
    for fp32 in (False, True):
        p, _ = _pair(cfg["L"], cfg["n_cells"], cfg["dt"], cfg["sigma_fm2"], cfg["n_test"], fp32, 3, mass=0.5, mu=0.4)
        sim = cuba.Sim(p, 20000)
        try:
            sim.init_riemann(20000, 0.4, 0.32)
            E0 = sim.totals()[0][0]
            Eprev = E0
            for k in range(50):
                sim.step(1)
                E1 = sim.totals()[0][0]
                assert abs(E1 - Eprev) / E0 < (1e-6 if fp32 else 1e-13), "step %d" % k
                assert abs(E1 - E0) / E0 < (1e-6 * (k + 1) if fp32 else 1e-12)
                Eprev = E1
            assert sim.stats()["executed"] > 0
        finally:
            sim.close()
