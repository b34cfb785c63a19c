"""Ensemble parity: multi-step energy-density profiles of the
GPU (FP32 state, one batch of R independent runs) and of the FP64 oracle (R
other independent runs) agree cell by cell within 3 standard errors: at most
1 % of the (cell, time) points may exceed 3 sigma and the chi^2 of every
profile must have p > 1e-3.  Initial states and random keys differ between
the two ensembles, so the comparison is statistical, not a replay."""
import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
from paper_1208_0961_gb300 import cuba
from paper_1208_0961_gb300 import workloads as W

pytestmark = pytest.mark.gpu

R = 32
N = 10000
CELLS = 50
L = (5.0, 1.0, 1.0)
DT = 0.05
SNAP = (10, 20)


def _cfg():
    return W.riemann_1d(N, CELLS, DT, 10.0, L=L)


def _gpu_profiles(cfg):
    b = cuba.Batch(cuba.make_batch_config(cuba.CUBA_FP32, max_sims=R, max_particles=R * N, max_cells=R * CELLS))
    out = {t: [] for t in SNAP}
    try:
        ids = []
        for r in range(R):
            p = cuba.make_params(L=cfg["L"], n_cells=cfg["n_cells"], dt=DT, sigma_fm2=cfg["sigma_fm2"],
                                 n_test=cfg["n_test"], precision=cuba.CUBA_FP32, seed=100 + r)
            st = W.thermal_state(N, cfg["regions"], seed=100 + r).astype(np.float32)
            ids.append(b.add_state(p, st))
        done = 0
        for t in SNAP:
            b.step(t - done)
            done = t
            for i in ids:
                out[t].append(b.observables(i)[0])
    finally:
        b.close()
    return {t: np.array(v) for t, v in out.items()}


def _oracle_profiles(cfg):
    out = {t: [] for t in SNAP}
    for r in range(R):
        p = O.make_params(L=cfg["L"], n=cfg["n_cells"], dt=DT, sigma_fm2=cfg["sigma_fm2"], n_test=cfg["n_test"],
                          seed=200 + r)
        st = W.thermal_state(N, cfg["regions"], seed=200 + r)
        st, _, _, cs = O.sort(p, st)
        for k in range(max(SNAP)):
            st, res = O.step(p, k, st, trace=False)
            if k + 1 in SNAP:
                _, _, _, cs = O.sort(p, st)
                out[k + 1].append(O.observables(p, st, cs)[0])
    return {t: np.array(v) for t, v in out.items()}


def test_energy_density_profiles_agree_within_three_standard_errors():
    cfg = _cfg()
    g = _gpu_profiles(cfg)
    o = _oracle_profiles(cfg)
    zs = []
    for t in SNAP:
        mg, mo = g[t].mean(axis=0), o[t].mean(axis=0)
        se = np.sqrt(g[t].var(axis=0, ddof=1) / R + o[t].var(axis=0, ddof=1) / R)
        z = (mg - mo) / se
        zs.append(z)
        assert stats.chi2.sf(np.sum(z * z), len(z)) > 1e-3, t
    zs = np.concatenate(zs)
    assert np.mean(np.abs(zs) > 3.0) <= 0.01
    # the profiles evolve: the shock region differs from the initial step
    assert np.ptp(g[SNAP[-1]].mean(axis=0)) > 0.2 * g[SNAP[-1]].mean()
