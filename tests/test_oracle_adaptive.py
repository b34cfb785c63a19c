"""Pins of the oracle's adaptive time step (the paper's future work, Sec. 6).

Reading: each step's dt is chosen at its start so that a particle of the most
populated cell expects kappa collisions: (n_max - 1) C <v_rel> = kappa with
C = sigma dt / (N_test V_cell) and <v_rel> = 1, capped by the given dt.

* the rule's special cases (no cross section, fewer than two particles per
  cell, the cap) and its value for a largest population counted here with
  numpy from the positions (not with the oracle's keys);
* physics: the relaxation of a mono-energetic gas, measured against the
  simulated time (the sum of the chosen steps), is the same with adaptive
  steps as with a fixed small step; a wrong time bookkeeping or a wrong
  scale of C between the two would separate the curves;
* the densest cell's collision rate per particle and step is kappa.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O


def test_rule_special_cases():
    p = O.make_params(L=(1.0, 1.0, 1.0), n=(2, 1, 1), dt=0.3, sigma_fm2=0.5, n_test=2.0, kappa=0.2)
    V = 0.5
    assert O.adaptive_dt(p, 1) == 0.3 and O.adaptive_dt(p, 0) == 0.3
    assert O.adaptive_dt(p, 2) == 0.3                      # 0.2 * 2 * 0.5 / (0.5 * 1) = 0.4: capped
    big = O.adaptive_dt(p, 1001)
    assert big == pytest.approx(0.2 * 2.0 * V / (0.5 * 1000), rel=1e-15)
    p0 = O.make_params(L=(1.0, 1.0, 1.0), n=(2, 1, 1), dt=0.3, sigma_fm2=0.0, n_test=2.0, kappa=0.2)
    assert O.adaptive_dt(p0, 5000) == 0.3
    pf = O.make_params(L=(1.0, 1.0, 1.0), n=(2, 1, 1), dt=0.3, sigma_fm2=0.5, n_test=2.0)
    assert O.adaptive_dt(pf, 5000) == 0.3                  # kappa = 0: fixed steps
    with pytest.raises(ValueError):
        O.step(O.make_params(L=(1.0, 1.0, 1.0), n=(2, 1, 1), dt=0.3, sigma_fm2=0.5, n_test=2.0, kappa=0.6),
               0, np.zeros((6, 4)))


def test_rule_value_small_cap():
    # 0.2 * 2 * 0.5 / (0.5 * 2) = 0.2 < 0.3: not capped at n_max = 3
    p = O.make_params(L=(1.0, 1.0, 1.0), n=(2, 1, 1), dt=0.45, sigma_fm2=0.5, n_test=2.0, kappa=0.2)
    assert O.adaptive_dt(p, 3) == pytest.approx(0.2, rel=1e-15)


def _mono_gas(N, seed):
    rng = np.random.default_rng(seed)
    st = np.zeros((6, N))
    st[:3] = rng.uniform(0, 1, (3, N))
    d = rng.normal(size=(3, N))
    st[3:] = 1.2 * d / np.linalg.norm(d, axis=0)[None, :]
    return st


def test_step_uses_the_rule_on_the_largest_cell():
    N = 3000
    p = O.make_params(L=(1.0, 1.0, 1.0), n=(2, 2, 2), dt=0.4, sigma_fm2=7.5e-4, n_test=3.0, seed=3, kappa=0.1)
    st, _, _, _ = O.sort(p, _mono_gas(N, 1))
    for k in range(3):
        idx = np.minimum((st[:3] / 0.5).astype(np.int64), 1)
        key = idx[0] + 2 * (idx[1] + 2 * idx[2])
        nmax = np.bincount(key, minlength=8).max()
        st, res = O.step(p, k, st, trace=False)
        assert res.dt == O.adaptive_dt(p, nmax)
        assert res.dt < 0.4


def _relaxation(p, steps, seeds, N=3000):
    curves = []
    for s in seeds:
        st, _, _, _ = O.sort(p, _mono_gas(N, s))
        t, ts, rs = 0.0, [0.0], [0.0]
        for k in range(steps):
            st, res = O.step(p, k, st, trace=False)
            t += res.dt
            E = np.sqrt((st[3:] ** 2).sum(axis=0))
            ts.append(t)
            rs.append(E.var() / E.mean() ** 2)
        curves.append((np.array(ts), np.array(rs)))
    return curves


def test_relaxation_in_simulated_time_matches_fixed_small_steps():
    grid = np.linspace(0.0, 4.0, 17)
    seeds = [11, 12, 13]
    fixed = O.make_params(L=(1.0, 1.0, 1.0), n=(2, 2, 2), dt=0.025, sigma_fm2=7.5e-4, n_test=3.0, seed=5)
    adapt = O.make_params(L=(1.0, 1.0, 1.0), n=(2, 2, 2), dt=0.4, sigma_fm2=7.5e-4, n_test=3.0, seed=6, kappa=0.1)
    cf = _relaxation(fixed, 161, seeds)
    ca = _relaxation(adapt, 40, seeds)
    rf = np.mean([np.interp(grid, t, r) for t, r in cf], axis=0)
    ra = np.mean([np.interp(grid, t, r) for t, r in ca], axis=0)
    assert all(t[-1] >= 4.0 for t, _ in ca)
    # the gas relaxes (towards 1/3 for E ~ Gamma(3)) over the window ...
    assert rf[0] < 1e-12 and rf[-1] > 0.2
    # ... along the same curve in simulated time, step sizes 5x apart
    assert np.max(np.abs(ra - rf)) < 0.035


def test_densest_cell_collision_rate_is_kappa():
    N = 3000
    kappa = 0.1
    p = O.make_params(L=(1.0, 1.0, 1.0), n=(2, 2, 2), dt=0.4, sigma_fm2=7.5e-4, n_test=3.0, seed=8, kappa=kappa)
    st, _, _, _ = O.sort(p, _mono_gas(N, 2))
    ratios = []
    for k in range(40):
        before = np.diff(O.sort(p, st)[3])
        nmax = before.max()
        st, res = O.step(p, k, st)
        cs = res.cell_start
        counts = np.diff(cs)
        # collisions per particle of the cells at the largest population
        for c in np.nonzero(counts == counts.max())[0]:
            acc = np.sum(res.accepted[:, 0] == c)
            ratios.append(2.0 * acc / counts[c] * (nmax - 1) / (counts[c] - 1))
    r = np.array(ratios)
    # <v_rel> = 1 for an isotropic gas: the mean rate is kappa
    assert abs(r.mean() / kappa - 1.0) < 4 * r.std() / kappa / math.sqrt(len(r)) + 0.02
