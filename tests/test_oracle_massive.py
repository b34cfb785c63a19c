"""Pins of the oracle's massive particles and screened angular distribution
(the third NEXT row: the paper treats massless gluons with isotropic cross
sections only).

* Thermal sampling of particles of mass m: momentum magnitudes follow the
  Juttner density p^2 exp(-sqrt(p^2 + m^2)/T), its CDF integrated here with
  scipy (KS test).
* Acceptance: per-pair frequencies of a fixed cell against C v_rel with the
  Moller velocity written with 3-velocities, sqrt(|v1 - v2|^2 - |v1 x v2|^2)
  (not the four-vector form the oracle uses), chi-square over all pairs.
* Kinematics: energy and momentum conserved, both outgoing particles on the
  mass shell; in the CM frame (an independent Lorentz matrix) the scattering
  angle is uniform in cos for mu = 0 and follows dsigma/dt ~ 1/(t - mu^2)^2,
  t = -2 |p*|^2 (1 - cos), for mu > 0 (its CDF integrated with scipy), with a
  uniform azimuth about the incoming direction.
* Relaxation: a mono-energetic massive gas becomes a Juttner gas with energy
  conserved every step.
"""
import math

import numpy as np
import pytest
from scipy import integrate, stats

from oracle import oracle as O

from test_oracle_collisions import _boost_matrix


def _juttner_cdf(m, T):
    norm = integrate.quad(lambda q: q * q * math.exp(-math.sqrt(q * q + m * m) / T), 0, 60 * T)[0]

    def cdf(p):
        p = np.atleast_1d(p)
        out = np.empty(len(p))
        # cumulative integration on a grid, interpolated
        grid = np.linspace(0.0, 60 * T, 6001)
        dens = grid ** 2 * np.exp(-np.sqrt(grid ** 2 + m * m) / T)
        cum = np.concatenate([[0.0], np.cumsum(0.5 * (dens[1:] + dens[:-1]) * np.diff(grid))])
        out[:] = np.interp(p, grid, cum / cum[-1])
        return out
    assert norm > 0
    return cdf


@pytest.mark.parametrize("m", [0.2, 0.5, 0.8])
def test_thermal_sampling_is_juttner(m):
    T, N = 0.4, 40000
    p = O.make_params(L=(1.0, 1.0, 1.0), n=(1, 1, 1), dt=0.1, sigma_fm2=0.0, n_test=1.0, seed=3, mass=m)
    st = O.init_thermal(p, N, [((0.0, 0.0, 0.0), (1.0, 1.0, 1.0), T)])
    q = np.linalg.norm(st[3:], axis=0)
    assert stats.kstest(q, _juttner_cdf(m, T)).pvalue > 1e-4
    # and not the massless spectrum (distinguishable from m ~ T on)
    if m >= 0.5:
        assert stats.kstest(q, _juttner_cdf(0.0, T)).pvalue < 1e-6


def _moller(pi, pj, m):
    Ei = math.sqrt(pi @ pi + m * m)
    Ej = math.sqrt(pj @ pj + m * m)
    vi, vj = pi / Ei, pj / Ej
    d = vi - vj
    c = np.cross(vi, vj)
    return math.sqrt(max(0.0, d @ d - c @ c))


def test_massive_pair_frequencies_follow_moller_velocity():
    n, steps, m = 18, 3000, 0.6
    rng = np.random.default_rng(4)
    v = rng.normal(size=(3, n))
    mom = v / np.linalg.norm(v, axis=0) * rng.gamma(3.0, 0.4, size=n)
    p = O.make_params(L=(1.0, 1.0, 1.0), n=(1, 1, 1), dt=0.1, sigma_fm2=0.6, n_test=1.0, seed=4, mass=m)
    C = O.p22_scale(p)
    P = np.zeros((n, n))
    for i in range(n):
        for j in range(i + 1, n):
            P[i, j] = C * _moller(mom[:, i], mom[:, j], m)
    cnt = np.zeros((n, n))
    for k in range(steps):
        acc = O.cell_accept(p, k, 0, mom)
        np.add.at(cnt, (acc[:, 0], acc[:, 1]), 1)
    iu = np.triu_indices(n, 1)
    e, o = steps * P[iu], cnt[iu]
    chi2 = np.sum((o - e) ** 2 / (e * (1 - P[iu])))
    assert stats.chi2.sf(chi2, len(e)) > 1e-4
    # the massless formula would be far off for these momenta
    Pm0 = np.array([C * 0.5 * np.sum((mom[:, i] / np.linalg.norm(mom[:, i]) - mom[:, j] / np.linalg.norm(mom[:, j])) ** 2)
                    for i, j in zip(*iu)])
    chi2_0 = np.sum((o - steps * Pm0) ** 2 / (steps * Pm0 * (1 - Pm0)))
    assert stats.chi2.sf(chi2_0, len(e)) < 1e-6


def _screened_x_cdf(a, mu):
    """CDF of x = 1 - cos(theta) for dsigma/dt ~ 1/(t - mu^2)^2, t = -a x."""
    tot = integrate.quad(lambda x: 1.0 / (a * x + mu * mu) ** 2, 0.0, 2.0)[0]

    def cdf(x):
        x = np.atleast_1d(x)
        return np.array([integrate.quad(lambda y: 1.0 / (a * y + mu * mu) ** 2, 0.0, min(max(v, 0.0), 2.0))[0] / tot
                         for v in x])
    return cdf


@pytest.mark.parametrize("m,mu", [(0.0, 0.0), (0.5, 0.0), (0.0, 0.4), (0.5, 0.3)])
def test_kinematics_conservation_shell_and_cm_angles(m, mu):
    rng = np.random.default_rng(7)
    key = [5, 6]
    pi = rng.normal(size=3) * 0.8
    pj = rng.normal(size=3) * 0.8
    Ei, Ej = math.sqrt(pi @ pi + m * m), math.sqrt(pj @ pj + m * m)
    Et, P = Ei + Ej, pi + pj
    s = Et ** 2 - P @ P
    beta = P / Et
    L = _boost_matrix(beta)
    qin = (L @ np.concatenate([[Ei], pi]))[1:]
    ein = qin / np.linalg.norm(qin)
    pstar2 = s / 4 - m * m
    xs, phis = [], []
    ref = np.cross(ein, [1.0, 0.0, 0.0] if abs(ein[0]) < 0.9 else [0.0, 1.0, 0.0])
    ref /= np.linalg.norm(ref)
    ref2 = np.cross(ein, ref)
    for step in range(2500):
        ok, a, b = O.kinematics_ex(key, m, mu, step, 3, 1, 2, pi, pj)
        assert ok
        Ea, Eb = math.sqrt(a @ a + m * m), math.sqrt(b @ b + m * m)
        assert abs(Ea + Eb - Et) < 1e-12 * Et
        assert np.max(np.abs(a + b - P)) < 1e-12 * Et
        q4 = L @ np.concatenate([[Ea], a])
        assert abs(q4[0] - math.sqrt(s) / 2) < 1e-9 * Et          # on shell: E* = sqrt(s)/2 for equal masses
        q = q4[1:] / np.linalg.norm(q4[1:])
        xs.append(1.0 - q @ ein)
        phis.append(math.atan2(q @ ref2, q @ ref))
    xs = np.array(xs)
    if mu == 0.0:
        assert stats.kstest(1.0 - xs, "uniform", args=(-1, 2)).pvalue > 1e-4
    else:
        assert stats.kstest(xs, _screened_x_cdf(2.0 * pstar2, mu)).pvalue > 1e-4
        # forward peaked: far more small angles than isotropic
        assert np.mean(xs < 0.5) > 0.5
    assert stats.kstest(np.array(phis), "uniform", args=(-math.pi, 2 * math.pi)).pvalue > 1e-4


def test_massive_gas_relaxes_to_juttner():
    rng = np.random.default_rng(12)
    N, T0, m = 4000, 0.4, 0.5
    p = O.make_params(L=(1.0, 1.0, 1.0), n=(2, 2, 2), dt=0.1, sigma_fm2=7.5e-4, n_test=3.0, seed=21, mass=m)
    st = np.zeros((6, N))
    st[:3] = rng.uniform(0, 1, (3, N))
    d = rng.normal(size=(3, N))
    # mono-energetic: every particle at the mean Juttner energy of T0
    grid = np.linspace(0, 30 * T0, 30001)
    w = grid ** 2 * np.exp(-np.sqrt(grid ** 2 + m * m) / T0)
    Emean = np.sum(w * np.sqrt(grid ** 2 + m * m)) / np.sum(w)
    pmag = math.sqrt(Emean ** 2 - m * m)
    st[3:] = pmag * d / np.linalg.norm(d, axis=0)[None, :]
    st, _, _, _ = O.sort(p, st)
    E0 = O.totals(st, m)[0]
    for k in range(200):
        st, res = O.step(p, k, st, trace=False)
        assert abs(O.totals(st, m)[0] - E0) / E0 < 1e-13
    q = np.linalg.norm(st[3:], axis=0)
    assert stats.kstest(q, _juttner_cdf(m, T0)).pvalue > 1e-3
