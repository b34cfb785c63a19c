"""Pins of the oracle's collision step (A5-A7).

* Acceptance (Eq. 3): given the momenta, the expected number of accepted pairs
  of a cell is sum_{i<j} P22_ij = C [n(n-1)/2 - (|sum n|^2 - n)/2] (closed form
  of sum (1 - n_i.n_j), independent of the pair loop); counts are tested with
  a z-score over many cells and steps.  For an isotropic gas <v_rel> = 1.
* Conflicts: the executed set is the lexicographic greedy matching of the
  accepted pairs, characterised without replaying the greedy loop: it is a
  matching, and every accepted pair outside it meets an executed pair that
  precedes it.
* Kinematics (Sec. 2): energy and momentum conserved per collision, massless
  outgoing particles (|p_i'| + |p_j'| = E_i + E_j), isotropic direction in the
  CM frame (checked with an independent Lorentz matrix), back-to-back limit.
* Relaxation: a mono-energetic gas becomes a Boltzmann gas, E/T ~ Gamma(3),
  with energy conserved to rounding every step.
"""
import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
import physics as PH


def _thermal_box(N, T, L, ncell, dt, sigma, seed, n_test=1.0):
    regs = [((0.0, 0.0, 0.0), L, T)]
    p = O.make_params(L=L, n=ncell, dt=dt, sigma_fm2=sigma, n_test=n_test, seed=seed)
    st = O.init_thermal(p, N, regs)
    st, _, _, cs = O.sort(p, st)
    return p, st, cs


def test_acceptance_count_matches_conditional_expectation():
    L = (1.0, 1.0, 1.0)
    zs = []
    tot_obs = tot_exp = 0.0
    for seed in range(3):
        p, st, _ = _thermal_box(3000, 0.4, L, (2, 2, 2), 0.1, sigma=0.4, seed=seed, n_test=20.0)
        p0 = O.make_params(L=L, n=(2, 2, 2), dt=0.1, sigma_fm2=0.0, n_test=20.0, seed=seed)
        C = O.p22_scale(p)
        for k in range(6):
            mid, r0 = O.step(p0, k, st)          # streamed and sorted, no collisions
            st, res = O.step(p, k, st)          # same stream, then collisions
            cs = r0.cell_start
            u = mid[3:] / np.sqrt((mid[3:] ** 2).sum(axis=0))[None, :]
            for c in range(len(cs) - 1):
                a, b = cs[c], cs[c + 1]
                n = b - a
                S = u[:, a:b].sum(axis=1)
                mu = C * (n * (n - 1) / 2 - (S @ S - n) / 2)
                obs = np.sum(res.accepted[:, 0] == c)
                # variance of a sum of Bernoulli(P): <= mu; use mu (1 - 2C) as a bound check
                zs.append((obs - mu) / np.sqrt(mu))
                tot_obs += obs
                tot_exp += mu
    zs = np.array(zs)
    assert np.max(np.abs(zs)) < 5
    ztot = (tot_obs - tot_exp) / np.sqrt(tot_exp)
    assert abs(ztot) < 4
    # mean relative velocity of an isotropic gas is 1 (massless: <1 - cos> = 1)
    assert abs(tot_exp / (C * 3 * 6 * 8 * (375 * 374 / 2)) - 1.0) < 0.05


def _is_lex_greedy(acc, exe):
    acc = [tuple(x) for x in acc]
    exe_set = set(tuple(x) for x in exe)
    acc_set = set(acc)
    assert acc == sorted(acc)
    used = {}
    for (i, j) in sorted(exe_set):
        assert (i, j) in acc_set
        assert i not in used and j not in used
        used[i] = (i, j)
        used[j] = (i, j)
    for e in acc:
        if e in exe_set:
            continue
        blockers = [used[q] for q in e if q in used]
        if not any(f < e for f in blockers):
            return False
    return True


def test_executed_pairs_are_the_lexicographic_greedy_matching():
    L = (1.0, 1.0, 1.0)
    p, st, _ = _thermal_box(1200, 0.4, L, (2, 1, 1), 0.2, sigma=3.0, seed=5, n_test=1.0)
    checked = 0
    for k in range(3):
        st, res = O.step(p, k, st)
        for c in range(2):
            acc = res.accepted[res.accepted[:, 0] == c][:, 1:]
            exe = res.executed[res.executed[:, 0] == c][:, 1:]
            assert len(acc) > len(exe) > 0
            assert _is_lex_greedy(acc, exe)
            # maximal: no accepted pair has both ends free
            used = set(exe.ravel().tolist())
            assert all((i in used) or (j in used) for i, j in acc)
            checked += len(acc)
    assert checked > 1000


def _boost_matrix(beta):
    """Lorentz matrix taking lab 4-vectors to the frame moving with velocity beta."""
    b2 = beta @ beta
    g = 1.0 / np.sqrt(1.0 - b2)
    M = np.eye(4)
    M[0, 0] = g
    M[0, 1:] = -g * beta
    M[1:, 0] = -g * beta
    M[1:, 1:] += (g - 1.0) * np.outer(beta, beta) / b2
    return M


@pytest.mark.parametrize("case", ["random", "high_gamma", "back_to_back"])
def test_kinematics_conservation_and_cm_isotropy(case):
    rng = np.random.default_rng(9)
    key = [77, 88]
    if case == "back_to_back":
        pi = np.array([0.0, 0.0, 0.7])
        pj = np.array([0.0, 0.0, -0.7])
    elif case == "high_gamma":
        pi = np.array([3.0, 0.05, 0.0])
        pj = np.array([2.0, -0.02, 0.01])
    else:
        pi = rng.normal(size=3)
        pj = rng.normal(size=3)
    Ei, Ej = np.linalg.norm(pi), np.linalg.norm(pj)
    Et, P = Ei + Ej, pi + pj
    s = Et ** 2 - P @ P
    beta = P / Et
    cos_t, phi = [], []
    for step in range(3000):
        ok, a, b = O.kinematics(key, step, 1, 2, 3, pi, pj)
        assert ok
        Ea, Eb = np.linalg.norm(a), np.linalg.norm(b)
        tol = 1e-12 * Et * (1.0 if case != "high_gamma" else 1e3)
        assert abs((Ea + Eb) - Et) < tol
        assert np.max(np.abs((a + b) - P)) < tol
        if case == "back_to_back":
            assert np.max(np.abs(a + b)) < 1e-15
            assert abs(Ea - 0.7) < 1e-14
            q = a
        else:
            q4 = _boost_matrix(beta) @ np.concatenate([[Ea], a])
            assert abs(q4[0] - np.sqrt(s) / 2) < 1e-9 * Et
            q = q4[1:]
        qn = q / np.linalg.norm(q)
        cos_t.append(qn[2])
        phi.append(np.arctan2(qn[1], qn[0]))
    assert stats.kstest(np.array(cos_t), "uniform", args=(-1, 2)).pvalue > 1e-4
    assert stats.kstest(np.array(phi), "uniform", args=(-np.pi, 2 * np.pi)).pvalue > 1e-4


def test_collinear_pair_is_never_accepted_or_moved():
    key = [1, 1]
    pi = np.array([1.0, 0.0, 0.0])
    pj = np.array([2.5, 0.0, 0.0])
    ok, a, b = O.kinematics(key, 0, 0, 0, 1, pi, pj)
    assert not ok
    p = O.make_params(L=(1, 1, 1), n=(1, 1, 1), dt=0.1, sigma_fm2=50.0, n_test=1.0)
    mom = np.array([[1.0, 2.0, 0.5], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    assert len(O.cell_accept(p, 0, 0, mom)) == 0


def test_monoenergetic_gas_relaxes_to_boltzmann_and_conserves_energy():
    """Small dt / lambda (about 0.1 collisions per particle per step), so that
    the one-collision-per-step conflict rule does not distort the rate; at
    saturation the selected-pair rate is no longer proportional to v_rel and
    the fixed point need not be Boltzmann."""
    rng = np.random.default_rng(12)
    L = (1.0, 1.0, 1.0)
    N = 4000
    T = 0.4
    p = O.make_params(L=L, n=(2, 2, 2), dt=0.1, sigma_fm2=7.5e-4, n_test=3.0, seed=21)
    st = np.zeros((6, N))
    st[:3] = rng.uniform(0, 1, (3, N))
    d = rng.normal(size=(3, N))
    st[3:] = 3.0 * T * d / np.linalg.norm(d, axis=0)[None, :]
    st, _, _, _ = O.sort(p, st)
    E0 = O.totals(st)[0]
    assert stats.kstest(np.sqrt((st[3:] ** 2).sum(axis=0)) / T, PH.gamma3_cdf).pvalue < 1e-10
    executed = 0
    for k in range(200):
        st, res = O.step(p, k, st, trace=False)
        executed += res.n_exe
        E1 = O.totals(st)[0]
        assert abs(E1 - E0) / E0 < 1e-13
        assert st.shape[1] == N
    assert executed > 6 * N
    E = np.sqrt((st[3:] ** 2).sum(axis=0))
    assert stats.kstest(E / T, PH.gamma3_cdf).pvalue > 1e-3
    # isotropy of the relaxed gas
    for a in range(3):
        assert abs(np.mean(st[3 + a])) < 5 * np.std(st[3 + a]) / np.sqrt(N)
