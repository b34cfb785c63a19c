"""Pins of the oracle's skip-ahead acceptance mode (A5, alternative sampling).

The skip-ahead mode draws candidate pairs along each row with geometric gaps
at rate P_max and keeps a candidate with probability P22 / P_max.  Pinned
without the oracle's own arithmetic:

* the fixed-point gap sampler against the exact inverse CDF of the geometric
  distribution, evaluated with 40-digit decimal logarithms, draw by draw;
* the gap histogram against the geometric pmf (chi-square);
* per-pair acceptance frequencies of a cell with fixed momenta against
  P22_ij = C |n_i - n_j|^2 / 2 computed here with numpy (chi-square over all
  pairs), FP64 and the FP32 mirror;
* the number of candidates per step against P_max n(n-1)/2 (z-test), and the
  accepted count against the closed form C [n(n-1)/2 - (|sum n|^2 - n)/2];
* the executed set is the lexicographic greedy matching, as in the all-pairs
  mode; the two modes agree in distribution on the same cell.
"""
import decimal
import math

import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O

from test_oracle_collisions import _is_lex_greedy


def _exact_gap(P_fix, U):
    """max{k >= 0 : (1 - P)^k >= U 2^-64} with P = P_fix 2^-64, exactly."""
    ctx = decimal.Context(prec=40)
    D = decimal.Decimal
    lq = ctx.ln(ctx.divide(D(2 ** 64 - P_fix), D(2 ** 64)))
    lu = ctx.ln(ctx.divide(D(int(U)), D(2 ** 64)))
    return int(ctx.divide(lu, lq).to_integral_value(rounding=decimal.ROUND_FLOOR))


@pytest.mark.parametrize("C_scale", [5e-5, 0.01, 0.15])
def test_gap_is_the_exact_geometric_inverse_cdf(C_scale):
    P_fix, Q = O.skip_table(C_scale)
    assert P_fix == math.floor(2.0001 * C_scale * 2 ** 64)
    rng = np.random.default_rng(11)
    U = rng.integers(1, 2 ** 64, size=4000, dtype=np.uint64)
    M = 1 << 31
    diff = 0
    for u in U:
        g = O.skip_gap(Q, int(u), M)
        e = _exact_gap(P_fix, int(u))
        if e >= M:
            assert g >= M
            continue
        assert abs(g - e) <= 1
        diff += g != e
    assert diff <= 2


def test_gap_histogram_is_geometric():
    C_scale = 0.025
    P_fix, Q = O.skip_table(C_scale)
    P = P_fix / 2 ** 64
    rng = np.random.default_rng(3)
    U = rng.integers(1, 2 ** 64, size=60000, dtype=np.uint64)
    g = np.array([O.skip_gap(Q, int(u), 1 << 20) for u in U])
    kmax = 150
    obs = np.bincount(np.minimum(g, kmax), minlength=kmax + 1)
    k = np.arange(kmax + 1)
    pmf = (1 - P) ** k * P
    pmf[kmax] = (1 - P) ** kmax
    exp = pmf * len(U)
    chi2 = np.sum((obs - exp) ** 2 / exp)
    assert stats.chi2.sf(chi2, kmax) > 1e-4


def test_row_end_and_short_rows():
    P_fix, Q = O.skip_table(0.2)
    # M = 1: G is 0 (candidate at the last column) or >= 1 (row ends); the
    # candidate probability is P_max
    rng = np.random.default_rng(5)
    U = rng.integers(1, 2 ** 64, size=20000, dtype=np.uint64)
    hits = sum(O.skip_gap(Q, int(u), 1) == 0 for u in U)
    P = P_fix / 2 ** 64
    z = (hits - len(U) * P) / math.sqrt(len(U) * P * (1 - P))
    assert abs(z) < 4.5


def _fixed_cell(n, seed, C_target, fp32=False):
    rng = np.random.default_rng(seed)
    v = rng.normal(size=(3, n))
    E = rng.gamma(3.0, 0.4, size=n)
    mom = v / np.linalg.norm(v, axis=0) * E
    if fp32:
        mom = mom.astype(np.float32).astype(np.float64)
    # C = sigma dt / (n_test V_cell) with a unit cell
    p = O.make_params(L=(1.0, 1.0, 1.0), n=(1, 1, 1), dt=0.1, sigma_fm2=C_target * 10.0, n_test=1.0,
                      seed=seed, skip=True, fp32=fp32)
    return p, mom


@pytest.mark.parametrize("fp32", [False, True])
def test_pair_frequencies_match_p22(fp32):
    n, steps = 22, 3000
    p, mom = _fixed_cell(n, 21, 0.06, fp32)
    C = O.p22_scale(p)
    u = mom / np.linalg.norm(mom, axis=0)
    P = np.zeros((n, n))
    for i in range(n):
        for j in range(i + 1, n):
            d = u[:, i] - u[:, j]
            P[i, j] = C * 0.5 * (d @ d)
    cnt = np.zeros((n, n))
    for k in range(steps):
        acc = O.cell_accept(p, k, 0, mom)
        # lexicographic, inside the cell, i < j
        if len(acc):
            assert np.all(acc[:, 0] < acc[:, 1]) and acc[:, 1].max() < n
            keys = acc[:, 0].astype(np.int64) * n + acc[:, 1]
            assert np.all(np.diff(keys) > 0)
        np.add.at(cnt, (acc[:, 0], acc[:, 1]), 1)
    iu = np.triu_indices(n, 1)
    e = steps * P[iu]
    o = cnt[iu]
    chi2 = np.sum((o - e) ** 2 / (e * (1 - P[iu])))
    assert stats.chi2.sf(chi2, len(e)) > 1e-4
    assert abs(o.sum() - e.sum()) / math.sqrt(e.sum()) < 4


def test_candidate_count_and_closed_form_acceptance():
    L = (1.0, 1.0, 1.0)
    regs = [((0.0, 0.0, 0.0), L, 0.4)]
    zc, za = [], []
    for seed in range(2):
        p = O.make_params(L=L, n=(2, 2, 1), dt=0.1, sigma_fm2=0.4, n_test=20.0, seed=seed, skip=True)
        p0 = O.make_params(L=L, n=(2, 2, 1), dt=0.1, sigma_fm2=0.0, n_test=20.0, seed=seed)
        st = O.init_thermal(p, 2400, regs)
        st, _, _, _ = O.sort(p, st)
        C = O.p22_scale(p)
        P_fix, _ = O.skip_table(C)
        Pm = P_fix / 2 ** 64
        for k in range(5):
            mid, r0 = O.step(p0, k, st)
            st, res = O.step(p, k, st)
            cs = r0.cell_start
            npairs = sum((cs[c + 1] - cs[c]) * (cs[c + 1] - cs[c] - 1) // 2 for c in range(len(cs) - 1))
            zc.append((res.n_candidates - Pm * npairs) / math.sqrt(Pm * npairs))
            u = mid[3:] / np.sqrt((mid[3:] ** 2).sum(axis=0))[None, :]
            mu = 0.0
            for c in range(len(cs) - 1):
                a, b = cs[c], cs[c + 1]
                m = b - a
                S = u[:, a:b].sum(axis=1)
                mu += C * (m * (m - 1) / 2 - (S @ S - m) / 2)
            za.append((res.n_acc - mu) / math.sqrt(mu))
            for c in range(len(cs) - 1):
                acc = res.accepted[res.accepted[:, 0] == c][:, 1:]
                exe = res.executed[res.executed[:, 0] == c][:, 1:]
                assert _is_lex_greedy(acc, exe)
    assert max(abs(z) for z in zc) < 4.5 and abs(np.sum(zc) / math.sqrt(len(zc))) < 4
    assert max(abs(z) for z in za) < 4.5 and abs(np.sum(za) / math.sqrt(len(za))) < 4


def test_modes_agree_in_distribution():
    n, steps = 30, 1500
    p, mom = _fixed_cell(n, 8, 0.02)
    pa = O.make_params(L=(1.0, 1.0, 1.0), n=(1, 1, 1), dt=0.1, sigma_fm2=0.2, n_test=1.0, seed=8)
    a = np.array([len(O.cell_accept(p, k, 0, mom)) for k in range(steps)])
    b = np.array([len(O.cell_accept(pa, k, 0, mom)) for k in range(steps)])
    # same Poisson-binomial law: means and variances agree
    se = math.sqrt(a.var() / steps + b.var() / steps)
    assert abs(a.mean() - b.mean()) < 4 * se
    assert stats.ks_2samp(a, b).pvalue > 1e-4


def test_zero_cross_section_draws_nothing():
    p, mom = _fixed_cell(10, 1, 0.0)
    assert len(O.cell_accept(p, 0, 0, mom)) == 0
