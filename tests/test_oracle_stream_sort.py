"""Pins of the oracle's streaming, reflection, cell keys and sort (A1-A4, A8).

* Single-particle trajectories against the exact straight-line motion between
  specular walls (Eq. 2 plus the reflection rule of Sec. 2), unfolded onto the
  even 2L-periodic extension of the box.
* Reflections conserve every |p_a| bit for bit; number of particles is exact.
* Keys: each particle lies inside the cell its key names (an invariant, not
  the formula retyped); the sort is the stable argsort of numpy (a library
  routine) and cell_start is the bincount prefix sum.
* sigma = 0 energy-density and momentum-density profiles of the 1D Riemann
  initial state against the closed-form collisionless solution (chi^2).
"""
import numpy as np
import pytest
from scipy import stats

from oracle import oracle as O
import physics as PH


def _params(**kw):
    d = dict(L=(1.0, 1.0, 1.0), n=(10, 10, 10), dt=0.04, sigma_fm2=0.0, n_test=1.0, seed=3)
    d.update(kw)
    return O.make_params(**d)


def _rand_state(rng, n, L):
    st = np.zeros((6, n))
    for a in range(3):
        st[a] = rng.uniform(0, L[a], n)
    st[3:] = rng.normal(size=(3, n)) * rng.exponential(1.0, n)[None, :]
    return st


def test_trajectories_match_unfolded_straight_lines():
    rng = np.random.default_rng(1)
    L = (1.0, 0.8, 1.3)
    p = _params(L=L, n=(10, 8, 13), dt=0.07)
    n = 500
    st0, _, _, _ = O.sort(p, _rand_state(rng, n, L))
    ident = np.arange(n)
    st = st0.copy()
    v = st0[3:] / np.sqrt((st0[3:] ** 2).sum(axis=0))[None, :]
    for k in range(1, 301):
        st, res = O.step(p, k, st)
        ident = ident[res.perm]
        if k % 50 == 0:
            for a in range(3):
                expect = PH.fold(st0[a, ident] + v[a, ident] * (k * p.dt), L[a])
                assert np.max(np.abs(st[a] - expect)) < 1e-12 * k
            # momentum components only flip sign
            assert np.array_equal(np.abs(st[3:]), np.abs(st0[3:, ident]))


def test_reflection_count_and_energy_bitwise():
    rng = np.random.default_rng(2)
    L = (0.5, 0.5, 0.5)
    p = _params(L=L, n=(5, 5, 5), dt=0.09)
    st, _, _, _ = O.sort(p, _rand_state(rng, 2000, L))
    E0 = np.sort(np.sqrt((st[3:] ** 2).sum(axis=0)))
    total_ref = 0
    for k in range(40):
        st, res = O.step(p, k, st)
        total_ref += res.n_reflections
    assert total_ref > 1000
    E1 = np.sort(np.sqrt((st[3:] ** 2).sum(axis=0)))
    assert np.array_equal(E0, E1)


def test_keys_name_the_containing_cell_and_sort_is_stable():
    rng = np.random.default_rng(3)
    L = (2.0, 1.5, 1.0)
    p = _params(L=L, n=(20, 15, 10), dt=0.05)
    st = _rand_state(rng, 20000, L)
    # a few particles exactly on faces and walls
    st[0, :5] = [0.0, 2.0, 0.1, 1.0, 1.9]
    keys = O.keys(p, st)
    ix = keys % 20
    iy = (keys // 20) % 15
    iz = keys // 300
    dx = np.array([0.1, 0.1, 0.1])
    for a, ia in enumerate((ix, iy, iz)):
        lo = ia * dx[a]
        hi = (ia + 1) * dx[a]
        assert np.all(st[a] >= lo - 1e-12) and np.all(st[a] <= hi + 1e-12)
    assert keys.max() < 20 * 15 * 10
    sst, k2, perm, cs = O.sort(p, st)
    assert np.array_equal(perm, np.argsort(keys, kind="stable"))
    assert np.array_equal(cs, np.concatenate([[0], np.cumsum(np.bincount(keys, minlength=3000))]))
    assert np.array_equal(sst, st[:, perm])


def test_fp32_mirror_keys_agree_with_fp64_away_from_faces():
    rng = np.random.default_rng(4)
    L = (10.0, 1.0, 1.0)
    p64 = _params(L=L, n=(100, 1, 1), dt=0.05)
    p32 = _params(L=L, n=(100, 1, 1), dt=0.05, fp32=True)
    st = _rand_state(rng, 50000, L).astype(np.float32).astype(np.float64)
    k64 = O.keys(p64, st)
    k32 = O.keys(p32, st)
    frac = np.abs(st[0] / 0.1 - np.round(st[0] / 0.1))
    far = frac > 1e-5
    assert np.array_equal(k64[far], k32[far])
    assert np.mean(k64 != k32) < 1e-3


@pytest.mark.parametrize("t_end", [1.5, 7.0])
def test_sigma0_riemann_profile_matches_free_streaming(t_end):
    L = (10.0, 1.0, 1.0)
    TL, TR = 0.4, 0.32
    regs = O.riemann_regions(L, TL, TR)
    N = 200000
    ntest = O.n_test_for(N, regs)
    dt = 0.05
    p = O.make_params(L=L, n=(100, 1, 1), dt=dt, sigma_fm2=0.0, n_test=ntest, seed=11)
    st = O.init_thermal(p, N, regs)
    counts = O.region_counts(N, regs)
    E = np.sqrt((st[3:] ** 2).sum(axis=0))
    vol_half = 5.0
    epsL = E[:counts[0]].sum() / (ntest * vol_half)
    epsR = E[counts[0]:].sum() / (ntest * vol_half)
    st, _, _, cs = O.sort(p, st)
    nsteps = int(round(t_end / dt))
    for k in range(nsteps):
        st, res = O.step(p, k, st)
        cs = res.cell_start
    T00, T0x, cnt = O.observables(p, st, cs)
    assert cnt.sum() == N
    edges = np.linspace(0, 10.0, 101)
    A00, A0x = PH.free_stream_profile(edges, nsteps * dt, 10.0,
                                      lambda x: np.where(x < 5.0, epsL, epsR), nmu=2001, nsub=8)
    # per-cell standard errors from the particles themselves
    E = np.sqrt((st[3:] ** 2).sum(axis=0))
    norm = ntest * 0.1
    s00 = np.sqrt(np.add.reduceat(E * E, cs[:-1])) / norm
    s0x = np.sqrt(np.add.reduceat(st[3] ** 2, cs[:-1])) / norm
    z00 = (T00 - A00) / s00
    z0x = (T0x - A0x) / s0x
    for z in (z00, z0x):
        assert np.max(np.abs(z)) < 5.0
        assert stats.chi2.sf(np.sum(z * z), len(z)) > 1e-4
    # the profile is not trivially flat: the analytic solution varies by > 10 sigma
    assert np.ptp(A00) / np.median(s00) > 10


def test_threads_do_not_change_results():
    """The oracle parallelises over particles and cells only: one thread and
    all threads give identical bits (state, accepted and executed pairs),
    in FP64, in the FP32 mirror and in the skip-ahead mode."""
    from paper_1208_0961_gb300 import workloads as W
    cfg = W.riemann_1d(20000, 100, 0.05, 10.0)
    st0 = W.thermal_state(20000, cfg["regions"], seed=3)
    keep = O.threads()
    try:
        for fp32, skip in ((False, False), (True, False), (False, True)):
            op = O.make_params(L=cfg["L"], n=cfg["n_cells"], dt=cfg["dt"], sigma_fm2=cfg["sigma_fm2"],
                               n_test=cfg["n_test"], fp32=fp32, seed=7, skip=skip)
            s = st0.astype(np.float32).astype(np.float64) if fp32 else st0
            out = []
            for t in (1, max(2, keep)):
                O.set_threads(t)
                o, _, _, _ = O.sort(op, s)
                for k in range(2):
                    o, res = O.step(op, k, o)
                out.append((o, res.accepted, res.executed))
            assert np.array_equal(out[0][0], out[1][0])
            assert np.array_equal(out[0][1], out[1][1])
            assert np.array_equal(out[0][2], out[1][2])
    finally:
        O.set_threads(keep)
