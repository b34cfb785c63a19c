"""Large-cross-section limit of the oracle's 1D Riemann problem (Sec. 5, Figs. 2-3).

The paper shows that the energy-density profile steepens towards the ideal
fluid solution as sigma grows (Fig. 3).  Pins: the ideal-fluid solver itself
satisfies the jump conditions and its limits; the oracle's T00 profile at
t = 2 fm/c approaches the ideal profile monotonically in sigma (L1 distance).
"""
import numpy as np

from oracle import oracle as O
import physics as PH


def test_ideal_solver_invariants():
    eL, eR = 16.204, 6.637
    e, v, vsh = PH.ideal_riemann(eL, eR)
    # invariants of the exact solution: jump conditions hold, plateau between
    # the two states, shock faster than sound, slower than light
    T00, T0x, Txx = PH._fluid_T(e, v)
    assert abs(vsh * (T00 - eR) - T0x) < 1e-12 * eL
    assert abs(vsh * T0x - (Txx - eR / 3)) < 1e-9 * eL
    assert eR < e < eL and 0 < v < 1 and PH.CS < vsh < 1
    # weak-shock limit: shock speed tends to the speed of sound
    e2, v2, vsh2 = PH.ideal_riemann(1.0 + 1e-6, 1.0)
    assert abs(vsh2 - PH.CS) < 1e-5 and v2 < 1e-6
    # 400 / 320 MeV gluon gas: plateau 10.37 GeV/fm^3, v* = 0.191, v_sh = 0.645
    assert abs(e - 10.37) < 0.01 and abs(v - 0.191) < 1e-3 and abs(vsh - 0.645) < 1e-3


def _profile(sigma_fm2, seed, N=20000, t_end=2.0, dt=0.05):
    L = (10.0, 1.0, 1.0)
    regs = O.riemann_regions(L, 0.4, 0.32)
    ntest = O.n_test_for(N, regs)
    p = O.make_params(L=L, n=(100, 1, 1), dt=dt, sigma_fm2=sigma_fm2, n_test=ntest, seed=seed)
    st = O.init_thermal(p, N, regs)
    st, _, _, cs = O.sort(p, st)
    for k in range(int(round(t_end / dt))):
        st, res = O.step(p, k, st, trace=False)
    _, _, _, cs = O.sort(p, st)
    T00, _, _ = O.observables(p, st, cs)
    return T00


def test_profile_approaches_ideal_fluid_as_sigma_grows():
    t = 2.0
    x = (np.arange(100) + 0.5) * 0.1
    eL = 3 * O.gluon_density(0.4) * 0.4
    eR = 3 * O.gluon_density(0.32) * 0.32
    _, _, ideal, _ = PH.ideal_profile((x - 5.0) / t, eL, eR)
    win = np.abs(x - 5.0) < 1.0 * t
    dists = []
    for sigma_mb in (0.0, 3.0, 30.0):
        prof = np.mean([_profile(sigma_mb * O.FM2_PER_MB, seed) for seed in (0, 1)], axis=0)
        # smooth over 5 cells (0.5 fm) to damp the test-particle noise
        k = np.ones(5) / 5
        ps = np.convolve(prof, k, mode="same")
        ids = np.convolve(ideal, k, mode="same")
        dists.append(np.mean(np.abs(ps - ids)[win]))
    assert dists[0] > dists[1] > dists[2]
    assert dists[2] < 0.5 * dists[0]
