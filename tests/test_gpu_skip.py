"""GPU parity of the skip-ahead acceptance mode (CUBA_ACCEPT_SKIP) against the
oracle's skip-ahead mode, on the same seeded inputs: keys, permutation,
cell_start and positions bit-exact; candidate count, accepted and executed
sets identical (FP64 and the FP32 mirror); momenta within 1e-12 / 1e-5 of the
pair energy.  Both cell paths (warp per small cell, 32-row items), a cell with
a global-memory accepted list, tiny and ragged sizes, the full-size 16 M
workload on sampled rows and one whole cell, several steps (energy), and a
batch that mixes both modes (each member identical alone and in the mix)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1208_0961_gb300 import cuba
from paper_1208_0961_gb300 import workloads as W

from test_gpu_parity import _one_step_compare, _pair

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("fp32", [False, True])
def test_skip_single_step_riemann_small(fp32):
    cfg = W.riemann_1d(20000, 100, 0.05, 10.0)
    st0 = W.thermal_state(20000, cfg["regions"], seed=1)
    na, ne = _one_step_compare(cfg["L"], cfg["n_cells"], cfg["dt"], cfg["sigma_fm2"], cfg["n_test"], fp32, 0, st0,
                               skip=True)
    assert na > 1000 and ne > 500


@pytest.mark.parametrize("small_max", [0, 32, 1024])
@pytest.mark.parametrize("fp32", [False, True])
def test_skip_small_cells_both_paths(fp32, small_max):
    L = (1.6, 1.6, 1.6)
    regs = [((0.0, 0.0, 0.0), L, 0.4)]
    st0 = W.thermal_state(81920, regs, seed=8)
    na, ne = _one_step_compare(L, (16, 16, 16), 0.05, 5e-4, 2.0, fp32, 31, st0, step_index=2, small_max=small_max,
                               skip=True)
    assert na > 1000


def test_skip_large_accepted_list():
    L = (0.5, 0.5, 0.5)
    regs = [((0.0, 0.0, 0.0), L, 0.4)]
    st0 = W.thermal_state(2500, regs, seed=3)
    na, ne = _one_step_compare(L, (1, 1, 1), 0.1, 0.0042, 1.0, False, 5, st0, skip=True)
    assert na > 4096


@pytest.mark.parametrize("n", [0, 1, 2, 33, 4097])
def test_skip_tiny_and_ragged_sizes(n):
    L = (1.0, 1.0, 1.0)
    regs = [((0.0, 0.0, 0.0), L, 0.4)]
    st0 = W.thermal_state(n, regs, seed=4) if n else np.zeros((6, 0))
    _one_step_compare(L, (2, 2, 1), 0.2, 0.5, 1.0, False, 9, st0, skip=True)


def test_skip_near_maximal_probability():
    # 2.0001 C close to 1: a candidate at almost every pair
    L = (1.0, 1.0, 1.0)
    regs = [((0.0, 0.0, 0.0), L, 0.4)]
    st0 = W.thermal_state(900, regs, seed=6)
    # C = sigma dt / (n_test V_cell) = 0.45 with one cell
    na, ne = _one_step_compare(L, (1, 1, 1), 0.5, 0.9, 1.0, False, 3, st0, skip=True)
    assert na > 10000


def test_skip_rejects_too_large_c():
    L = (1.0, 1.0, 1.0)
    p = cuba.make_params(L=L, n_cells=(1, 1, 1), dt=0.5, sigma_fm2=0.99999, n_test=1.0,
                         precision=cuba.CUBA_FP64, acceptance=cuba.CUBA_ACCEPT_SKIP)
    with pytest.raises(cuba.CubaError):
        cuba.Sim(p, 10).close()
    p.acceptance = 7
    with pytest.raises(cuba.CubaError):
        cuba.Sim(p, 10).close()


def test_skip_multi_step_energy():
    cfg = W.riemann_1d(20000, 100, 0.05, 10.0)
    for fp32 in (False, True):
        p, _ = _pair(cfg["L"], cfg["n_cells"], cfg["dt"], cfg["sigma_fm2"], cfg["n_test"], fp32, 4, skip=True)
        sim = cuba.Sim(p, 20000)
        try:
            sim.init_riemann(20000, 0.4, 0.32)
            E0 = sim.totals()[0][0]
            Eprev = E0
            for k in range(50):
                sim.step(1)
                E1, n = sim.totals()
                assert n == 20000
                assert abs(E1[0] - Eprev) / E0 < (1e-6 if fp32 else 1e-13), "step %d" % k
                assert abs(E1[0] - E0) / E0 < (1e-6 * (k + 1) if fp32 else 1e-12)
                Eprev = E1[0]
            st = sim.stats()
            assert st["steps"] == 50 and st["overflow"] == 0
            # candidates of 50 steps: P_max n(n - 1) / 2 summed over cells
            P_fix, _ = O.skip_table(O.p22_scale(_pair(cfg["L"], cfg["n_cells"], cfg["dt"], cfg["sigma_fm2"],
                                                      cfg["n_test"], fp32, 4, skip=True)[1]))
            mu = P_fix / 2 ** 64 * st["pair_tests"]
            assert abs(st["candidates"] - mu) < 6 * np.sqrt(mu)
            assert st["candidates"] > st["accepted"] > st["executed"] > 0
        finally:
            sim.close()


def test_skip_full_size_riemann_16M_sampled():
    """The 16 M workload in the skip-ahead mode, one step: sort of every
    particle, sampled rows and one whole cell against the oracle."""
    cfg = W.riemann_1d(16_000_000, 2000, 0.0025, 10.0)
    st0 = W.thermal_state(16_000_000, cfg["regions"], seed=21).astype(np.float32)
    p, op = _pair(cfg["L"], cfg["n_cells"], cfg["dt"], cfg["sigma_fm2"], cfg["n_test"], True, 0, skip=True)
    sim = cuba.Sim(p, 16_000_000)
    try:
        sim.set_state(st0)
        cuba.cuba_trace_enable(sim.h, True)
        sim.step(1)
        g = sim.get_state()
        keys, perm, cs, pairs, exe = sim.trace()
        stats = sim.stats()
    finally:
        sim.close()
    op0 = O.make_params(L=cfg["L"], n=cfg["n_cells"], dt=cfg["dt"], sigma_fm2=0.0, n_test=cfg["n_test"],
                        fp32=True, seed=0)
    o_in, _, _, _ = O.sort(op0, st0.astype(np.float64))
    mid, r0 = O.step(op0, 0, o_in)
    assert np.array_equal(cs.astype(np.int64), r0.cell_start)
    assert np.array_equal(g[:3].astype(np.float64), mid[:3])
    # about P_max n (n - 1) / 2 candidates
    P_fix, _ = O.skip_table(O.p22_scale(op))
    npairs = float(np.sum(np.diff(r0.cell_start) * (np.diff(r0.cell_start) - 1) / 2))
    mu = P_fix / 2 ** 64 * npairs
    assert abs(stats["candidates"] - mu) < 6 * np.sqrt(mu)
    rng = np.random.default_rng(5)
    for c in np.concatenate([rng.integers(0, 1000, 3), rng.integers(1000, 2000, 3)]):
        b, e = int(cs[c]), int(cs[c + 1])
        mom = mid[3:, b:e]
        gp = pairs[pairs[:, 0] == c]
        for i in rng.integers(0, e - b - 1, 40):
            want = O.row_accept(op, 0, int(c), mom, int(i), 0, e - b)
            got = gp[gp[:, 1] == i][:, 2]
            assert np.array_equal(np.sort(got), want), (c, i)
    c = 700
    b, e = int(cs[c]), int(cs[c + 1])
    acc = O.cell_accept(op, 0, c, mid[3:, b:e])
    sel = pairs[:, 0] == c
    assert np.array_equal(pairs[sel][:, 1:], acc)
    assert len(acc) > 20


@pytest.mark.parametrize("prec", [cuba.CUBA_FP64, cuba.CUBA_FP32])
def test_skip_and_all_pairs_members_in_one_batch(prec):
    dtype = np.float64 if prec == cuba.CUBA_FP64 else np.float32
    members = []
    for k, (n, cells, sigma, skip) in enumerate([(20000, 100, 10.0, True), (15000, 60, 30.0, False),
                                                 (9000, 300, 3.0, True)]):
        cfg = W.riemann_1d(n, cells, 0.5 * 10.0 / cells, sigma)
        p = cuba.make_params(L=cfg["L"], n_cells=cfg["n_cells"], dt=cfg["dt"], sigma_fm2=cfg["sigma_fm2"],
                             n_test=cfg["n_test"], precision=prec, seed=40 + k,
                             acceptance=cuba.CUBA_ACCEPT_SKIP if skip else cuba.CUBA_ACCEPT_ALL_PAIRS)
        st = W.thermal_state(n, cfg["regions"], seed=50 + k).astype(dtype)
        members.append((p, st))
    alone = []
    for p, st in members:
        sim = cuba.Sim(p, st.shape[1])
        try:
            sim.set_state(st)
            sim.step(4)
            alone.append((sim.get_state(), sim.stats()))
        finally:
            sim.close()
    b = cuba.Batch(cuba.make_batch_config(prec, max_sims=4, max_particles=60000, max_cells=600))
    try:
        ids = [b.add_state(p, st) for p, st in members]
        b.step(4)
        for (ref, rs), i in zip(alone, ids):
            assert np.array_equal(b.get_state(i), ref)
            s = b.stats(i)
            assert s["accepted"] == rs["accepted"] and s["candidates"] == rs["candidates"]
    finally:
        b.close()
