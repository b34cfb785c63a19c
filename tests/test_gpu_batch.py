"""Batched execution (A9): many simulations in one arena and one launch
sequence per step.  Each member's result must be bit-identical to the same
simulation run alone (its random numbers are keyed by its own seed, step and
local indices), also when other members are admitted and retired (with arena
compaction) while it runs, and a member's step must match the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1208_0961_gb300 import cuba
from paper_1208_0961_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _riemann(n, cells, sigma_mb, seed, prec, L=(10.0, 1.0, 1.0), dt=None):
    cfg = W.riemann_1d(n, cells, dt or 0.5 * L[0] / cells, sigma_mb, L=L)
    p = cuba.make_params(L=cfg["L"], n_cells=cfg["n_cells"], dt=cfg["dt"], sigma_fm2=cfg["sigma_fm2"],
                         n_test=cfg["n_test"], precision=prec, seed=seed)
    return cfg, p


def _alone(p, st, steps, prec):
    sim = cuba.Sim(p, st.shape[1])
    try:
        sim.set_state(st)
        sim.step(steps)
        return sim.get_state(), sim.observables(), sim.stats()
    finally:
        sim.close()


@pytest.mark.parametrize("prec", [cuba.CUBA_FP64, cuba.CUBA_FP32])
def test_member_identical_alone_and_in_the_mix(prec):
    dtype = np.float64 if prec == cuba.CUBA_FP64 else np.float32
    cfgA, pA = _riemann(20000, 100, 10.0, seed=11, prec=prec)
    cfgB, pB = _riemann(35000, 80, 30.0, seed=12, prec=prec, L=(8.0, 1.0, 1.0))
    cfgC, pC = _riemann(9000, 300, 3.0, seed=13, prec=prec, L=(12.0, 2.0, 1.0))
    stA = W.thermal_state(20000, cfgA["regions"], seed=1).astype(dtype)
    stB = W.thermal_state(35000, cfgB["regions"], seed=2).astype(dtype)
    stC = W.thermal_state(9000, cfgC["regions"], seed=3).astype(dtype)
    refA, obsA, statA = _alone(pA, stA, 6, prec)
    refC, obsC, statC = _alone(pC, stC, 3, prec)

    b = cuba.Batch(cuba.make_batch_config(prec, max_sims=8, max_particles=100000, max_cells=1000))
    try:
        idB = b.add_state(pB, stB)
        idA = b.add_state(pA, stA)
        b.step(3)
        b.remove(idB)          # A moves down: compaction
        idC = b.add_state(pC, stC)
        b.step(3)
        assert b.get_step(idA) == 6 and b.get_step(idC) == 3
        gA = b.get_state(idA)
        gC = b.get_state(idC)
        oA = b.observables(idA)
        sA = b.stats(idA)
        assert b.usage() == (2, 29000, 400)
    finally:
        b.close()
    assert np.array_equal(gA, refA)
    assert np.array_equal(gC, refC)
    for x, y in zip(oA, obsA):
        assert np.array_equal(x, y)
    assert sA == statA and sA["executed"] > 0


def test_batch_member_matches_oracle_one_step():
    cfg, p = _riemann(20000, 100, 10.0, seed=5, prec=cuba.CUBA_FP64)
    _, pO = _riemann(15000, 60, 20.0, seed=6, prec=cuba.CUBA_FP64, L=(6.0, 1.0, 1.0))
    st = W.thermal_state(20000, cfg["regions"], seed=7)
    stO = W.thermal_state(15000, W.riemann_regions((6.0, 1.0, 1.0), 0.4, 0.32), seed=8)
    b = cuba.Batch(cuba.make_batch_config(cuba.CUBA_FP64, max_sims=4, max_particles=50000, max_cells=500))
    try:
        b.add_state(pO, stO)
        i = b.add_state(p, st)
        b.step(1)
        g = b.get_state(i)
        s = b.stats(i)
    finally:
        b.close()
    op = O.make_params(L=cfg["L"], n=cfg["n_cells"], dt=cfg["dt"], sigma_fm2=cfg["sigma_fm2"],
                       n_test=cfg["n_test"], seed=5)
    o, _, _, _ = O.sort(op, st)
    o, res = O.step(op, 0, o)
    assert np.array_equal(g[:3], o[:3])
    E = np.sqrt((o[3:] ** 2).sum(axis=0))
    assert np.max(np.abs(g[3:] - o[3:]).max(axis=0) / E) < 1e-9
    assert s["accepted"] == res.n_acc and s["executed"] == res.n_exe


def test_batch_capacity_is_enforced():
    _, p = _riemann(20000, 100, 10.0, seed=5, prec=cuba.CUBA_FP32)
    b = cuba.Batch(cuba.make_batch_config(cuba.CUBA_FP32, max_sims=2, max_particles=30000, max_cells=150))
    try:
        b.add(p, 20000, W.riemann_regions((10.0, 1.0, 1.0), 0.4, 0.32))
        with pytest.raises(cuba.CubaError) as e:
            b.add(p, 20000, W.riemann_regions((10.0, 1.0, 1.0), 0.4, 0.32))
        assert e.value.code == cuba.CUBA_ERR_CAPACITY
        assert b.usage() == (1, 20000, 100)
        b.step(2)
    finally:
        b.close()


def test_full_size_ensemble_sampled_members():
    """The batched ensemble at full size (256 Riemann runs, 2.4e8 particles,
    FP32), one step of the whole batch: the members the oracle can step in
    seconds (the fewest pair tests) start from host-sampled states and must
    match the oracle's single-precision mirror — positions bit-exact (hence
    the same sort), the same accepted and executed counts, momenta of
    colliding particles within 1e-5 of the pair energy and untouched ones
    exact; the other members are sampled on the device."""
    import bench
    members = bench.ensemble(256, 0)
    cost = [m["n"] ** 2 / m["n_cells"][0] for m in members]
    sampled = set(np.argsort(cost)[:3].tolist())
    N = sum(m["n"] for m in members)
    C = sum(m["n_cells"][0] for m in members)
    b = cuba.Batch(cuba.make_batch_config(cuba.CUBA_FP32, max_sims=256, max_particles=N, max_cells=C))
    want = {}
    try:
        ids = {}
        for k, m in enumerate(members):
            p = cuba.make_params(L=m["L"], n_cells=m["n_cells"], dt=m["dt"], sigma_fm2=m["sigma_fm2"],
                                 n_test=m["n_test"], precision=cuba.CUBA_FP32, seed=m["seed"])
            if k in sampled:
                st = W.thermal_state(m["n"], m["regions"], seed=100 + k).astype(np.float32)
                ids[k] = b.add_state(p, st)
                want[k] = st
            else:
                b.add(p, m["n"], m["regions"])
        b.step(1)
        got = {k: (b.get_state(ids[k]), b.stats(ids[k])) for k in sampled}
    finally:
        b.close()
    for k in sorted(sampled):
        m = members[k]
        op = O.make_params(L=m["L"], n=m["n_cells"], dt=m["dt"], sigma_fm2=m["sigma_fm2"], n_test=m["n_test"],
                           fp32=True, seed=m["seed"])
        o, _, _, _ = O.sort(op, want[k].astype(np.float64))
        o, res = O.step(op, 0, o)
        g, s = got[k]
        assert np.array_equal(g[:3].astype(np.float64), o[:3]), k
        assert s["accepted"] == res.n_acc and s["executed"] == res.n_exe, k
        E = np.sqrt((o[3:] ** 2).sum(axis=0))
        tol = np.zeros(o.shape[1])
        for c, i, j in res.executed.tolist():
            bb = res.cell_start[c]
            tol[bb + i] = tol[bb + j] = E[bb + i] + E[bb + j]
        d = np.abs(g[3:].astype(np.float64) - o[3:]).max(axis=0)
        moved = tol > 0
        assert np.all(d[~moved] == 0), k
        assert np.all(d[moved] <= 1e-5 * tol[moved]), k
        assert res.n_exe > 0, k


def test_removal_keeps_later_members_exact_on_the_neighbour_sort():
    """3D boxes of about 30 particles per cell (more than 2048 cells in the
    arena: the step sorts by neighbour moves, which reads the previous
    cell_start).  Removing a middle member shifts the later ones; their
    observables read right after the removal, and the steps after it, must
    equal the same simulations run alone."""
    def box(k, seed):
        L = (0.1 * k,) * 3
        regs = [((0.0, 0.0, 0.0), L, 0.4)]
        n = 30 * k ** 3
        nt = W.n_test_for(n, regs)
        p = cuba.make_params(L=L, n_cells=(k, k, k), dt=0.05, sigma_fm2=3.0, n_test=nt, precision=cuba.CUBA_FP32,
                             seed=seed)
        return p, W.thermal_state(n, regs, seed=seed).astype(np.float32)

    pA, sA = box(14, 21)
    pB, sB = box(12, 22)
    pC, sC = box(13, 23)
    refC1 = _alone(pC, sC, 2, cuba.CUBA_FP32)
    refC2 = _alone(pC, sC, 5, cuba.CUBA_FP32)
    refA = _alone(pA, sA, 5, cuba.CUBA_FP32)
    b = cuba.Batch(cuba.make_batch_config(cuba.CUBA_FP32, max_sims=4, max_particles=300000, max_cells=9000))
    try:
        iA = b.add_state(pA, sA)
        iB = b.add_state(pB, sB)
        iC = b.add_state(pC, sC)
        b.step(2)
        b.remove(iB)                          # C moves down
        oC1 = b.observables(iC)               # before any further step
        b.step(3)
        gC = b.get_state(iC)
        gA = b.get_state(iA)
        oC2 = b.observables(iC)
    finally:
        b.close()
    for x, y in zip(oC1, refC1[1]):
        assert np.array_equal(x, y)
    assert np.array_equal(gC, refC2[0]) and np.array_equal(gA, refA[0])
    for x, y in zip(oC2, refC2[1]):
        assert np.array_equal(x, y)
