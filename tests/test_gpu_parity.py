"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle.

Bars (per the method's reading of the single-step comparison):
  * cell keys, sort permutation, cell_start, particle counts: bit-exact;
  * positions: bit-exact (streaming and reflection are separately rounded
    IEEE operations on both sides);
  * accepted pair set and executed (greedy) set: identical in FP64 and in FP32
    against the oracle's single-precision mirror;
  * momenta after collisions: |dp|_inf <= 1e-12 (E_i + E_j) in FP64 (only the
    libm/CUDA sin, cos, log differ), <= 1e-5 (E_i + E_j) in FP32;
  * observables: relative 1e-12 (FP64 sums in a different order).
Inputs come from the seeded numpy sampler in paper_1208_0961_gb300.workloads,
never from the GPU.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1208_0961_gb300 import cuba
from paper_1208_0961_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _pair(L, n_cells, dt, sigma_fm2, n_test, fp32, seed, gamma_fp64=0.0, skip=False, kappa=0.0, mass=0.0, mu=0.0):
    p = cuba.make_params(L=L, n_cells=n_cells, dt=dt, sigma_fm2=sigma_fm2, n_test=n_test,
                         precision=cuba.CUBA_FP32 if fp32 else cuba.CUBA_FP64, seed=seed, gamma_fp64=gamma_fp64,
                         acceptance=cuba.CUBA_ACCEPT_SKIP if skip else cuba.CUBA_ACCEPT_ALL_PAIRS, kappa=kappa,
                         mass=mass, mu=mu)
    op = O.make_params(L=L, n=n_cells, dt=dt, sigma_fm2=sigma_fm2, n_test=n_test, fp32=fp32, seed=seed, skip=skip,
                       kappa=kappa, mass=mass, mu=mu)
    return p, op


def _one_step_compare(L, n_cells, dt, sigma_fm2, n_test, fp32, seed, st0, step_index=3, small_max=None,
                      skip=False, kappa=0.0, mass=0.0, mu=0.0):
    p, op = _pair(L, n_cells, dt, sigma_fm2, n_test, fp32, seed, skip=skip, kappa=kappa, mass=mass, mu=mu)
    dtype = np.float32 if fp32 else np.float64
    st0 = st0.astype(dtype)
    n = st0.shape[1]
    sim = cuba.Sim(p, max(n, 1))
    try:
        if small_max is not None:
            cuba.cuba_set_small_max(sim.h, small_max)
        sim.set_state(st0)
        cuba.cuba_trace_enable(sim.h, True)
        cuba.cuba_set_step(sim.h, step_index)
        g_in = sim.get_state()
        sim.step(1)
        g_out = sim.get_state()
        keys, perm, cs, pairs, exe = sim.trace()
        stats = sim.stats()
        t_gpu, dt_gpu = sim.time()
        assert cuba.cuba_get_step(sim.h) == step_index + 1
    finally:
        sim.close()
    # oracle: same input, same stable sort, one step
    o_in, _, _, _ = O.sort(op, st0.astype(np.float64))
    assert np.array_equal(g_in.astype(np.float64), o_in), "set_state sort differs"
    o_out, res = O.step(op, step_index, o_in)
    assert dt_gpu == res.dt and t_gpu == res.dt, "time step differs"
    assert np.array_equal(keys, res.keys.astype(np.uint32)), "keys differ"
    assert np.array_equal(perm.astype(np.int64), res.perm), "permutation differs"
    assert np.array_equal(cs.astype(np.int64), res.cell_start), "cell_start differs"
    assert np.array_equal(g_out[:3].astype(np.float64), o_out[:3]), "positions differ"
    acc_o = [tuple(x) for x in res.accepted.tolist()]
    acc_g = [tuple(x) for x in pairs.tolist()]
    assert acc_g == acc_o, "accepted pairs differ (%d vs %d)" % (len(acc_g), len(acc_o))
    exe_o = set(tuple(x) for x in res.executed.tolist())
    exe_g = set(tuple(x) for x in pairs[exe].tolist())
    assert exe_g == exe_o, "executed pairs differ"
    # momenta
    E = np.sqrt((o_out[3:] ** 2).sum(axis=0) + mass * mass)
    tol = np.zeros(n)
    for c, i, j in res.executed.tolist():
        b = res.cell_start[c]
        s = E[b + i] + E[b + j]
        tol[b + i] = s
        tol[b + j] = s
    rel = 1e-5 if fp32 else 1e-12
    d = np.abs(g_out[3:].astype(np.float64) - o_out[3:]).max(axis=0)
    moved = tol > 0
    assert np.all(d[~moved] == 0), "momenta of non-colliding particles differ"
    if moved.any():
        assert np.all(d[moved] <= rel * tol[moved]), "max rel dp %.3g" % (d[moved] / tol[moved]).max()
    assert stats["accepted"] == len(acc_o)
    assert stats["executed"] == len(exe_o)
    assert stats["reflections"] == res.n_reflections
    assert stats["pair_tests"] == res.n_pairs_tested
    assert stats["candidates"] == res.n_candidates
    return len(acc_o), len(exe_o)


@pytest.mark.parametrize("fp32", [False, True])
def test_single_step_riemann_small(fp32):
    cfg = W.riemann_1d(20000, 100, 0.05, 10.0)
    st0 = W.thermal_state(20000, cfg["regions"], seed=1)
    na, ne = _one_step_compare(cfg["L"], cfg["n_cells"], cfg["dt"], cfg["sigma_fm2"], cfg["n_test"], fp32, 0, st0)
    assert na > 1000 and ne > 500


@pytest.mark.parametrize("fp32", [False, True])
def test_single_step_3d_ragged(fp32):
    L = (1.2, 0.9, 0.6)
    regs = [((0.0, 0.0, 0.0), L, 0.4)]
    st0 = W.thermal_state(12345, regs, seed=2)
    na, ne = _one_step_compare(L, (6, 5, 4), 0.1, 0.02, 3.0, fp32, 77, st0, step_index=11)
    assert na > 100


@pytest.mark.parametrize("dt", [0.05, 0.0985])
@pytest.mark.parametrize("fp32", [False, True])
def test_single_step_3d_many_small_cells(fp32, dt):
    # 16 x 12 x 12 = 2304 cells (more than one 11-bit digit), about 17
    # particles per cell: dt = 0.05 takes the neighbour-move sort (dt below
    # 0.98 of the 0.1 fm cell edge), dt = 0.0985 the two-pass radix sort
    L = (1.6, 1.2, 1.2)
    regs = [((0.0, 0.0, 0.0), (0.8, 1.2, 1.2), 0.45), ((0.8, 0.0, 0.0), L, 0.35)]
    st0 = W.thermal_state(40000, regs, seed=17)
    na, ne = _one_step_compare(L, (16, 12, 12), dt, 0.002, 5.0, fp32, 19, st0, step_index=5)
    assert na > 200 and ne > 100


def test_neighbour_sort_several_steps():
    """Four steps in FP64 on 3072 small cells (every step after the first
    sorts from the previous step's order and cell_start): keys, permutation
    and cell_start of the last step equal the oracle's, positions agree to
    1e-12 fm and momenta to 1e-10 of the particle energy."""
    L = (1.6, 1.6, 1.2)
    regs = [((0.0, 0.0, 0.0), L, 0.4)]
    st0 = W.thermal_state(50000, regs, seed=29)
    p, op = _pair(L, (16, 16, 12), 0.06, 0.002, 5.0, False, 31)
    sim = cuba.Sim(p, 50000)
    try:
        sim.set_state(st0)
        sim.step(3)
        cuba.cuba_trace_enable(sim.h, True)
        sim.step(1)
        g = sim.get_state()
        keys, perm, cs, pairs, exe = sim.trace()
        stats = sim.stats()
    finally:
        sim.close()
    o, _, _, _ = O.sort(op, st0)
    for k in range(3):
        o, _ = O.step(op, k, o)
    o, res = O.step(op, 3, o)
    assert np.array_equal(keys, res.keys.astype(np.uint32))
    assert np.array_equal(perm.astype(np.int64), res.perm)
    assert np.array_equal(cs.astype(np.int64), res.cell_start)
    assert np.max(np.abs(g[:3] - o[:3])) <= 1e-12
    E = np.sqrt((o[3:] ** 2).sum(axis=0))
    assert np.max(np.abs(g[3:] - o[3:]).max(axis=0) / E) <= 1e-10
    assert stats["reflections"] > 0 and stats["executed"] > 0


def test_large_accepted_list_uses_global_sort_path():
    # one cell, ~10^4 accepted pairs: beyond the shared-memory list size
    L = (0.5, 0.5, 0.5)
    regs = [((0.0, 0.0, 0.0), L, 0.4)]
    st0 = W.thermal_state(2500, regs, seed=3)
    na, ne = _one_step_compare(L, (1, 1, 1), 0.1, 0.0042, 1.0, False, 5, st0)
    assert na > 4096


def test_survivors_beyond_the_global_list():
    # one cell, C = 0.45: the byte filters pass about 90 % of the 2.9 M pairs,
    # more survivors than the 2^21-record list holds, so the pair kernel also
    # evaluates the overflow in place (shared-memory and global)
    L = (0.5, 0.5, 0.5)
    regs = [((0.0, 0.0, 0.0), L, 0.4)]
    st0 = W.thermal_state(2400, regs, seed=13)
    C = 0.45
    dt, n_test = 0.1, 1.0
    sigma = C * n_test * (0.5 ** 3) / dt
    for fp32 in (False, True):
        na, ne = _one_step_compare(L, (1, 1, 1), dt, sigma, n_test, fp32, 21, st0)
        assert na > 2 ** 20 and ne > 1000


@pytest.mark.parametrize("n", [0, 1, 2, 33, 4097])
def test_tiny_and_ragged_sizes(n):
    L = (1.0, 1.0, 1.0)
    regs = [((0.0, 0.0, 0.0), L, 0.4)]
    st0 = W.thermal_state(n, regs, seed=4) if n else np.zeros((6, 0))
    _one_step_compare(L, (2, 2, 1), 0.2, 0.5, 1.0, False, 9, st0)


def test_sigma_zero_is_free_streaming():
    cfg = W.riemann_1d(5000, 50, 0.05, 0.0)
    st0 = W.thermal_state(5000, cfg["regions"], seed=5)
    na, ne = _one_step_compare(cfg["L"], cfg["n_cells"], cfg["dt"], 0.0, cfg["n_test"], False, 0, st0)
    assert na == 0 and ne == 0


def test_init_thermal_matches_oracle_sampling():
    cfg = W.riemann_1d(30000, 100, 0.05, 10.0)
    p, op = _pair(cfg["L"], cfg["n_cells"], cfg["dt"], cfg["sigma_fm2"], cfg["n_test"], False, 1234)
    sim = cuba.Sim(p, 30000)
    try:
        sim.init_riemann(30000, 0.4, 0.32)
        g = sim.get_state()
        assert cuba.cuba_get_step(sim.h) == 0
    finally:
        sim.close()
    o = O.init_thermal(op, 30000, O.riemann_regions(cfg["L"], 0.4, 0.32))
    o, _, _, _ = O.sort(op, o)
    # positions are exact arithmetic; momenta go through log/sin/cos
    assert np.array_equal(g[:3], o[:3])
    E = np.sqrt((o[3:] ** 2).sum(axis=0))
    assert np.max(np.abs(g[3:] - o[3:]).max(axis=0) / E) < 1e-13


def test_observables_and_totals_match_oracle():
    cfg = W.riemann_1d(40000, 100, 0.05, 10.0)
    p, op = _pair(cfg["L"], cfg["n_cells"], cfg["dt"], cfg["sigma_fm2"], cfg["n_test"], False, 3)
    st0 = W.thermal_state(40000, cfg["regions"], seed=6)
    sim = cuba.Sim(p, 40000)
    try:
        sim.set_state(st0)
        sim.step(2)
        g = sim.get_state()
        T00, T0x, cnt = sim.observables()
        tot, n = sim.totals()
    finally:
        sim.close()
    _, _, _, cs = O.sort(op, g.astype(np.float64))
    oT00, oT0x, ocnt = O.observables(op, g, cs)
    assert np.array_equal(cnt, ocnt) and cnt.sum() == 40000 and n == 40000
    assert np.allclose(T00, oT00, rtol=1e-12, atol=0)
    assert np.allclose(T0x, oT0x, rtol=1e-12, atol=1e-12 * np.abs(oT00).max())
    ot = O.totals(g)
    assert abs(tot[0] - ot[0]) <= 1e-12 * ot[0]
    assert np.max(np.abs(np.array(tot[1:]) - ot[1:])) <= 1e-12 * ot[0]


def test_multi_step_energy_conservation_fp64_and_fp32():
    cfg = W.riemann_1d(20000, 100, 0.05, 10.0)
    for fp32 in (False, True):
        p, _ = _pair(cfg["L"], cfg["n_cells"], cfg["dt"], cfg["sigma_fm2"], cfg["n_test"], fp32, 0)
        sim = cuba.Sim(p, 20000)
        try:
            sim.init_riemann(20000, 0.4, 0.32)
            E0 = sim.totals()[0][0]
            # relative drift below 1e-6 in every single step (FP32 state; FP64:
            # rounding only), checked after each of the 100 steps
            Eprev = E0
            for k in range(100):
                sim.step(1)
                E1, n = sim.totals()
                assert n == 20000
                assert abs(E1[0] - Eprev) / E0 < (1e-6 if fp32 else 1e-13), "step %d" % k
                assert abs(E1[0] - E0) / E0 < (1e-6 * (k + 1) if fp32 else 1e-12)
                Eprev = E1[0]
            st = sim.stats()
            assert st["steps"] == 100 and st["overflow"] == 0 and st["executed"] > 0
        finally:
            sim.close()


def test_init_hotspot_matches_oracle_sampling():
    L = (6.4, 6.4, 6.4)
    n = 200000
    p, op = _pair(L, (32, 32, 32), 0.05, 0.5, 100.0, False, 77)
    sim = cuba.Sim(p, n)
    try:
        sim.init_hotspot(n, 0.4, 0.2, 1.0)
        g = sim.get_state()
    finally:
        sim.close()
    o = O.init_hotspot(op, n, 0.4, 0.2, 1.0)
    o, _, _, _ = O.sort(op, o)
    # positions are exact arithmetic; only an acceptance decision that falls
    # within an ulp of exp() could differ between the two math libraries
    differ = np.any(g[:3] != o[:3], axis=0)
    assert differ.sum() <= max(2, n // 100000)
    E = np.sqrt((o[3:] ** 2).sum(axis=0))
    ok = ~differ
    assert np.max(np.abs(g[3:, ok] - o[3:, ok]).max(axis=0) / E[ok]) < 1e-12


def test_full_size_riemann_16M_sampled():
    """The bench workload at full size (16 M particles, 2000 cells, FP32), one
    step in the bench's launch configuration: keys, permutation, cell_start and
    positions of all particles against the oracle's single-precision mirror;
    accepted pairs of sampled rows and of one whole cell; the executed set of
    that cell is the greedy matching of its accepted pairs; its momenta follow
    the oracle's kinematics to 1e-5 of the pair energy."""
    cfg = W.riemann_1d(16_000_000, 2000, 0.0025, 10.0)
    st0 = W.thermal_state(16_000_000, cfg["regions"], seed=21).astype(np.float32)
    p, op = _pair(cfg["L"], cfg["n_cells"], cfg["dt"], cfg["sigma_fm2"], cfg["n_test"], True, 0)
    sim = cuba.Sim(p, 16_000_000)
    try:
        sim.set_state(st0)
        # the shape the autotuner picks for this workload: 32-row items only,
        # eight Philox blocks per lane and iteration
        cuba.cuba_set_launch_shape(sim.h, 0, 2, 8)
        cuba.cuba_trace_enable(sim.h, True)
        sim.step(1)
        g = sim.get_state()
        keys, perm, cs, pairs, exe = sim.trace()
    finally:
        sim.close()
    # stream + key + sort of every particle: the oracle's step with sigma = 0
    op0 = O.make_params(L=cfg["L"], n=cfg["n_cells"], dt=cfg["dt"], sigma_fm2=0.0, n_test=cfg["n_test"],
                        fp32=True, seed=0)
    o_in, _, _, _ = O.sort(op0, st0.astype(np.float64))
    mid, r0 = O.step(op0, 0, o_in)
    assert np.array_equal(keys, r0.keys.astype(np.uint32))
    assert np.array_equal(perm.astype(np.int64), r0.perm)
    assert np.array_equal(cs.astype(np.int64), r0.cell_start)
    assert np.array_equal(g[:3].astype(np.float64), mid[:3])
    # sampled rows of several cells
    rng = np.random.default_rng(5)
    cells = np.concatenate([rng.integers(0, 1000, 3), rng.integers(1000, 2000, 3)])
    for c in cells:
        b, e = int(cs[c]), int(cs[c + 1])
        mom = mid[3:, b:e]
        gp = pairs[pairs[:, 0] == c]
        for i in rng.integers(0, e - b - 1, 20):
            want = O.row_accept(op, 0, int(c), mom, int(i), 0, e - b)
            got = gp[gp[:, 1] == i][:, 2]
            assert np.array_equal(np.sort(got), want), (c, i)
    # one whole cell of the right half: accepted set, greedy matching, momenta
    c = 1500
    b, e = int(cs[c]), int(cs[c + 1])
    mom = mid[3:, b:e]
    acc = O.cell_accept(op, 0, c, mom)
    sel = pairs[:, 0] == c
    assert np.array_equal(pairs[sel][:, 1:], acc)
    used = set()
    for (i, j), x in zip(acc.tolist(), exe[sel].tolist()):
        want = i not in used and j not in used
        assert x == want
        if want:
            used.update((i, j))
            ok, pi, pj = O.kinematics([0, 0], 0, c, i, j, mom[:, i], mom[:, j])
            s = np.linalg.norm(mom[:, i]) + np.linalg.norm(mom[:, j])
            assert np.max(np.abs(g[3:, b + i] - pi)) <= 1e-5 * s
            assert np.max(np.abs(g[3:, b + j] - pj)) <= 1e-5 * s
    assert len(used) > 0


def _check_cell(op, c, mom, pairs, exe, g, b):
    """All accepted pairs of cell c, its greedy matching and the momenta of
    its executed pairs (1e-5 of the pair energy) against the oracle."""
    acc = O.cell_accept(op, 0, c, mom)
    sel = pairs[:, 0] == c
    assert np.array_equal(pairs[sel][:, 1:], acc), c
    used = set()
    for (i, j), x in zip(acc.tolist(), exe[sel].tolist()):
        want = i not in used and j not in used
        assert x == want
        if want:
            used.update((i, j))
            ok, pi, pj = O.kinematics([0, 0], 0, c, i, j, mom[:, i], mom[:, j])
            s = np.linalg.norm(mom[:, i]) + np.linalg.norm(mom[:, j])
            assert np.max(np.abs(g[3:, b + i] - pi)) <= 1e-5 * s
            assert np.max(np.abs(g[3:, b + j] - pj)) <= 1e-5 * s
    return len(acc), len(used) // 2


def test_full_size_hotspot_64M_sampled():
    """The 3D hot spot at full size (64 M particles, 128^3 cells, sigma = 5 mb,
    dt = 0.01, FP32), one step in the launch shape the autotuner picks for it
    (warp-per-cell kernels for cells up to 256 particles, two Philox blocks per
    iteration of the 32-row item kernel): keys, permutation, cell_start and
    positions of every particle against the oracle's single-precision mirror;
    accepted pairs, greedy matching and momenta of the fullest cells and of
    random ones."""
    n = 64_000_000
    cfg = W.hotspot_3d(n, 128, 0.01, 5.0)
    st0 = W.hotspot_state(n, cfg, seed=23).astype(np.float32)
    p, op = _pair(cfg["L"], cfg["n_cells"], cfg["dt"], cfg["sigma_fm2"], cfg["n_test"], True, 0)
    sim = cuba.Sim(p, n)
    try:
        sim.set_state(st0)
        cuba.cuba_set_launch_shape(sim.h, 256, 1, 2)
        cuba.cuba_trace_enable(sim.h, True)
        sim.step(1)
        g = sim.get_state()
        keys, perm, cs, pairs, exe = sim.trace()
    finally:
        sim.close()
    op0 = O.make_params(L=cfg["L"], n=cfg["n_cells"], dt=cfg["dt"], sigma_fm2=0.0, n_test=cfg["n_test"],
                        fp32=True, seed=0)
    o_in, _, _, _ = O.sort(op0, st0.astype(np.float64))
    del st0
    mid, r0 = O.step(op0, 0, o_in)
    del o_in
    assert np.array_equal(keys, r0.keys.astype(np.uint32))
    assert np.array_equal(perm.astype(np.int64), r0.perm)
    assert np.array_equal(cs.astype(np.int64), r0.cell_start)
    assert np.array_equal(g[:3].astype(np.float64), mid[:3])
    occ = np.diff(r0.cell_start)
    rng = np.random.default_rng(7)
    cells = np.concatenate([np.argsort(occ)[-3:], rng.integers(0, len(occ), 40)])
    na = ne = 0
    for c in cells.tolist():
        b, e = int(cs[c]), int(cs[c + 1])
        a, x = _check_cell(op, c, mid[3:, b:e], pairs, exe, g, b)
        na += a
        ne += x
    assert na > 20 and ne > 10


@pytest.mark.parametrize("small_max", [0, 32, 1024])
@pytest.mark.parametrize("fp32", [False, True])
def test_small_cells_both_paths(fp32, small_max):
    """About 20 particles per cell (3D): the warp-per-cell pair and resolve
    kernels (small_max >= 32) and the item path (0) give the oracle's step."""
    L = (1.6, 1.6, 1.6)
    regs = [((0.0, 0.0, 0.0), L, 0.4)]
    st0 = W.thermal_state(81920, regs, seed=8)
    # C = sigma dt / (N_test V_cell) = 0.0125
    na, ne = _one_step_compare(L, (16, 16, 16), 0.05, 5e-4, 2.0, fp32, 31, st0, step_index=2, small_max=small_max)
    assert na > 1000


def test_small_cells_with_many_accepted_pairs_hand_over():
    """Small cells whose accepted lists exceed 32 pairs go to the block path."""
    L = (0.8, 0.8, 0.8)
    regs = [((0.0, 0.0, 0.0), L, 0.4)]
    st0 = W.thermal_state(15000, regs, seed=9)
    # about 29 particles per cell, C = 0.15: about 60 accepted pairs per cell
    na, ne = _one_step_compare(L, (8, 8, 8), 0.09, 1.0 / 3.0 * 1e-3, 0.2, False, 13, st0, small_max=64)
    assert na > 32 * 512 * 0.5


@pytest.mark.parametrize("fp32", [False, True])
@pytest.mark.parametrize("L,cells", [((10.0, 1.0, 1.0), (2000, 1, 1)), ((1.3, 0.7, 2.9), (7, 5, 3)),
                                     ((12.8, 12.8, 12.8), (128, 128, 128))])
def test_cell_keys_on_and_next_to_every_face(fp32, L, cells):
    """Positions exactly on each cell face and one ulp either side (the cases
    where the quotient x / dx sits on an integer or rounds onto one): the
    library's keys equal the oracle's correctly rounded floor(x / dx)."""
    dtype = np.float32 if fp32 else np.float64
    rng = np.random.default_rng(5)
    cols = []
    for a in range(3):
        dx = dtype(L[a] / cells[a]) if fp32 else L[a] / cells[a]
        faces = np.arange(cells[a] + 1, dtype=dtype) * dtype(dx)
        faces = np.minimum(faces, dtype(L[a]))
        near = np.concatenate([faces, np.nextafter(faces, dtype(np.inf)), np.nextafter(faces, dtype(0))])
        near = near[(near >= 0) & (near <= dtype(L[a]))]
        cols.append(near)
    n = max(len(c) for c in cols) * 3
    st = np.zeros((6, n), dtype=dtype)
    for a in range(3):
        c = cols[a]
        st[a] = np.concatenate([c] * (n // len(c) + 1))[:n]
        st[a] = st[a][rng.permutation(n)]
        st[3 + a] = rng.normal(size=n).astype(dtype)
    p, op = _pair(L, cells, 0.5 * min(L[a] / cells[a] for a in range(3)), 0.0, 1.0, fp32, 0)
    sim = cuba.Sim(p, n)
    try:
        cuba.cuba_trace_enable(sim.h, True)
        sim.set_state(st)
        keys, perm, cs, _, _ = sim.trace()
    finally:
        sim.close()
    _, okeys, operm, ocs = O.sort(op, st.astype(np.float64))
    assert np.array_equal(keys, okeys)
    assert np.array_equal(perm.astype(np.int64), operm)
    assert np.array_equal(cs.astype(np.int64), ocs)


@pytest.mark.parametrize("fp32", [False, True])
def test_neighbour_sort_sparse_cells(fp32):
    """Three small dense boxes in a 16x16x12 grid (most cells empty): five
    steps in one call through the neighbour-move sort, whose count pass reads
    each particle's old cell off cell_start across the empty cells.  The
    stable order, keys and cell_start of the last step equal the oracle's;
    FP64 with collisions (positions to 1e-12 fm), FP32 without (sigma = 0:
    streaming and sorting only, positions bit-exact)."""
    L = (1.6, 1.6, 1.2)
    regs = [((0.0, 0.0, 0.0), (0.3, 0.3, 0.3), 0.4), ((1.0, 1.2, 0.5), (1.3, 1.5, 0.8), 0.5),
            ((0.7, 0.1, 0.9), (0.9, 0.3, 1.2), 0.3)]
    st0 = W.thermal_state(20000, regs, seed=61)
    sigma = 0.0 if fp32 else 0.002
    p, op = _pair(L, (16, 16, 12), 0.06, sigma, 5.0, fp32, 67)
    dtype = np.float32 if fp32 else np.float64
    st0 = st0.astype(dtype)
    sim = cuba.Sim(p, st0.shape[1])
    try:
        sim.set_state(st0)
        sim.step(4)
        cuba.cuba_trace_enable(sim.h, True)
        sim.step(1)
        g = sim.get_state()
        keys, perm, cs, pairs, exe = sim.trace()
        stats = sim.stats()
    finally:
        sim.close()
    o, _, _, _ = O.sort(op, st0.astype(np.float64))
    refl = 0
    for k in range(4):
        o, r = O.step(op, k, o)
        refl += r.n_reflections
    o, res = O.step(op, 4, o)
    refl += res.n_reflections
    assert np.array_equal(keys, res.keys.astype(np.uint32))
    assert np.array_equal(perm.astype(np.int64), res.perm)
    assert np.array_equal(cs.astype(np.int64), res.cell_start)
    assert int(np.count_nonzero(np.diff(res.cell_start) == 0)) > 1000  # most cells are empty
    assert stats["reflections"] == refl
    if fp32:
        assert np.array_equal(g[:3].astype(np.float64), o[:3])
    else:
        assert np.max(np.abs(g[:3] - o[:3])) <= 1e-12
        E = np.sqrt((o[3:] ** 2).sum(axis=0))
        assert np.max(np.abs(g[3:] - o[3:]).max(axis=0) / E) <= 1e-10
        assert stats["executed"] > 0
