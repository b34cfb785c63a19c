"""ctypes wrapper of the CPU oracle (``cuba_oracle.c``).

Test infrastructure only: the test suite, the smoke check and the CPU baseline
leg of the benchmark call it; the product path never does.  Everything here is
argument marshalling; the arithmetic is in the C file, which follows the
paper's Eq. 2 (streaming), Eq. 3 (P22) and Sec. 2 (reflection, CM kinematics).

State arrays are float64 numpy arrays of shape (6, n): rows x, y, z, px, py, pz.
"""
import ctypes as C
import math

import numpy as np

from . import build as _build

HBARC_GEV_FM = 0.1973269804   # hbar c in GeV fm
FM2_PER_MB = 0.1              # 1 mb = 0.1 fm^2


class Params(C.Structure):
    _fields_ = [
        ("L", C.c_double * 3),
        ("n", C.c_int32 * 3),
        ("dt", C.c_double),
        ("sigma", C.c_double),
        ("n_test", C.c_double),
        ("fp32", C.c_int32),
        ("key", C.c_uint32 * 2),
        ("skip", C.c_int32),
        ("kappa", C.c_double),
        ("mass", C.c_double),
        ("mu", C.c_double),
    ]


class Region(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3), ("T", C.c_double)]


class Trace(C.Structure):
    _fields_ = [
        ("keys", C.POINTER(C.c_uint32)),
        ("perm", C.POINTER(C.c_int64)),
        ("cell_start", C.POINTER(C.c_int64)),
        ("acc", C.POINTER(C.c_uint32)),
        ("acc_cap", C.c_int64),
        ("n_acc", C.c_int64),
        ("exe", C.POINTER(C.c_uint32)),
        ("exe_cap", C.c_int64),
        ("n_exe", C.c_int64),
        ("n_reflections", C.c_int64),
        ("n_pairs_tested", C.c_int64),
        ("n_candidates", C.c_int64),
        ("dt", C.c_double),
    ]


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        dp = C.POINTER(C.c_double)
        u32p = C.POINTER(C.c_uint32)
        i64p = C.POINTER(C.c_int64)
        L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
        L.orc_philox4x32_10.restype = None
        L.orc_p22_scale.argtypes = [C.POINTER(Params)]
        L.orc_p22_scale.restype = C.c_double
        L.orc_ncells.argtypes = [C.POINTER(Params)]
        L.orc_ncells.restype = C.c_int64
        L.orc_region_counts.argtypes = [C.c_int64, C.POINTER(Region), C.c_int, i64p]
        L.orc_region_counts.restype = C.c_int
        L.orc_init_thermal.argtypes = [C.POINTER(Params), C.c_int64, C.POINTER(Region), C.c_int, dp]
        L.orc_init_thermal.restype = C.c_int
        L.orc_init_hotspot.argtypes = [C.POINTER(Params), C.c_int64, C.c_double, C.c_double, C.c_double, dp]
        L.orc_init_hotspot.restype = C.c_int
        L.orc_keys.argtypes = [C.POINTER(Params), C.c_int64, dp, u32p]
        L.orc_keys.restype = C.c_int
        L.orc_sort.argtypes = [C.POINTER(Params), C.c_int64, dp, u32p, i64p, i64p]
        L.orc_sort.restype = C.c_int
        L.orc_pair_word.argtypes = [u32p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32]
        L.orc_pair_word.restype = C.c_uint32
        L.orc_kinematics.argtypes = [u32p, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32, dp, dp]
        L.orc_kinematics.restype = C.c_int
        L.orc_kinematics_ex.argtypes = [u32p, C.c_double, C.c_double, C.c_uint32, C.c_uint32, C.c_uint32,
                                        C.c_uint32, dp, dp]
        L.orc_kinematics_ex.restype = C.c_int
        L.orc_cell_accept.argtypes = [C.POINTER(Params), C.c_uint32, C.c_uint32, C.c_int64,
                                      dp, dp, dp, u32p, C.c_int64]
        L.orc_cell_accept.restype = C.c_int64
        L.orc_row_accept.argtypes = [C.POINTER(Params), C.c_uint32, C.c_uint32, C.c_int64,
                                     C.c_int64, C.c_int64, C.c_int64, dp, dp, dp, u32p, C.c_int64]
        L.orc_row_accept.restype = C.c_int64
        L.orc_step.argtypes = [C.POINTER(Params), C.c_uint32, C.c_int64, dp, C.POINTER(Trace)]
        L.orc_step.restype = C.c_int
        L.orc_observables.argtypes = [C.POINTER(Params), C.c_int64, dp, i64p, dp, dp,
                                      C.POINTER(C.c_int32)]
        L.orc_observables.restype = C.c_int
        L.orc_totals.argtypes = [C.c_int64, dp, C.c_double, dp]
        L.orc_totals.restype = None
        u64p = C.POINTER(C.c_uint64)
        L.orc_skip_table.argtypes = [C.c_double, u64p, u64p]
        L.orc_skip_table.restype = C.c_int
        L.orc_skip_gap.argtypes = [u64p, C.c_uint64, C.c_uint64]
        L.orc_skip_gap.restype = C.c_uint64
        L.orc_adaptive_dt.argtypes = [C.POINTER(Params), C.c_int64]
        L.orc_adaptive_dt.restype = C.c_double
        L.orc_threads.argtypes = []
        L.orc_threads.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_set_threads.restype = None
        _lib = L
    return _lib


def _ptr(a, ct):
    return a.ctypes.data_as(C.POINTER(ct))


def make_params(L=(10.0, 1.0, 1.0), n=(100, 1, 1), dt=0.05, sigma_fm2=1.0, n_test=1.0,
                fp32=False, seed=0, skip=False, kappa=0.0, mass=0.0, mu=0.0):
    p = Params()
    for a in range(3):
        p.L[a] = float(L[a])
        p.n[a] = int(n[a])
    p.dt = float(dt)
    p.sigma = float(sigma_fm2)
    p.n_test = float(n_test)
    p.fp32 = 1 if fp32 else 0
    p.key[0] = int(seed) & 0xFFFFFFFF
    p.key[1] = (int(seed) >> 32) & 0xFFFFFFFF
    p.skip = 1 if skip else 0
    p.kappa = float(kappa)
    p.mass = float(mass)
    p.mu = float(mu)
    return p


def make_regions(regions):
    """regions: iterable of (lo[3], hi[3], T)."""
    regions = list(regions)
    arr = (Region * len(regions))()
    for k, (lo, hi, T) in enumerate(regions):
        for a in range(3):
            arr[k].lo[a] = float(lo[a])
            arr[k].hi[a] = float(hi[a])
        arr[k].T = float(T)
    return arr


def riemann_regions(L, T_left, T_right):
    """Left and right halves of the box along x (the 1D Riemann problem)."""
    half = 0.5 * L[0]
    return [((0.0, 0.0, 0.0), (half, L[1], L[2]), T_left),
            ((half, 0.0, 0.0), (L[0], L[1], L[2]), T_right)]


def philox(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().orc_philox4x32_10(_ptr(c, C.c_uint32), _ptr(k, C.c_uint32), _ptr(out, C.c_uint32))
    return out


def p22_scale(p):
    return lib().orc_p22_scale(C.byref(p))


def ncells(p):
    return int(lib().orc_ncells(C.byref(p)))


def region_counts(n, regions):
    R = make_regions(regions)
    out = np.zeros(len(R), dtype=np.int64)
    rc = lib().orc_region_counts(int(n), R, len(R), _ptr(out, C.c_int64))
    if rc != 0:
        raise ValueError("orc_region_counts failed: %d" % rc)
    return out


def init_thermal(p, n, regions):
    """Sampled state in generation order (unsorted), shape (6, n)."""
    R = make_regions(regions)
    st = np.zeros((6, int(n)), dtype=np.float64)
    rc = lib().orc_init_thermal(C.byref(p), int(n), R, len(R), _ptr(st, C.c_double))
    if rc != 0:
        raise ValueError("orc_init_thermal failed: %d" % rc)
    return st


def init_hotspot(p, n, T0, dT, width):
    """Hot-spot state in generation order (unsorted), shape (6, n)."""
    st = np.zeros((6, int(n)), dtype=np.float64)
    rc = lib().orc_init_hotspot(C.byref(p), int(n), float(T0), float(dT), float(width), _ptr(st, C.c_double))
    if rc != 0:
        raise ValueError("orc_init_hotspot failed: %d" % rc)
    return st


def keys(p, st):
    st = np.ascontiguousarray(st, dtype=np.float64)
    n = st.shape[1]
    out = np.zeros(n, dtype=np.uint32)
    rc = lib().orc_keys(C.byref(p), n, _ptr(st, C.c_double), _ptr(out, C.c_uint32))
    if rc != 0:
        raise ValueError("orc_keys failed: %d" % rc)
    return out


def sort(p, st):
    """Stable sort by cell key. Returns (sorted state, keys, perm, cell_start)."""
    st = np.array(st, dtype=np.float64, order="C", copy=True)
    n = st.shape[1]
    k = np.zeros(n, dtype=np.uint32)
    perm = np.zeros(n, dtype=np.int64)
    cs = np.zeros(ncells(p) + 1, dtype=np.int64)
    rc = lib().orc_sort(C.byref(p), n, _ptr(st, C.c_double), _ptr(k, C.c_uint32),
                        _ptr(perm, C.c_int64), _ptr(cs, C.c_int64))
    if rc != 0:
        raise ValueError("orc_sort failed: %d" % rc)
    return st, k, perm, cs


def pair_word(key, step, cell, i, j):
    k = np.ascontiguousarray(key, dtype=np.uint32)
    return int(lib().orc_pair_word(_ptr(k, C.c_uint32), step, cell, i, j))


def kinematics(key, step, cell, i, j, pi, pj):
    k = np.ascontiguousarray(key, dtype=np.uint32)
    a = np.array(pi, dtype=np.float64)
    b = np.array(pj, dtype=np.float64)
    ok = lib().orc_kinematics(_ptr(k, C.c_uint32), step, cell, i, j, _ptr(a, C.c_double),
                              _ptr(b, C.c_double))
    return bool(ok), a, b


def adaptive_dt(p, n_max):
    """The time step the adaptive rule takes for a largest cell population n_max."""
    return float(lib().orc_adaptive_dt(C.byref(p), int(n_max)))


def skip_table(C_scale):
    """(P_fix, Q[0..32]) of the skip-ahead mode for the P22 scale C."""
    Q = np.zeros(33, dtype=np.uint64)
    pf = C.c_uint64()
    rc = lib().orc_skip_table(float(C_scale), C.byref(pf), _ptr(Q, C.c_uint64))
    if rc != 0:
        raise ValueError("orc_skip_table failed: %d" % rc)
    return int(pf.value), Q


def skip_gap(Q, U, M):
    """Geometric gap of the skip-ahead mode for the 64-bit uniform U with M
    columns left in the row (a result >= M ends the row)."""
    Q = np.ascontiguousarray(Q, dtype=np.uint64)
    return int(lib().orc_skip_gap(_ptr(Q, C.c_uint64), int(U), int(M)))


def kinematics_ex(key, mass, mu, step, cell, i, j, pi, pj):
    """Kinematics of an executed pair for any mass and angular distribution."""
    k = np.ascontiguousarray(key, dtype=np.uint32)
    a = np.array(pi, dtype=np.float64)
    b = np.array(pj, dtype=np.float64)
    ok = lib().orc_kinematics_ex(_ptr(k, C.c_uint32), float(mass), float(mu), step, cell, i, j,
                                 _ptr(a, C.c_double), _ptr(b, C.c_double))
    return bool(ok), a, b


def cell_accept(p, step, cell, mom):
    """Accepted (i, j) pairs of one cell; mom has shape (3, nc) in sorted order."""
    mom = np.ascontiguousarray(mom, dtype=np.float64)
    nc = mom.shape[1]
    cap = 1024
    while True:
        out = np.zeros(2 * cap, dtype=np.uint32)
        cnt = lib().orc_cell_accept(C.byref(p), step, cell, nc, _ptr(mom[0], C.c_double),
                                    _ptr(mom[1], C.c_double), _ptr(mom[2], C.c_double),
                                    _ptr(out, C.c_uint32), cap)
        if cnt < 0:
            raise ValueError("orc_cell_accept failed: %d" % cnt)
        if cnt <= cap:
            return out[:2 * cnt].reshape(-1, 2)
        cap = int(cnt)


def row_accept(p, step, cell, mom, i, j0, j1):
    """Accepted columns j of row i of a cell, j in [max(j0, i+1), min(j1, nc))."""
    mom = np.ascontiguousarray(mom, dtype=np.float64)
    nc = mom.shape[1]
    cap = max(16, min(1 << 16, nc))
    while True:
        out = np.zeros(cap, dtype=np.uint32)
        cnt = lib().orc_row_accept(C.byref(p), step, cell, nc, int(i), int(j0), int(j1),
                                   _ptr(mom[0], C.c_double), _ptr(mom[1], C.c_double),
                                   _ptr(mom[2], C.c_double), _ptr(out, C.c_uint32), cap)
        if cnt < 0:
            raise ValueError("orc_row_accept failed: %d" % cnt)
        if cnt <= cap:
            return out[:cnt].copy()
        cap = int(cnt)


class StepResult:
    pass


def step(p, step_index, st, trace=True):
    """One time step of a sorted state. Returns (new state, StepResult)."""
    st = np.array(st, dtype=np.float64, order="C", copy=True)
    n = st.shape[1]
    res = StepResult()
    tr = Trace()
    if trace:
        res.keys = np.zeros(n, dtype=np.uint32)
        res.perm = np.zeros(n, dtype=np.int64)
        res.cell_start = np.zeros(ncells(p) + 1, dtype=np.int64)
        cap = 1 << 16
        res._acc = np.zeros(3 * cap, dtype=np.uint32)
        res._exe = np.zeros(3 * cap, dtype=np.uint32)
        tr.keys = _ptr(res.keys, C.c_uint32)
        tr.perm = _ptr(res.perm, C.c_int64)
        tr.cell_start = _ptr(res.cell_start, C.c_int64)
        tr.acc = _ptr(res._acc, C.c_uint32)
        tr.acc_cap = cap
        tr.exe = _ptr(res._exe, C.c_uint32)
        tr.exe_cap = cap
    st_in = st.copy() if trace else None
    rc = lib().orc_step(C.byref(p), int(step_index), n, _ptr(st, C.c_double), C.byref(tr))
    if rc != 0:
        raise ValueError("orc_step failed: %d" % rc)
    if trace and (tr.n_acc > tr.acc_cap or tr.n_exe > tr.exe_cap):
        # Rerun from the saved input with room for every pair.
        cap = max(tr.n_acc, tr.n_exe)
        res._acc = np.zeros(3 * cap, dtype=np.uint32)
        res._exe = np.zeros(3 * cap, dtype=np.uint32)
        tr = Trace()
        tr.keys = _ptr(res.keys, C.c_uint32)
        tr.perm = _ptr(res.perm, C.c_int64)
        tr.cell_start = _ptr(res.cell_start, C.c_int64)
        tr.acc = _ptr(res._acc, C.c_uint32)
        tr.acc_cap = cap
        tr.exe = _ptr(res._exe, C.c_uint32)
        tr.exe_cap = cap
        st = st_in
        rc = lib().orc_step(C.byref(p), int(step_index), n, _ptr(st, C.c_double), C.byref(tr))
        if rc != 0:
            raise ValueError("orc_step failed: %d" % rc)
    res.n_acc = tr.n_acc
    res.n_exe = tr.n_exe
    res.n_reflections = tr.n_reflections
    res.n_pairs_tested = tr.n_pairs_tested
    res.n_candidates = tr.n_candidates
    res.dt = tr.dt
    if trace:
        res.accepted = res._acc[:3 * tr.n_acc].reshape(-1, 3).copy()
        res.executed = res._exe[:3 * tr.n_exe].reshape(-1, 3).copy()
        del res._acc, res._exe
    return st, res


def observables(p, st, cell_start):
    st = np.ascontiguousarray(st, dtype=np.float64)
    cs = np.ascontiguousarray(cell_start, dtype=np.int64)
    nc = ncells(p)
    T00 = np.zeros(nc)
    T0x = np.zeros(nc)
    cnt = np.zeros(nc, dtype=np.int32)
    rc = lib().orc_observables(C.byref(p), st.shape[1], _ptr(st, C.c_double), _ptr(cs, C.c_int64),
                               _ptr(T00, C.c_double), _ptr(T0x, C.c_double), _ptr(cnt, C.c_int32))
    if rc != 0:
        raise ValueError("orc_observables failed: %d" % rc)
    return T00, T0x, cnt


def totals(st, mass=0.0):
    st = np.ascontiguousarray(st, dtype=np.float64)
    out = np.zeros(4)
    lib().orc_totals(st.shape[1], _ptr(st, C.c_double), float(mass), _ptr(out, C.c_double))
    return out


def threads():
    return int(lib().orc_threads())


def set_threads(t):
    lib().orc_set_threads(int(t))


def gluon_density(T, g=16.0):
    """Boltzmann number density g T^3 / (pi^2 (hbar c)^3) in fm^-3 (T in GeV)."""
    return g * T ** 3 / (math.pi ** 2 * HBARC_GEV_FM ** 3)


def n_test_for(n_particles, regions, g=16.0):
    """Test particles per physical particle for a thermal gas filling `regions`."""
    nphys = 0.0
    for lo, hi, T in regions:
        vol = (hi[0] - lo[0]) * (hi[1] - lo[1]) * (hi[2] - lo[2])
        nphys += gluon_density(T, g) * vol
    return n_particles / nphys
