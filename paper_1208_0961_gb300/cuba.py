"""Python binding of the C ABI in ``include/cuba.h`` (argument marshalling only).

Every entry point keeps its C name.  Device buffers are torch tensors (their
``data_ptr()`` is passed through); streams are torch CUDA streams.  All work
runs in ``libcuba.so``; if the library cannot be loaded the import of this
module's functions raises — there is no other implementation behind them.

Units: fm, fm/c, GeV; cross sections in fm^2 (1 mb = 0.1 fm^2).
"""
import ctypes as C
import os

from . import _build

CUBA_OK = 0
CUBA_ERR_INVALID = -1
CUBA_ERR_OOM = -2
CUBA_ERR_CUDA = -3
CUBA_ERR_OVERFLOW = -4
CUBA_ERR_P22 = -5
CUBA_ERR_CAPACITY = -6
CUBA_FP32 = 0
CUBA_FP64 = 1
CUBA_ACCEPT_ALL_PAIRS = 0
CUBA_ACCEPT_SKIP = 1

FM2_PER_MB = 0.1


class cuba_params(C.Structure):
    _fields_ = [
        ("L", C.c_double * 3),
        ("n_cells", C.c_int32 * 3),
        ("dt", C.c_double),
        ("sigma_fm2", C.c_double),
        ("n_test", C.c_double),
        ("precision", C.c_int32),
        ("seed", C.c_uint64),
        ("gamma_fp64", C.c_double),
        ("acceptance", C.c_int32),
        ("kappa", C.c_double),
        ("mass", C.c_double),
        ("mu", C.c_double),
    ]


class cuba_region(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3), ("T", C.c_double)]


class cuba_counters(C.Structure):
    _fields_ = [(name, C.c_int64) for name in
                ("steps", "pair_tests", "accepted", "executed", "reflections", "fp64_boosts", "overflow",
                 "candidates")]


class cuba_batch_config(C.Structure):
    _fields_ = [("precision", C.c_int32), ("max_sims", C.c_int32), ("max_particles", C.c_int64),
                ("max_cells", C.c_int64)]


class cuba_launch_shape(C.Structure):
    _fields_ = [("small_max", C.c_int32), ("small_blocks", C.c_int32), ("tile_blocks", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class cuba_allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("free", FREE_FN), ("ctx", C.c_void_p)]


class CubaError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("cuba error %d: %s" % (code, msg))
        self.code = code


_lib = None


def library_path():
    return _build.LIB


def load(build_if_missing=True):
    """Load libcuba.so (building it first if asked and missing)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and not os.path.exists(path):
        _build.build()
    if not os.path.exists(path):
        raise ImportError("libcuba.so is not built (run __graft_entry__.build())")
    L = C.CDLL(path)
    vp = C.c_void_p
    i64p = C.POINTER(C.c_int64)
    u32p = C.POINTER(C.c_uint32)
    sig = {
        "cuba_create": (C.c_int, [C.POINTER(cuba_params), C.c_int64, C.POINTER(vp)]),
        "cuba_destroy": (None, [vp]),
        "cuba_init_thermal": (C.c_int, [vp, C.c_int64, C.POINTER(cuba_region), C.c_int, vp]),
        "cuba_init_riemann": (C.c_int, [vp, C.c_int64, C.c_double, C.c_double, vp]),
        "cuba_init_hotspot": (C.c_int, [vp, C.c_int64, C.c_double, C.c_double, C.c_double, vp]),
        "cuba_set_state": (C.c_int, [vp, vp, C.c_int64, vp]),
        "cuba_get_state": (C.c_int, [vp, vp, vp]),
        "cuba_sizes": (C.c_int, [vp, i64p, i64p]),
        "cuba_get_step": (C.c_int, [vp, u32p]),
        "cuba_set_step": (C.c_int, [vp, C.c_uint32]),
        "cuba_get_time": (C.c_int, [vp, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "cuba_step": (C.c_int, [vp, C.c_int, vp]),
        "cuba_observables": (C.c_int, [vp, vp, vp, vp, vp]),
        "cuba_totals": (C.c_int, [vp, C.POINTER(C.c_double), i64p, vp]),
        "cuba_stats": (C.c_int, [vp, C.POINTER(cuba_counters)]),
        "cuba_last_error": (C.c_char_p, []),
        "cuba_trace_enable": (C.c_int, [vp, C.c_int]),
        "cuba_trace_get": (C.c_int, [vp, vp, vp, vp, vp, vp, C.c_int64, i64p]),
        "cuba_philox": (C.c_int, [vp, C.c_int64, C.c_uint64, vp, vp]),
        "cuba_step_profiled": (C.c_int, [vp, C.c_int, C.POINTER(C.c_double), vp]),
        "cuba_bin_noalloc": (C.c_int, [C.POINTER(cuba_params), vp, C.c_int64, vp, vp, vp]),
        "cuba_batch_create": (C.c_int, [C.POINTER(cuba_batch_config), C.POINTER(vp)]),
        "cuba_create_with_allocator": (C.c_int, [C.POINTER(cuba_params), C.c_int64, C.POINTER(cuba_allocator),
                                                 C.POINTER(vp)]),
        "cuba_batch_create_with_allocator": (C.c_int, [C.POINTER(cuba_batch_config), C.POINTER(cuba_allocator),
                                                       C.POINTER(vp)]),
        "cuba_sim_bytes": (C.c_int64, [C.POINTER(cuba_params), C.c_int64]),
        "cuba_batch_destroy": (None, [vp]),
        "cuba_batch_add": (C.c_int, [vp, C.POINTER(cuba_params), C.c_int64, C.POINTER(cuba_region), C.c_int,
                                     C.POINTER(C.c_int32), vp]),
        "cuba_batch_add_state": (C.c_int, [vp, C.POINTER(cuba_params), vp, C.c_int64, C.POINTER(C.c_int32), vp]),
        "cuba_batch_remove": (C.c_int, [vp, C.c_int32]),
        "cuba_batch_step": (C.c_int, [vp, C.c_int, vp]),
        "cuba_batch_observables": (C.c_int, [vp, C.c_int32, vp, vp, vp, vp]),
        "cuba_batch_totals": (C.c_int, [vp, C.c_int32, C.POINTER(C.c_double), i64p, vp]),
        "cuba_batch_stats": (C.c_int, [vp, C.c_int32, C.POINTER(cuba_counters)]),
        "cuba_batch_get_state": (C.c_int, [vp, C.c_int32, vp, vp]),
        "cuba_batch_get_step": (C.c_int, [vp, C.c_int32, u32p]),
        "cuba_batch_get_time": (C.c_int, [vp, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
        "cuba_batch_usage": (C.c_int, [vp, C.POINTER(C.c_int32), i64p, i64p]),
        "cuba_batch_bytes": (C.c_int64, [C.POINTER(cuba_batch_config)]),
        "cuba_kinematics_fp32": (C.c_int, [vp, C.c_int64, C.c_uint64, C.c_uint32, C.c_double, vp, vp, vp]),
        "cuba_set_small_max": (C.c_int, [vp, C.c_int32]),
        "cuba_get_small_max": (C.c_int, [vp, C.POINTER(C.c_int32)]),
        "cuba_autotune": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_double), vp]),
        "cuba_batch_autotune": (C.c_int, [vp, C.c_int, C.POINTER(C.c_int32), C.POINTER(C.c_double), vp]),
        "cuba_set_launch_shape": (C.c_int, [vp, C.POINTER(cuba_launch_shape)]),
        "cuba_get_launch_shape": (C.c_int, [vp, C.POINTER(cuba_launch_shape)]),
        "cuba_autotune_shape": (C.c_int, [vp, C.c_int, C.POINTER(cuba_launch_shape), C.POINTER(C.c_double), vp]),
        "cuba_batch_set_launch_shape": (C.c_int, [vp, C.POINTER(cuba_launch_shape)]),
        "cuba_batch_get_launch_shape": (C.c_int, [vp, C.POINTER(cuba_launch_shape)]),
        "cuba_batch_autotune_shape": (C.c_int, [vp, C.c_int, C.POINTER(cuba_launch_shape), C.POINTER(C.c_double),
                                                vp]),
        "cuba_batch_set_small_max": (C.c_int, [vp, C.c_int32]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def _check(rc):
    if rc != CUBA_OK:
        msg = load().cuba_last_error()
        raise CubaError(rc, msg.decode() if msg else "")
    return rc


def _stream_ptr(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def _ptr(x):
    """Raw address of a torch tensor or numpy array (or None)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return C.c_void_p(x.data_ptr())
    if hasattr(x, "ctypes"):
        return C.c_void_p(x.ctypes.data)
    return C.c_void_p(int(x))


def make_params(L=(10.0, 1.0, 1.0), n_cells=(100, 1, 1), dt=0.05, sigma_fm2=1.0, n_test=1.0,
                precision=CUBA_FP64, seed=0, gamma_fp64=0.0, acceptance=0, kappa=0.0, mass=0.0, mu=0.0):
    p = cuba_params()
    for a in range(3):
        p.L[a] = float(L[a])
        p.n_cells[a] = int(n_cells[a])
    p.dt = float(dt)
    p.sigma_fm2 = float(sigma_fm2)
    p.n_test = float(n_test)
    p.precision = int(precision)
    p.seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    p.gamma_fp64 = float(gamma_fp64)
    p.acceptance = int(acceptance)
    p.kappa = float(kappa)
    p.mass = float(mass)
    p.mu = float(mu)
    return p


def make_regions(regions):
    regions = list(regions)
    arr = (cuba_region * len(regions))()
    for k, (lo, hi, T) in enumerate(regions):
        for a in range(3):
            arr[k].lo[a] = float(lo[a])
            arr[k].hi[a] = float(hi[a])
        arr[k].T = float(T)
    return arr


# ---- thin wrappers with the C names ------------------------------------------

def cuba_create(params, max_particles):
    h = C.c_void_p()
    _check(load().cuba_create(C.byref(params), int(max_particles), C.byref(h)))
    return h


def cuba_create_with_allocator(params, max_particles, allocator):
    """allocator: a DeviceAllocator (its C struct must outlive the handle)."""
    h = C.c_void_p()
    _check(load().cuba_create_with_allocator(C.byref(params), int(max_particles), C.byref(allocator.c_struct),
                                             C.byref(h)))
    return h


def cuba_sim_bytes(params, max_particles):
    return int(load().cuba_sim_bytes(C.byref(params), int(max_particles)))


class DeviceAllocator:
    """A cuba_allocator whose callbacks are Python callables:
    alloc(nbytes) -> device address (int, 256-byte aligned) or 0, and
    free(address, nbytes).  Keeps the ctypes callbacks alive and counts the
    bytes handed out (live_bytes, peak_bytes, calls)."""

    def __init__(self, alloc, free):
        self._alloc, self._free = alloc, free
        self.live = {}
        self.live_bytes = 0
        self.peak_bytes = 0
        self.calls = 0

        def _a(nbytes, _ctx):
            ptr = int(self._alloc(int(nbytes)) or 0)
            if ptr:
                self.live[ptr] = int(nbytes)
                self.live_bytes += int(nbytes)
                self.peak_bytes = max(self.peak_bytes, self.live_bytes)
                self.calls += 1
            return ptr

        def _f(ptr, nbytes, _ctx):
            self.live_bytes -= self.live.pop(int(ptr), 0)
            self._free(int(ptr), int(nbytes))

        self._cb_alloc = ALLOC_FN(_a)
        self._cb_free = FREE_FN(_f)
        self.c_struct = cuba_allocator(self._cb_alloc, self._cb_free, None)


def torch_allocator(device=None):
    """Device memory from PyTorch's caching allocator: freed blocks return to
    torch's cache, so the library's HBM counts against what torch manages."""
    import torch
    dev = torch.cuda.current_device() if device is None else device
    return DeviceAllocator(lambda n: torch.cuda.caching_allocator_alloc(n, dev),
                           lambda ptr, n: torch.cuda.caching_allocator_delete(ptr))


def cuba_destroy(sim):
    load().cuba_destroy(sim)


def cuba_init_thermal(sim, n, regions, stream=None):
    R = make_regions(regions)
    _check(load().cuba_init_thermal(sim, int(n), R, len(R), _stream_ptr(stream)))


def cuba_init_riemann(sim, n, T_left, T_right, stream=None):
    _check(load().cuba_init_riemann(sim, int(n), float(T_left), float(T_right), _stream_ptr(stream)))


def cuba_init_hotspot(sim, n, T0, dT, width, stream=None):
    _check(load().cuba_init_hotspot(sim, int(n), float(T0), float(dT), float(width), _stream_ptr(stream)))


def cuba_set_state(sim, soa, n, stream=None):
    _check(load().cuba_set_state(sim, _ptr(soa), int(n), _stream_ptr(stream)))


def cuba_get_state(sim, out, stream=None):
    _check(load().cuba_get_state(sim, _ptr(out), _stream_ptr(stream)))


def cuba_sizes(sim):
    n = C.c_int64()
    c = C.c_int64()
    _check(load().cuba_sizes(sim, C.byref(n), C.byref(c)))
    return n.value, c.value


def cuba_get_step(sim):
    s = C.c_uint32()
    _check(load().cuba_get_step(sim, C.byref(s)))
    return s.value


def cuba_get_time(sim):
    """(simulated time, dt of the last step)."""
    t = C.c_double()
    dt = C.c_double()
    _check(load().cuba_get_time(sim, C.byref(t), C.byref(dt)))
    return t.value, dt.value


def cuba_set_step(sim, step):
    _check(load().cuba_set_step(sim, int(step)))


def cuba_step(sim, n_steps, stream=None):
    _check(load().cuba_step(sim, int(n_steps), _stream_ptr(stream)))


def cuba_step_profiled(sim, n_steps, stream=None):
    """Per-phase device milliseconds summed over n_steps (see include/cuba.h)."""
    out = (C.c_double * 6)()
    _check(load().cuba_step_profiled(sim, int(n_steps), out, _stream_ptr(stream)))
    return list(out)


def cuba_observables(sim, T00=None, T0x=None, counts=None, stream=None):
    _check(load().cuba_observables(sim, _ptr(T00), _ptr(T0x), _ptr(counts), _stream_ptr(stream)))


def cuba_totals(sim, stream=None):
    out = (C.c_double * 4)()
    n = C.c_int64()
    _check(load().cuba_totals(sim, out, C.byref(n), _stream_ptr(stream)))
    return list(out), n.value


def cuba_stats(sim):
    c = cuba_counters()
    _check(load().cuba_stats(sim, C.byref(c)))
    return {name: getattr(c, name) for name, _ in cuba_counters._fields_}


def cuba_trace_enable(sim, on=True):
    _check(load().cuba_trace_enable(sim, 1 if on else 0))


def cuba_trace_get(sim, keys=None, perm=None, cell_start=None, pairs=None, executed=None, cap=0):
    n = C.c_int64()
    _check(load().cuba_trace_get(sim, _ptr(keys), _ptr(perm), _ptr(cell_start), _ptr(pairs), _ptr(executed),
                                 int(cap), C.byref(n)))
    return n.value


def cuba_philox(ctr, n, key, out, stream=None):
    _check(load().cuba_philox(_ptr(ctr), int(n), int(key) & 0xFFFFFFFFFFFFFFFF, _ptr(out), _stream_ptr(stream)))


CUBA_NOALLOC_MAX_PARTICLES = 1 << 18


def cuba_bin_noalloc(params, xyz, n, perm, cell_start, stream=None):
    """Cell keys and stable sort of device positions into caller buffers,
    with no allocation inside the library (see include/cuba.h)."""
    _check(load().cuba_bin_noalloc(C.byref(params), _ptr(xyz), int(n), _ptr(perm), _ptr(cell_start),
                                   _stream_ptr(stream)))


# ---- launch shape and autotuner ---------------------------------------------

TUNE_CANDIDATES = (0, 16, 32, 64, 128, 256, 512, 1024)


def cuba_set_small_max(sim, v):
    _check(load().cuba_set_small_max(sim, int(v)))


def cuba_get_small_max(sim):
    v = C.c_int32()
    _check(load().cuba_get_small_max(sim, C.byref(v)))
    return v.value


SHAPE_CANDIDATES = tuple("small_max=%d" % v for v in TUNE_CANDIDATES) + (
    "small_blocks=1", "small_blocks=2", "tile_blocks=2", "tile_blocks=4", "tile_blocks=8")


def _shape_dict(sh):
    return {"small_max": sh.small_max, "small_blocks": sh.small_blocks, "tile_blocks": sh.tile_blocks}


def cuba_set_launch_shape(sim, small_max, small_blocks=2, tile_blocks=4):
    sh = cuba_launch_shape(int(small_max), int(small_blocks), int(tile_blocks))
    _check(load().cuba_set_launch_shape(sim, C.byref(sh)))


def cuba_get_launch_shape(sim):
    sh = cuba_launch_shape()
    _check(load().cuba_get_launch_shape(sim, C.byref(sh)))
    return _shape_dict(sh)


def cuba_autotune_shape(sim, n_steps=2, stream=None):
    """Tune small_max, then the small-cell and the item kernel's blocks per
    iteration; returns (shape dict, {candidate: ms per step})."""
    sh = cuba_launch_shape()
    ms = (C.c_double * len(SHAPE_CANDIDATES))()
    _check(load().cuba_autotune_shape(sim, int(n_steps), C.byref(sh), ms, _stream_ptr(stream)))
    return _shape_dict(sh), dict(zip(SHAPE_CANDIDATES, list(ms)))


def cuba_batch_autotune_shape(b, n_steps=2, stream=None):
    sh = cuba_launch_shape()
    ms = (C.c_double * len(SHAPE_CANDIDATES))()
    _check(load().cuba_batch_autotune_shape(b, int(n_steps), C.byref(sh), ms, _stream_ptr(stream)))
    return _shape_dict(sh), dict(zip(SHAPE_CANDIDATES, list(ms)))


def cuba_autotune(sim, n_steps=2, stream=None):
    """Returns (chosen small_max, {candidate: ms per step})."""
    v = C.c_int32()
    ms = (C.c_double * len(TUNE_CANDIDATES))()
    _check(load().cuba_autotune(sim, int(n_steps), C.byref(v), ms, _stream_ptr(stream)))
    return v.value, dict(zip(TUNE_CANDIDATES, list(ms)))


def cuba_batch_autotune(b, n_steps=2, stream=None):
    v = C.c_int32()
    ms = (C.c_double * len(TUNE_CANDIDATES))()
    _check(load().cuba_batch_autotune(b, int(n_steps), C.byref(v), ms, _stream_ptr(stream)))
    return v.value, dict(zip(TUNE_CANDIDATES, list(ms)))


def cuba_batch_set_small_max(b, v):
    _check(load().cuba_batch_set_small_max(b, int(v)))


# ---- batches ---------------------------------------------------------------

def make_batch_config(precision=CUBA_FP32, max_sims=16, max_particles=1 << 20, max_cells=1 << 16):
    c = cuba_batch_config()
    c.precision = int(precision)
    c.max_sims = int(max_sims)
    c.max_particles = int(max_particles)
    c.max_cells = int(max_cells)
    return c


def cuba_batch_create(cfg):
    h = C.c_void_p()
    _check(load().cuba_batch_create(C.byref(cfg), C.byref(h)))
    return h


def cuba_batch_create_with_allocator(cfg, allocator):
    h = C.c_void_p()
    _check(load().cuba_batch_create_with_allocator(C.byref(cfg), C.byref(allocator.c_struct), C.byref(h)))
    return h


def cuba_batch_destroy(b):
    load().cuba_batch_destroy(b)


def cuba_batch_add(b, params, n, regions, stream=None):
    R = make_regions(regions)
    i = C.c_int32()
    _check(load().cuba_batch_add(b, C.byref(params), int(n), R, len(R), C.byref(i), _stream_ptr(stream)))
    return i.value


def cuba_batch_add_state(b, params, soa, n, stream=None):
    i = C.c_int32()
    _check(load().cuba_batch_add_state(b, C.byref(params), _ptr(soa), int(n), C.byref(i), _stream_ptr(stream)))
    return i.value


def cuba_batch_remove(b, sim_id):
    _check(load().cuba_batch_remove(b, int(sim_id)))


def cuba_batch_step(b, n_steps, stream=None):
    _check(load().cuba_batch_step(b, int(n_steps), _stream_ptr(stream)))


def cuba_batch_observables(b, sim_id, T00=None, T0x=None, counts=None, stream=None):
    _check(load().cuba_batch_observables(b, int(sim_id), _ptr(T00), _ptr(T0x), _ptr(counts), _stream_ptr(stream)))


def cuba_batch_totals(b, sim_id, stream=None):
    out = (C.c_double * 4)()
    n = C.c_int64()
    _check(load().cuba_batch_totals(b, int(sim_id), out, C.byref(n), _stream_ptr(stream)))
    return list(out), n.value


def cuba_batch_stats(b, sim_id):
    c = cuba_counters()
    _check(load().cuba_batch_stats(b, int(sim_id), C.byref(c)))
    return {name: getattr(c, name) for name, _ in cuba_counters._fields_}


def cuba_batch_get_state(b, sim_id, out, stream=None):
    _check(load().cuba_batch_get_state(b, int(sim_id), _ptr(out), _stream_ptr(stream)))


def cuba_batch_get_time(b, sim_id):
    t = C.c_double()
    dt = C.c_double()
    _check(load().cuba_batch_get_time(b, int(sim_id), C.byref(t), C.byref(dt)))
    return t.value, dt.value


def cuba_batch_get_step(b, sim_id):
    s = C.c_uint32()
    _check(load().cuba_batch_get_step(b, int(sim_id), C.byref(s)))
    return s.value


def cuba_batch_usage(b):
    n = C.c_int32()
    p = C.c_int64()
    c = C.c_int64()
    _check(load().cuba_batch_usage(b, C.byref(n), C.byref(p), C.byref(c)))
    return n.value, p.value, c.value


def cuba_batch_bytes(cfg):
    return int(load().cuba_batch_bytes(C.byref(cfg)))


class Batch:
    """Owns one batch handle; members are addressed by the ids cuba returns."""

    def __init__(self, cfg, allocator=None):
        self.cfg = cfg
        self.allocator = allocator
        self.h = cuba_batch_create(cfg) if allocator is None else cuba_batch_create_with_allocator(cfg, allocator)
        self.dtype = "float64" if cfg.precision == CUBA_FP64 else "float32"
        self.members = {}

    def close(self):
        if self.h:
            cuba_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add(self, params, n, regions, stream=None):
        i = cuba_batch_add(self.h, params, n, regions, stream)
        self.members[i] = params
        return i

    def add_state(self, params, st, stream=None):
        import numpy as np
        st = np.ascontiguousarray(st, dtype=self.dtype)
        i = cuba_batch_add_state(self.h, params, st, st.shape[1], stream)
        self.members[i] = params
        return i

    def remove(self, sim_id):
        cuba_batch_remove(self.h, sim_id)
        self.members.pop(sim_id, None)

    def step(self, n_steps=1, stream=None):
        cuba_batch_step(self.h, n_steps, stream)

    def n_cells(self, sim_id):
        p = self.members[sim_id]
        return p.n_cells[0] * p.n_cells[1] * p.n_cells[2]

    def observables(self, sim_id, stream=None):
        import numpy as np
        nc = self.n_cells(sim_id)
        T00 = np.zeros(nc)
        T0x = np.zeros(nc)
        cnt = np.zeros(nc, dtype=np.int32)
        cuba_batch_observables(self.h, sim_id, T00, T0x, cnt, stream)
        return T00, T0x, cnt

    def totals(self, sim_id, stream=None):
        return cuba_batch_totals(self.h, sim_id, stream)

    def stats(self, sim_id):
        return cuba_batch_stats(self.h, sim_id)

    def get_state(self, sim_id, stream=None):
        import numpy as np
        n = self.totals(sim_id)[1]
        out = np.zeros((6, n), dtype=self.dtype)
        cuba_batch_get_state(self.h, sim_id, out, stream)
        return out

    def get_step(self, sim_id):
        return cuba_batch_get_step(self.h, sim_id)

    def get_time(self, sim_id):
        return cuba_batch_get_time(self.h, sim_id)

    def usage(self):
        return cuba_batch_usage(self.h)


def cuba_kinematics_fp32(pin, npairs, key, step, gamma_fp64, pout, used_fp64, stream=None):
    _check(load().cuba_kinematics_fp32(_ptr(pin), int(npairs), int(key) & 0xFFFFFFFFFFFFFFFF, int(step),
                                       float(gamma_fp64), _ptr(pout), _ptr(used_fp64), _stream_ptr(stream)))


def cuba_last_error():
    return load().cuba_last_error().decode()


# ---- a small object wrapper -------------------------------------------------

class Sim:
    """Owns one simulation handle; state exchange via numpy (host) arrays."""

    def __init__(self, params, max_particles, allocator=None):
        self.params = params
        self.allocator = allocator
        self.h = (cuba_create(params, max_particles) if allocator is None
                  else cuba_create_with_allocator(params, max_particles, allocator))
        self.dtype = "float64" if params.precision == CUBA_FP64 else "float32"

    def close(self):
        if self.h:
            cuba_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n_cells(self):
        return cuba_sizes(self.h)[1]

    @property
    def n(self):
        return cuba_sizes(self.h)[0]

    def init_thermal(self, n, regions, stream=None):
        cuba_init_thermal(self.h, n, regions, stream)

    def init_riemann(self, n, T_left, T_right, stream=None):
        cuba_init_riemann(self.h, n, T_left, T_right, stream)

    def init_hotspot(self, n, T0, dT, width, stream=None):
        cuba_init_hotspot(self.h, n, T0, dT, width, stream)

    def set_state(self, st, stream=None):
        import numpy as np
        st = np.ascontiguousarray(st, dtype=self.dtype)
        cuba_set_state(self.h, st, st.shape[1], stream)

    def get_state(self, stream=None):
        import numpy as np
        out = np.zeros((6, self.n), dtype=self.dtype)
        cuba_get_state(self.h, out, stream)
        return out

    def step(self, n_steps=1, stream=None):
        cuba_step(self.h, n_steps, stream)

    def time(self):
        return cuba_get_time(self.h)

    def observables(self, stream=None):
        import numpy as np
        nc = self.n_cells
        T00 = np.zeros(nc)
        T0x = np.zeros(nc)
        cnt = np.zeros(nc, dtype=np.int32)
        cuba_observables(self.h, T00, T0x, cnt, stream)
        return T00, T0x, cnt

    def totals(self, stream=None):
        return cuba_totals(self.h, stream)

    def stats(self):
        return cuba_stats(self.h)

    def trace(self):
        import numpy as np
        n, nc = cuba_sizes(self.h)
        keys = np.zeros(n, dtype=np.uint32)
        perm = np.zeros(n, dtype=np.uint32)
        cs = np.zeros(nc + 1, dtype=np.uint32)
        total = cuba_trace_get(self.h, keys, perm, cs, None, None, 0)
        pairs = np.zeros((max(total, 1), 3), dtype=np.uint32)
        exe = np.zeros(max(total, 1), dtype=np.uint8)
        cuba_trace_get(self.h, None, None, None, pairs, exe, total)
        return keys, perm, cs, pairs[:total], exe[:total].astype(bool)
