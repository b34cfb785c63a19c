"""Continuous-batching server for whole test-particle simulations.

Requests (a box, cells, dt, sigma, N_test, particle count, step count, seed and
an initial state description) arrive over time.  The server keeps every
admitted simulation's particle state resident on the device, in one batch
(`cuba_batch_*`) per cost class, admits queued requests whenever particles,
cells and member slots of their class free up (the batches are sized from an
HBM budget), advances the residents of each class together in quanta of
steps (one captured graph per step, all simulations of the class in each
launch; the classes run on their own streams and overlap on the device), and
retires a simulation when it has taken its steps: its observables (per-cell
T^00, T^0x, counts) are read back and its latency (arrival to observables on
the host) recorded.  Cost classes keep a small request from advancing at the
pace of the largest resident: each class's quantum is sized from an estimate
of its step time.

Each result is the same as the same request run alone: a simulation's random
numbers depend only on its own seed, step counter and local indices.

The scheduling logic is independent of the device: `Server` takes backend
objects (the real one wraps `cuba.Batch`) and a clock, so that it can be
tested on the CPU with a fake backend and a fake clock.
"""
import dataclasses
import math
import time
from typing import Callable, List, Optional

import numpy as np

from . import workloads as W


@dataclasses.dataclass
class Request:
    rid: int
    arrival: float             # seconds after the start of the stream
    kind: str                  # "riemann" or "thermal"
    n: int                     # test particles
    L: tuple
    n_cells: tuple
    dt: float
    sigma_fm2: float
    n_test: float
    steps: int
    regions: list              # [(lo, hi, T), ...]
    seed: int


@dataclasses.dataclass
class Result:
    rid: int
    arrival: float
    admitted: float
    finished: float
    n: int
    steps: int
    observables: Optional[tuple] = None

    @property
    def latency(self):
        return self.finished - self.arrival


def list_room(req):
    """Accepted-pair list entries the library reserves for a request's cells
    at admission (per cell mu + 8 sqrt(mu) + 16, mu = 2.0001 C n (n - 1) / 2,
    C = sigma dt / (N_test V_cell)), with each region's cells at their mean
    occupancy plus one standard deviation (Poisson)."""
    nc = req.n_cells[0] * req.n_cells[1] * req.n_cells[2]
    V = (req.L[0] / req.n_cells[0]) * (req.L[1] / req.n_cells[1]) * (req.L[2] / req.n_cells[2])
    C = req.sigma_fm2 * req.dt / (req.n_test * V)
    if C <= 0.0 or req.n == 0:
        return 0
    wsum = sum(T ** 3 * np.prod(np.subtract(hi, lo)) for lo, hi, T in req.regions)
    room = 0.0
    for lo, hi, T in req.regions:
        vol = float(np.prod(np.subtract(hi, lo)))
        cells_r = max(1.0, nc * vol / float(np.prod(req.L)))
        n_r = req.n * (T ** 3 * vol) / wsum
        occ = n_r / cells_r
        occ += math.sqrt(occ)
        mu = 2.0001 * C * occ * max(occ - 1.0, 0.0) / 2.0
        room += cells_r * (mu + 8.0 * math.sqrt(mu) + 16.0)
    return int(math.ceil(room))


# the library allocates four times the residents' list room plus 2^20 entries
LIST_FACTOR = 4
LIST_MIN_ENTRIES = 1 << 20

# ---------------------------------------------------------------------------
# Synthetic request streams (stand-ins for a real request log)
# ---------------------------------------------------------------------------

def _dt_for(dx_min, density, sigma_fm2):
    """dt = min(dx/2, 0.1 lambda) with lambda = 1 / (n sigma) (0.1 mean free
    path per step keeps the one-collision-per-step cap from distorting the
    rate); dx/2 when sigma = 0."""
    dt = 0.5 * dx_min
    if sigma_fm2 > 0.0:
        dt = min(dt, 0.1 / (density * sigma_fm2))
    return dt


def poisson_stream(n_requests=400, rate_hz=20.0, seed=7, n_min=1e4, n_max=8e6, steps_min=50, steps_max=500,
                   sigma_mb_max=100.0, T_pairs=((0.4, 0.32), (0.5, 0.3), (0.35, 0.25))):
    """Poisson arrivals; half 1D Riemann problems (cells along x, about 1000
    particles per cell, between 100 and 2000 cells), half 3D thermal boxes
    (n^3 cells of 0.1 fm with about 30 particles per cell, T = 0.4 GeV);
    particle counts log-uniform, step counts and sigma uniform."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for rid in range(n_requests):
        t += rng.exponential(1.0 / rate_hz)
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        steps = int(rng.integers(steps_min, steps_max + 1))
        sigma_fm2 = float(rng.uniform(0.0, sigma_mb_max)) * W.FM2_PER_MB
        if rng.random() < 0.5:
            cells = int(min(2000, max(100, round(n / 1000))))
            TL, TR = T_pairs[int(rng.integers(len(T_pairs)))]
            L = (10.0, 1.0, 1.0)
            regs = W.riemann_regions(L, TL, TR)
            n_test = W.n_test_for(n, regs)
            dt = _dt_for(L[0] / cells, W.gluon_density(TL), sigma_fm2)
            out.append(Request(rid, t, "riemann", n, L, (cells, 1, 1), dt, sigma_fm2, n_test, steps, regs,
                               1000 + rid))
        else:
            k = max(2, int(round((n / 30.0) ** (1.0 / 3.0))))
            L = (0.1 * k, 0.1 * k, 0.1 * k)
            regs = [((0.0, 0.0, 0.0), L, 0.4)]
            n_test = W.n_test_for(n, regs)
            dt = _dt_for(0.1, W.gluon_density(0.4), sigma_fm2)
            out.append(Request(rid, t, "thermal", n, L, (k, k, k), dt, sigma_fm2, n_test, steps, regs, 1000 + rid))
    return out


# ---------------------------------------------------------------------------
# Backends
# ---------------------------------------------------------------------------

class CudaBackend:
    """The device: one cuba batch sized from an HBM budget.

    The arena (everything the batch allocates at creation, cuba_batch_bytes)
    takes the budget minus a reserve for the accepted-pair list, which the
    library sizes from the residents' occupancy at each admission; a request
    is admitted only while the list room of all residents fits that reserve.
    """

    def __init__(self, budget_bytes, precision=None, max_sims=256, cells_per_particle=0.01, stream=None,
                 list_fraction=0.15, allocator=None, sizes=None):
        from . import cuba
        self.cuba = cuba
        precision = cuba.CUBA_FP32 if precision is None else precision
        if sizes is None:
            reserve = max(16 << 20, int(list_fraction * budget_bytes))
            self.max_particles, self.max_cells = self.size_for(cuba, precision, max_sims, budget_bytes - reserve,
                                                               cells_per_particle)
            if self.max_particles < 1:
                raise ValueError("budget of %d bytes is too small for a batch" % budget_bytes)
            self.list_entries = (reserve // 8 - LIST_MIN_ENTRIES) // LIST_FACTOR
        else:
            self.max_particles, self.max_cells, self.list_entries = sizes
        cfg = cuba.make_batch_config(precision, max_sims=max_sims, max_particles=self.max_particles,
                                     max_cells=self.max_cells)
        self.arena_bytes = cuba.cuba_batch_bytes(cfg)
        self.room_used = 0
        self._room = {}
        self.admit_s = 0.0    # host seconds in admissions (sampling and the settling sort)
        self.finish_s = 0.0   # host seconds in retirements (observables and compaction)
        self.batch = cuba.Batch(cfg, allocator=allocator)
        self.precision = precision
        self.stream = stream
        self.max_sims = max_sims

    @classmethod
    def for_request(cls, req, precision=None, stream=None, allocator=None):
        """A backend holding exactly one request (the plain one-at-a-time
        loop): its particles, its cells and its list room."""
        nc = req.n_cells[0] * req.n_cells[1] * req.n_cells[2]
        return cls(0, precision=precision, max_sims=1, stream=stream, allocator=allocator,
                   sizes=(max(1, req.n), nc, list_room(req)))

    @staticmethod
    def size_for(cuba, precision, max_sims, arena_budget, cells_per_particle):
        """Largest (max_particles, max_cells) whose batch fits arena_budget."""
        def cells(p):
            return int(min(1 << 30, max(1 << 16, p * cells_per_particle)))

        def nbytes(p):
            cfg = cuba.make_batch_config(precision, max_sims=max_sims, max_particles=p, max_cells=cells(p))
            return cuba.cuba_batch_bytes(cfg)
        lo, hi = 0, 0x7FFFFFF0
        while lo < hi:
            mid = (lo + hi + 1) // 2
            if nbytes(mid) <= arena_budget:
                lo = mid
            else:
                hi = mid - 1
        return lo, cells(lo) if lo else 0

    def fits(self, req, used_particles, used_cells, used_sims):
        nc = req.n_cells[0] * req.n_cells[1] * req.n_cells[2]
        room_used = self.room_used if used_sims else 0
        return (used_particles + req.n <= self.max_particles and used_cells + nc <= self.max_cells
                and used_sims < self.max_sims and room_used + list_room(req) <= self.list_entries)

    def admit(self, req):
        p = self.cuba.make_params(L=req.L, n_cells=req.n_cells, dt=req.dt, sigma_fm2=req.sigma_fm2,
                                  n_test=req.n_test, precision=self.precision, seed=req.seed)
        t0 = time.perf_counter()
        h = self.batch.add(p, req.n, req.regions, self.stream)
        self.admit_s += time.perf_counter() - t0
        self._room[h] = list_room(req)
        self.room_used += self._room[h]
        return h

    def step(self, k):
        self.batch.step(k, self.stream)

    def step_time(self, requests):
        """Estimated device seconds of one batch step with these residents."""
        return STEP_FIXED_S + sum(step_cost(r) for r in requests)

    def sync(self):
        if self.stream is not None:
            self.stream.synchronize()
        else:
            import torch
            torch.cuda.synchronize()

    def finish(self, handle):
        t0 = time.perf_counter()
        obs = self.batch.observables(handle, self.stream)
        self.batch.remove(handle)
        self.finish_s += time.perf_counter() - t0
        self.room_used -= self._room.pop(handle, 0)
        return obs

    def close(self):
        self.batch.close()


# ---------------------------------------------------------------------------
# Cost model and classes
# ---------------------------------------------------------------------------

# Device time of one step of a simulation, from the measured rates of the
# kernels: a fixed launch cost, HBM-bound streaming and binning per particle,
# and the all-pairs test per pair.
STEP_FIXED_S = 4e-5
STEP_PER_PARTICLE_S = 4e-11
STEP_PER_PAIR_S = 2.5e-13


def pairs_per_step(r):
    cells = r.n_cells[0] * r.n_cells[1] * r.n_cells[2]
    return 0.0 if r.sigma_fm2 <= 0.0 else 0.5 * r.n * r.n / cells


def step_cost(r):
    """Estimated device seconds one step of request r adds to a batch step."""
    return STEP_PER_PARTICLE_S * r.n + STEP_PER_PAIR_S * pairs_per_step(r)


def cost_class(r, bounds=(1e-4, 1e-3)):
    """0: steps under 0.1 ms, 1: under 1 ms, 2: larger."""
    c = step_cost(r)
    for k, b in enumerate(bounds):
        if c < b:
            return k
    return len(bounds)


# ---------------------------------------------------------------------------
# Scheduler
# ---------------------------------------------------------------------------

class Server:
    """Continuous batching over cost classes that share the device in turn.

    Requests go to the class of their estimated step cost (promoted to a
    larger class if they do not fit an empty one; rejected if they fit none).
    Each round visits the classes in order, smallest first.  A class admits
    queued requests while its backend has room and its resident limit allows
    -- in arrival order, or (order "sjf") shortest remaining work first with
    aging: a request's work is divided by 1 + waiting time / aging_s, so a
    large request waiting long enough is served before newer small ones --
    then advances all its residents by a quantum of steps worth about its
    budget of device time -- the budget grows with the age of the class's
    oldest resident, budget (1 + age / budget_aging_s), so that a class whose
    requests have waited long catches up -- (at most the smallest remaining
    step count, so a finished resident leaves at once), waits for it and
    retires the finished residents.  While large requests wait for admission
    and the queued work is small (no overload), the large class's budget is
    doubled: its requests' waits set the tail of the latency distribution.
    Classes take turns instead of running concurrently because a
    large simulation's pair kernel occupies every SM for its whole duration:
    a small request's kernels queued beside it would wait for it at every
    step.  With one large resident at a time the large requests run nearly
    at full speed, and small ones never wait behind them.
    """

    def __init__(self, backend, quantum=256, clock: Callable[[], float] = time.perf_counter,
                 sleep: Callable[[float], None] = time.sleep, classify=None, round_s=0.01, budgets=None,
                 max_resident=None, order=None, aging_s=2.0, budget_aging_s=0.2, budget_cap=4.0,
                 queue_boost=2.0, boost_backlog_s=2.0):
        self.backends = list(backend) if isinstance(backend, (list, tuple)) else [backend]
        nb = len(self.backends)
        self.classify = classify or (lambda r: 0)
        self.quantum = quantum
        self.clock = clock
        self.sleep = sleep
        if nb == 1:
            self.budgets = [round_s]
            self.max_resident = [None]
            self.order = ["fifo"]
        else:
            # device seconds per round: the small class's steps are short and
            # its requests finish in a few rounds; medium and large share
            self.budgets = budgets or [round_s * f for f in ((0.2, 1.0, 1.0) if nb == 3 else [1.0] * nb)]
            # the large class runs one simulation at a time and the medium
            # class a few: their batches stay small, so a step's time and the
            # cost of an admission (a sort of the class's arena) or a
            # retirement (its compaction) stay small too
            self.max_resident = max_resident or ([None] * (nb - 2) + [8, 1] if nb >= 2 else [None])
            self.order = order or (["fifo"] * (nb - 2) + ["sjf", "sjf"] if nb >= 2 else ["fifo"])
        self.aging_s = aging_s
        self.budget_aging_s = budget_aging_s
        self.budget_cap = budget_cap
        # the largest class's budget is multiplied by queue_boost while requests
        # of that class wait for admission and the estimated work queued in all
        # classes is at most boost_backlog_s (not under overload, where it
        # would starve the smaller classes)
        self.queue_boost = queue_boost
        self.boost_backlog_s = boost_backlog_s
        self._boost = False

    def _steps(self, k, residents, now):
        reqs = [v[0] for v in residents.values()]
        be = self.backends[k]
        cost = be.step_time(reqs) if hasattr(be, "step_time") else STEP_FIXED_S + sum(step_cost(r) for r in reqs)
        budget = self.budgets[k]
        if k == len(self.backends) - 1 and len(self.backends) > 1 and self._boost:
            budget *= self.queue_boost
        if self.budget_aging_s:
            age = max(now - v[2] for v in residents.values())   # time since admission
            budget *= min(self.budget_cap, 1.0 + age / self.budget_aging_s)
        q = int(max(1, min(self.quantum, round(budget / max(cost, 1e-9)))))
        return min(q, min(v[1] for v in residents.values()))

    def _next(self, k, queue, now):
        if self.order[k] != "sjf":
            return 0
        key = [(work(r) / (1.0 + max(0.0, now - r.arrival) / self.aging_s), r.arrival) for r in queue]
        return min(range(len(queue)), key=lambda i: key[i])

    def run(self, requests: List[Request], keep_observables=False):
        reqs = sorted(requests, key=lambda r: r.arrival)
        nb = len(self.backends)
        t0 = self.clock()
        now = lambda: self.clock() - t0  # noqa: E731
        queues = [[] for _ in range(nb)]
        resident = [dict() for _ in range(nb)]  # handle -> [request, remaining, admitted_at]
        used = [[0, 0] for _ in range(nb)]
        results, rejected = [], []
        nxt = 0
        while nxt < len(reqs) or any(queues) or any(resident):
            t = now()
            while nxt < len(reqs) and reqs[nxt].arrival <= t:
                r = reqs[nxt]
                nxt += 1
                k = min(max(0, int(self.classify(r))), nb - 1)
                while k < nb and not self.backends[k].fits(r, 0, 0, 0):
                    k += 1
                if k == nb:
                    rejected.append(r)
                else:
                    queues[k].append(r)
            ran = False
            for k in range(nb):
                be, q, res, u = self.backends[k], queues[k], resident[k], used[k]
                lim = self.max_resident[k]
                while q and (lim is None or len(res) < lim):
                    i = self._next(k, q, now())
                    r = q[i]
                    if not be.fits(r, u[0], u[1], len(res)):
                        break
                    h = be.admit(r)
                    res[h] = [r, r.steps, now()]
                    u[0] += r.n
                    u[1] += r.n_cells[0] * r.n_cells[1] * r.n_cells[2]
                    q.pop(i)
                if not res:
                    continue
                self._boost = bool(queues[nb - 1]) and \
                    sum(work(r) for q_ in queues for r in q_) <= self.boost_backlog_s
                ks = self._steps(k, res, now())
                be.step(ks)
                if hasattr(be, "sync"):
                    be.sync()
                ran = True
                for h in list(res):
                    v = res[h]
                    v[1] -= ks
                    if v[1] == 0:
                        r = v[0]
                        obs = be.finish(h)
                        results.append(Result(r.rid, r.arrival, v[2], now(), r.n, r.steps,
                                              obs if keep_observables else None))
                        u[0] -= r.n
                        u[1] -= r.n_cells[0] * r.n_cells[1] * r.n_cells[2]
                        del res[h]
            if not ran and not any(queues) and nxt < len(reqs):
                wait = reqs[nxt].arrival - now()
                if wait > 0:
                    self.sleep(wait)
        return summarize(results, rejected, now(), reqs)


def work(r):
    """Estimated device seconds of a whole request run alone."""
    return (STEP_FIXED_S + step_cost(r)) * r.steps


def run_alone(backend_factory, requests: List[Request], clock=time.perf_counter, sleep=time.sleep,
              keep_observables=False):
    """The plain loop: one simulation at a time, in arrival order, each in a
    backend of its own, stepped to completion before the next starts."""
    reqs = sorted(requests, key=lambda r: r.arrival)
    t0 = clock()
    now = lambda: clock() - t0  # noqa: E731
    results = []
    for r in reqs:
        wait = r.arrival - now()
        if wait > 0:
            sleep(wait)
        be = backend_factory(r)
        t_adm = now()
        h = be.admit(r)
        left = r.steps
        while left:
            k = min(64, left)
            be.step(k)
            left -= k
        obs = be.finish(h)
        be.close()
        results.append(Result(r.rid, r.arrival, t_adm, now(), r.n, r.steps, obs if keep_observables else None))
    return summarize(results, [], now(), reqs)


def summarize(results, rejected, makespan, requests):
    lat = np.array(sorted(r.latency for r in results)) if results else np.zeros(0)
    updates = float(sum(r.n * r.steps for r in results))
    offered = float(sum(r.n * r.steps for r in requests))
    span = max(makespan, 1e-12)
    arrival_span = max((requests[-1].arrival - requests[0].arrival) if len(requests) > 1 else span, 1e-12)
    return {
        "served": len(results),
        "rejected": len(rejected),
        "p50_s": float(np.percentile(lat, 50)) if len(lat) else None,
        "p99_s": float(np.percentile(lat, 99)) if len(lat) else None,
        "mean_s": float(lat.mean()) if len(lat) else None,
        "makespan_s": makespan,
        "updates_per_s": updates / span,
        "offered_updates_per_s": offered / arrival_span,
        "results": results,
    }
