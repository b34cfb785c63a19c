"""Scheduling logic of the continuous-batching server, on the CPU with a fake
device backend and a fake clock: admission in arrival order against the
backend's capacity, no over-commit, rejection of requests larger than the
whole device, latency accounting, that batching shortens the makespan of a
burst compared with the one-at-a-time loop, the large class's one resident
at a time in shortest-work-first order with aging, and latency percentiles
against the one-at-a-time loop under the cost model."""
import numpy as np

from paper_1208_0961_gb300 import serve as S


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        return self.t

    def sleep(self, dt):
        self.t += max(0.0, dt)


class FakeBackend:
    """Capacity in particles/cells/members; a step of k costs k * (a + b * resident particles)
    seconds of fake time (a fixed launch cost plus a per-particle cost)."""

    def __init__(self, clock, max_particles=1000, max_cells=100, max_sims=4, a=1e-3, b=1e-6):
        self.clock, self.max_particles, self.max_cells, self.max_sims = clock, max_particles, max_cells, max_sims
        self.a, self.b = a, b
        self.res = {}
        self.next = 1
        self.peak = (0, 0, 0)
        self.log = []

    def fits(self, r, p, c, s):
        nc = r.n_cells[0] * r.n_cells[1] * r.n_cells[2]
        return p + r.n <= self.max_particles and c + nc <= self.max_cells and s < self.max_sims

    def admit(self, r):
        h = self.next
        self.next += 1
        self.res[h] = r
        p = sum(x.n for x in self.res.values())
        c = sum(np.prod(x.n_cells) for x in self.res.values())
        assert p <= self.max_particles and c <= self.max_cells and len(self.res) <= self.max_sims
        self.peak = (max(self.peak[0], p), max(self.peak[1], c), max(self.peak[2], len(self.res)))
        self.log.append(("admit", r.rid, self.clock()))
        return h

    def step(self, k):
        p = sum(x.n for x in self.res.values())
        self.clock.t += k * (self.a + self.b * p)

    def step_time(self, reqs):
        return self.a + self.b * sum(r.n for r in reqs)

    def finish(self, h):
        r = self.res.pop(h)
        self.log.append(("done", r.rid, self.clock()))
        return (r.rid,)

    def close(self):
        pass


def _req(rid, t, n, cells, steps):
    return S.Request(rid, t, "riemann", n, (1.0, 1.0, 1.0), (cells, 1, 1), 0.01, 0.1, 1.0, steps,
                     [((0, 0, 0), (1, 1, 1), 0.4)], rid)


def test_all_served_in_capacity_and_fifo_admission():
    clk = FakeClock()
    be = FakeBackend(clk)
    reqs = [_req(k, 0.001 * k, 200 + 50 * (k % 5), 10 + k % 7, 10 + 7 * (k % 4)) for k in range(30)]
    reqs.append(_req(99, 0.005, 5000, 10, 5))  # larger than the whole device
    out = S.Server(be, quantum=8, clock=clk, sleep=clk.sleep).run(reqs)
    assert out["served"] == 30 and out["rejected"] == 1
    admits = [rid for kind, rid, _ in be.log if kind == "admit"]
    assert admits == sorted(admits)          # arrival order
    assert be.peak[0] <= 1000 and be.peak[2] <= 4
    for r in out["results"]:
        assert r.finished >= r.admitted >= r.arrival
        assert r.latency > 0


def test_batching_beats_one_at_a_time_on_a_burst():
    reqs = [_req(k, 0.0, 100, 10, 50) for k in range(8)]
    clk = FakeClock()
    batched = S.Server(FakeBackend(clk, max_sims=8), quantum=16, clock=clk, sleep=clk.sleep).run(reqs)
    clk2 = FakeClock()
    alone = S.run_alone(lambda r: FakeBackend(clk2, max_sims=1), reqs, clock=clk2, sleep=clk2.sleep)
    assert batched["served"] == alone["served"] == 8
    # eight launches' fixed cost shared: the burst finishes far earlier
    assert batched["makespan_s"] < 0.5 * alone["makespan_s"]
    assert batched["p99_s"] < alone["p99_s"]


def test_poisson_stream_shape():
    reqs = S.poisson_stream(n_requests=200, seed=7)
    kinds = [r.kind for r in reqs]
    assert 60 < kinds.count("riemann") < 140
    ns = np.array([r.n for r in reqs])
    assert ns.min() >= 1e4 and ns.max() <= 8e6
    gaps = np.diff([r.arrival for r in reqs])
    assert abs(gaps.mean() - 1 / 20.0) < 0.015
    for r in reqs:
        dx = min(r.L[a] / r.n_cells[a] for a in range(3))
        assert r.dt < dx


def test_cost_classes_keep_small_requests_fast():
    big = S.Request(0, 0.0, "riemann", 900, (1.0, 1.0, 1.0), (2, 1, 1), 0.01, 0.1, 1.0, 200,
                    [((0, 0, 0), (1, 1, 1), 0.4)], 0)
    small = [_req(k, 0.001 + 0.001 * k, 20, 10, 200) for k in range(1, 6)]
    reqs = [big] + small

    def run(nclasses):
        clk = FakeClock()
        if nclasses == 1:
            srv = S.Server(FakeBackend(clk, max_particles=2000, max_cells=200, max_sims=8, a=1e-5, b=1e-5),
                           quantum=200, clock=clk, sleep=clk.sleep)
        else:
            bes = [FakeBackend(clk, max_particles=2000, max_cells=200, max_sims=8, a=1e-5, b=1e-5) for _ in range(2)]
            srv = S.Server(bes, quantum=200, clock=clk, sleep=clk.sleep, classify=lambda r: 1 if r.n > 100 else 0,
                           round_s=0.02)
        out = srv.run(reqs)
        return {r.rid: r.latency for r in out["results"]}

    one, two = run(1), run(2)
    assert len(one) == len(two) == 6
    small_one = max(one[k] for k in range(1, 6))
    small_two = max(two[k] for k in range(1, 6))
    assert small_two < 0.5 * small_one


def test_cost_model_orders_requests():
    a = S.Request(0, 0.0, "riemann", 8_000_000, (10, 1, 1), (2000, 1, 1), 0.002, 1.0, 1e5, 100, [], 0)
    b = S.Request(1, 0.0, "thermal", 20_000, (1, 1, 1), (9, 9, 9), 0.01, 1.0, 1e3, 100, [], 1)
    assert S.step_cost(a) > 1e-3 > 1e-4 > S.step_cost(b)
    assert S.cost_class(a) == 2 and S.cost_class(b) == 0


class CostBackend(FakeBackend):
    """Fake device whose step takes the server's own cost model in fake time:
    a fixed launch cost plus each resident's estimated step cost."""

    def __init__(self, clock, **kw):
        kw.setdefault("max_particles", 10 ** 9)
        kw.setdefault("max_cells", 10 ** 9)
        kw.setdefault("max_sims", 256)
        super().__init__(clock, **kw)

    def step_time(self, reqs):
        return S.STEP_FIXED_S + sum(S.step_cost(r) for r in reqs)

    def step(self, k):
        self.clock.t += k * self.step_time(list(self.res.values()))


def _classes(clk):
    return [CostBackend(clk) for _ in range(3)]


def test_large_class_runs_one_at_a_time_shortest_first():
    big = lambda rid, t, steps: S.Request(rid, t, "riemann", 4_000_000, (10.0, 1.0, 1.0), (2000, 1, 1), 0.002,  # noqa
                                          1.0, 1e5, steps, [((0, 0, 0), (10, 1, 1), 0.4)], rid)
    reqs = [big(0, 0.0, 400), big(1, 0.01, 300), big(2, 0.02, 60), big(3, 0.03, 200)]
    assert all(S.cost_class(r) == 2 for r in reqs)
    clk = FakeClock()
    bes = _classes(clk)
    out = S.Server(bes, clock=clk, sleep=clk.sleep, classify=S.cost_class).run(reqs)
    assert out["served"] == 4
    assert bes[2].peak[2] == 1                       # never two large residents
    done = [rid for kind, rid, _ in bes[2].log if kind == "done"]
    assert done == [0, 2, 3, 1]                     # first come, then shortest work first


def test_aging_serves_a_long_waiting_large_request():
    big = lambda rid, t, steps: S.Request(rid, t, "riemann", 4_000_000, (10.0, 1.0, 1.0), (2000, 1, 1), 0.002,  # noqa
                                          1.0, 1e5, steps, [((0, 0, 0), (10, 1, 1), 0.4)], rid)
    # request 1 is long; shorter ones keep arriving behind it
    reqs = [big(0, 0.0, 100), big(1, 0.01, 500)] + [big(2 + k, 0.02 + 0.2 * k, 100) for k in range(40)]
    clk = FakeClock()
    bes = _classes(clk)
    out = S.Server(bes, clock=clk, sleep=clk.sleep, classify=S.cost_class, aging_s=1.0).run(reqs)
    done = [rid for kind, rid, _ in bes[2].log if kind == "done"]
    # without aging request 1 would finish last
    assert done.index(1) < len(done) - 5


def test_small_requests_do_not_wait_for_a_large_one():
    big = S.Request(0, 0.0, "riemann", 8_000_000, (10.0, 1.0, 1.0), (2000, 1, 1), 0.002, 1.0, 1e5, 500,
                    [((0, 0, 0), (10, 1, 1), 0.4)], 0)
    small = [S.Request(k, 0.05 * k, "thermal", 20_000, (0.9, 0.9, 0.9), (9, 9, 9), 0.01, 1.0, 1e3, 200,
                       [((0, 0, 0), (0.9, 0.9, 0.9), 0.4)], k) for k in range(1, 8)]
    assert S.cost_class(big) == 2 and all(S.cost_class(r) == 0 for r in small)
    clk = FakeClock()
    out = S.Server(_classes(clk), clock=clk, sleep=clk.sleep, classify=S.cost_class).run([big] + small)
    lat = {r.rid: r.latency for r in out["results"]}
    alone_small = S.work(small[0])
    # each small request takes about its own run time plus a few rounds of
    # the large class's budget, far below the large request's run time
    assert max(lat[k] for k in range(1, 8)) < alone_small + 0.2
    assert lat[0] > 10 * max(lat[k] for k in range(1, 8))


def test_served_beats_one_at_a_time_on_p50_and_p99():
    """At a rate where the fake device is busy about 60-75 % of the time (the
    cost model's estimate of the real one), serving lowers the mean, the
    median and the 99th percentile of the latency below the one-at-a-time
    loop's."""
    for rate in (8.0, 10.0):
        reqs = S.poisson_stream(n_requests=300, rate_hz=rate, seed=7)
        clk = FakeClock()
        served = S.Server(_classes(clk), clock=clk, sleep=clk.sleep, classify=S.cost_class).run(reqs)
        clk2 = FakeClock()
        alone = S.run_alone(lambda r: CostBackend(clk2, max_sims=1), reqs, clock=clk2, sleep=clk2.sleep)
        assert served["served"] == alone["served"] == 300
        assert served["p50_s"] < 0.8 * alone["p50_s"]
        assert served["p99_s"] < alone["p99_s"]
        assert served["mean_s"] < 0.8 * alone["mean_s"]


class StepLog(CostBackend):
    """CostBackend that records the step count of every advance."""

    def __init__(self, clock, **kw):
        super().__init__(clock, **kw)
        self.steps = []

    def step(self, k):
        self.steps.append(k)
        super().step(k)


def _large_pair(backlog_steps):
    big = lambda rid, t, steps: S.Request(rid, t, "riemann", 4_000_000, (10.0, 1.0, 1.0), (2000, 1, 1), 0.002,  # noqa
                                          1.0, 1e5, steps, [((0, 0, 0), (10, 1, 1), 0.4)], rid)
    return [big(0, 0.0, 400), big(1, 0.0, backlog_steps)]


def test_large_class_budget_doubles_while_large_requests_wait():
    """The largest class's quanta double while a large request waits for
    admission and the queued work is small, and not once the queued work
    exceeds boost_backlog_s (overload)."""
    out = {}
    for boost, steps in ((1.0, 50), (2.0, 50), (2.0, 5000)):
        clk = FakeClock()
        bes = [StepLog(clk) for _ in range(3)]
        reqs = _large_pair(steps)
        assert S.work(reqs[1]) < 2.0 if steps == 50 else S.work(reqs[1]) > 2.0
        S.Server(bes, clock=clk, sleep=clk.sleep, classify=S.cost_class, queue_boost=boost).run(reqs)
        out[(boost, steps)] = bes[2].steps[0]   # the first resident's first quantum, request 1 queued
    assert abs(out[(2.0, 50)] - 2 * out[(1.0, 50)]) <= 1   # quanta are rounded budgets / step cost
    assert out[(2.0, 5000)] == out[(1.0, 50)]
