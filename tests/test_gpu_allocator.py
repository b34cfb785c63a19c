"""Simulations and batches whose device memory comes from the caller's
allocator (cuba_create_with_allocator, cuba_batch_create_with_allocator).

Every buffer goes through the allocator: what it hands out at creation is
exactly what cuba_sim_bytes / cuba_batch_bytes state (less the accepted-pair
list, which the first state load allocates), everything comes back at
destroy, and the physics is bit-identical to the cudaMalloc path and equal to
the oracle's step.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1208_0961_gb300 import cuba
from paper_1208_0961_gb300 import workloads as W

pytestmark = pytest.mark.gpu

LIST_MIN_BYTES = 8 << 20


def _cfg(n=20000, cells=100, sigma_mb=10.0, seed=42, prec=cuba.CUBA_FP64):
    cfg = W.riemann_1d(n, cells, 0.05, sigma_mb)
    p = cuba.make_params(L=cfg["L"], n_cells=cfg["n_cells"], dt=cfg["dt"], sigma_fm2=cfg["sigma_fm2"],
                         n_test=cfg["n_test"], precision=prec, seed=seed)
    op = O.make_params(L=cfg["L"], n=cfg["n_cells"], dt=cfg["dt"], sigma_fm2=cfg["sigma_fm2"],
                       n_test=cfg["n_test"], seed=seed)
    return cfg, p, op


def test_sim_with_torch_allocator_matches_oracle_and_default_path():
    import torch
    cfg, p, op = _cfg()
    st0 = W.thermal_state(20000, cfg["regions"], seed=7)
    alloc = cuba.torch_allocator()
    before = torch.cuda.memory_allocated()
    sim = cuba.Sim(p, 20000, allocator=alloc)
    try:
        assert alloc.live_bytes == cuba.cuba_sim_bytes(p, 20000) - LIST_MIN_BYTES
        assert torch.cuda.memory_allocated() - before >= alloc.live_bytes
        sim.set_state(st0)
        assert alloc.live_bytes >= cuba.cuba_sim_bytes(p, 20000)
        cuba.cuba_trace_enable(sim.h, True)
        sim.step(1)
        g = sim.get_state()
        keys, perm, cs, pairs, exe = sim.trace()
        obs = sim.observables()
    finally:
        sim.close()
    assert alloc.live_bytes == 0 and not alloc.live
    assert torch.cuda.memory_allocated() == before
    o, _, _, _ = O.sort(op, st0)
    o, res = O.step(op, 0, o)
    assert np.array_equal(keys, res.keys)
    assert np.array_equal(perm.astype(np.int64), res.perm)
    assert np.array_equal(pairs, res.accepted) and len(pairs) > 0
    assert set(map(tuple, pairs[exe].tolist())) == set(map(tuple, res.executed.tolist()))
    assert np.array_equal(g[:3], o[:3])
    # the same simulation through cudaMalloc: bit-identical
    ref = cuba.Sim(p, 20000)
    try:
        ref.set_state(st0)
        ref.step(1)
        assert np.array_equal(ref.get_state(), g)
        for x, y in zip(ref.observables(), obs):
            assert np.array_equal(x, y)
    finally:
        ref.close()


def test_batch_with_allocator_bytes_and_results():
    cfg_b = cuba.make_batch_config(cuba.CUBA_FP32, max_sims=4, max_particles=100000, max_cells=1000)
    alloc = cuba.torch_allocator()
    b = cuba.Batch(cfg_b, allocator=alloc)
    plain = cuba.Batch(cfg_b)
    try:
        assert alloc.live_bytes == cuba.cuba_batch_bytes(cfg_b) - LIST_MIN_BYTES
        ids = []
        for k, (n, cells, s) in enumerate([(30000, 100, 10.0), (20000, 200, 30.0)]):
            c = W.riemann_1d(n, cells, 0.02, s)
            p = cuba.make_params(L=c["L"], n_cells=c["n_cells"], dt=c["dt"], sigma_fm2=c["sigma_fm2"],
                                 n_test=c["n_test"], precision=cuba.CUBA_FP32, seed=100 + k)
            ids.append((b.add(p, n, c["regions"]), plain.add(p, n, c["regions"])))
        b.step(5)
        plain.step(5)
        for ia, ip in ids:
            assert np.array_equal(b.get_state(ia), plain.get_state(ip))
            for x, y in zip(b.observables(ia), plain.observables(ip)):
                assert np.array_equal(x, y)
        b.remove(ids[0][0])
        b.step(2)
    finally:
        b.close()
        plain.close()
    assert alloc.live_bytes == 0 and not alloc.live


def test_allocator_failure_is_reported_not_fatal():
    cfg, p, _ = _cfg()
    budget = {"left": 3}

    def alloc(n):
        import torch
        if budget["left"] == 0:
            return 0
        budget["left"] -= 1
        return torch.cuda.caching_allocator_alloc(n)

    a = cuba.DeviceAllocator(alloc, lambda ptr, n: __import__("torch").cuda.caching_allocator_delete(ptr))
    with pytest.raises(cuba.CubaError) as e:
        cuba.Sim(p, 20000, allocator=a)
    assert e.value.code == cuba.CUBA_ERR_OOM
    assert a.live_bytes == 0 and not a.live
