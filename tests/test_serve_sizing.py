"""Sizing of the serving batches against an HBM budget (no GPU needed).

The arena a backend creates must fit the budget minus the accepted-list
reserve, and the list room the server charges per request must cover the
room the library reserves for an actual initial state: per cell with n >= 2
particles mu + 8 sqrt(mu) + 16 entries, mu = 2.0001 C n (n - 1) / 2 (the
cell preparation's rule), counted here from a sampled state with numpy.
"""
import math

import numpy as np
import pytest

from paper_1208_0961_gb300 import cuba
from paper_1208_0961_gb300 import serve as S
from paper_1208_0961_gb300 import workloads as W


@pytest.mark.parametrize("budget_gb,cpp", [(150.0, 0.01), (15.0, 0.01), (0.3, 0.05)])
def test_arena_fits_budget_minus_reserve(budget_gb, cpp):
    budget = int(budget_gb * 1e9)
    reserve = max(16 << 20, int(0.15 * budget))
    P, Cc = S.CudaBackend.size_for(cuba, cuba.CUBA_FP32, 256, budget - reserve, cpp)
    assert P > 0
    cfg = cuba.make_batch_config(cuba.CUBA_FP32, max_sims=256, max_particles=P, max_cells=Cc)
    assert cuba.cuba_batch_bytes(cfg) <= budget - reserve
    cfg = cuba.make_batch_config(cuba.CUBA_FP32, max_sims=256, max_particles=P + 1,
                                 max_cells=int(min(1 << 30, max(1 << 16, (P + 1) * cpp))))
    assert cuba.cuba_batch_bytes(cfg) > budget - reserve   # largest that fits


def _room_of_state(req):
    st = W.thermal_state(req.n, req.regions, seed=req.seed)
    nx, ny, nz = req.n_cells
    dx = [req.L[a] / req.n_cells[a] for a in range(3)]
    ix = [np.clip(np.floor(st[a] / dx[a]).astype(np.int64), 0, req.n_cells[a] - 1) for a in range(3)]
    key = ix[0] + nx * (ix[1] + ny * ix[2])
    n = np.bincount(key, minlength=nx * ny * nz).astype(np.float64)
    V = dx[0] * dx[1] * dx[2]
    C = req.sigma_fm2 * req.dt / (req.n_test * V)
    mu = 2.0001 * C * 0.5 * n * (n - 1)
    room = np.where(n >= 2, np.ceil(mu + 8 * np.sqrt(mu) + 16), 0)
    return room.sum()


def test_list_room_covers_the_librarys_reservation():
    reqs = S.poisson_stream(n_requests=40, rate_hz=20.0, seed=11, n_min=1e4, n_max=4e5)
    for r in reqs:
        if r.sigma_fm2 <= 0.0:
            assert S.list_room(r) == 0
            continue
        got = S.list_room(r)
        need = _room_of_state(r)
        assert got >= need, (r.rid, r.kind, got, need)
        assert got <= 3 * need + 16 * math.prod(r.n_cells), (r.rid, got, need)
