"""cuba_bin_noalloc against the library's allocating path.

Some callers cannot allocate device memory (a loop with a fixed memory budget,
a pool that must not grow, code without an allocator of its own).  For them
the library offers cell keys and the stable sort by cell through
cuba_bin_noalloc, whose scratch is a fixed array inside the library.  Its
permutation and cell_start must equal, bit for bit, those of the sort that
cuba_set_state performs on the same positions; two calls in a row (different
sizes, precisions and grids) check that the shared scratch keeps no stale
state between calls.  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_1208_0961_gb300 import cuba
from paper_1208_0961_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _reference(p, st):
    """Permutation and cell_start of the sort done by cuba_set_state."""
    n = st.shape[1]
    sim = cuba.Sim(p, max(n, 1))
    try:
        cuba.cuba_trace_enable(sim.h, True)
        sim.set_state(st)
        _, perm, cs, _, _ = sim.trace()
    finally:
        sim.close()
    return perm, cs


def _run_cases(cases):
    import torch
    for call, (n, L, cells, prec) in enumerate(cases):
        regs = [((0.0, 0.0, 0.0), L, 0.4)]
        dtype = np.float64 if prec == cuba.CUBA_FP64 else np.float32
        st = W.thermal_state(n, regs, seed=100 + call).astype(dtype) if n else np.zeros((6, 0), dtype)
        dt = 0.5 * min(L[a] / cells[a] for a in range(3))
        p = cuba.make_params(L=L, n_cells=cells, dt=dt, sigma_fm2=0.0, n_test=1.0, precision=prec, seed=call)
        ref_perm, ref_cs = _reference(p, st)
        ncells = cells[0] * cells[1] * cells[2]
        xyz = torch.from_numpy(np.ascontiguousarray(st[:3])).cuda()
        perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device="cuda")
        cs = torch.full((ncells + 1,), -1, dtype=torch.int32, device="cuda")
        cuba.cuba_bin_noalloc(p, xyz, n, perm, cs)
        torch.cuda.synchronize()
        got_perm = perm.cpu().numpy().view(np.uint32)[:n]
        got_cs = cs.cpu().numpy().view(np.uint32)
        assert np.array_equal(got_perm, ref_perm), "call %d: permutation differs" % call
        assert np.array_equal(got_cs, ref_cs), "call %d: cell_start differs" % call


def test_noalloc_binning_matches_allocating_sort_twice():
    _run_cases([
        # n, L, cells, precision: two radix passes of 8-bit digits
        (200000, (1.0, 0.8, 0.4), (50, 4, 2), cuba.CUBA_FP64),
        (77777, (10.0, 1.0, 1.0), (300, 1, 1), cuba.CUBA_FP32),
    ])


@pytest.mark.parametrize("cases", [
    # one cell (no radix pass: identity permutation), then one pass (<= 256
    # cells: the result sits in the second buffer)
    [(5000, (1.0, 1.0, 1.0), (1, 1, 1), cuba.CUBA_FP32), (123457, (10.0, 1.0, 1.0), (200, 1, 1), cuba.CUBA_FP64)],
    # three passes (more than 65536 cells, most of them empty), then no
    # particles at all
    [(262144, (6.4, 6.4, 3.2), (64, 64, 32), cuba.CUBA_FP32), (0, (1.0, 1.0, 1.0), (7, 3, 2), cuba.CUBA_FP64)],
    # no particles first, then the largest size the scratch holds
    [(0, (2.0, 1.0, 1.0), (300, 1, 1), cuba.CUBA_FP32), (262144, (2.0, 1.0, 1.0), (300, 2, 1), cuba.CUBA_FP32)],
])
def test_noalloc_every_pass_count_and_empty_input(cases):
    _run_cases(cases)


def test_noalloc_rejects_sizes_beyond_its_scratch():
    p = cuba.make_params(L=(1.0, 1.0, 1.0), n_cells=(4, 4, 4), dt=0.01, sigma_fm2=0.1, n_test=1.0)
    with pytest.raises(cuba.CubaError) as e:
        cuba.cuba_bin_noalloc(p, None, cuba.CUBA_NOALLOC_MAX_PARTICLES + 1, None, None)
    assert e.value.code == cuba.CUBA_ERR_CAPACITY
    assert "at most" in cuba.cuba_last_error()
