"""Multi-process (gloo, CPU) checks of the benchmark's N > 1 logic: one
independent replica per rank, the slowest rank's time, the whole-job rate, the
round-robin split of an ensemble, and the reference arm on ranks other than 0.
No GPU: the collectives run over gloo on the host."""
import contextlib
import io
import multiprocessing as mp
import os
import socket
import sys
import types

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench as B
    w, r, _ = B.dist_setup(None, backend="gloo")
    t = B.max_over_ranks(1.0 + 0.5 * r, w)          # per-rank "time"
    s = B.sum_over_ranks(10 * (r + 1), w)
    B.barrier(w)
    q.put({"rank": r, "world": w, "max": t, "sum": s, "seed": B.replica_seed(7, r),
           "shard": B.shard_members(list(range(11)), r, w)})
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_replica_collectives_gloo(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = [q.get(timeout=120) for _ in range(world)]
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    res.sort(key=lambda d: d["rank"])
    slowest = 1.0 + 0.5 * (world - 1)
    for d in res:
        assert d["world"] == world
        assert d["max"] == pytest.approx(slowest)
        assert d["sum"] == pytest.approx(sum(10 * (k + 1) for k in range(world)))
    # independent replicas: distinct seeds
    assert len({d["seed"] for d in res}) == world
    # the shards partition the ensemble
    got = sorted(m for d in res for m in d["shard"])
    assert got == list(range(11))
    # whole-job rate: all ranks' updates over the slowest rank's time
    assert bench.replica_rate(16_000_000 * 20, world, slowest) == pytest.approx(16e6 * 20 * world / slowest)


def test_reference_arm_other_ranks_exit(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = types.SimpleNamespace(steps=3, warmup=3)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.run_reference(args) == 0
    assert buf.getvalue() == ""


def test_launch_count():
    # one 11-bit pass up to 2048 cells, two up to 2^22
    assert bench.bin_passes(1) == 1 and bench.bin_passes(2000) == 1 and bench.bin_passes(2048) == 1
    assert bench.bin_passes(2049) == 2 and bench.bin_passes(128 ** 3) == 2 and bench.bin_passes(1 << 23) == 3
    # counted against the ncu launch lists of one step: 11 (16 M, 2000 cells,
    # no small-cell kernels; the cell table's scan is one kernel up to 4095
    # cells), 14 (20 k FP64 particles in 100 cells: a streaming kernel before
    # the histogram) and 21 (64 M, 128^3 cells, small-cell kernels)
    assert bench.launches_per_step(2000, 0) == 11
    assert bench.launches_per_step(100, 32, split_stream=True) == 14
    assert bench.launches_per_step(128 ** 3, 64) == 21
    # the neighbour-move sort of the 64 M hot spot: 16 per step
    assert bench.launches_per_step(128 ** 3, 256, neighbour=True) == 16
    hs = {"n_cells": (128, 128, 128), "L": (12.8, 12.8, 12.8), "dt": 0.01}
    assert bench.neighbour_sort(64_000_000, hs) and not bench.neighbour_sort(300_000_000, hs)
    rm = {"n_cells": (2000, 1, 1), "L": (10.0, 1.0, 1.0), "dt": 0.0025}
    assert not bench.neighbour_sort(16_000_000, rm)
    # skip-ahead: 11 per step of the 16 M workload (both scans one kernel)
    assert bench.launches_per_step(2000, 0, skip=True) == 11
