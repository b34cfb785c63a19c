#!/usr/bin/env python
"""Throughput of the per-time-step test-particle update (stream + reflect + bin +
2->2 collide) on one GB300, in particle updates per second.

Workload (default): the 1D Riemann problem of the paper's Results section scaled
up — box 10 x 1 x 1 fm, 2000 cells along x (dx = 0.005 fm), dt = 0.0025 fm/c,
16M test particles (left half T = 400 MeV, right half 320 MeV, density ~ T^3),
sigma = 10 mb, FP32 state with FP64 reductions.  One bench step = one time step
of the whole state.  The state (384 MB) is larger than L2, so no flush is needed
between steps.

Printed: one JSON line (rank 0).  Under torchrun each rank advances its own
independent replica (seed + rank); the value is the sum over ranks divided by
the slowest rank's time.

--impl reference times the CPU oracle (the plain FP64/FP32 C definition of the
same step) on the host cores, on a bounded sample of the workload: a strip of
cells of the same box with the same cell occupancies, time step and N_test.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="cuba", choices=["cuba", "reference"])
    ap.add_argument("--mode", default="step", choices=["step", "batch", "serve"],
                    help="step: the headline single-workload line; batch: the batched ensemble; "
                         "serve: the continuous-batching request stream")
    ap.add_argument("--batch-sims", type=int, default=256)
    ap.add_argument("--serve-requests", type=int, default=400)
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--serve-alone", type=int, default=1, help="also run the one-at-a-time loop")
    ap.add_argument("--serve-classes", type=int, default=3, choices=[1, 3])
    ap.add_argument("--workload", default="riemann1d", choices=["riemann1d", "hotspot3d"],
                    help="riemann1d: the headline 1D Riemann problem; hotspot3d: 3D thermal box with a hot spot")
    ap.add_argument("--n", type=int, default=16_000_000)
    ap.add_argument("--cells", type=int, default=2000)
    ap.add_argument("--dt", type=float, default=0.0025)
    ap.add_argument("--sigma-mb", type=float, default=10.0)
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--acceptance", default="all-pairs", choices=["all-pairs", "skip"],
                    help="pair test of the paper (every pair draws its uniform) or skip-ahead sampling")
    ap.add_argument("--mass", type=float, default=0.0, help="particle mass, GeV (0: massless gluons)")
    ap.add_argument("--mu", type=float, default=0.0, help="> 0: screened forward-peaked scattering, GeV")
    ap.add_argument("--kappa", type=float, default=0.0,
                    help="> 0: adaptive time step (kappa collisions per particle of the fullest cell per "
                         "step, dt as its cap)")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--profile-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune", type=int, default=1, help="pick the collision launch shape before timing")
    ap.add_argument("--shape", default=None,
                    help="small_max,small_blocks,tile_blocks: set the collision launch shape (no autotuning)")
    ap.add_argument("--cpu-sample-cells", type=int, default=16)
    ap.add_argument("--cpu-sample-steps", type=int, default=2)
    return ap.parse_args()


def workload(args):
    from paper_1208_0961_gb300 import workloads as W
    if args.workload == "hotspot3d":
        cfg = W.hotspot_3d(args.n, args.cells, args.dt, args.sigma_mb)
        cfg["name"] = "hotspot-3d-%dM-%d^3cells-%gmb" % (round(args.n / 1e6), args.cells, args.sigma_mb)
        return cfg
    cfg = W.riemann_1d(args.n, args.cells, args.dt, args.sigma_mb)
    cfg["name"] = "riemann-1d-%dM-%dcells-%gmb" % (round(args.n / 1e6), args.cells, args.sigma_mb)
    return cfg


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm_sorted = sorted(sm)
        return {"sm_mhz": sm_sorted[len(sm_sorted) // 2], "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(args, backend=None):
    """Join the process group of a torchrun launch (one rank per GPU, NCCL);
    backend "gloo" joins on the CPU (multi-process tests of the replica
    logic)."""
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    backend = backend or "nccl"
    if world > 1:
        import torch.distributed as dist
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend)
    elif backend == "nccl":
        torch.cuda.set_device(0)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x, world):
    """Largest x over the ranks (the slowest rank's time)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x, world):
    """Sum of x over the ranks."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def replica_seed(seed, rank):
    """Each rank advances an independent replica with its own seed."""
    return seed + rank


def replica_rate(units_per_rank, world, seconds_max):
    """Whole-job throughput: the units all ranks processed over the slowest
    rank's time (weak scaling: every rank holds the same workload)."""
    return units_per_rank * world / seconds_max


def bin_passes(ncells):
    """Radix passes of the in-step sort (11-bit digits)."""
    bits = 0
    while bits < 32 and (ncells - 1) >> bits:
        bits += 1
    return max(1, (bits + 10) // 11)


def neighbour_sort(n, cfg):
    """Whether a step of this single-simulation workload sorts by neighbour
    moves (the library's rule: more than 2048 cells, at most 64 particles per
    cell on average, dt at most 0.98 of the cell edge on every axis with more
    than one cell)."""
    cells = cfg["n_cells"][0] * cfg["n_cells"][1] * cfg["n_cells"][2]
    edges_ok = all(cfg["n_cells"][a] == 1 or cfg["dt"] <= 0.98 * cfg["L"][a] / cfg["n_cells"][a] for a in range(3))
    return cells > 2048 and n <= 64 * cells and edges_ok


def launches_per_step(ncells, small_max, skip=False, adaptive=False, neighbour=False):
    """Kernels of one step: the stream/sort kernels — radix: streaming
    histogram; per radix pass the digit histogram (passes after the first), 3
    scan kernels and the ranking kernel, then (two passes or more) the gather;
    neighbour-move sort: count pass, offsets, 3 scan kernels, scatter pass —;
    cell preparation + 3 scan kernels; small-cell and tiled pair kernels and
    the survivor kernel (skip-ahead: 3 scan kernels of its row blocks and its
    pair kernel); small-cell and per-cell resolve kernels; the step counter."""
    p = bin_passes(ncells)
    sort = 6 if neighbour else 1 + 4 * p + (p - 1) + (1 if p > 1 else 0)
    small = 1 if small_max else 0
    pairs = 3 + 1 if skip else 1 + small + 1
    return (1 if adaptive else 0) + sort + 4 + pairs + (1 + small) + 1


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def pair_tile_traffic():
    """DRAM bytes of one full-size pair-tile launch from the committed ncu
    summary, if the kernel's sources are unchanged since the capture."""
    import hashlib
    import re
    prof = os.path.join(ROOT, "profiles", "k_pair_tile_riemann1d_fp32.md")
    srcs = ["kernels_pairs.cu", "engine.cuh", "philox.cuh", "fp.cuh"]
    try:
        text = open(prof).read()
        h = hashlib.sha256()
        for f in srcs:
            with open(os.path.join(ROOT, "paper_1208_0961_gb300", "csrc", f), "rb") as fh:
                h.update(fh.read())
        m = re.search(r"source-sha256[^:]*:\s*([0-9a-f]{64})", text)
        t = re.search(r"traffic_bytes_per_launch \| (\d+)", text)
        if m and t and m.group(1) == h.hexdigest():
            return int(t.group(1))
    except OSError:
        pass
    return None


def strip_sample(args, cfg):
    """A strip of cells with the workload's occupancy: it keeps dx, dt, sigma,
    N_test and the per-cell particle numbers of the left and right halves (m
    cells, half of them at the left occupancy and half at the right one), so
    per-update cost matches the full workload's mix.  Returns the box, the
    cell count, the seeded state (FP32-representable for an FP32 run) and the
    two particle numbers."""
    import numpy as np
    from paper_1208_0961_gb300 import workloads as W
    m = max(2, args.cpu_sample_cells - args.cpu_sample_cells % 2)
    dx = cfg["L"][0] / cfg["n_cells"][0]
    counts = W.region_split(cfg["n"], cfg["regions"])
    per_l = counts[0] / (cfg["n_cells"][0] / 2)
    per_r = counts[1] / (cfg["n_cells"][0] / 2)
    Ls = (m * dx, cfg["L"][1], cfg["L"][2])
    n_l = int(round(per_l * m / 2))
    n_r = int(round(per_r * m / 2))
    regs = [((0.0, 0.0, 0.0), (Ls[0] / 2, Ls[1], Ls[2]), cfg["T_left"]),
            ((Ls[0] / 2, 0.0, 0.0), Ls, cfg["T_right"])]
    st = np.concatenate([W.thermal_state(n_l, regs[:1], seed=args.seed),
                         W.thermal_state(n_r, regs[1:], seed=args.seed + 1)], axis=1)
    if args.precision == "fp32":
        st = st.astype(np.float32).astype(np.float64)
    return Ls, m, st, n_l, n_r


def cpu_sample(args, cfg, steps):
    """Time the oracle on a strip of cells with the workload's occupancy
    (strip_sample)."""
    from oracle import oracle as O
    Ls, m, st, n_l, n_r = strip_sample(args, cfg)
    op = O.make_params(L=Ls, n=(m, 1, 1), dt=cfg["dt"], sigma_fm2=cfg["sigma_fm2"], n_test=cfg["n_test"],
                       fp32=args.precision == "fp32", seed=args.seed)
    st, _, _, _ = O.sort(op, st)
    n = st.shape[1]
    t0 = time.perf_counter()
    for k in range(steps):
        st, _ = O.step(op, k, st, trace=False)
    dt = time.perf_counter() - t0
    sample = ("%d-cell strip of the same box (%d + %d particles at the workload's left/right cell "
              "occupancy, same dx, dt, sigma, N_test), %d oracle steps" % (m, n_l, n_r, steps))
    return n * steps / dt, O.threads(), sample, dt


def fp32_vs_fp64_oracle(args, cfg):
    """The FP32 path against the FP64 oracle on the strip of cpu_sample: one
    step on the GPU in FP32 and one oracle step in FP64 from the same
    FP32-representable state.  Keys may differ only by rounding near a cell
    face; accepted pairs are compared in the cells whose sorted order agrees,
    each pair accepted on one side only measured by |u - P22_FP64| / C (the
    band where FP32 rounding of v_rel can flip a decision); momenta of the
    pairs executed on both sides against the pair energy."""
    import numpy as np
    from oracle import oracle as O
    from paper_1208_0961_gb300 import cuba
    Ls, m, st, _, _ = strip_sample(args, cfg)
    op = O.make_params(L=Ls, n=(m, 1, 1), dt=cfg["dt"], sigma_fm2=cfg["sigma_fm2"], n_test=cfg["n_test"],
                       seed=args.seed)
    o_in, _, _, _ = O.sort(op, st)
    o_out, res = O.step(op, 0, o_in)
    n = o_in.shape[1]
    p = cuba.make_params(L=Ls, n_cells=(m, 1, 1), dt=cfg["dt"], sigma_fm2=cfg["sigma_fm2"], n_test=cfg["n_test"],
                         precision=cuba.CUBA_FP32, seed=args.seed)
    sim = cuba.Sim(p, n)
    try:
        sim.set_state(o_in.astype(np.float32))
        cuba.cuba_trace_enable(sim.h, True)
        cuba.cuba_set_step(sim.h, 0)
        sim.step(1)
        g = sim.get_state().astype(np.float64)
        keys, perm, cs, pairs, exe = sim.trace()
    finally:
        sim.close()
    keys_differ = int(np.count_nonzero(keys != res.keys))
    same = np.array([np.array_equal(perm[cs[c]:cs[c + 1]], res.perm[res.cell_start[c]:res.cell_start[c + 1]])
                     for c in range(m)])
    cells = np.nonzero(same)[0]
    acc_g = set(map(tuple, pairs[np.isin(pairs[:, 0], cells)].tolist()))
    acc_o = set(map(tuple, res.accepted[np.isin(res.accepted[:, 0], cells)].tolist()))
    flips = acc_g ^ acc_o
    band = 0.0
    if flips:
        C = O.p22_scale(op)
        free = O.make_params(L=Ls, n=(m, 1, 1), dt=cfg["dt"], sigma_fm2=0.0, n_test=cfg["n_test"], seed=args.seed)
        mid, _ = O.step(free, 0, o_in)
        key = [args.seed & 0xFFFFFFFF, (args.seed >> 32) & 0xFFFFFFFF]
        for c, i, j in flips:
            b = res.cell_start[c]
            ni = mid[3:, b + i] / np.linalg.norm(mid[3:, b + i])
            nj = mid[3:, b + j] / np.linalg.norm(mid[3:, b + j])
            u = O.pair_word(key, 0, c, i, j) * 2.0 ** -32
            band = max(band, abs(u - C * 0.5 * float(np.sum((ni - nj) ** 2))) / C)
    ex_g = set(map(tuple, pairs[exe].tolist()))
    both = [e for e in map(tuple, res.executed.tolist()) if e in ex_g and same[e[0]]]
    worst = 0.0
    for c, i, j in both:
        bo, bg = res.cell_start[c], cs[c]
        s = np.linalg.norm(o_out[3:, bo + i]) + np.linalg.norm(o_out[3:, bo + j])
        worst = max(worst, np.abs(g[3:, bg + i] - o_out[3:, bo + i]).max() / s,
                    np.abs(g[3:, bg + j] - o_out[3:, bo + j]).max() / s)
    return {"particles": n, "keys_differ": keys_differ, "cells_compared": int(same.sum()), "cells": m,
            "accepted": int(len(acc_o)), "accepted_differ": len(flips), "max_abs_u_minus_p22_over_C": band,
            "pairs_compared": len(both), "max_dp_over_pair_energy": worst}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    cfg = workload(args)
    from oracle import oracle as O
    O.lib()
    # one bounded sample per step: the bench's step count, each a 1-step strip run
    rate_steps = max(1, args.steps)
    times = []
    n_upd = 0
    for _ in range(args.warmup and 1):
        cpu_sample(args, cfg, 1)
    for _ in range(rate_steps):
        r, cores, sample, dt = cpu_sample(args, cfg, 1)
        times.append(dt)
        n_upd += r * dt
    tot = sum(times)
    value = n_upd / tot
    line = {
        "impl": "reference", "metric": "particle-updates/s (stream+bin+collide)", "value": value,
        "unit": "particle-updates/s", "n_gpus": world, "steps": rate_steps, "warmup": args.warmup,
        "ms_per_step": 1000.0 * tot / rate_steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f32", "data": "synthetic",
        "config": {"workload": cfg["name"], "n_particles": args.n, "n_cells": args.cells, "dt": args.dt,
                   "sigma_mb": args.sigma_mb, "precision": args.precision},
        "cpu_baseline": {"value": value, "unit": "particle-updates/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "particle-updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def ensemble(n_sims, seed=0):
    """Batched ensemble: independent 1D Riemann runs with particle counts
    log-uniform in [5e4, 4e6], cell counts log-uniform in [100, 2000], sigma
    log-uniform in [0.5, 50] mb, (T_L, T_R) from {400/320, 500/300, 350/250}
    MeV; dt = min(dx/2, 0.1 lambda(T_L)); member k has seed 1000 + k."""
    import numpy as np
    from paper_1208_0961_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    pairs = [(0.4, 0.32), (0.5, 0.3), (0.35, 0.25)]
    out = []
    for k in range(n_sims):
        n = int(round(math.exp(rng.uniform(math.log(5e4), math.log(4e6)))))
        cells = int(round(math.exp(rng.uniform(math.log(100), math.log(2000)))))
        sigma_mb = float(math.exp(rng.uniform(math.log(0.5), math.log(50.0))))
        TL, TR = pairs[int(rng.integers(3))]
        L = (10.0, 1.0, 1.0)
        lam = 1.0 / (W.gluon_density(TL) * sigma_mb * W.FM2_PER_MB)
        dt = min(0.5 * L[0] / cells, 0.1 * lam)
        cfg = W.riemann_1d(n, cells, dt, sigma_mb, T_left=TL, T_right=TR, L=L)
        cfg["seed"] = 1000 + k
        out.append(cfg)
    return out


def shard_members(members, rank, world):
    """Members of an ensemble that rank advances (round robin: independent
    simulations need no exchange, so ranks share nothing on the data path)."""
    return members[rank::world]


def run_batch_mode(args):
    import torch
    from paper_1208_0961_gb300 import cuba
    world, rank, local = dist_setup(args)
    cuba.load()
    prec = cuba.CUBA_FP32 if args.precision == "fp32" else cuba.CUBA_FP64
    members = shard_members(ensemble(args.batch_sims, args.seed), rank, world)
    N = sum(m["n"] for m in members)
    C = sum(m["n_cells"][0] for m in members)
    cfg = cuba.make_batch_config(prec, max_sims=len(members), max_particles=N, max_cells=C)
    b = cuba.Batch(cfg)
    stream = torch.cuda.Stream()
    params = []
    for m in members:
        p = cuba.make_params(L=m["L"], n_cells=m["n_cells"], dt=m["dt"], sigma_fm2=m["sigma_fm2"],
                             n_test=m["n_test"], precision=prec, seed=m["seed"])
        params.append(p)
        b.add(p, m["n"], m["regions"], stream)
    torch.cuda.synchronize()
    b.step(args.warmup, stream)
    torch.cuda.synchronize()
    # the launch shape for the whole batch (timed on its live state, which is
    # restored); the one-at-a-time loop below keeps the library's default
    # shape, which is faster for it than the batch's
    shape, tune_ms = (cuba.cuba_batch_autotune_shape(b.h, 1, stream) if args.autotune
                      else (None, None))
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    b.step(args.steps, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    ids = list(b.members)
    pair_tests = sum(b.stats(i)["pair_tests"] for i in ids) / (args.warmup + args.steps)
    b.close()
    # the plain loop: each member alone (single-simulation API), same steps
    alone_ms = 0.0
    for m, p in zip(members, params):
        sim = cuba.Sim(p, m["n"])
        sim.init_thermal(m["n"], m["regions"], stream)
        cuba.cuba_step(sim.h, 1, stream)
        torch.cuda.synchronize()
        a0 = torch.cuda.Event(enable_timing=True)
        a1 = torch.cuda.Event(enable_timing=True)
        a0.record(stream)
        cuba.cuba_step(sim.h, args.steps, stream)
        a1.record(stream)
        torch.cuda.synchronize()
        alone_ms += a0.elapsed_time(a1)
        sim.close()
    alone_ms = max_over_ranks(alone_ms, world)
    # the updates of all ranks over the slowest rank's time
    tot = sum_over_ranks(N, world)
    if rank == 0:
        line = {"mode": "batch", "metric": "particle-updates/s (stream+bin+collide), batched ensemble",
                "value": tot * args.steps / (ms / 1000.0), "unit": "particle-updates/s", "steps": args.steps,
                "n_gpus": world, "scaling": "weak", "ms_per_step": ms / args.steps, "members": args.batch_sims,
                "particles": int(tot), "cells": int(sum_over_ranks(C, world)) if world > 1 else C,
                "pair_tests_per_step": pair_tests,
                "alone": {"value": tot * args.steps / (alone_ms / 1000.0), "ms_per_step": alone_ms / args.steps},
                "launch_shape": shape, "autotune_ms": tune_ms,
                "dtype": "f32" if prec == cuba.CUBA_FP32 else "f64", "data": "synthetic"}
        line["speedup_vs_alone"] = line["value"] / line["alone"]["value"]
        print(json.dumps(line), flush=True)
    elif world > 1:
        sum_over_ranks(C, world)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0





def run_serve_mode(args):
    """One server on one GPU; under torchrun only rank 0 serves (the request
    stream is one queue) and the other ranks exit at once."""
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    import torch
    from paper_1208_0961_gb300 import cuba
    from paper_1208_0961_gb300 import serve as S
    torch.cuda.set_device(0)
    cuba.load()
    prec = cuba.CUBA_FP32 if args.precision == "fp32" else cuba.CUBA_FP64
    reqs = S.poisson_stream(n_requests=args.serve_requests, rate_hz=args.serve_rate, seed=7)
    stream = torch.cuda.Stream()
    budget = int(args.serve_budget_gb * 1e9)
    if args.serve_classes == 1:
        backends = [S.CudaBackend(budget, precision=prec, max_sims=256, stream=stream)]
        srv = S.Server(backends, quantum=32)
    else:
        # cost classes (step under 0.1 ms, under 1 ms, larger), each its own
        # batch and stream; the HBM budget split 10 / 30 / 60 %
        fractions = (0.1, 0.3, 0.6)
        backends = [S.CudaBackend(budget * f, precision=prec, max_sims=256, stream=torch.cuda.Stream())
                    for f in fractions]
        srv = S.Server(backends, quantum=256, classify=S.cost_class, round_s=0.02)
    out = srv.run(reqs)
    for be in backends:
        be.close()
    line = {"mode": "serve", "metric": "served p50/p99 latency and particle-updates/s",
            "requests": len(reqs), "rate_hz": args.serve_rate, "budget_gb": args.serve_budget_gb,
            "served": out["served"], "rejected": out["rejected"], "p50_s": out["p50_s"], "p99_s": out["p99_s"],
            "updates_per_s": out["updates_per_s"], "offered_updates_per_s": out["offered_updates_per_s"],
            "makespan_s": out["makespan_s"], "classes": args.serve_classes,
            "dtype": "f32" if prec == cuba.CUBA_FP32 else "f64", "data": "synthetic"}
    if args.serve_alone:
        alone = S.run_alone(lambda r: S.CudaBackend.for_request(r, precision=prec, stream=stream), reqs)
        line["alone"] = {"p50_s": alone["p50_s"], "p99_s": alone["p99_s"], "updates_per_s": alone["updates_per_s"],
                         "makespan_s": alone["makespan_s"]}
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batch":
        return run_batch_mode(args)
    if args.mode == "serve":
        return run_serve_mode(args)
    import numpy as np
    import torch
    world, rank, local = dist_setup(args)
    from paper_1208_0961_gb300 import cuba
    from paper_1208_0961_gb300 import workloads as W
    cuba.load()
    cfg = workload(args)
    prec = cuba.CUBA_FP32 if args.precision == "fp32" else cuba.CUBA_FP64
    p = cuba.make_params(L=cfg["L"], n_cells=cfg["n_cells"], dt=cfg["dt"], sigma_fm2=cfg["sigma_fm2"],
                         n_test=cfg["n_test"], precision=prec, seed=replica_seed(args.seed, rank),
                         acceptance=cuba.CUBA_ACCEPT_SKIP if args.acceptance == "skip" else cuba.CUBA_ACCEPT_ALL_PAIRS,
                         kappa=args.kappa, mass=args.mass, mu=args.mu)
    sim = cuba.Sim(p, args.n)
    stream = torch.cuda.Stream()
    if args.workload == "hotspot3d":
        sim.init_hotspot(args.n, cfg["T0"], cfg["dT"], cfg["width"], stream)
        args.no_cpu_baseline = True
    else:
        sim.init_riemann(args.n, cfg["T_left"], cfg["T_right"], stream)
    torch.cuda.synchronize()
    cuba.cuba_step(sim.h, args.warmup, stream)
    torch.cuda.synchronize()
    tuned = None
    tune_ms = None
    if args.shape:
        sm, sb, tb = (int(v) for v in args.shape.split(","))
        cuba.cuba_set_launch_shape(sim.h, sm, sb, tb)
    elif args.autotune:
        tuned, tune_ms = cuba.cuba_autotune_shape(sim.h, 2, stream)

    t_sim0 = cuba.cuba_get_time(sim.h)[0]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    cuba.cuba_step(sim.h, args.steps, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    sim_fm_per_step = (cuba.cuba_get_time(sim.h)[0] - t_sim0) / args.steps
    ms_max = max_over_ranks(ms, world)
    value = replica_rate(args.n * args.steps, world, ms_max / 1000.0)

    # per-phase device times, kernel by kernel with events on the same stream
    phase = cuba.cuba_step_profiled(sim.h, args.profile_steps, stream)
    phase_names = ["stream_key", "sort_bin", "cell_prep", "pair_tile", "resolve", "advance"]
    stats = sim.stats()
    pk, pk_kind = peaks()
    nsteps_total = args.warmup + args.steps + args.profile_steps
    pairs_per_step = stats["pair_tests"] / max(1, stats["steps"])
    pair_ms = phase[3] / max(1, args.profile_steps)
    sm_mhz = clk.get("sm_mhz") or pk.get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(0).multi_processor_count
    # pair tile: bound by the integer multiply pipe.  Every pair test costs
    # one 32x32->64 multiply (16 per 16-pair Philox block once the
    # row-invariant part of rounds 1-3 is hoisted); the FMA-heavy pipe issues
    # them at 32 lanes per clock per SM, so the ceiling is n_SM x 32 x f_SM
    # pair tests/s.  The issue-slot view (43 algorithmic lane-ops per block:
    # 16 multiplies, 18 xors, 9 for the byte test, against 128 lanes per clock
    # per SM) and the FP32 view are reported beside it.
    ops_per_pair = 43.0 / 16.0
    pair_s = pair_ms / 1000.0
    peak_tops = n_sm * 128 * sm_mhz * 1e6 / 1e12
    achieved_tops = pairs_per_step * ops_per_pair / pair_s / 1e12
    pipe_peak = n_sm * 32 * sm_mhz * 1e6
    roofline = {"bound": "alu", "achieved": pairs_per_step / pair_s / 1e12, "peak": pipe_peak / 1e12,
                "unit": "T pair tests/s (one 32x32->64 integer multiply each)",
                "frac": pairs_per_step / pair_s / pipe_peak, "traffic": pair_tile_traffic(),
                "kernel": "k_pair_tile (+ k_pair_finish)",
                "peak_basis": "%d SMs x 32 multiplies/clk x %.0f MHz (sampled median)" % (n_sm, sm_mhz),
                "issue_lane_ops": {"ops_per_pair": ops_per_pair, "achieved_tops": achieved_tops,
                                   "peak_tops": peak_tops, "frac": achieved_tops / peak_tops},
                # the pair-test rate against the FP32 peak, at the 9 flops per
                # pair an FP32 all-pairs tile would spend (dot product, P22,
                # uniform conversion, compare)
                "fp32_equivalent": {"flops_per_pair": 9,
                                    "achieved_tflops": 9.0 * pairs_per_step / pair_s / 1e12,
                                    "peak_tflops": n_sm * 128 * 2 * sm_mhz * 1e6 / 1e12,
                                    "frac": 9.0 * pairs_per_step / pair_s / (n_sm * 128 * 2 * sm_mhz * 1e6)}}
    # stream/bin phases against HBM: 56 algorithmic bytes per update (FP32)
    bpu = 56.0 if prec == cuba.CUBA_FP32 else 104.0
    sb_ms = (phase[0] + phase[1]) / max(1, args.profile_steps)
    hbm = {"phases": "stream_key+sort_bin", "achieved_gbs": args.n * bpu / (sb_ms / 1000.0) / 1e9,
           "peak_gbs": pk.get("hbm_gbs"), "bytes_per_update": bpu}
    hbm["frac"] = hbm["achieved_gbs"] / hbm["peak_gbs"] if hbm["peak_gbs"] else None
    if args.acceptance == "skip":
        # skip-ahead: the pair phase draws one Philox block per row plus one
        # per candidate, far below the stream/bin phases; those (HBM) are the
        # dominant work and the roofline reported
        roofline = {"bound": "hbm", "achieved": hbm["achieved_gbs"], "peak": hbm["peak_gbs"], "unit": "GB/s",
                    "frac": hbm["frac"], "traffic": None,
                    "kernel": "k_stream_hist + histogram scan + k_bin_final (stream/bin phases)",
                    "bytes_per_update": bpu}

    # end to end through the C ABI with host buffers: H2D state, one step,
    # D2H observables, every step
    e2e = None
    if args.e2e_steps > 0:
        host = torch.empty((6, args.n), dtype=torch.float32 if prec == cuba.CUBA_FP32 else torch.float64,
                           pin_memory=True)
        cuba.cuba_get_state(sim.h, host.data_ptr(), stream)
        nc = cfg["n_cells"][0] * cfg["n_cells"][1] * cfg["n_cells"][2]
        T00 = torch.empty(nc, dtype=torch.float64, pin_memory=True)
        T0x = torch.empty(nc, dtype=torch.float64, pin_memory=True)
        cnt = torch.empty(nc, dtype=torch.int32, pin_memory=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            cuba.cuba_set_state(sim.h, host.data_ptr(), args.n, stream)
            cuba.cuba_step(sim.h, 1, stream)
            cuba.cuba_observables(sim.h, T00.data_ptr(), T0x.data_ptr(), cnt.data_ptr(), stream)
        t1 = time.perf_counter()
        e2e_s = max_over_ranks(t1 - t0, world)
        e2e = {"value": replica_rate(args.n * args.e2e_steps, world, e2e_s), "unit": "particle-updates/s",
               "h2d_bytes_per_step": host.numel() * host.element_size(),
               "d2h_bytes_per_step": nc * (8 + 8 + 4), "steps": args.e2e_steps}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r, cores, sample, dt = cpu_sample(args, cfg, args.cpu_sample_steps)
        cpu = {"value": r, "unit": "particle-updates/s", "cores": cores, "kind": "oracle", "sample": sample,
               "seconds": dt}
        if (prec == cuba.CUBA_FP32 and args.workload == "riemann1d" and args.acceptance == "all-pairs"
                and args.mass == 0.0 and args.mu == 0.0 and args.kappa == 0.0):
            # the FP32-vs-FP64-oracle error of this result, on the same strip
            cpu["fp32_vs_fp64_oracle"] = fp32_vs_fp64_oracle(args, cfg)

    if rank == 0:
        line = {
            "metric": "particle-updates/s (stream+bin+collide)", "value": value, "unit": "particle-updates/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_max / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32" if prec == cuba.CUBA_FP32 else "f64", "data": "synthetic",
            "config": {"workload": cfg["name"], "n_particles": args.n, "n_cells": args.cells, "dt": args.dt,
                       "sigma_mb": args.sigma_mb, "precision": args.precision, "n_test": cfg["n_test"],
                       "acceptance": args.acceptance, "kappa": args.kappa, "mass": args.mass, "mu": args.mu,
                       "simulated_fm_per_step": sim_fm_per_step,
                       "l2": "state %.0f MB > L2, no flush" % (args.n * 24 / 1e6 * (2 if prec else 1)),
                       "parallelism": "replicas" if world > 1 else "single",
                       "launch_shape": cuba.cuba_get_launch_shape(sim.h), "autotune_ms": tune_ms},
            "clocks": clk,
            "gpu_launches": launches_per_step(cfg["n_cells"][0] * cfg["n_cells"][1] * cfg["n_cells"][2],
                                              cuba.cuba_get_small_max(sim.h), args.acceptance == "skip",
                                              args.kappa > 0, neighbour_sort(args.n, cfg)) * args.steps,
            "roofline": roofline,
            "hbm_phases": hbm,
            "phase_ms_per_step": {k: v / max(1, args.profile_steps) for k, v in zip(phase_names, phase)},
            "pair_tests_per_step": pairs_per_step,
            "candidates_per_step": stats["candidates"] / max(1, stats["steps"]),
            "accepted_per_step": stats["accepted"] / max(1, stats["steps"]),
            "executed_per_step": stats["executed"] / max(1, stats["steps"]),
            "e2e": e2e,
            "cpu_baseline": cpu,
            "peaks": pk_kind,
        }
        print(json.dumps(line), flush=True)
    sim.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
