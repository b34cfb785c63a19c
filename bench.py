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


def parse(argv=None):
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
    ap.add_argument("--extras", type=int, default=1,
                    help="on one GPU, add the other workloads to the line: config1 (20 k particles, FP64, "
                         "100 steps), hotspot3d (64 M particles, 128^3 cells), batch (256-member ensemble) and "
                         "serve (400 Poisson requests at 20/s, and a sustainable rate)")
    ap.add_argument("--extra-steps", type=int, default=20, help="timed steps of the hotspot3d and batch extras")
    return ap.parse_args(argv)


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


def launches_per_step(ncells, small_max, skip=False, adaptive=False, neighbour=False, split_stream=False):
    """Kernels of one step: the stream/sort kernels — radix: streaming
    histogram (FP64 with fewer 4096-particle tiles than SMs: a streaming
    kernel first, split_stream); per radix pass the digit histogram (passes
    after the first), 3 scan kernels and the ranking kernel, then (two passes
    or more) the gather;
    neighbour-move sort: count pass, offsets, 3 scan kernels, scatter pass —;
    cell preparation + its scan (one kernel up to 4095 cells, else 3);
    small-cell and tiled pair kernels and the survivor kernel (skip-ahead: the
    scan of its row blocks and its pair kernel); small-cell and per-cell
    resolve kernels; the step counter."""
    p = bin_passes(ncells)
    scan = 1 if ncells + 1 <= 4096 else 3   # one-block scan of up to two 2048-entry tiles
    sort = 3 + scan if neighbour else 1 + 4 * p + (p - 1) + (1 if p > 1 else 0) + (1 if split_stream else 0)
    small = 1 if small_max else 0
    pairs = scan + 1 if skip else 1 + small + 1
    return (1 if adaptive else 0) + sort + 1 + scan + pairs + (1 + small) + 1


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def pair_tile_traffic(cfg, pairs_per_step):
    """DRAM bytes of one pair-tile launch from ncu_traffic.json (written by
    ncu_traffic.py from a one-pass ncu capture of this workload), or None if
    the kernel's sources or the workload differ from the capture's."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "ncu_traffic.json")) as f:
            rec = json.load(f)["k_pair_tile"]
        h = hashlib.sha256()
        for name in ["kernels_pairs.cu", "engine.cuh", "philox.cuh", "fp.cuh"]:
            with open(os.path.join(ROOT, "paper_1208_0961_gb300", "csrc", name), "rb") as fh:
                h.update(fh.read())
        if rec["source_sha256"] == h.hexdigest() and rec["workload"] == cfg["name"]:
            return rec["dram_bytes_per_launch"]
    except (OSError, KeyError, ValueError):
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


def batch_result(args, world, rank):
    """The batched ensemble (256 independent 1D Riemann runs in one arena, one
    captured graph per step) against the plain loop (each member alone through
    the single-simulation API, same steps).  Returns the line on rank 0."""
    import torch
    from paper_1208_0961_gb300 import cuba
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
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize()
    e0.record(stream)
    b.step(args.steps, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), world)
    ids = list(b.members)
    pair_tests = sum(b.stats(i)["pair_tests"] for i in ids) / (args.warmup + args.steps)
    b.close()
    # the plain loop: each member alone (single-simulation API), same steps
    alone_ms = 0.0
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
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
    clk_alone = clocks.stop()
    alone_ms = max_over_ranks(alone_ms, world)
    # the updates of all ranks over the slowest rank's time
    tot = sum_over_ranks(N, world)
    cells = sum_over_ranks(C, world)
    if rank != 0:
        return None
    line = {"mode": "batch", "metric": "particle-updates/s (stream+bin+collide), batched ensemble",
            "config": {"workload": "ensemble-%d-riemann-1d" % args.batch_sims, "members": args.batch_sims,
                       "particles": int(tot), "cells": int(cells),
                       "members_drawn": "N log-uniform 5e4-4e6, cells log-uniform 100-2000, sigma log-uniform "
                                        "0.5-50 mb, T_L/T_R from 400/320, 500/300, 350/250 MeV, "
                                        "dt = min(dx/2, 0.1 lambda), seed 1000 + k",
                       "timed_steps": args.steps, "steps_per_member_in_config": 300},
            "value": tot * args.steps / (ms / 1000.0), "unit": "particle-updates/s", "steps": args.steps,
            "warmup": args.warmup, "n_gpus": world, "scaling": "weak", "ms_per_step": ms / args.steps,
            "pair_tests_per_step": pair_tests, "clocks": clk,
            "alone": {"value": tot * args.steps / (alone_ms / 1000.0), "ms_per_step": alone_ms / args.steps,
                      "clocks": clk_alone, "what": "each member alone, single-simulation API, default shape"},
            "launch_shape": shape, "autotune_ms": tune_ms,
            "dtype": "f32" if prec == cuba.CUBA_FP32 else "f64", "data": "synthetic"}
    line["speedup_vs_alone"] = line["value"] / line["alone"]["value"]
    return line


def run_batch_mode(args):
    world, rank, local = dist_setup(args)
    line = batch_result(args, world, rank)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def serve_result(args, rate_hz, n_requests, alone=True):
    """The served request stream (Poisson arrivals at rate_hz, n_requests,
    seed 7) through cost-class batches under the HBM budget, and the plain
    one-at-a-time loop on the same requests; clocks sampled during each."""
    import torch
    from paper_1208_0961_gb300 import cuba
    from paper_1208_0961_gb300 import serve as S
    cuba.load()
    prec = cuba.CUBA_FP32 if args.precision == "fp32" else cuba.CUBA_FP64
    reqs = S.poisson_stream(n_requests=n_requests, rate_hz=rate_hz, seed=7)
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
        srv = S.Server(backends, classify=S.cost_class)
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    out = srv.run(reqs)
    clk = clocks.stop()
    host = {"admit_s": [round(be.admit_s, 3) for be in backends], "retire_s": [round(be.finish_s, 3) for be in backends]}
    for be in backends:
        be.close()
    line = {"mode": "serve", "metric": "served p50/p99 latency and particle-updates/s",
            "config": {"workload": "poisson-%d-requests-%gHz" % (n_requests, rate_hz), "requests": n_requests,
                       "rate_hz": rate_hz, "seed": 7, "budget_gb": args.serve_budget_gb,
                       "mix": "half 1D Riemann (about 1000 particles per cell), half 3D thermal boxes (0.1 fm "
                              "cells, about 30 per cell); N log-uniform 1e4-8e6, 50-500 steps, sigma 0-100 mb"},
            "served": out["served"], "rejected": out["rejected"], "p50_s": out["p50_s"], "p99_s": out["p99_s"],
            "mean_s": out["mean_s"], "updates_per_s": out["updates_per_s"],
            "offered_updates_per_s": out["offered_updates_per_s"], "makespan_s": out["makespan_s"],
            "classes": args.serve_classes, "host_seconds_per_class": host, "clocks": clk,
            "dtype": "f32" if prec == cuba.CUBA_FP32 else "f64", "data": "synthetic"}
    if alone:
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        a = S.run_alone(lambda r: S.CudaBackend.for_request(r, precision=prec, stream=stream), reqs)
        line["alone"] = {"p50_s": a["p50_s"], "p99_s": a["p99_s"], "mean_s": a["mean_s"],
                         "updates_per_s": a["updates_per_s"], "makespan_s": a["makespan_s"],
                         "clocks": clocks.stop(), "what": "one request at a time, in arrival order, each in a "
                                                          "batch of its own"}
    return line


def run_serve_mode(args):
    """One server on one GPU; under torchrun only rank 0 serves (the request
    stream is one queue) and the other ranks exit at once."""
    if int(os.environ.get("RANK", "0")) != 0:
        return 0
    import torch
    torch.cuda.set_device(0)
    line = serve_result(args, args.serve_rate, args.serve_requests, alone=bool(args.serve_alone))
    print(json.dumps(line), flush=True)
    return 0


def run_step(args, world, rank):
    """One simulation (the workload args name) advanced K graph-replayed steps;
    returns the JSON line (rank 0) with its roofline, phase split, end-to-end
    rate and CPU baseline."""
    import torch
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
    # pair tile (the dominant kernel): the FP32 view is the headline
    # roofline -- 9 flops per pair test (dot product, P22, uniform conversion,
    # compare) against n_SM x 128 FP32 lanes x 2 x f_SM.  Beside it, the units
    # that bind this integer kernel: the 32x32->64 multiply pipe (one multiply
    # per pair test: 16 per 16-pair Philox block once the row-invariant part
    # of rounds 1-3 is hoisted, issued at 32 lanes per clock per SM), and the
    # issue slots (43 algorithmic lane-ops per block: 16 multiplies, 18 xors,
    # 9 for the byte test, against 128 lanes per clock per SM).
    ops_per_pair = 43.0 / 16.0
    pair_s = pair_ms / 1000.0
    rate = pairs_per_step / pair_s
    fp32_peak = n_sm * 128 * 2 * sm_mhz * 1e6
    peak_tops = n_sm * 128 * sm_mhz * 1e6 / 1e12
    pipe_peak = n_sm * 32 * sm_mhz * 1e6
    roofline = {"bound": "alu", "achieved": 9.0 * rate / 1e12, "peak": fp32_peak / 1e12,
                "unit": "TFLOP/s FP32-equivalent (9 flops per pair test)", "frac": 9.0 * rate / fp32_peak,
                "traffic": pair_tile_traffic(cfg, pairs_per_step), "kernel": "k_pair_tile (+ k_pair_finish)",
                "peak_basis": "%d SMs x 128 FP32 lanes x 2 x %.0f MHz (sampled median)" % (n_sm, sm_mhz),
                "pair_tests_per_s": rate,
                "multiply_pipe": {"achieved": rate / 1e12, "peak": pipe_peak / 1e12,
                                  "unit": "T pair tests/s (one 32x32->64 integer multiply each)",
                                  "frac": rate / pipe_peak,
                                  "peak_basis": "%d SMs x 32 multiplies/clk x %.0f MHz" % (n_sm, sm_mhz)},
                "issue_lane_ops": {"ops_per_pair": ops_per_pair, "achieved_tops": rate * ops_per_pair / 1e12,
                                   "peak_tops": peak_tops, "frac": rate * ops_per_pair / 1e12 / peak_tops}}
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

    line = None
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
                                              args.kappa > 0, neighbour_sort(args.n, cfg),
                                              prec == cuba.CUBA_FP64 and (args.n + 4095) // 4096 < n_sm) * args.steps,
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
    sim.close()
    return line


def extras(args):
    """The other workloads of the benchmark, each timed on its own with its
    own clock record: config1 (the paper-sized 1D Riemann run, FP64, with the
    oracle timed on the whole run), hotspot3d, the batched ensemble and the
    served request stream (config rate, then 85 % and 95 % of the rate the
    server carried at it)."""
    import copy
    out = {}
    # config 1: 20 k particles, 100 cells, dt = 0.05, 100 steps, FP64
    a = copy.copy(args)
    a.workload, a.n, a.cells, a.dt, a.sigma_mb, a.precision = "riemann1d", 20000, 100, 0.05, 10.0, "fp64"
    a.steps, a.warmup, a.e2e_steps, a.no_cpu_baseline, a.profile_steps = 100, 5, 0, True, 3
    line = run_step(a, 1, 0)
    out["config1"] = _sub(line, "20 k particles, 10x1x1 fm, 100 cells, dt 0.05 fm/c, sigma 10 mb, FP64, 100 steps")
    out["config1"]["oracle_full_run"] = oracle_full_run(a)
    # config 3: 64 M particles, 128^3 cells, hot spot, sigma 5 mb, dt 0.01
    a = copy.copy(args)
    a.workload, a.n, a.cells, a.dt, a.sigma_mb, a.precision = "hotspot3d", 64_000_000, 128, 0.01, 5.0, "fp32"
    a.steps, a.e2e_steps, a.no_cpu_baseline = args.extra_steps, 0, True
    line = run_step(a, 1, 0)
    out["hotspot3d"] = _sub(line, "12.8^3 fm box, 128^3 cells, 64 M particles at T = 400 MeV plus a hot spot "
                                  "(600 MeV peak, width 1 fm), sigma 5 mb, dt 0.01 fm/c, FP32; %d timed steps "
                                  "of the config's 200" % a.steps)
    # config 4: the batched ensemble
    a = copy.copy(args)
    a.steps, a.precision = args.extra_steps, "fp32"
    out["batch"] = batch_result(a, 1, 0)
    # config 5: the served stream at its rate, then at a rate the server sustains
    a = copy.copy(args)
    a.precision = "fp32"
    s5 = serve_result(a, args.serve_rate, args.serve_requests)
    out["serve"] = s5
    cap = s5["updates_per_s"]
    for key, frac in (("serve_sustainable", 0.85), ("serve_near_capacity", 0.95)):
        sustain = min(args.serve_rate, args.serve_rate * frac * cap / max(s5["offered_updates_per_s"], 1.0))
        if sustain < args.serve_rate:
            s_low = serve_result(a, round(sustain, 2), 200)
            s_low["config"]["why"] = ("the config's rate offers more than the server carries: %d %% of the carried "
                                      "rate, 200 requests" % round(100 * frac))
            out[key] = s_low
    return out


def default_workload(args):
    """Whether args name the headline workload (the extras run beside it
    only, so that a run of another workload, e.g. under a profiler, times
    that workload alone)."""
    d = parse([])
    keys = ("workload", "n", "cells", "dt", "sigma_mb", "precision", "acceptance", "mass", "mu", "kappa", "seed")
    return all(getattr(args, k) == getattr(d, k) for k in keys)


def _sub(line, desc):
    keep = ("metric", "value", "unit", "steps", "warmup", "ms_per_step", "dtype", "config", "clocks",
            "gpu_launches", "roofline", "hbm_phases", "phase_ms_per_step", "pair_tests_per_step",
            "accepted_per_step", "executed_per_step")
    sub = {k: line[k] for k in keep if k in line}
    sub["config"] = dict(sub["config"], description=desc)
    return sub


def oracle_full_run(a):
    """The oracle on the whole config-1 run (20 k particles, 100 steps, FP64)
    on the host cores."""
    from oracle import oracle as O
    cfg = workload(a)
    op = O.make_params(L=cfg["L"], n=cfg["n_cells"], dt=cfg["dt"], sigma_fm2=cfg["sigma_fm2"], n_test=cfg["n_test"],
                       seed=a.seed)
    st = O.init_thermal(op, a.n, cfg["regions"])
    st, _, _, _ = O.sort(op, st)
    t0 = time.perf_counter()
    for k in range(a.steps):
        st, _ = O.step(op, k, st, trace=False)
    dt = time.perf_counter() - t0
    return {"value": a.n * a.steps / dt, "unit": "particle-updates/s", "cores": O.threads(), "kind": "oracle",
            "seconds": dt, "sample": "the whole run: %d particles, %d steps" % (a.n, a.steps)}


def main(argv=None):
    args = parse(argv)
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batch":
        return run_batch_mode(args)
    if args.mode == "serve":
        return run_serve_mode(args)
    world, rank, local = dist_setup(args)
    line = run_step(args, world, rank)
    if line is not None and world == 1 and args.extras and default_workload(args):
        line["extras"] = extras(args)
    if line is not None:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
