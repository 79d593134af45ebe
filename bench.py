#!/usr/bin/env python3
"""Benchmark of the bit-sliced Gillespie hot path on GB300.

Workload (one "step" = one full pass of the hot path over one batch): Frank's
model with unit rates, N_tot = 1024 from (L, D, A) = (256, 256, 512), 2^20 runs
per GPU (32768 groups of 32 runs), seed 0, fp64 clock, t_end = 50, 10
log-spaced snapshot times 50 * 10^(4 (s - 9) / 9) with the 65-bin
enantiomeric-excess histogram at each, the absorption time of every run.  Every
step restarts from t = 0, so all steps do the same work.

Prints one JSON line: lane-reactions/s (real reactions only) as `value`, with
absorbed runs/s, lane-steps/s, the roofline of the kernel against the
integer-ALU issue peak, the end-to-end figure through the C ABI with host
buffers, the one-thread-per-run GPU baseline on the same workload, and the CPU
oracle timed on a bounded sample.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU: launched by torch.distributed.run, one rank per GPU; rank r holds
runs [r 2^20, (r+1) 2^20) of one ensemble (weak scaling, no data-path
collective; the per-rank histograms are summed after the timed region).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "lane-reactions/s and absorbed runs/s on 1 GB300, bit-sliced vs 1-thread-per-run SSA"
N_TOT = 1024
INIT = (256, 256, 512)
RUNS_PER_GPU = 1 << 20
SEED = 0
T_END = 50.0
N_SNAP = 10
SNAPS = [T_END * 10.0 ** (4.0 * (s - (N_SNAP - 1)) / (N_SNAP - 1)) for s in range(N_SNAP)]
L2_BYTES = 129 * 2**20
# DRAM bytes (read + write) of one launch of the one-thread bit-sliced kernel on the default
# workload, from one ncu capture, keyed by a fingerprint of the kernel's sources (below): a
# kernel changed since its capture has no entry and reports null.
KERNEL_SOURCES = ("frank_kernel.cuh", "frank_tail.cuh", "bitslice.cuh", "philox.cuh", "internal.h",
                  "frank_instance.cu")
TRAFFIC_BYTES_PER_LAUNCH = {"c23af68050df54d3": 3_193_344 + 1_005_056,
                            "995f30d5dca30e9a": 3_229_696 + 931_584}


def kernel_fingerprint() -> str:
    """sha256 (16 hex digits) of the one-thread kernel's source files."""
    import hashlib
    h = hashlib.sha256()
    for name in KERNEL_SOURCES:
        with open(os.path.join(ROOT, "paper_2412_16613_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def device_sm_count_and_max_mhz(index: int):
    """SM count from the device properties; the maximum SM clock from nvidia-smi (MHz)."""
    import torch
    sms = torch.cuda.get_device_properties(index).multi_processor_count
    mhz, basis = None, "nvidia-smi clocks.max.sm"
    try:
        out = subprocess.run(["nvidia-smi", "-i", str(index), "--query-gpu=clocks.max.sm",
                              "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=30).stdout
        mhz = float(out.strip().splitlines()[0])
    except Exception:
        khz = getattr(torch.cuda.get_device_properties(index), "clock_rate", None)
        if khz:
            mhz, basis = khz / 1e3, "device property clock_rate"
    if not mhz:
        mhz, basis = 2070.0, "not readable: GB300's listed maximum"
    return sms, mhz, basis


def layout_name(bits: int) -> str:
    """The layouts counter 9 reports: one thread / three warps, and the general kernel's mode."""
    names = [n for bit, n in ((1, "thread"), (2, "warps"), (4, "general incremental"), (8, "general products"),
                              (16, "tail one run per thread"), (32, "planes in registers")) if bits & bit]
    return "+".join(names) or "none"


def general_ops_per_group_step(K: int, b: int, products: bool) -> int:
    """Word operations of one group step of Frank's model on the general kernel.  Per reaction:
    the selection of its changer word (3K: the running sum and the comparison, or the subtraction
    of h_r from what is left of n and its borrow, 2K, as the kernel does it), and either a b x b
    schoolbook product (3 b^2: AND, sum, carry) or the change of h_r (two scaled counts, 4 ops a
    plane, and a small constant, 2 ops a plane: 10K).  Per species the change planes (3R) and the
    masked add (2b).  The Philox calls (20 LOP3 each).  The per-unit figure keeps 3K so that it
    does not move with the kernel's way of doing the selection."""
    per_reaction = 3 * K + (3 * b * b if products else 10 * K)
    return 3 * per_reaction + 3 * (2 * b + 3 * 3) + 20 * ((K + 2 + 3) // 4)


def algorithmic_ops_per_group_step(K: int, b: int, pad: int = 0) -> int:
    """Word operations one group step must do (27K + 6b logic plus 20 LOP3 per Philox call
    for the ceil((K+2)/4) calls of n and tau); a bound padded to 2^K has no rejection test
    (K fewer); the state-following bound (pad 2) adds the reduction of S_R's planes over the
    live lanes and the mask of n's planes above it (2K more)."""
    return {0: 27, 1: 26, 2: 28}[int(pad)] * K + 6 * b + 20 * ((K + 2 + 3) // 4)


def lattice_ops_per_group_step(K: int, B: int, rho_r: int) -> int:
    """Word operations of one group step of the lattice kernel, with B count planes (the bit length
    of the cap m) and K planes of n: the hop test (K), the molecule's species by two
    adds and three comparisons over B planes (7B), the three products A L, A (L + D) and L D by
    schoolbook (3 x 3B^2: AND, sum, carry) and S_3's add (4B), n minus the hop slots (2K), rho_r S_r
    for the three sums (2K an add per further set bit of rho_r), three comparisons over K planes
    (3K), the changer words (6), the masked updates of three counts (12B), and 20 LOP3 per Philox
    call for the ceil((K + 3) / 4) calls of the step's words."""
    extra_bits = max(0, bin(int(rho_r)).count("1") - 1)
    return (K + 7 * B + 9 * B * B + 4 * B + 2 * K + 3 * 2 * K * extra_bits + 3 * K + 6 + 12 * B
            + 20 * ((K + 3 + 3) // 4))


def bit_length(v: int) -> int:
    return int(v).bit_length()


def env_rank():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int, path: str):
        self.path, self.proc = path, None
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.f = open(path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(sample_runs: int, threads: int):
    """The oracle as it stands, on the host cores, on runs 0..sample_runs-1 of the workload."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    r = oracle.run(oracle.frank(), INIT, sample_runs, seed=SEED, t_end=T_END, snap_times=SNAPS,
                   threads=threads, pad_pow2=PAD, ensemble_runs=0)
    dt = time.perf_counter() - t0
    reactions = int(r["reactions"].sum())
    return {"value": reactions / dt, "unit": "lane-reactions/s", "cores": threads, "kind": "oracle",
            "sample": f"runs 0..{sample_runs - 1} of the workload (all snapshots, to absorption or t_end), "
                      f"{dt:.1f} s wall on {threads} threads",
            "absorbed_runs_per_s": int((r["outcome"] >= 0).sum()) / dt, "seconds": dt}


def run_reference(args, rank, world):
    """The reference arm: the CPU oracle on the same workload and metric, bounded samples."""
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    per_step = args.ref_runs
    import oracle
    oracle.build()
    for _ in range(args.warmup):
        oracle.run(oracle.frank(), INIT, 64, seed=SEED, t_end=T_END, snap_times=SNAPS, threads=threads,
                   pad_pow2=PAD, ensemble_runs=0)
    total_react, total_abs, total_t = 0, 0, 0.0
    for k in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.run(oracle.frank(), INIT, per_step, first_run=k * per_step, seed=SEED, t_end=T_END,
                       snap_times=SNAPS, threads=threads, pad_pow2=PAD, ensemble_runs=0)
        total_t += time.perf_counter() - t0
        total_react += int(r["reactions"].sum())
        total_abs += int((r["outcome"] >= 0).sum())
    value = total_react / total_t
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "lane-reactions/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * total_t / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": workload_config(world),
            "absorbed_runs_per_s": total_abs / total_t,
            "cpu_baseline": {"value": value, "unit": "lane-reactions/s", "cores": threads, "kind": "oracle",
                             "sample": f"{per_step} runs per step of the workload (runs k*{per_step}.. for "
                                       f"step k), host threads"},
            "e2e": {"value": value, "unit": "lane-reactions/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


WORKLOAD = "c2"
BATCH = None
PRECISION = 0
PAD = 1  # 1: uniformisation bound padded to 2^K (no rejected draws of n); --pad 0 for N(N-1)/2
ENGINE = 0  # 0: Frank's kernels; 2: the general-network kernel
PRECISION_NAMES = {0: "p64", 1: "p32kahan", 2: "p32d64acc", 3: "p64logsum", 4: "p32plain"}


def set_workload(name, runs):
    """Workload constants: the metric's workload (c2) or the other configurations."""
    global WORKLOAD, N_TOT, INIT, RUNS_PER_GPU, T_END, SNAPS, BATCH
    WORKLOAD = name
    if name == "c4":
        N_TOT, INIT, RUNS_PER_GPU = 10000, (2500, 2500, 5000), 1 << 22
    if name == "c3":
        from paper_2412_16613_gb300 import workloads
        BATCH = workloads.batch_ensembles()
        RUNS_PER_GPU = int(BATCH["runs"].sum())
    if runs:
        RUNS_PER_GPU = runs


def workload_config(world):
    if WORKLOAD == "c3":
        return {"workload": f"frank_batch{len(BATCH['runs'])}ens_N16-65536loguniform_rates0.5-2_runs1024_tend{T_END:g}"
                            f"_snap{N_SNAP}log",
                "model": "Frank, per-ensemble rates", "ensembles": len(BATCH["runs"]),
                "runs": RUNS_PER_GPU * world, "runs_per_gpu": RUNS_PER_GPU, "t_end": T_END,
                "global_batch": RUNS_PER_GPU * world, "parallelism": f"replicas x{world}",
                "bound": BOUND_NAMES[PAD], "l2": "L2 flushed between timed steps (256 MiB write)"}
    return workload_config_single(world)


BOUND_NAMES = ["lambda_int = N(N-1)/2, rejected draws redrawn", "lambda_int padded to 2^K with null events",
               "2^p per step, p = bit length of the largest S_R over the group's live runs"]


def workload_config_single(world):
    return {"workload": f"frank_N{N_TOT}_{INIT[0]}-{INIT[1]}-{INIT[2]}_runs{RUNS_PER_GPU}xgpu_tend{T_END:g}"
                        f"_snap{N_SNAP}log_{PRECISION_NAMES[PRECISION]}",
            "model": "Frank (A+L->2L, A+D->2D, L+D->2A), k=(1,1,1)", "N_tot": N_TOT, "init": list(INIT),
            "runs": RUNS_PER_GPU * world, "runs_per_gpu": RUNS_PER_GPU, "groups_per_gpu": RUNS_PER_GPU // 32,
            "seed": SEED, "t_end": T_END, "snapshots": SNAPS, "precision": PRECISION_NAMES[PRECISION],
            "global_batch": RUNS_PER_GPU * world, "parallelism": f"replicas x{world} (run shards)",
            "bound": BOUND_NAMES[PAD], "engine": ENGINE_NAMES[ENGINE],
            "l2": "L2 flushed between timed steps (256 MiB write)"}


C5_SIDE, C5_RUNS, C5_HOP = 64, 4096, 0.1


def lattice_leg(pkg, stream, local, t_end, rank, world, flush, runs=C5_RUNS, timed=2, warm=True):
    """Frank's model on the 64 x 64 periodic lattice: 4096 runs per GPU from per-site Poisson
    counts of means (8, 8, 16), unit rates, hops at d = 0.1, fp32 Kahan clock, snapshots at
    t_end / 2 and t_end; one warm-up run, then two runs timed with CUDA events after an L2 flush
    (a run to the workload's own t_end = 50 is timed once, without the warm-up).  Lane
    steps count every run of every group step; the roofline counts the word operations of each
    group's steps at its final cap."""
    import torch
    from paper_2412_16613_gb300 import sharding, workloads
    M = C5_SIDE * C5_SIDE
    init = workloads.lattice_init(C5_SIDE, C5_SIDE, runs)
    o = pkg.ssa_default_options(cuda_stream=stream, device=local, precision=pkg.SSA_P32_KAHAN,
                                first_run=sharding.weak_shard(runs, rank)[0])
    ctx = pkg.ssa_lattice_create(C5_SIDE, C5_SIDE, [1.0, 1.0, 1.0], C5_HOP, init, runs, SEED, o)
    snaps = [t_end / 2, t_end]
    if warm:
        pkg.ssa_lattice_run(ctx, t_end, snaps)
    ms, steps_total, react, hops, ops = [], 0, 0, 0, 0.0
    rho_r = int(round(1.0 / C5_HOP))
    for k in range(timed):
        flush.fill_(k + 11)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pkg.ssa_lattice_run(ctx, t_end, snaps)
        b.record(stream)
        torch.cuda.synchronize()
        ms.append(a.elapsed_time(b))
        cnt = pkg.ssa_lattice_fetch(ctx, pkg.SSA_LAT_COUNTERS)
        groups = pkg.ssa_lattice_fetch(ctx, pkg.SSA_LAT_GROUPS).reshape(-1, 3)
        steps_total += int(cnt[0])
        react += int(cnt[3])
        hops += int(cnt[4])
        for steps_g, m, _ in groups.tolist():
            K = bit_length(4 * (1 << bit_length(m - 1)) + rho_r * (m * (m - 1) // 2) - 1)
            ops += steps_g * lattice_ops_per_group_step(K, bit_length(m), rho_r)
    # the workload's outputs at the last snapshot: global ee of every run and its domain counts
    tot = pkg.ssa_lattice_fetch(ctx, pkg.SSA_LAT_SNAP_TOTALS).reshape(len(snaps), -1, 3)[-1].astype(np.float64)
    dom = pkg.ssa_lattice_fetch(ctx, pkg.SSA_LAT_SNAP_DOMAINS).reshape(len(snaps), -1, 2)[-1]
    th = pkg.ssa_lattice_fetch(ctx, pkg.SSA_LAT_HOMOCHIRAL_TIME)
    ld = tot[:, 0] + tot[:, 1]
    ee = np.where(ld > 0, (tot[:, 0] - tot[:, 1]) / np.maximum(ld, 1), 0.0)
    outputs = {"at_t": snaps[-1], "mean_abs_ee": float(np.abs(ee).mean()), "mean_ee": float(ee.mean()),
               "mean_L_domains": float(dom[:, 0].mean()), "mean_D_domains": float(dom[:, 1].mean()),
               "runs_single_species_by_t_end": int(np.isfinite(th).sum())}
    pkg.ssa_lattice_destroy(ctx)
    t = sum(ms) / 1e3
    sms, max_mhz, basis = device_sm_count_and_max_mhz(local)
    peak = sms * 64 * max_mhz * 1e6 / 1e9
    caps = {int(m): int(c) for m, c in zip(*np.unique(groups[:, 1], return_counts=True))}
    return {"workload": f"lattice_{C5_SIDE}x{C5_SIDE}_poisson8-8-16_runs{runs}xgpu_d{C5_HOP:g}_tend{t_end:g}_p32kahan",
            "t_end": t_end, "t_end_of_the_workload": 50.0, "steps": timed, "warmup": int(warm),
            "ms_per_step": statistics.mean(ms), "group_steps_per_s": steps_total * world / t,
            "lane_steps_per_s": 32 * steps_total * world / t, "lane_reactions_per_s": react * world / t,
            "lane_hops_per_s": hops * world / t, "groups_by_cap": caps,
            "rounds_per_group": int(cnt[1]) / max(1, len(groups)), "outputs": outputs,
            "roofline": {"bound": "alu", "achieved": ops / t / 1e9, "peak": peak, "unit": "Gop/s",
                         "frac": ops / t / 1e9 / peak,
                         "ops_per_group_step_at_cap_64": lattice_ops_per_group_step(15, 7, rho_r),
                         "peak_basis": f"{sms} SMs x 64 LOP3 lanes/clk/SM x {max_mhz:g} MHz ({basis})"}}


ENGINE_NAMES = {0: "Frank kernels (cumulative propensities, App. A increments)",
                2: "general kernel (propensities by bit-sliced products every step)"}


def main():
    global RUNS_PER_GPU
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-runs", type=int, default=4096)
    ap.add_argument("--cpu-sample", type=int, default=8192)
    ap.add_argument("--no-baselines", action="store_true", help="skip the K7 and CPU legs")
    ap.add_argument("--c4-steps", type=int, default=3,
                    help="timed runs of the N_tot = 10 000, 2^22-run workload per bound after the main "
                         "measurement (0: skip)")
    ap.add_argument("--c5-tend", type=float, default=0.05,
                    help="t_end of the lattice leg (64 x 64 sites, 4096 runs, d = 0.1, fp32 Kahan clock) "
                         "timed after the main measurement (0: skip); the workload's own t_end is 50")
    ap.add_argument("--block", type=int, default=0)
    ap.add_argument("--layout", type=int, default=0,
                    help="0 auto, 1 one thread per group of 32 runs, 2 three warps per 32 groups")
    ap.add_argument("--no-tune", action="store_true",
                    help="skip ssa_tune (by default it times every launch configuration on the "
                         "workload during warm-up and keeps the fastest; c3 keeps the per-bucket rule)")
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--tail", type=int, default=0,
                    help="ssa_options.tail_groups: 0 the library's choice, -1 never hand the last groups of "
                         "a warp to one run per thread, 1..4 the threshold")
    ap.add_argument("--pad", type=int, default=1, choices=[0, 1, 2],
                    help="1: pad the uniformisation bound to 2^K with null events, so that no draw of n "
                         "is rejected (the same process, sampled through a different draw); 2: a "
                         "power-of-two bound that follows each group's state")
    ap.add_argument("--engine", type=int, default=0, choices=[0, 2],
                    help="0: Frank's kernels; 2: the general-network kernel on the same workload")
    ap.add_argument("--recompute", type=int, default=0, choices=[0, 1, 2, 3],
                    help="ssa_options.recompute on the general engine: 0 the library's choice (planes in "
                         "registers where the network fits), 1 products every step, 2 incremental, 3 "
                         "incremental with the planes in shared memory")
    ap.add_argument("--budget", type=int, default=0,
                    help="stop every group after this many steps (profiling one phase of a launch; the "
                         "line then covers that phase only and says so)")
    ap.add_argument("--runs", type=int, default=0,
                    help="runs per GPU (smaller cases are for profiling; the metric is quoted at 2^20)")
    ap.add_argument("--workload", default="c2", choices=["c2", "c3", "c4", "c5"],
                    help="c2: N_tot=1024, 2^20 runs (the metric's workload); c3: 4096 ensembles "
                         "with log-uniform N_tot in [16, 65536] and rates in [0.5, 2], 1024 runs each; "
                         "c4: N_tot=10000, 2^22 runs; c5: the lattice leg alone (--c5-tend, --c5-runs), "
                         "for profiling it")
    ap.add_argument("--c5-runs", type=int, default=0, help="runs of the lattice leg (default 4096)")
    args = ap.parse_args()
    rank, world, local = env_rank()
    set_workload(args.workload, args.runs)
    global PRECISION, PAD, ENGINE
    PRECISION = args.precision
    PAD = args.pad
    ENGINE = args.engine

    if args.impl == "reference":
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group("gloo")
        run_reference(args, rank, world)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
            dist.destroy_process_group()
        return

    import torch
    import paper_2412_16613_gb300 as pkg
    torch.cuda.set_device(local)
    if WORKLOAD == "c5":  # the lattice leg alone, on rank 0's GPU (a profiling line)
        pkg.build()
        pkg.use_torch_allocator()
        flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")
        long_run = (args.c5_tend or 0.05) > 1.0  # a run to the workload's t_end: once, no warm-up
        line = lattice_leg(pkg, torch.cuda.current_stream(), local, args.c5_tend or 0.05, 0, 1, flush,
                           runs=args.c5_runs or C5_RUNS, timed=1 if long_run else 2, warm=not long_run)
        if rank == 0:
            print(json.dumps(line), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    pkg.build()
    pkg.use_torch_allocator()
    stream = torch.cuda.current_stream()
    from paper_2412_16613_gb300 import sharding
    first_run = sharding.weak_shard(RUNS_PER_GPU, rank)[0] if WORKLOAD != "c3" else 0
    opt = pkg.ssa_default_options(cuda_stream=stream, device=local, precision=args.precision,
                                  block_size=args.block, first_run=first_run, layout=args.layout,
                                  pad_pow2=PAD, engine=ENGINE, tail_groups=args.tail, step_budget=args.budget,
                                  recompute=args.recompute)
    if WORKLOAD == "c3":
        opt.first_run = 0
        ctx = pkg.ssa_create_batch(pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS, BATCH["init"], BATCH["rates"],
                                   BATCH["runs"], BATCH["seeds"] + np.uint64(rank * len(BATCH["runs"])), opt)
    else:
        ctx = pkg.ssa_create(pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS, [1.0, 1.0, 1.0], np.array(INIT),
                             RUNS_PER_GPU, SEED, opt)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.int32, device="cuda")

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    def run(ctx_, snaps=None):
        """ssa_run; with --budget every group stops at its budget, which the library reports."""
        try:
            pkg.ssa_run(ctx_, T_END, SNAPS if snaps is None else snaps)
        except pkg.SSAError as e:
            if not (args.budget and e.status == pkg.SSA_ETIMEOUT):
                raise

    def time_runs(ctx_, steps, snaps=None):
        """One warm-up run, then `steps` runs each timed with CUDA events after an L2 flush:
        mean ms per run, lane-reactions/s, the counters of the last run."""
        snaps = SNAPS if snaps is None else snaps
        run(ctx_, snaps)
        ms, react = [], 0
        for k in range(steps):
            flush.fill_(k + 7)
            a_, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a_.record(stream)
            run(ctx_, snaps)
            b_.record(stream)
            torch.cuda.synchronize()
            ms.append(a_.elapsed_time(b_))
            cnt = pkg.ssa_fetch(ctx_, pkg.SSA_FIELD_COUNTERS)
            react += int(cnt[2])
        return statistics.mean(ms), react / (sum(ms) / 1e3), cnt

    tuned = None
    if not args.no_tune and not args.budget and WORKLOAD != "c3" and args.layout == 0 and args.block == 0:
        tuned = pkg.ssa_tune(ctx, T_END, SNAPS, probe_steps=0)
    for _ in range(args.warmup):
        run(ctx)
    barrier()
    # the raw samples go to BENCH_CLOCKS_DIR when it is set (a summary is in the JSON line)
    clocks_dir = os.environ.get("BENCH_CLOCKS_DIR") or tempfile.gettempdir()
    os.makedirs(clocks_dir, exist_ok=True)
    clocks = Clocks(local, os.path.join(clocks_dir, f"clocks_rank{rank}.csv"))
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    reactions = absorbed = lane_steps = group_steps = max_group_steps = layout_used = 0
    barrier()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        flush.fill_(k)  # L2 flush, outside the kernel's event pair
        ev[k][0].record(stream)
        run(ctx)
        ev[k][1].record(stream)
        c = pkg.ssa_fetch(ctx, pkg.SSA_FIELD_COUNTERS)
        reactions += int(c[2])
        lane_steps += int(c[1])
        group_steps += int(c[0])
        absorbed += int(c[5])
        max_group_steps = max(max_group_steps, int(c[8]))
        layout_used = int(c[9])
    barrier()
    wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    kernel_ms = [a.elapsed_time(b) for a, b in ev]
    t_dev = sum(kernel_ms) / 1e3
    hist = pkg.ssa_fetch(ctx, pkg.SSA_FIELD_EE_HIST).reshape(-1, N_SNAP, 65).sum(0)
    # max over ranks of the device time; totals over ranks
    totals = torch.tensor([reactions, absorbed, lane_steps, group_steps], dtype=torch.float64, device="cuda")
    tmax = torch.tensor([t_dev], dtype=torch.float64, device="cuda")
    htot = torch.from_numpy(hist.astype(np.float64)).cuda()
    if dist is not None:
        dist.all_reduce(totals)
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        dist.all_reduce(htot)
    reactions, absorbed, lane_steps, group_steps = [float(x) for x in totals.tolist()]
    t_dev = float(tmax.item())

    # ---- roofline of the bit-sliced kernel (one launch per step; a batch runs one launch per
    # number of planes K, so its per-unit count is not a single figure and is not reported)
    sms, max_mhz, mhz_basis = device_sm_count_and_max_mhz(local)
    micro = None
    try:
        micro = pkg.bitssa_bench_alu(local, 4000)[0] / 1e9
    except Exception:
        pass

    def roofline_of(n_tot, pad, gs_per_launch, launch_ms, engine=ENGINE, layout_bits=1):
        K, b = bit_length(n_tot * (n_tot - 1) // 2), bit_length(n_tot)
        # the per-unit figure of the method (27K + 6b logic, 20 LOP3 per Philox call), whatever the
        # bound; the count of the mode that ran is reported beside it
        ops_unit = (general_ops_per_group_step(K, b, bool(layout_bits & 8)) if engine == 2
                    else algorithmic_ops_per_group_step(K, b, 0))
        ops_mode = ops_unit if engine == 2 else algorithmic_ops_per_group_step(K, b, pad)
        achieved = ops_unit * gs_per_launch / (launch_ms / 1e3) / 1e9
        peak_ops_per_clk = float(os.environ.get("BITSSA_ALU_OPS_PER_CLK_PER_SM", "64"))
        peak = sms * peak_ops_per_clk * max_mhz * 1e6 / 1e9
        return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s", "frac": achieved / peak,
                "ops_per_group_step": ops_unit, "ops_per_group_step_of_the_mode": ops_mode,
                "frac_at_the_mode_count": achieved * ops_mode / ops_unit / peak,
                "group_steps_per_launch": gs_per_launch,
                "peak_basis": f"{sms} SMs x {peak_ops_per_clk:g} LOP3 lanes/clk/SM x {max_mhz:g} MHz "
                              f"(SM count from the device, clock from {mhz_basis}); derived, not measured",
                "lop3_microbench_gops": micro}

    roofline = roofline_of(N_TOT, PAD, group_steps / world / args.steps, statistics.mean(kernel_ms),
                           layout_bits=layout_used)
    fp = kernel_fingerprint()
    roofline["traffic"] = (TRAFFIC_BYTES_PER_LAUNCH.get(fp) if (WORKLOAD == "c2" and RUNS_PER_GPU == 1 << 20
                                                                 and PRECISION == 0 and PAD == 1 and ENGINE == 0
                                                                 and (layout_used & 3) == 1) else None)
    roofline["kernel_sources_sha"] = fp
    if WORKLOAD == "c3":
        roofline = None

    result = {"metric": METRIC, "value": reactions / t_dev, "unit": "lane-reactions/s", "n_gpus": world,
              "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_dev / args.steps,
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
              "data": "synthetic", "config": workload_config(world),
              "absorbed_runs_per_s": absorbed / t_dev, "lane_steps_per_s": lane_steps / t_dev,
              "reactions_per_step": reactions / args.steps, "wall_s": wall,
              "group_steps_per_step": group_steps / args.steps, "max_group_steps": max_group_steps,
              "roofline": roofline, "clocks": clk, "gpu_launches": args.steps,
              "hist_checksum": float(htot.sum().item()),
              "layout": layout_name(layout_used), "layout_bits": layout_used,
              "tuned": None if tuned is None else {"layout": {0: "rule", 1: "thread", 2: "warps"}[tuned[0]],
                                                   "block": tuned[1]}}

    if args.budget:  # a profiling line: the first args.budget steps of every group only
        result["config"]["step_budget"] = args.budget
        result["config"]["workload"] += f"_first{args.budget}steps"

    # ---- end to end through the C ABI with host buffers (create from host arrays, run, read every
    # per-run output into pinned host memory, destroy), rank-local
    pinned = {f: torch.empty(pkg.ssa_field_bytes(ctx, f), dtype=torch.uint8, pin_memory=True)
              for f in (pkg.SSA_FIELD_FINAL_COUNTS, pkg.SSA_FIELD_ABSORB_TIME, pkg.SSA_FIELD_ABSORB_OUTCOME,
                        pkg.SSA_FIELD_EE_HIST)}
    host_in = {"reac": pkg.FRANK_REACTANTS, "prod": pkg.FRANK_PRODUCTS, "rates": np.ones(3),
               "init": np.array(INIT, dtype=np.int64)}
    h2d = sum(v.nbytes for v in host_in.values()) + 8 * (N_SNAP + 1)
    d2h = sum(t.numel() for t in pinned.values())
    if WORKLOAD == "c3":
        h2d = sum(np.asarray(BATCH[k]).nbytes for k in ("init", "rates", "runs", "seeds")) + 144
    e2e_steps = max(1, min(args.steps, 3))
    if tuned is not None:  # the end-to-end contexts run the configuration the tuner chose
        opt.layout, opt.block_size = tuned[0], (tuned[1] if tuned[0] == pkg.SSA_LAYOUT_THREAD else 0)
    barrier()
    t0 = time.perf_counter()
    e2e_react = 0
    for _ in range(e2e_steps):
        if WORKLOAD == "c3":
            c2 = pkg.ssa_create_batch(host_in["reac"], host_in["prod"], BATCH["init"], BATCH["rates"], BATCH["runs"],
                                      BATCH["seeds"] + np.uint64(rank * len(BATCH["runs"])), opt)
        else:
            c2 = pkg.ssa_create(host_in["reac"], host_in["prod"], host_in["rates"], host_in["init"], RUNS_PER_GPU,
                                SEED, opt)
        run(c2)
        for f, t in pinned.items():
            pkg.ssa_fetch(c2, f, t.numpy())
        e2e_react += int(pkg.ssa_fetch(c2, pkg.SSA_FIELD_COUNTERS)[2])
        pkg.ssa_destroy(c2)
    barrier()
    e2e_t = time.perf_counter() - t0
    result["e2e"] = {"value": e2e_react * world / e2e_t, "unit": "lane-reactions/s", "h2d_bytes_per_step": h2d,
                     "d2h_bytes_per_step": d2h, "steps": e2e_steps}
    pkg.ssa_destroy(ctx)

    # ---- the per-run snapshot dump (int32[snap][runs][3]) on the same workload: its HBM bytes and
    # what it adds to the step, outside the timed region
    if not args.no_baselines and WORKLOAD != "c3":
        od = pkg.ssa_default_options(cuda_stream=stream, device=local, precision=args.precision,
                                     keep_snap_counts=1, first_run=first_run, layout=opt.layout,
                                     block_size=opt.block_size, pad_pow2=PAD, engine=ENGINE)
        cd = pkg.ssa_create(pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS, [1.0, 1.0, 1.0], np.array(INIT),
                            RUNS_PER_GPU, SEED, od)
        pkg.ssa_run(cd, T_END, SNAPS)
        torch.cuda.synchronize()
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(2)
        a.record(stream)
        pkg.ssa_run(cd, T_END, SNAPS)
        b2.record(stream)
        torch.cuda.synchronize()
        msd = a.elapsed_time(b2)
        dump_bytes = pkg.ssa_field_bytes(cd, pkg.SSA_FIELD_SNAP_COUNTS)
        pkg.ssa_destroy(cd)
        result["snapshot_dump"] = {"bytes_per_step": dump_bytes, "ms_per_step": msd,
                                   "hbm_gbs_over_step": dump_bytes / (msd / 1e3) / 1e9,
                                   "added_ms": msd - result["ms_per_step"]}

    # ---- the one-thread-per-run GPU baseline on the same workload and precision
    if not args.no_baselines and WORKLOAD != "c3":
        o7 = pkg.ssa_default_options(cuda_stream=stream, device=local, precision=args.precision,
                                     engine=pkg.SSA_ENGINE_THREAD_PER_RUN, first_run=first_run)
        c7 = pkg.ssa_create(pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS, [1.0, 1.0, 1.0], np.array(INIT),
                            RUNS_PER_GPU, SEED, o7)
        pkg.ssa_run(c7, T_END, SNAPS)
        torch.cuda.synchronize()
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1)
        a.record(stream)
        pkg.ssa_run(c7, T_END, SNAPS)
        b2.record(stream)
        c = pkg.ssa_fetch(c7, pkg.SSA_FIELD_COUNTERS)
        ms7 = a.elapsed_time(b2)
        pkg.ssa_destroy(c7)
        r7 = int(c[2]) / (ms7 / 1e3)
        result["thread_per_run"] = {"value": r7 * world, "unit": "lane-reactions/s", "ms_per_step": ms7,
                                    "absorbed_runs_per_s": int(c[5]) * world / (ms7 / 1e3),
                                    "speedup_bitsliced_over_thread_per_run": (reactions / t_dev) / (r7 * world),
                                    "precision": PRECISION_NAMES[PRECISION]}
        # the same pairing with fp32 Kahan clocks on both sides: the baseline's fp64 clock takes a
        # logarithm and a division per reaction, the bit-sliced product clock none
        if PRECISION == 0:
            pair = {}
            for name, eng in (("bitsliced", ENGINE), ("thread_per_run", pkg.SSA_ENGINE_THREAD_PER_RUN)):
                kw = dict(pad_pow2=PAD, layout=opt.layout, block_size=opt.block_size) if eng != 1 else {}
                of = pkg.ssa_default_options(cuda_stream=stream, device=local, precision=pkg.SSA_P32_KAHAN,
                                             engine=eng, first_run=first_run, **kw)
                cf = pkg.ssa_create(pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS, [1.0, 1.0, 1.0], np.array(INIT),
                                    RUNS_PER_GPU, SEED, of)
                pair[name] = time_runs(cf, 3)
                pkg.ssa_destroy(cf)
            result["thread_per_run_fp32"] = {
                "precision": "p32kahan", "bitsliced_ms_per_step": pair["bitsliced"][0],
                "thread_per_run_ms_per_step": pair["thread_per_run"][0],
                "bitsliced_value": pair["bitsliced"][1] * world, "thread_per_run_value": pair["thread_per_run"][1] * world,
                "unit": "lane-reactions/s",
                "speedup_bitsliced_over_thread_per_run": pair["thread_per_run"][0] / pair["bitsliced"][0]}
        if rank == 0:
            sample = args.cpu_sample if WORKLOAD == "c2" else max(64, args.cpu_sample // 8)
            result["cpu_baseline"] = cpu_baseline(sample, os.cpu_count() or 1)
    # ---- the same workload with a clock per run (SSA_CLOCK_LANE): what independent runs in a group cost
    if not args.no_baselines and WORKLOAD == "c2" and ENGINE == 0 and PAD in (0, 1):
        ol = pkg.ssa_default_options(cuda_stream=stream, device=local, precision=args.precision, pad_pow2=PAD,
                                     first_run=first_run, clock=pkg.SSA_CLOCK_LANE)
        cl = pkg.ssa_create(pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS, [1.0, 1.0, 1.0], np.array(INIT), RUNS_PER_GPU,
                            SEED, ol)
        msl, vall, cntl = time_runs(cl, 2)
        pkg.ssa_destroy(cl)
        result["lane_clock"] = {"ms_per_step": msl, "value": vall * world, "unit": "lane-reactions/s",
                                "relative_to_group_clock": result["ms_per_step"] / msl,
                                "layout": layout_name(int(cntl[9]))}

    # ---- the precision workload (N_tot = 10 000, 2^22 runs), a few steps per bound, with its roofline
    if args.c4_steps > 0 and WORKLOAD == "c2" and ENGINE == 0 and PRECISION == 0:
        result["c4"] = {}
        for pad in (1, 2):
            o4 = pkg.ssa_default_options(cuda_stream=stream, device=local, pad_pow2=pad,
                                         first_run=sharding.weak_shard(1 << 22, rank)[0])
            c4 = pkg.ssa_create(pkg.FRANK_REACTANTS, pkg.FRANK_PRODUCTS, [1.0, 1.0, 1.0], np.array([2500, 2500, 5000]),
                                1 << 22, SEED, o4)
            ms4, val4, cnt4 = time_runs(c4, args.c4_steps, snaps=SNAPS)
            pkg.ssa_destroy(c4)
            result["c4"][f"pad{pad}"] = {
                "workload": f"frank_N10000_2500-2500-5000_runs{1 << 22}xgpu_tend50_snap10log_p64",
                "bound": BOUND_NAMES[pad], "steps": args.c4_steps, "warmup": 1, "ms_per_step": ms4,
                "value": val4 * world, "unit": "lane-reactions/s", "max_group_steps": int(cnt4[8]),
                "layout": layout_name(int(cnt4[9])),
                "roofline": roofline_of(10000, pad, float(cnt4[0]), ms4, engine=0, layout_bits=int(cnt4[9]))}
    # ---- the lattice workload (Frank's model on a 64 x 64 torus with hops), to a short t_end
    if args.c5_tend > 0 and WORKLOAD == "c2" and ENGINE == 0 and PRECISION == 0:
        result["c5"] = lattice_leg(pkg, stream, local, args.c5_tend, rank, world, flush)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
