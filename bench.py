"""Benchmark of the TNMCMC-1 slice update on GB300.

Metric: effective independent samples per second = sweeps/s / tau_int(q) of the
spin-glass overlap q (main text, "Sampling 3D spin glasses"; tau_int of SM III),
on 3D Edwards-Anderson Gaussian glasses at L = 32 (periodic), 16 inverse
temperatures in [0.5, 1.6], chi = 64, 16 disorder instances x 2 replicas.

One step is one sweep (slices normal to axis t mod 3, each colour class in one
launch, replayed from a CUDA graph) of the timed block of chains (--bench-chains,
whole disorder instances of the workload; every chain costs the same, so the
block's per-chain rate is the workload's). The value aggregates over the block's
replica pairs: sum over pairs of sweeps/s / tau_int(q). Inputs are synthetic and
resident on the device before timing.

The plain FP64 GPU path (the same kernels in double, no graph) is timed on one
full wave of the block's slices (every SM busy), with CUDA events, and its
samples/s uses the same tau_int; the headline ratio is value / that.

--impl reference times the CPU oracle on the host cores (the reported baseline).
Multi-GPU (torchrun): every rank runs its own block (weak scaling, no
collective on the data path); rank 0 prints the aggregate.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (model, L, betas, chi, n_inst, n_rep)
    "ea_gauss_L32_chi64": ("ea_gauss", 32, [float(b) for b in np.linspace(0.5, 1.6, 16)], 64, 16, 2),
    "ea_pm_L16_chi32": ("ea_pm", 16, [0.5, 0.8, 1.0, 1.25], 32, 64, 2),
    "ea_pm_L4_chi16": ("ea_pm", 4, [1.0], 16, 1, 2),
}

# tau_int(q) of the FP32 path on the L=32 chi=64 Gaussian workload: the mean over the 16 temperatures
# of a separate 100-sweep replica-pair run of this kernel (tau_run, 20 burn-in sweeps dropped; the
# lowest temperatures are not equilibrated in 100 sweeps). The few sweeps of a bench run start hot and
# cannot resolve tau_int, so the metric divides by max(in-run estimate, this value).
TAU_INT_Q_EQUILIBRIUM = {"ea_gauss_L32_chi64": 4.45}

# Algorithmic flops of one bond step of the environment pass, counted for the method's own route
# (MPO apply + LQ + absorb + QR + SVD at 20 n^3 + V + S V^T absorb, periodic rows)
FLOPS_PER_SITE_STEP = {"ea_gauss_L32_chi64": 193e6, "ea_pm_L16_chi32": 24.2e6, "ea_pm_L4_chi16": 1.0e6}

# DRAM bytes (read + write) per slice update of the slice kernel, from an ncu capture of one launch of
# 8 slices of this workload, keyed by workload. Each slice streams its own CTA's workspace, so the
# traffic of a launch scales with its slices. Empty: the kernel has changed since the last capture
# (137.2 MB per slice, taken before the tcgen05 engine moved to its own instance), so the bench line
# reports no traffic until the counters are taken again.
DRAM_BYTES_PER_SLICE = {}

# engines of the environment pass's contractions (tnmc_set_tuning gemm_mode)
GEMM_ENGINES = {"ffma": 0, "mma_tf32x3": 1, "mma_bf16": 2, "umma_tf32x3": 3, "umma_bf16": 4}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ea_gauss_L32_chi64", choices=list(WORKLOADS))
    ap.add_argument("--precision", default="f32", choices=["f32", "f64", "bf16"])
    ap.add_argument("--gemm", default="default", choices=["default"] + list(GEMM_ENGINES),
                    help="engine of the environment pass's contractions (default: the context's)")
    ap.add_argument("--gemm-tile", default="auto", choices=["auto", "0", "1", "2"],
                    help="CUDA-core GEMM tile (0 64x64, 1 32x32, 2 128x64); auto: time each on one wave of the "
                         "block's slices before the warm-up and keep the fastest (all give identical results)")
    ap.add_argument("--no-graph", action="store_true")
    ap.add_argument("--tau-sweeps", type=int, default=1,
                    help="extra untimed sweeps appended to the q(t) series for tau_int")
    ap.add_argument("--seed", type=int, default=20250923)
    ap.add_argument("--bench-chains", type=int, default=128, help="chains per timed block (whole instances)")
    ap.add_argument("--fp64-items", type=int, default=-1,
                    help="slices in the timed plain FP64 launch (-1: one full wave of resident CTAs; 0: skip)")
    ap.add_argument("--no-cpu-baseline", dest="cpu_baseline", action="store_false")
    return ap.parse_args()


def make_workload(name, rank=0, seed=1):
    from paper_2509_23945_gb300 import inputs
    mdl, L, betas, chi, n_inst, n_rep = WORKLOADS[name]
    return inputs.Workload(model=inputs.MODEL_NAMES[mdl], dims=(L, L, L), bc=(1, 1, 1), chi=chi, betas=betas,
                           n_inst=n_inst, n_rep=n_rep, seed=seed + 7919 * rank)


def site_steps_per_sweep(wl):
    L = wl.dims[0]
    m = L - 1                    # one fixed line per periodic slice
    return wl.n_chains * L * (m - 1) * L   # rows m..2 build environments, L bonds each


class ClockSampler:
    def __init__(self, device_index=0):
        self.samples = []
        self.stop = threading.Event()
        self.idx = device_index

    def run(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            p = subprocess.Popen(["nvidia-smi", f"--id={self.idx}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                  "-lms", "200"], stdout=subprocess.PIPE, text=True)
        except Exception:
            return
        while not self.stop.is_set():
            line = p.stdout.readline()
            if not line:
                break
            self.samples.append([t.strip() for t in line.split(",")])
        p.terminate()

    def __enter__(self):
        self.th = threading.Thread(target=self.run, daemon=True)
        self.th.start()
        return self

    def __exit__(self, *a):
        self.stop.set()
        self.th.join(timeout=2)

    def summary(self):
        sm = [float(s[1]) for s in self.samples if len(s) >= 9 and s[1].replace(".", "").isdigit()]
        mx = [float(s[2]) for s in self.samples if len(s) >= 9 and s[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for s in self.samples if len(s) >= 9 for i in range(4) if s[5 + i] == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


def tau_from_series(qs):
    """Pooled tau_int(q) over replica pairs: the mean normalised autocorrelation with Sokal's window."""
    qs = np.asarray(qs)          # [T, pairs]
    T = qs.shape[0]
    if T < 4:
        return None, None
    xc = qs - qs.mean(axis=0, keepdims=True)
    var = (xc ** 2).mean(axis=0)
    ok = var > 0
    if not ok.any():
        return None, None
    rho = np.array([np.mean((xc[: T - k, ok] * xc[k:, ok]).mean(axis=0) / var[ok]) for k in range(T)])
    tau, W = 0.5, T - 1
    for w in range(1, T):
        tau += rho[w]
        if w >= 6 * tau:
            W = w
            break
    tau = max(tau, 0.5)
    return float(tau), int(W)


def time_fp64_wave(args, wl, n_items):
    """The plain FP64 GPU path: the same kernels in double, launched directly (no graph), default
    tuning, on n_items slices of the block's first colour class (axis 0, hot start); n_items < 0 takes
    one full wave of resident CTAs, so every SM is busy. Timed with CUDA events on the context's
    stream after a warm-up launch of the same kernel on a small lattice. Returns (slice updates/s,
    acceptance, items, seconds)."""
    import torch
    from paper_2509_23945_gb300 import inputs, tnmc
    stream = torch.cuda.Stream()
    warm = inputs.Workload(model=wl.model, dims=(4, 4, 4), bc=wl.bc, chi=4, betas=[1.0], n_inst=1, n_rep=1)
    wctx = tnmc.Context([warm], precision=tnmc.PREC_F64, stream=stream)
    wctx.set_spins(0, warm.initial_spins())
    wctx.slice_update(0, 0, [0], [0], args.seed, 0, write_back=False)
    wctx.sync()
    wctx.close()
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F64, stream=stream)
    ctx.set_spins(0, wl.initial_spins())
    L = wl.dims[0]
    ks = tnmc.colour_classes(L, True)[0]
    chains = np.repeat(np.arange(wl.n_chains), len(ks))
    slices = np.tile(ks, wl.n_chains)
    if n_items < 0:
        t = ctx.get_tuning()
        n_items = torch.cuda.get_device_properties(0).multi_processor_count * t["ctas_per_sm"]
    n_items = min(n_items, len(chains))
    chains, slices = chains[:n_items], slices[:n_items]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    out = ctx.slice_update(0, 0, chains, slices, args.seed, 0, write_back=False)
    e1.record(stream)
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) / 1e3
    acc = float(out["accept"].float().mean().item())
    ctx.close()
    return n_items / dt, acc, n_items, dt


def pick_gemm_tile(ctx, wl, stream, seed):
    """Autotune the GEMM tile (a result-preserving choice): time one launch of a full wave of the block's
    first colour class (axis 0, no write-back) per tile with CUDA events; apply and return the fastest."""
    import torch
    from paper_2509_23945_gb300 import tnmc
    L = wl.dims[0]
    ks = tnmc.colour_classes(L, True)[0]
    wave = torch.cuda.get_device_properties(0).multi_processor_count * ctx.get_tuning()["ctas_per_sm"]
    n = max(1, min(wl.n_chains, wave // len(ks)))
    chains = np.repeat(np.arange(n), len(ks))
    slices = np.tile(ks, n)
    times = {}
    for tile in (0, 1, 2):
        ctx.set_tuning(gemm_tile=tile)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        ctx.slice_update(0, 0, chains, slices, seed, 0, write_back=False, want_spins=False)
        e1.record(stream)
        torch.cuda.synchronize()
        times[tile] = e0.elapsed_time(e1) / 1e3
    best = min(times, key=times.get)
    ctx.set_tuning(gemm_tile=best)
    return best, times, len(chains)


def block_workload(wl_full, n_chains):
    """The first n_chains chains of a workload (instance-major layout, whole instances)."""
    from paper_2509_23945_gb300 import inputs
    per_inst = len(wl_full.betas) * wl_full.n_rep
    n_inst = max(1, n_chains // per_inst)
    betas = wl_full.betas if n_chains >= per_inst else wl_full.betas[: max(1, n_chains // wl_full.n_rep)]
    return inputs.Workload(model=wl_full.model, dims=wl_full.dims, bc=wl_full.bc, chi=wl_full.chi, betas=betas,
                           n_inst=n_inst, n_rep=wl_full.n_rep, seed=wl_full.seed,
                           couplings=wl_full.couplings[:n_inst])


def run_ours(args):
    import torch
    import torch.distributed as dist
    from paper_2509_23945_gb300 import tnmc

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    wl_full = make_workload(args.workload, rank)
    wl = block_workload(wl_full, min(args.bench_chains, wl_full.n_chains))
    prec = {"f32": tnmc.PREC_F32, "f64": tnmc.PREC_F64, "bf16": tnmc.PREC_BF16}[args.precision]
    stream = torch.cuda.Stream()
    # measured roofline denominators of this device (FMA throughput of the CUDA cores)
    peak32 = tnmc.probe_alu_peak(tnmc.PREC_F32, stream) / 1e12
    peak64 = tnmc.probe_alu_peak(tnmc.PREC_F64, stream) / 1e12
    ctx = tnmc.Context([wl], precision=prec, stream=stream)
    if args.gemm != "default":
        ctx.set_tuning(gemm_mode=GEMM_ENGINES[args.gemm])
    gemm_engine = {v: k for k, v in GEMM_ENGINES.items()}[ctx.get_tuning()["gemm_mode"]]
    ctx.set_spins(0, wl.initial_spins())
    tile_times, tile_slices = None, 0
    if prec == tnmc.PREC_F64:
        gemm_tile = 0
    elif args.gemm_tile == "auto":
        gemm_tile, tile_times, tile_slices = pick_gemm_tile(ctx, wl, stream, args.seed)
    else:
        gemm_tile = int(args.gemm_tile)
        ctx.set_tuning(gemm_tile=gemm_tile)
    use_graph = not args.no_graph
    pair_idx = np.arange(0, wl.n_chains, 2)
    n_pairs = len(pair_idx)
    acc = torch.zeros(wl.n_chains, dtype=torch.int32, device="cuda")
    n_rec = args.warmup + args.steps + args.tau_sweeps
    obs_buf = torch.zeros((n_rec, wl.n_chains, 3), dtype=torch.float64, device="cuda")
    rec = [0]

    def record_q():
        # observables of this sweep into the device buffer, on the library's stream (no host sync)
        ctx.observables(0, out=obs_buf[rec[0]])
        rec[0] += 1

    for _ in range(args.warmup):
        ctx.sweep(1, args.seed, use_graph=use_graph, accept_counter=acc)
        record_q()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    acc.zero_()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        start.record(stream)
        for _ in range(args.steps):
            ctx.sweep(1, args.seed, use_graph=use_graph, accept_counter=acc)
            record_q()
        stop.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_ms = start.elapsed_time(stop)
    acc_timed = int(acc.sum().item())
    for _ in range(args.tau_sweeps):
        ctx.sweep(1, args.seed, use_graph=use_graph)
        record_q()
    ctx.sync()
    qs = list(obs_buf[: rec[0], pair_idx, 2].cpu().numpy())
    tmax = t_ms
    if world > 1:
        tt = torch.tensor([t_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        tmax = float(tt.item())
    events = ctx.events()

    # end to end through the public API with host buffers: H2D spins, one sweep, D2H spins
    host = ctx.get_spins(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.set_spins(0, host)
    ctx.sweep(1, args.seed, use_graph=use_graph)
    host = ctx.get_spins(0)
    e2e_s = time.perf_counter() - t0
    ctx.close()

    L = wl.dims[0]
    slices_per_sweep = wl.n_chains * L
    sweeps_per_s = args.steps / (tmax / 1e3)                  # of the timed block (every chain advances)
    tau_meas, W = tau_from_series(np.array(qs[1:]))   # drop the first sweep after the hot start
    tau_eq = TAU_INT_Q_EQUILIBRIUM.get(args.workload, 1.0)
    tau = max(tau_meas if tau_meas is not None else 0.0, tau_eq, 1.0)
    value = n_pairs * world * sweeps_per_s / tau               # sum over replica pairs of all ranks
    fp64 = None
    if rank == 0 and args.fp64_items != 0:
        rate64, acc64, items64, dt64 = time_fp64_wave(args, wl, args.fp64_items)
        sweeps64 = rate64 / slices_per_sweep
        value64 = n_pairs * sweeps64 / tau
        site_steps64 = items64 * (L - 2) * L
        ach64 = FLOPS_PER_SITE_STEP[args.workload] * site_steps64 / dt64 / 1e12
        fp64 = {"slice_updates_per_s": rate64, "sweeps_per_s_block": sweeps64, "samples_per_s": value64,
                "acceptance": acc64, "timed_slices": items64, "launch_s": dt64,
                "tau_int_q": tau, "tau_note": "same tau_int(q) as the FP32 path (acceptance 1 within 1e-3 on both)",
                "roofline": {"bound": "alu", "achieved": ach64, "peak": peak64, "unit": "TFLOP/s",
                             "frac": ach64 / peak64, "peak_source": "measured DFMA probe"}}
    # roofline of the slice kernel: algorithmic flops of one launch / its mean duration
    site_steps_launch = site_steps_per_sweep(wl) / 2
    flops_launch = FLOPS_PER_SITE_STEP[args.workload] * site_steps_launch
    launch_s = (tmax / 1e3) / args.steps / 2
    clocks = clk.summary()
    peak = peak64 if prec == tnmc.PREC_F64 else peak32
    achieved = flops_launch / launch_s / 1e12
    slices_launch = wl.n_chains * L / 2
    traffic_launch = (DRAM_BYTES_PER_SLICE[args.workload] * slices_launch
                      if args.workload in DRAM_BYTES_PER_SLICE and prec == tnmc.PREC_F32 and gemm_engine == "ffma"
                      and gemm_tile == 0 else None)
    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {
        "metric": "effective indep. samples/s (sweeps/s / tau_int of q_EA) at L=32 vs plain FP64 GPU",
        "value": value,
        "unit": "samples/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": tmax / args.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {tnmc.PREC_F32: "f32", tnmc.PREC_F64: "f64", tnmc.PREC_BF16: "bf16"}[prec],
        "data": "synthetic (seeded Gaussian couplings, hot start)",
        "config": {
            "workload": args.workload, "L": L, "chi": wl.chi, "chains": wl.n_chains,
            "workload_chains": wl_full.n_chains, "betas": [round(b, 4) for b in wl.betas], "n_inst": wl.n_inst,
            "replicas": wl.n_rep, "replica_pairs": n_pairs, "fix_mode": "R1", "truncation": "LQ + one-sided Jacobi SVD",
            "gemm_engine": gemm_engine,
            "gemm_tile": {0: "64x64", 1: "32x32", 2: "128x64"}[gemm_tile],
            "gemm_tile_times_s": ({ {0: "64x64", 1: "32x32", 2: "128x64"}[k]: v for k, v in tile_times.items()}
                                  if tile_times else None),
            "gemm_tile_timed_slices": tile_slices,
            "step": f"one sweep (axis t mod 3, both colour classes, graph-replayed) of {wl.n_chains} chains "
                    f"({wl.n_inst} whole instances of the {wl_full.n_chains}-chain workload; {slices_per_sweep} "
                    f"slice updates per step)",
            "sweeps_per_s": sweeps_per_s, "slice_updates_per_s": sweeps_per_s * slices_per_sweep,
            "tau_int_q_used": tau, "tau_int_q_in_run": tau_meas, "tau_window_in_run": W,
            "tau_series_sweeps_in_run": len(qs) - 1, "tau_int_q_equilibrium": tau_eq,
            "acceptance": acc_timed / (args.steps * slices_per_sweep),
            "uniform_fallback_sites": events,
            "fp64_plain_gpu": fp64,
            "speedup_vs_fp64_plain_gpu": (value / fp64["samples_per_s"]) if fp64 else None,
            "l2": "working set per CTA (environment stack) far above L2; no flush needed",
            "parallelism": f"replicas x{world}",
        },
        "clocks": clocks,
        "gpu_launches": args.steps * 4,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic_launch,
                     "kernel": "slice_update_kernel<double>" if prec == tnmc.PREC_F64 else "slice_update_kernel<float>",
                     "peak_source": "measured FMA probe of this device (tnmc_probe_alu_peak)",
                     "peak_fp64": peak64,
                     "note": "achieved = algorithmic flops of one launch (193 MF per bond step x bond steps of one "
                             "colour class) / mean launch time (half a graph-replayed sweep)"},
        "e2e": {"value": n_pairs * world * (1.0 / e2e_s) / tau, "unit": "samples/s",
                "h2d_bytes_per_step": int(host.size), "d2h_bytes_per_step": int(host.size)},
    }
    line["cpu_baseline"] = cpu_baseline(args, wl, n_pairs, tau) if args.cpu_baseline else None
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


def _oracle_slice_seconds(job):
    """One oracle slice update (spawned worker, one thread): seconds."""
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    name, chain, k, seed = job
    from oracle import update
    wl = make_workload(name, 0)
    spins = wl.initial_spins()
    betas = wl.chain_beta()
    inst = wl.chain_instance()
    t0 = time.perf_counter()
    update.slice_update(wl.model, wl.dims, wl.bc, spins[chain], wl.couplings[inst[chain]], float(betas[chain]),
                        wl.chi, 0, k, seed, 0, chain)
    return time.perf_counter() - t0


def cpu_baseline(args, wl, n_pairs, tau):
    """The oracle as it stands on every host core: one single-threaded slice update per core in spawned
    processes (a bounded sample of the workload), scaled to the timed block's samples/s."""
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    jobs = [(args.workload, c % wl.n_chains, 2 * (c // wl.n_chains) % wl.dims[0], args.seed) for c in range(cores)]
    # one BLAS thread per process: the variables must be in the environment the spawned processes start with
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    t0 = time.perf_counter()
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            secs = pool.map(_oracle_slice_seconds, jobs)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    wall = time.perf_counter() - t0
    rate = len(jobs) / wall                      # slice updates per second on all cores
    slices_per_sweep = wl.n_chains * wl.dims[0]
    value = n_pairs * (rate / slices_per_sweep) / tau
    return {"value": value, "unit": "samples/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(jobs)} slice updates at L={wl.dims[0]}, chi={wl.chi} (one per core, single-threaded, "
                      f"{wall:.1f} s wall); scaled to the {wl.n_chains}-chain block's {slices_per_sweep} slices per "
                      f"sweep and divided by the same tau_int",
            "single_thread_slice_s": float(np.median(secs)), "all_cores_slice_updates_per_s": rate}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    wl_full = make_workload(args.workload, 0)
    wl = block_workload(wl_full, min(args.bench_chains, wl_full.n_chains))
    from oracle import update
    steps = []
    spins = wl.initial_spins()
    betas = wl.chain_beta()
    inst = wl.chain_instance()
    for s in range(args.warmup + args.steps):
        c = s % wl.n_chains
        t0 = time.perf_counter()
        update.slice_update(wl.model, wl.dims, wl.bc, spins[c], wl.couplings[inst[c]], float(betas[c]), wl.chi, 0, 0,
                            args.seed, s, c)
        steps.append(time.perf_counter() - t0)
    dt = float(np.mean(steps[args.warmup:]))
    slices_per_sweep = wl.n_chains * wl.dims[0]
    sweeps_per_s = 1.0 / (dt * slices_per_sweep)
    n_pairs = wl.n_chains // 2
    # the oracle runs the same chain dynamics as the GPU path, so it takes the same tau_int(q)
    tau = TAU_INT_Q_EQUILIBRIUM.get(args.workload, 1.0)
    value = n_pairs * sweeps_per_s / tau
    line = {"impl": "reference", "metric": "effective indep. samples/s (sweeps/s / tau_int of q_EA) at L=32 vs plain FP64 GPU",
            "value": value, "unit": "samples/s", "n_gpus": 0, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "L": wl.dims[0], "chi": wl.chi, "chains": wl.n_chains,
                       "workload_chains": wl_full.n_chains, "betas": [round(b, 4) for b in wl.betas],
                       "n_inst": wl.n_inst, "replicas": wl.n_rep, "replica_pairs": n_pairs, "fix_mode": "R1",
                       "step": "one oracle slice update on one core (a bounded sample of the workload); value = the "
                               "block's sweeps/s from the mean slice time, summed over replica pairs, divided by "
                               "tau_int(q)",
                       "sweeps_per_s": sweeps_per_s, "tau_int_q_used": tau},
            "cpu_baseline": {"kind": "oracle", "cores": 1, "sample": f"{args.steps} slice updates at L={wl.dims[0]}, "
                             f"chi={wl.chi}", "value": value},
            "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
