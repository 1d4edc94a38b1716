"""Autotuner of the slice-update kernel configuration.

For a workload (chi, local dimension d, row topology, extents, precision) it
times each candidate kernel configuration (tnmc_tuning) on one colour class of
a sample of chains and keeps the fastest. By default only choices that leave
every result bitwise unchanged are candidates: where the factorisations' working
matrices live (shared or global memory), how many slice CTAs share an SM and,
for F32 and BF16, the output tile of the CUDA-core GEMMs (64 x 64, 32 x 32,
128 x 64; each its own compiled kernel).
allow_arith_changes=True adds the FP32 contraction engine (CUDA-core FMA or
3xTF32 tensor-core products), which changes results at the rounding level
(the chain stays exact; only log q moves). The truncation route and the
convergence floor of the density-matrix route are never tuned.
Results are cached in a JSON file keyed by (GPU name, chi, d, ring rows, extents,
precision), so a context is tuned once per machine:

    from paper_2509_23945_gb300 import autotune
    best = autotune.tune(ctx, group=0)          # or autotune.apply_cached(ctx, group=0)
"""
from __future__ import annotations

import itertools
import json
import os
import time

import numpy as np

from . import tnmc

CACHE = os.environ.get("TNMC_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "tnmc_tune.json"))


def _key(ctx, group, prec):
    import torch
    wl = ctx.workloads[group]
    ring = int(wl.bc[0] or wl.bc[1] or wl.bc[2])
    dims = "x".join(str(v) for v in wl.dims)
    return f"{torch.cuda.get_device_name()}|chi={wl.chi}|d={wl.d}|ring={ring}|L={dims}|prec={prec}"


def candidates(prec, allow_arith_changes=False):
    """Result-preserving choices (memory placement, CTAs per SM, GEMM tile of F32 / BF16 contexts); with
    allow_arith_changes the FP32 contraction engine as well."""
    gemms = [0, 1] if (prec == tnmc.PREC_F32 and allow_arith_changes) else [-1]
    tiles = [0, 1, 2] if prec != tnmc.PREC_F64 else [-1]
    return [dict(gemm_mode=g, eig_smem=e, ctas_per_sm=c, gemm_tile=t)
            for g, e, c, t in itertools.product(gemms, [1, 0], [2, 1], tiles)]


def time_config(ctx, group, n_chains, seed=11, repeats=1):
    import torch
    wl = ctx.workloads[group]
    L = wl.dims[0]
    ks = tnmc.colour_classes(L, bool(wl.bc[0]))[0]
    n = min(n_chains, wl.n_chains)
    chains = np.repeat(np.arange(n), len(ks))
    slices = np.tile(ks, n)
    best = float("inf")
    for _ in range(repeats):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.slice_update(group, 0, chains, slices, seed, 0, write_back=False, want_spins=False)
        ctx.sync()
        best = min(best, time.perf_counter() - t0)
    return best / len(chains)


def tune(ctx, group=0, n_chains=None, save=True, allow_arith_changes=False):
    """Time every candidate, apply the fastest, return {'best': cfg, 'times': [...]}."""
    import torch
    prec = ctx.precision
    n_chains = n_chains or max(1, (torch.cuda.get_device_properties(0).multi_processor_count * 2) //
                               max(1, ctx.workloads[group].dims[0] // 2))
    results = []
    for cfg in candidates(prec, allow_arith_changes):
        ctx.set_tuning(**cfg)
        results.append((time_config(ctx, group, n_chains), cfg))
    results.sort(key=lambda t: t[0])
    best = results[0][1]
    ctx.set_tuning(**best)
    out = {"best": best, "times": [{"s_per_slice": t, **c} for t, c in results]}
    if save:
        db = {}
        if os.path.exists(CACHE):
            with open(CACHE) as f:
                db = json.load(f)
        db[_key(ctx, group, prec)] = out
        os.makedirs(os.path.dirname(CACHE), exist_ok=True)
        with open(CACHE, "w") as f:
            json.dump(db, f, indent=1)
    return out


def apply_cached(ctx, group=0):
    """Apply a cached tuning for this context if one exists; returns it or None."""
    if not os.path.exists(CACHE):
        return None
    with open(CACHE) as f:
        db = json.load(f)
    entry = db.get(_key(ctx, group, ctx.precision))
    if entry:
        ctx.set_tuning(**entry["best"])
        return entry["best"]
    return None
