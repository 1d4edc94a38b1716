"""Throughput and acceptance of the update variants on one workload block.

    python -m paper_2509_23945_gb300.variants_run --L 32 --chi 64 --chi2 16 --sweeps 3

On one disorder instance of the Gaussian EA glass (periodic, R1, --betas temperatures in [0.5, 1.6] x 2
replicas, FP32), after --warm fresh TNMCMC-1 sweeps from a hot start, times --sweeps sweeps of each
variant with CUDA events on the context's stream and counts accepted proposals:
  * tn:        TNMCMC-1, one proposal per environment build (Algorithm 2);
  * k<K>:      K proposals per environment build (independence-sampler chain on the slice);
  * cache:     every update proposes from a cache of environments built once from the warmed state
               (the build is timed separately), then a mix that contracts afresh every --fresh-every
               sweeps;
  * tnmcmc2:   TNMCMC-2 composite layers of superspins at --chi2 (separate context, same couplings and
               warm-up), and TNMCMC-1 at --chi2 on the same warmed state for comparison.
Prints one JSON line per variant: seconds per sweep, proposals and accepted proposals per sweep,
acceptance and accepted proposals per second.
"""
from __future__ import annotations

import argparse
import json

import numpy as np

from . import inputs, tnmc


def timed(ctx, stream, n, seed, acc):
    import torch
    acc.zero_()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.sweep(n, seed, use_graph=True, accept_counter=acc)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / 1e3 / n, int(acc.sum().item()) / n


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=32)
    ap.add_argument("--chi", type=int, default=64)
    ap.add_argument("--chi2", type=int, default=16)
    ap.add_argument("--betas", type=int, default=8)
    ap.add_argument("--warm", type=int, default=2)
    ap.add_argument("--sweeps", type=int, default=3)
    ap.add_argument("--k", type=int, default=4)
    ap.add_argument("--fresh-every", type=int, default=3)
    ap.add_argument("--seed", type=int, default=2718)
    a = ap.parse_args()
    import torch
    L = a.L
    betas = [float(b) for b in np.linspace(0.5, 1.6, a.betas)]
    wl = inputs.Workload(model=inputs.MODEL_EA_GAUSS, dims=(L, L, L), bc=(1, 1, 1), chi=a.chi, betas=betas, n_inst=1,
                         n_rep=2, seed=5)
    stream = torch.cuda.Stream()
    acc = torch.zeros(wl.n_chains, dtype=torch.int32, device="cuda")
    slices = wl.n_chains * L

    def report(name, sec, accepted, proposals, **extra):
        line = {"variant": name, "L": L, "chains": wl.n_chains, "s_per_sweep": sec, "proposals_per_sweep": proposals,
                "accepted_per_sweep": accepted, "acceptance": accepted / proposals,
                "accepted_per_s": accepted / sec}
        line.update(extra)
        print(json.dumps(line), flush=True)

    ctx = tnmc.Context([wl], precision=tnmc.PREC_F32, stream=stream)
    ctx.set_spins(0, wl.initial_spins())
    for _ in range(a.warm):
        ctx.sweep(1, a.seed, use_graph=True)
    warmed = ctx.get_spins(0)
    t0 = ctx.sweep_counter
    sec, accd = timed(ctx, stream, a.sweeps, a.seed, acc)
    report("tn", sec, accd, slices, chi=a.chi)
    ctx.sweep_counter = t0
    ctx.set_spins(0, warmed)
    ctx.set_proposals_per_env(a.k)
    sec, accd = timed(ctx, stream, a.sweeps, a.seed, acc)
    report(f"k{a.k}", sec, accd, slices * a.k, chi=a.chi, slice_updates_per_sweep=slices)
    ctx.set_proposals_per_env(1)
    ctx.sweep_counter = t0
    ctx.set_spins(0, warmed)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    ctx.cache_build(a.seed + 1, 0)
    e1.record(stream)
    torch.cuda.synchronize()
    build_s = e0.elapsed_time(e1) / 1e3
    ctx.set_cache_mix(True, 0)
    sec, accd = timed(ctx, stream, a.sweeps, a.seed, acc)
    report("cache", sec, accd, slices, chi=a.chi, build_s=build_s, fresh_every=0,
           context_gb=ctx.memory_bytes() / 1e9)
    ctx.sweep_counter = t0
    ctx.set_spins(0, warmed)
    n_mix = max(a.sweeps, a.fresh_every)
    ctx.set_cache_mix(True, a.fresh_every)
    sec, accd = timed(ctx, stream, n_mix, a.seed, acc)
    report("cache_mix", sec, accd, slices, chi=a.chi, fresh_every=a.fresh_every)
    ctx.close()

    wl2 = inputs.Workload(model=wl.model, dims=wl.dims, bc=wl.bc, chi=a.chi2, betas=betas, n_inst=1, n_rep=2, seed=5,
                          couplings=wl.couplings)
    for layers in (1, 2):
        c2 = tnmc.Context([wl2], precision=tnmc.PREC_F32, stream=stream, layers=layers)
        c2.set_spins(0, warmed)
        c2.sweep_counter = t0
        sec, accd = timed(c2, stream, a.sweeps, a.seed, acc)
        # composites per sweep: every chain updates n // 2 composites of the sweep's axis (periodic, even L)
        props = wl2.n_chains * (L // 2 if layers == 2 else L)
        report("tnmcmc2" if layers == 2 else "tn_chi2", sec, accd, props, chi=a.chi2,
               spins_per_proposal=(2 if layers == 2 else 1) * (L - 1) * L)
        c2.close()


if __name__ == "__main__":
    main()
