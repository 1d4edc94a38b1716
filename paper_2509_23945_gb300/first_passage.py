"""First-passage time of the magnetisation, tau_fp,M (SM III): sweeps from the all-up start until M(t) <= 0.

    python -m paper_2509_23945_gb300.first_passage --L 4 6 8 --beta 1.0 --instances 16 --replicas 4 --chi 4

The paper measures how fast TNMCMC and single-spin Metropolis leave the all-up state of a 3D EA +-J
glass with free boundaries (main text, "Sampling 3D spin glasses": chains start at M = 1; SM III). For
each lattice size this creates a context of such glasses, puts every chain in the all-up state, and
advances it by TNMCMC-1 sweeps (tnmc_sweep) or by checkerboard Metropolis sweeps
(tnmc_metropolis_sweep), reading the magnetisation of every chain after each sweep
(tnmc_observables). The first-passage time of a chain is the first sweep t with M(t) <= 0; a chain
that has not got there by max_sweeps is reported as censored. Prints one JSON line per (L, method):
mean and median first-passage sweeps, the censored count, and the wall time per sweep.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs, tnmc


def first_crossing(m_series, max_sweeps):
    """m_series [T, chains] of M after sweeps 1..T -> first sweep (1-based) with M <= 0, or None."""
    m = np.asarray(m_series)
    out = []
    for c in range(m.shape[1]):
        hit = np.nonzero(m[:, c] <= 0.0)[0]
        out.append(int(hit[0]) + 1 if len(hit) else None)
    return out


def run_method(ctx, method, seed, max_sweeps, group=0, check_every=1):
    """Advance every chain of ``group`` from the all-up state; returns (first-passage sweeps, s per sweep)."""
    import torch
    wl = ctx.workloads[group]
    ctx.set_spins(group, np.zeros((wl.n_chains, wl.dims[2], wl.dims[1], wl.dims[0]), dtype=np.int8))
    ctx.sweep_counter = 0
    obs = torch.zeros((wl.n_chains, 3), dtype=torch.float64, device="cuda")
    series = []
    done = np.zeros(wl.n_chains, dtype=bool)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    t = 0
    while t < max_sweeps and not done.all():
        n = min(check_every, max_sweeps - t)
        for _ in range(n):
            if method == "tnmcmc":
                ctx.sweep(1, seed)
            else:
                ctx.metropolis_sweep(1, seed)
        t += n
        ctx.observables(group, out=obs)
        ctx.sync()
        m = obs[:, 1].cpu().numpy().copy()
        series.append(m)
        done |= m <= 0.0
    dt = (time.perf_counter() - t0) / max(t, 1)
    fp = first_crossing(np.array(series), t)
    return [None if v is None else v * check_every for v in fp], dt


def summary(fp):
    hit = [v for v in fp if v is not None]
    return {"chains": len(fp), "censored": len(fp) - len(hit),
            "mean_sweeps": float(np.mean(hit)) if hit else None,
            "median_sweeps": float(np.median(hit)) if hit else None}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, nargs="+", default=[4, 6, 8])
    ap.add_argument("--beta", type=float, default=1.0)
    ap.add_argument("--chi", type=int, default=4)
    ap.add_argument("--instances", type=int, default=16)
    ap.add_argument("--replicas", type=int, default=4)
    ap.add_argument("--max-sweeps", type=int, default=20000)
    ap.add_argument("--methods", nargs="+", default=["tnmcmc", "metropolis"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64"])
    ap.add_argument("--seed", type=int, default=7)
    a = ap.parse_args()
    prec = tnmc.PREC_F32 if a.precision == "f32" else tnmc.PREC_F64
    for L in a.L:
        wl = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(L, L, L), bc=(0, 0, 0), chi=a.chi, betas=[a.beta],
                             n_inst=a.instances, n_rep=a.replicas, seed=a.seed)
        ctx = tnmc.Context([wl], precision=prec)
        for method in a.methods:
            fp, dt = run_method(ctx, method, a.seed, a.max_sweeps)
            print(json.dumps({"L": L, "beta": a.beta, "method": method, "chi": a.chi if method == "tnmcmc" else None,
                              "s_per_sweep": dt, **summary(fp)}), flush=True)
        ctx.close()


if __name__ == "__main__":
    main()
