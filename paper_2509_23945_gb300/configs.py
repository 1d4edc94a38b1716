"""The five workload configurations and a short runner for each.

    python -m paper_2509_23945_gb300.configs [name ...] [--sweeps N]

prints one JSON line per configuration: sweeps/s of the timed sweeps,
acceptance (per proposal kind where the learned proposal is on), memory held
by the context, and for the exact configuration the largest |log A|.

Configurations (3D lattices, periodic):
  exact_L4     +/-J EA, L=4, beta=1, chi=16 (exact contraction), FP64, 1 instance x 2 replicas
  pm_L16       +/-J EA, L=16, beta in {0.5, 0.8, 1.0, 1.25}, chi=32, FP32, 64 instances x 4 beta x 2
  gauss_L32    Gaussian EA, L=32, 16 beta in [0.5, 1.6], chi=64, FP32, 16 instances x 16 beta x 2
  uneven_net   +/-J EA, L in {24, 32, 48} (8 instances each, 2 replicas) in one context, beta=1,
               chi=64, FP32, learned proposal (6 layers x 64 channels) trained on accepted TN slices
               and alternated 1:1 with the tensor network
  potts_L64    3-state ferromagnetic Potts, L=64, beta=0.5505, chi=64, FP32, 4 chains, learned proposal
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs, tnmc

CONFIGS = {
    "exact_L4": dict(groups=[dict(model="ea_pm", L=4, betas=[1.0], chi=16, n_inst=1)], prec="f64"),
    "pm_L16": dict(groups=[dict(model="ea_pm", L=16, betas=[0.5, 0.8, 1.0, 1.25], chi=32, n_inst=64)], prec="f32"),
    "gauss_L32": dict(groups=[dict(model="ea_gauss", L=32, betas=list(np.linspace(0.5, 1.6, 16)), chi=64,
                                   n_inst=16)], prec="f32"),
    "uneven_net": dict(groups=[dict(model="ea_pm", L=L, betas=[1.0], chi=64, n_inst=8) for L in (24, 32, 48)],
                       prec="f32", net=True),
    "potts_L64": dict(groups=[dict(model="potts", L=64, betas=[0.5505], chi=64, n_inst=1, n_rep=4)], prec="f32",
                      net=True),
}


def workloads(name, seed=1, scale_chains=1.0):
    out = []
    for i, g in enumerate(CONFIGS[name]["groups"]):
        n_inst = max(1, int(round(g["n_inst"] * scale_chains)))
        out.append(inputs.Workload(model=inputs.MODEL_NAMES[g["model"]], dims=(g["L"],) * 3, bc=(1, 1, 1),
                                   chi=g["chi"], betas=[float(b) for b in g["betas"]], n_inst=n_inst,
                                   n_rep=g.get("n_rep", 2), seed=seed + 101 * i))
    return out


def run(name, sweeps=3, scale_chains=1.0, net_train_steps=20, seed=7):
    import torch
    cfg = CONFIGS[name]
    wls = workloads(name, scale_chains=scale_chains)
    prec = tnmc.PREC_F64 if cfg["prec"] == "f64" else tnmc.PREC_F32
    ctx = tnmc.Context(wls, precision=prec)
    for gi, wl in enumerate(wls):
        ctx.set_spins(gi, wl.initial_spins())
    n_chains = sum(wl.n_chains for wl in wls)
    acc = torch.zeros(n_chains, dtype=torch.int32, device="cuda")
    res = {"config": name, "groups": [dict(L=wl.dims[0], chains=wl.n_chains, chi=wl.chi) for wl in wls],
           "precision": cfg["prec"]}
    if cfg.get("net"):
        ctx.net_init(channels=64, layers=6, seed=seed, buffer_slots=2048)
        ctx.set_proposal_mix(0, True)
        ctx.sweep(1, seed, use_graph=True, accept_counter=acc)     # TN sweep fills the replay buffer
        ctx.sync()
        losses = ctx.net_train(net_train_steps, 32, 1e-3, seed)
        res["net_loss_first_last"] = [float(losses[0]), float(losses[-1])]
        ctx.set_proposal_mix(2, True)                                # alternate TN / network 1:1
    acc.zero_()
    ctx.sync()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ctx.sweep(sweeps, seed, use_graph=True, accept_counter=acc)
    ctx.sync()
    dt = time.perf_counter() - t0
    slices = sum(wl.n_chains * wl.dims[0] for wl in wls) * sweeps
    res.update(sweeps=sweeps, seconds=dt, sweeps_per_s=sweeps / dt, acceptance=float(acc.sum().item()) / slices,
               device_bytes=ctx.memory_bytes())
    if name == "exact_L4":
        wl = wls[0]
        chains = [0, 0, 1, 1]
        out = ctx.slice_update(0, 0, chains, [0, 2, 1, 3], seed, 1000)
        la = (out["logq_old"] - out["logq_new"] - wl.chain_beta()[0] * out["dE"].double() * 2.0 ** -20).abs()
        res["max_abs_logA_exact"] = float(la.max().item())
    ctx.close()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("names", nargs="*", default=list(CONFIGS))
    ap.add_argument("--sweeps", type=int, default=2)
    ap.add_argument("--scale-chains", type=float, default=1.0)
    a = ap.parse_args()
    for n in a.names:
        print(json.dumps(run(n, sweeps=a.sweeps, scale_chains=a.scale_chains)), flush=True)


if __name__ == "__main__":
    main()
