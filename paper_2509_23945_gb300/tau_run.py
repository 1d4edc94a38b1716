"""Integrated autocorrelation time of the overlap q on a block of the L=32 workload.

    python -m paper_2509_23945_gb300.tau_run --sweeps 60 --burn 20 --instances 2

Runs replica pairs of the Gaussian EA workload (L=32 periodic, 16 beta in
[0.5, 1.6], chi=64, FP32 path) for the given number of sweeps, records
q(t) = (1/N) sum_i s_i^(1) s_i^(2) after every sweep (main text, "Sampling 3D
spin glasses"), drops the burn-in, and estimates tau_int(q) per beta with the
integrated autocorrelation of SM III truncated by Sokal's window (W >= 6 tau),
pooling the autocorrelation over the instances of each beta. Prints one JSON
object with the per-beta estimates, the sweep rate and the acceptance.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs, tnmc


def pooled_tau(series):
    """series: [T, k] independent chains of one observable -> (tau, window, error)."""
    x = np.asarray(series, dtype=np.float64)
    T = x.shape[0]
    xc = x - x.mean(axis=0, keepdims=True)
    var = (xc ** 2).mean(axis=0)
    ok = var > 0
    if T < 4 or not ok.any():
        return None, None, None
    rho = np.array([np.mean((xc[: T - k, ok] * xc[k:, ok]).mean(axis=0) / var[ok]) for k in range(T)])
    tau, W = 0.5, T - 1
    for w in range(1, T):
        tau += rho[w]
        if w >= 6 * tau:
            W = w
            break
    err = tau * np.sqrt(2.0 * (2 * W + 1) / (T * ok.sum()))
    return float(tau), int(W), float(err)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=32)
    ap.add_argument("--chi", type=int, default=64)
    ap.add_argument("--instances", type=int, default=2)
    ap.add_argument("--n-beta", type=int, default=16)
    ap.add_argument("--sweeps", type=int, default=60)
    ap.add_argument("--burn", type=int, default=20)
    ap.add_argument("--precision", default="f32", choices=["f32", "f64", "bf16"])
    ap.add_argument("--seed", type=int, default=4242)
    a = ap.parse_args()
    import torch
    betas = [float(b) for b in np.linspace(0.5, 1.6, a.n_beta)]
    wl = inputs.Workload(model=inputs.MODEL_EA_GAUSS, dims=(a.L,) * 3, bc=(1, 1, 1), chi=a.chi, betas=betas,
                         n_inst=a.instances, n_rep=2, seed=1)
    prec = {"f32": tnmc.PREC_F32, "f64": tnmc.PREC_F64, "bf16": tnmc.PREC_BF16}[a.precision]
    stream = torch.cuda.Stream()
    ctx = tnmc.Context([wl], precision=prec, stream=stream)
    ctx.set_spins(0, wl.initial_spins())
    obs = torch.zeros((a.sweeps, wl.n_chains, 3), dtype=torch.float64, device="cuda")
    acc = torch.zeros(wl.n_chains, dtype=torch.int32, device="cuda")
    t0 = time.perf_counter()
    for t in range(a.sweeps):
        ctx.sweep(1, a.seed, use_graph=True, accept_counter=acc)
        ctx.observables(0, out=obs[t])
    ctx.sync()
    dt = time.perf_counter() - t0
    q = obs[:, 0::2, 2].cpu().numpy()          # [T, pairs]; pair p = chains (2p, 2p+1)
    pair_beta = wl.chain_beta()[0::2]
    out = {"L": a.L, "chi": a.chi, "precision": a.precision, "chains": wl.n_chains, "sweeps": a.sweeps,
           "burn": a.burn, "seconds": dt, "sweeps_per_s": a.sweeps / dt,
           "acceptance": float(acc.sum().item()) / (a.sweeps * wl.n_chains * a.L), "per_beta": []}
    taus = []
    for b in betas:
        cols = np.where(np.isclose(pair_beta, b))[0]
        tau, W, err = pooled_tau(q[a.burn:, cols])
        out["per_beta"].append({"beta": round(b, 4), "tau_int_q": tau, "window": W, "error": err,
                                "q2": float(np.mean(q[a.burn:, cols] ** 2))})
        if tau is not None:
            taus.append(tau)
    out["tau_int_q_mean_over_beta"] = float(np.mean(taus)) if taus else None
    ctx.close()
    print(json.dumps(out))


if __name__ == "__main__":
    main()
