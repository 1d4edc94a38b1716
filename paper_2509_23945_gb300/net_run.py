"""The learned proposal on a workload: train on tensor-network-accepted slices, then compare.

    python -m paper_2509_23945_gb300.net_run --L 32 --chi 64 --tn-sweeps 6 --train-steps 1500

Builds the Gaussian EA workload (periodic, R1, one disorder instance x n_beta temperatures in
[0.5, 1.6] x 2 replicas) with a masked-convolution network (channels x layers), then:
  1. runs --tn-sweeps tensor-network sweeps that record every accepted slice in the replay buffer,
     timing them (accepted slices per second of the tensor network);
  2. trains the network for --train-steps Adam steps on the buffer, timing the training;
  3. runs --net-sweeps sweeps that propose with the network only, timing them (its acceptance and
     accepted slices per second);
  4. runs --mix-sweeps sweeps alternating the two proposals 1:1 (net_every = 2).
Prints one JSON line with the acceptances, sweep times, accepted slices per second and losses.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs, tnmc


def timed_sweeps(ctx, n, seed, acc, slices_per_sweep):
    import torch
    acc.zero_()
    ctx.sync()
    t0 = time.perf_counter()
    ctx.sweep(n, seed, use_graph=True, accept_counter=acc)
    ctx.sync()
    dt = (time.perf_counter() - t0) / max(n, 1)
    a = acc.sum().item() / (max(n, 1) * slices_per_sweep)
    return a, dt


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=32)
    ap.add_argument("--chi", type=int, default=64)
    ap.add_argument("--n-beta", type=int, default=16)
    ap.add_argument("--channels", type=int, default=64)
    ap.add_argument("--layers", type=int, default=6)
    ap.add_argument("--tn-sweeps", type=int, default=6)
    ap.add_argument("--train-steps", type=int, default=1500)
    ap.add_argument("--batch", type=int, default=64)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--net-sweeps", type=int, default=3)
    ap.add_argument("--mix-sweeps", type=int, default=6)
    ap.add_argument("--seed", type=int, default=5)
    a = ap.parse_args()
    import torch
    betas = inputs.linspace_betas(0.5, 1.6, a.n_beta)
    wl = inputs.Workload(model=inputs.MODEL_EA_GAUSS, dims=(a.L, a.L, a.L), bc=(1, 1, 1), chi=a.chi, betas=betas,
                         n_inst=1, n_rep=2, seed=a.seed)
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F32)
    ctx.set_spins(0, wl.initial_spins())
    ctx.net_init(channels=a.channels, layers=a.layers, seed=a.seed, buffer_slots=8192)
    acc = torch.zeros(wl.n_chains, dtype=torch.int32, device="cuda")
    per_sweep = wl.n_chains * a.L
    ctx.set_proposal_mix(0, True)
    acc_tn, t_tn = timed_sweeps(ctx, a.tn_sweeps, a.seed, acc, per_sweep)
    ctx.set_proposal_mix(1, False)
    acc_net0, t_net0 = timed_sweeps(ctx, 1, a.seed + 1, acc, per_sweep)
    ctx.sync()
    t0 = time.perf_counter()
    losses = ctx.net_train(a.train_steps, a.batch, a.lr, a.seed)
    t_train = time.perf_counter() - t0
    acc_net, t_net = timed_sweeps(ctx, a.net_sweeps, a.seed + 2, acc, per_sweep)
    ctx.set_proposal_mix(2, False)
    acc_mix, t_mix = timed_sweeps(ctx, a.mix_sweeps, a.seed + 3, acc, per_sweep)
    ctx.close()
    k = max(1, min(50, len(losses) // 10))
    print(json.dumps({
        "L": a.L, "chi": a.chi, "chains": wl.n_chains, "net": f"{a.layers} layers x {a.channels} channels",
        "buffer_positions": None, "tn": {"acceptance": acc_tn, "s_per_sweep": t_tn,
                                         "accepted_slices_per_s": acc_tn * per_sweep / t_tn},
        "net_before_training": {"acceptance": acc_net0, "s_per_sweep": t_net0},
        "training": {"steps": a.train_steps, "batch": a.batch, "seconds": t_train,
                     "loss_first": float(np.mean(losses[:k])), "loss_last": float(np.mean(losses[-k:]))},
        "net_after_training": {"acceptance": acc_net, "s_per_sweep": t_net,
                               "accepted_slices_per_s": acc_net * per_sweep / t_net},
        "mix_1_to_1": {"acceptance": acc_mix, "s_per_sweep": t_mix,
                       "accepted_slices_per_s": acc_mix * per_sweep / t_mix},
    }), flush=True)


if __name__ == "__main__":
    main()
