"""One launch of the slice-update kernel on a seeded workload, for profilers.

    python -m paper_2509_23945_gb300.profile_case --L 16 --chi 32 --slices 32 --precision f32

Builds a context of the Gaussian EA glass (periodic, R1) with enough replica chains, runs one
warm-up launch of two slices, then one launch of --slices slice updates (axis 0, even slices of
consecutive chains, hot start, no write-back) and prints the launch time measured with CUDA
events. Used to capture the kernel under ncu on a case of a chosen size.
"""
from __future__ import annotations

import argparse

from . import inputs, tnmc


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--L", type=int, default=16)
    ap.add_argument("--chi", type=int, default=32)
    ap.add_argument("--slices", type=int, default=32)
    ap.add_argument("--precision", default="f32", choices=["f32", "f64", "bf16"])
    ap.add_argument("--gemm", type=int, default=-1,
                    help="engine of the contractions, a TNMC_GEMM_* value (default: the context's)")
    ap.add_argument("--tile", type=int, default=-1, help="CUDA-core GEMM tile (0 64x64, 1 32x32, 2 128x64)")
    a = ap.parse_args()
    import torch
    prec = {"f32": tnmc.PREC_F32, "f64": tnmc.PREC_F64, "bf16": tnmc.PREC_BF16}[a.precision]
    per_chain = a.L // 2
    n_rep = max(2, -(-a.slices // per_chain))
    wl = inputs.Workload(model=inputs.MODEL_EA_GAUSS, dims=(a.L, a.L, a.L), bc=(1, 1, 1), chi=a.chi, betas=[1.0],
                         n_inst=1, n_rep=n_rep, seed=11)
    ctx = tnmc.Context([wl], precision=prec)
    if a.gemm >= 0:
        ctx.set_tuning(gemm_mode=a.gemm)
    if a.tile >= 0:
        ctx.set_tuning(gemm_tile=a.tile)
    ctx.set_spins(0, wl.initial_spins())
    chains = [c for c in range(wl.n_chains) for k in range(0, a.L, 2)][: a.slices]
    slices = [k for c in range(wl.n_chains) for k in range(0, a.L, 2)][: a.slices]
    ctx.slice_update(0, 0, chains[:2], slices[:2], 1, 1, write_back=False)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    ctx.slice_update(0, 0, chains, slices, 1, 2, write_back=False)
    e1.record()
    torch.cuda.synchronize()
    t = ctx.get_tuning()
    print(f"L={a.L} chi={a.chi} {a.precision} gemm_mode={t['gemm_mode']} gemm_tile={t['gemm_tile']}: {len(chains)} "
          f"slice updates in {e0.elapsed_time(e1) / 1e3:.3f} s")
    ctx.close()


if __name__ == "__main__":
    main()
