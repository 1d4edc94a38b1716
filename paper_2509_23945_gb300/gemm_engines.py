"""Throughput of the slice kernel's GEMM engines on their own (tnmc_cta_gemm), one CTA per matrix.

    python -m paper_2509_23945_gb300.gemm_engines --batch 304

Each engine runs the same batch of independent FP32 products (the shapes of the environment pass's
contractions at L = 32, chi = 64: the centre times a right factor, the products P, the trailing updates
of the LQ) with one CTA per product, as in the slice kernel (2 CTAs per SM at batch = 2 x SMs). Prints one
JSON line per (shape, engine): the mean time of one batched call (CUDA events around `reps` calls after
two untimed ones) and the flop rate 2 M N K batch / time.
"""
from __future__ import annotations

import argparse
import json

from . import tnmc

SHAPES = [(128, 256, 256), (64, 256, 64), (128, 64, 512), (256, 32, 512)]
ENGINES = {"ffma": tnmc.GEMM_FFMA, "mma_tf32x3": tnmc.GEMM_MMA_TF32X3, "mma_bf16": tnmc.GEMM_MMA_BF16,
           "umma_tf32x3": tnmc.GEMM_UMMA_TF32X3, "umma_bf16": tnmc.GEMM_UMMA_BF16}


def main(argv=None):
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--batch", type=int, default=304)
    ap.add_argument("--reps", type=int, default=5)
    ap.add_argument("--engines", nargs="+", default=list(ENGINES), choices=list(ENGINES))
    args = ap.parse_args(argv)
    tnmc.load_library()
    g = torch.Generator(device="cuda").manual_seed(1)
    for (M, N, K) in SHAPES:
        a = torch.randn(args.batch, M, K, device="cuda", generator=g)
        b = torch.randn(args.batch, K, N, device="cuda", generator=g)
        c = torch.zeros(args.batch, M, N, device="cuda")
        for name in args.engines:
            eng = ENGINES[name]
            for _ in range(2):
                tnmc.cta_gemm(eng, a, b, c)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            for _ in range(args.reps):
                tnmc.cta_gemm(eng, a, b, c)
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / args.reps
            print(json.dumps({"M": M, "N": N, "K": K, "batch": args.batch, "engine": name, "ms": ms,
                              "tflops": 2.0 * M * N * K * args.batch / (ms * 1e-3) / 1e12}), flush=True)


if __name__ == "__main__":
    main()
