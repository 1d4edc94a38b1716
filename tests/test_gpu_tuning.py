"""Kernel configurations that do not change the arithmetic (where the eigenproblem
lives, how many CTAs share an SM) give bitwise identical chains; the autotuner
times the candidates and applies the fastest."""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2509_23945_gb300 import autotune, inputs, tnmc  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_23945_gb300 import build_lib
    build_lib.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(wl, prec, **tuning):
    ctx = tnmc.Context([wl], precision=prec)
    ctx.set_spins(0, wl.initial_spins())
    if tuning:
        ctx.set_tuning(**tuning)
    ctx.sweep(4, 31)
    s = ctx.get_spins(0)
    t = ctx.get_tuning()
    ctx.close()
    return s, t


@pytest.mark.parametrize("prec", [tnmc.PREC_F32, tnmc.PREC_F64])
def test_layout_only_tunings_are_bitwise_identical(prec):
    wl = inputs.Workload(model=inputs.MODEL_EA_GAUSS, dims=(8, 8, 8), bc=(1, 1, 1), chi=12, betas=[0.9, 1.3],
                         n_inst=2, n_rep=2, seed=3)
    ref, t0 = _run(wl, prec)
    cfgs = [dict(eig_smem=0), dict(ctas_per_sm=1), dict(eig_smem=0, ctas_per_sm=1)]
    if prec != tnmc.PREC_F64:
        cfgs += [dict(gemm_tile=1), dict(gemm_tile=2), dict(gemm_tile=2, eig_smem=0)]
    for cfg in cfgs:
        got, t = _run(wl, prec, **cfg)
        for k, v in cfg.items():
            assert t[k] == v
        assert np.array_equal(got, ref), cfg


@pytest.mark.parametrize("prec", [tnmc.PREC_F32, tnmc.PREC_BF16])
def test_gemm_tiles_are_bitwise_identical_on_large_bonds(prec):
    """chi = 40 on ring rows (bond 160): the GEMMs span several tiles of every shape, with ragged edges,
    and the LQ trailing updates cover triangular (b_lower) operands. Every tile gives the same chain."""
    wl = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(6, 6, 6), bc=(1, 1, 1), chi=40, betas=[1.1], n_inst=1,
                         n_rep=2, seed=8)
    ref, _ = _run(wl, prec)
    for tile in (1, 2):
        got, t = _run(wl, prec, gemm_tile=tile)
        assert t["gemm_tile"] == tile
        assert np.array_equal(got, ref), tile


def test_gemm_tile_values_checked():
    wl = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(4, 4, 4), bc=(1, 1, 1), chi=4, betas=[1.0], n_inst=1,
                         n_rep=1, seed=1)
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F64)
    with pytest.raises(tnmc.TnmcError):
        ctx.set_tuning(gemm_tile=1)          # F64 has the default tile only
    ctx.close()
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F32)
    with pytest.raises(tnmc.TnmcError):
        ctx.set_tuning(gemm_tile=3)
    ctx.close()


def test_autotune_picks_and_applies(tmp_path):
    autotune.CACHE = str(tmp_path / "tune.json")
    wl = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(8, 8, 8), bc=(1, 1, 1), chi=8, betas=[1.0], n_inst=4,
                         n_rep=2, seed=5)
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F32)
    ctx.set_spins(0, wl.initial_spins())
    out = autotune.tune(ctx, 0, n_chains=8)
    assert len(out["times"]) == len(autotune.candidates(tnmc.PREC_F32))
    t = ctx.get_tuning()
    for k, v in out["best"].items():
        if k == "ctas_per_sm":          # a request: the kernel instance's occupancy caps it
            assert 1 <= t[k] <= v
        elif v >= 0:                    # -1 keeps the current setting
            assert t[k] == v
    assert autotune.apply_cached(ctx, 0) == out["best"]
    ctx.close()
