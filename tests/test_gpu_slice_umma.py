"""GPU parity of the slice update with the contractions on the tcgen05 engines (tensor memory
accumulators), against the CPU oracle, with the bars of the default engines: FP32 with the 3xTF32
engine 1e-4 per slice on typical slices (and the per-site bound on hot-start log q_old); BF16 with the
tcgen05 BF16 engine reported against 3e-2. Sampled spins, dE and accept decisions are compared
exactly away from CDF and Metropolis thresholds."""
import pytest

torch = pytest.importorskip("torch")

from paper_2509_23945_gb300 import tnmc  # noqa: E402
from test_gpu_slice import CASES, TOL_F32_HOT_OLD_PER_SITE, _compare_batch  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_23945_gb300 import build_lib
    build_lib.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("name", list(CASES))
def test_slice_update_parity_f32_umma(name):
    st = _compare_batch(name, tnmc.PREC_F32, warm=2, gemm_mode=tnmc.GEMM_UMMA_TF32X3)
    print("FP32 (tcgen05 3xTF32) log q error", name, st)


@pytest.mark.parametrize("name", ["L6_gauss_chi8", "L10_ragged_chi24"])
def test_slice_update_parity_f32_umma_hot_start(name):
    st = _compare_batch(name, tnmc.PREC_F32, hot_old_per_site=TOL_F32_HOT_OLD_PER_SITE,
                        gemm_mode=tnmc.GEMM_UMMA_TF32X3)
    print("FP32 (tcgen05 3xTF32) hot start", name, st)


@pytest.mark.parametrize("name", ["L6_gauss_chi8", "potts_L5", "L10_ragged_chi24"])
def test_slice_update_parity_bf16_umma_reported(name):
    st = _compare_batch(name, tnmc.PREC_BF16, warm=2, check_old=False, bf16_report=True,
                        gemm_mode=tnmc.GEMM_UMMA_BF16)
    worst = max(st["worst_old"], st["worst_new"])
    print(f"BF16 (tcgen05) log q error {name}: worst {worst:.3e} per slice "
          f"(bar 3e-2: {'met' if worst < 3e-2 else 'MISSED'}), {st}")


def test_umma_tuning_values_checked():
    """F32 takes only FP32-level engines, BF16 only BF16 engines."""
    from paper_2509_23945_gb300 import inputs
    wl = inputs.Workload(model=inputs.MODEL_EA_PM, dims=(4, 4, 4), bc=(1, 1, 1), chi=4, betas=[1.0], n_inst=1,
                         n_rep=1)
    ctx = tnmc.Context([wl], precision=tnmc.PREC_F32)
    for bad in (tnmc.GEMM_MMA_BF16, tnmc.GEMM_UMMA_BF16, 5):
        with pytest.raises(tnmc.TnmcError):
            ctx.set_tuning(gemm_mode=bad)
    ctx.set_tuning(gemm_mode=tnmc.GEMM_UMMA_TF32X3)
    assert ctx.get_tuning()["gemm_mode"] == tnmc.GEMM_UMMA_TF32X3
    ctx.close()
