"""The CTA-level GEMM engines of the slice kernel's contractions against an FP64 host product.

Every step of the environment pass is a product of small dense matrices (SM I.B); the slice kernel runs
them on one of these engines. Each case runs one CTA per matrix through tnmc_cta_gemm, on shapes that span
several output tiles with ragged edges, all four transpose combinations, beta = 0 and beta != 0, and K = 0.
Bounds (elementwise, relative to |op(A)| |op(B)|, the scale of the rounding errors of a length-K sum):
  FFMA and the 3xTF32 engines: 2e-6 (FP32 accumulation over K <= 300 terms; the TF32 split carries
  2^-22 per product);
  BF16 engines: the product of the BF16-rounded operands to 2e-6 (BF16 products are exact in FP32, the
  accumulation is FP32).
"""
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

SHAPES = [(128, 64, 16), (200, 100, 75), (64, 256, 128), (1, 1, 1), (130, 65, 300), (37, 129, 33)]


@pytest.fixture(scope="module")
def tn():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_2509_23945_gb300 import build_lib, tnmc
    build_lib.build()
    tnmc.load_library()
    return tnmc


def _bf16(x):
    return x.to(torch.bfloat16).to(torch.float64)


def _run(tn, engine, M, N, K, ta, tb, beta, batch=3, seed=0):
    g = torch.Generator().manual_seed(seed + 1000 * M + 7 * N + K)
    a = torch.randn(batch, *( (K, M) if ta else (M, K) ), generator=g)
    b = torch.randn(batch, *( (N, K) if tb else (K, N) ), generator=g)
    c0 = torch.randn(batch, M, N, generator=g)
    opa = a.transpose(1, 2) if ta else a
    opb = b.transpose(1, 2) if tb else b
    c = c0.clone().cuda()
    tn.cta_gemm(engine, a.cuda(), b.cuda(), c, alpha=1.5, beta=beta, trans_a=ta, trans_b=tb)
    torch.cuda.synchronize()
    bf = engine in (tn.GEMM_MMA_BF16, tn.GEMM_UMMA_BF16)
    A64 = _bf16(opa) if bf else opa.double()
    B64 = _bf16(opb) if bf else opb.double()
    ref = 1.5 * (A64 @ B64) + beta * c0.double()
    scale = 1.5 * (A64.abs() @ B64.abs()) + abs(beta) * c0.double().abs() + 1e-30
    err = ((c.cpu().double() - ref).abs() / scale).max().item()
    return err


ENGINES = ["GEMM_FFMA", "GEMM_MMA_TF32X3", "GEMM_MMA_BF16", "GEMM_UMMA_TF32X3", "GEMM_UMMA_BF16"]


@pytest.mark.parametrize("engine", ENGINES)
@pytest.mark.parametrize("ta,tb", [(False, False), (True, False), (False, True), (True, True)])
def test_gemm_engine_matches_fp64(tn, engine, ta, tb):
    worst = 0.0
    for (M, N, K) in SHAPES:
        for beta in (0.0, -0.75):
            err = _run(tn, getattr(tn, engine), M, N, K, ta, tb, beta)
            worst = max(worst, err)
            assert err < 2e-6, (engine, M, N, K, ta, tb, beta, err)
    print(f"{engine} ta={ta} tb={tb}: worst relative error {worst:.2e}")


@pytest.mark.parametrize("engine", ENGINES)
def test_gemm_engine_k_zero(tn, engine):
    """K = 0: C = beta C exactly (alpha times an empty sum)."""
    c0 = torch.randn(2, 70, 90)
    c = c0.clone().cuda()
    a = torch.zeros(2, 70, 1).cuda()[:, :, :0].contiguous()
    b = torch.zeros(2, 0, 90).cuda()
    tn.cta_gemm(getattr(tn, engine), a, b, c, alpha=2.0, beta=0.5)
    assert torch.equal(c.cpu(), c0 * 0.5)


def test_umma_bf16_differs_from_fp32_product(tn):
    """The BF16 engine really rounds its operands (its result is the BF16 product, not the FP32 one)."""
    g = torch.Generator().manual_seed(3)
    a = torch.randn(1, 128, 64, generator=g)
    b = torch.randn(1, 64, 64, generator=g)
    c = torch.zeros(1, 128, 64).cuda()
    tn.cta_gemm(tn.GEMM_UMMA_BF16, a.cuda(), b.cuda(), c)
    exact = a.double() @ b.double()
    rounded = _bf16(a) @ _bf16(b)
    got = c.cpu().double()
    assert (got - rounded).abs().max() < 1e-4
    assert (got - exact).abs().max() > 1e-3
