"""The tensor-core projection contraction C = B V^T (tcgen05, BF16 inputs,
FP32 accumulation) against an FP64 product of the same BF16 values."""
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def kp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2511_17634_gb300 import build
    build.build()
    from paper_2511_17634_gb300 import kp as K
    return K


@pytest.mark.parametrize("nt,nv,K", [(128, 48, 1024), (300, 41, 4096), (5, 7, 784),
                                     (1, 1, 64), (257, 16, 16384)])
def test_projection_gemm_matches_fp64(kp, nt, nv, K):
    g = torch.Generator(device="cuda").manual_seed(nt * 7 + nv)
    ld = (K + 7) // 8 * 8
    B = torch.randn(nt, ld, device="cuda", generator=g).to(torch.bfloat16)
    V = torch.randn(nv, ld, device="cuda", generator=g).to(torch.bfloat16)
    C = torch.full((nt, nv + 3), float("nan"), device="cuda", dtype=torch.float32)
    ctx = kp.Context(max_n=16384)
    ctx.project_gemm_bf16(B, V, C, K=K)
    torch.cuda.synchronize()
    ref = B[:, :K].double() @ V[:, :K].double().T
    scale = B[:, :K].double().abs() @ V[:, :K].double().abs().T
    err = (C[:, :nv].double() - ref).abs()
    assert torch.isfinite(C[:, :nv]).all()
    assert bool((err <= 2e-6 * scale + 1e-6).all()), float((err / (scale + 1e-30)).max())
    assert torch.isnan(C[:, nv:]).all()          # columns beyond nv untouched
