"""Tensor-core BF16 GEMM (tcgen05) through the C-ABI against a plain PyTorch FP32 product of
the same BF16 operands."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
DEV = "cuda:0"


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build()
    from paper_2301_04259_gb300 import soap
    torch.backends.cuda.matmul.allow_tf32 = False
    return soap


SHAPES = [(128, 128, 64), (300, 129, 8), (8192, 256, 256), (256, 8, 8192), (1000, 256, 136),
          (64, 64, 1000), (129, 200, 72), (4096, 144, 384)]


@pytest.mark.parametrize("M,N,K", SHAPES)
@pytest.mark.parametrize("act", [0, 1])
def test_gemm_matches_fp32_product(S, M, N, K, act):
    g = torch.Generator(device=DEV).manual_seed(M * 7 + N * 3 + K)
    lda = (K + 7) // 8 * 8 + (8 if K % 16 == 0 else 0)     # padded strides on some shapes
    A = torch.randn(M, lda, device=DEV, generator=g).to(torch.bfloat16)
    B = torch.randn(N, lda, device=DEV, generator=g).to(torch.bfloat16)
    bias = torch.randn(N, device=DEV, generator=g) if act else None
    C = torch.full((M, N + 3), float("nan"), device=DEV)
    S.soap_gemm_bf16_tn(A[:, :K], B[:, :K], C, bias=bias, activation=act)
    torch.cuda.synchronize()
    ref = A[:, :K].float() @ B[:, :K].float().T
    if bias is not None:
        ref = ref + bias
    bound = (A[:, :K].float().abs() @ B[:, :K].float().abs().T) * 2e-6 + 1e-6
    z = C[:, :N]
    if act:
        ref = torch.nn.functional.gelu(ref)
        bound = bound * 1.5 + 1e-6 * ref.abs()
    assert torch.isnan(C[:, N:]).all()                   # nothing written past N
    err = (z - ref).abs()
    assert bool((err <= bound).all()), float((err / bound).max())
