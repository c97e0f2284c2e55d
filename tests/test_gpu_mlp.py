"""BF16 tensor-core kernels of the learned-start network against CPU FP32
references computed from the same BF16-rounded inputs."""
import pytest
import torch

from paper_2203_06139_gb300 import cg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def dev():
    import __graft_entry__
    __graft_entry__.build()
    return torch.device("cuda:0")


def _bf(shape, seed, dev, scale=1.0):
    g = torch.Generator().manual_seed(seed)
    return (torch.randn(shape, generator=g) * scale).to(torch.bfloat16).to(dev)


@pytest.mark.parametrize("M,N,K,tA,tB", [(200, 512, 256, 0, 0), (300, 16, 512, 0, 0), (128, 128, 64, 0, 0),
                                         (257, 512, 320, 0, 1), (512, 256, 200, 1, 1), (96, 40, 130, 1, 0)])
def test_gemm_matches_fp32_reference(dev, M, N, K, tA, tB):
    A = _bf((K, M) if tA else (M, K), 1, dev)
    B = _bf((K, N) if tB else (N, K), 2, dev)
    C = torch.full((M, N), float("nan"), dtype=torch.float32, device=dev)
    err = torch.zeros(1, dtype=torch.int32, device=dev)
    cg.gemm_bf16(A, B, M, N, K, transA=tA, transB=tB, Cf=C, err=err)
    torch.cuda.synchronize()
    a = A.float().cpu()
    b = B.float().cpu()
    ref = (a.T if tA else a) @ (b if tB else b.T)
    assert int(err.item()) == 0
    torch.testing.assert_close(C.cpu(), ref, rtol=1e-4, atol=1e-4 * float(ref.abs().max()))


def test_gemm_epilogues(dev):
    M, N, K = 150, 96, 128
    A, B = _bf((M, K), 3, dev), _bf((N, K), 4, dev)
    bias = torch.randn(N, device=dev)
    z = torch.empty((M, N), device=dev)
    h = torch.empty((M, N), dtype=torch.bfloat16, device=dev)
    cg.gemm_bf16(A, B, M, N, K, Cb=h, bias=bias, aux_out=z, epilogue=cg.EPI_BIAS_GELU)
    ref_z = A.float() @ B.float().T + bias
    torch.testing.assert_close(z, ref_z, rtol=1e-4, atol=1e-3)
    torch.testing.assert_close(h.float(), torch.nn.functional.gelu(ref_z).bfloat16().float(), rtol=1e-2, atol=1e-2)
    dz = torch.empty((M, N), device=dev)
    cg.gemm_bf16(A, B, M, N, K, Cf=dz, aux_in=z, epilogue=cg.EPI_GELU_GRAD)
    zz = z.clone().requires_grad_(True)
    torch.nn.functional.gelu(zz).backward(A.float() @ B.float().T)
    torch.testing.assert_close(dz, zz.grad, rtol=1e-3, atol=1e-3)
