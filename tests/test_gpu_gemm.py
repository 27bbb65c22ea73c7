"""Tensor-core GEMM (tcgen05, BF16 in, FP32 accumulate) through the C ABI against the
same product computed in float64 from the same BF16 values.  The tolerance is that of
FP32 accumulation over K terms (a few units of 2^-24 times sqrt(K) of the magnitude)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def Q():
    from paper_2406_15632_gb300 import build as B
    from paper_2406_15632_gb300 import qmcrt

    B.build()
    qmcrt.load()
    return qmcrt


def _bf16(shape, seed, scale=1.0):
    import torch

    g = torch.Generator().manual_seed(seed)
    return (torch.randn(shape, generator=g) * scale).to(torch.bfloat16)


def _check(got, ref, K):
    tol = 4 * 2.0 ** -24 * np.sqrt(K) * np.abs(ref).max() + 1e-30
    assert np.abs(got - ref).max() <= tol * 8, (np.abs(got - ref).max(), tol)


# K <= 128 runs the persistent warp-specialised form (several tiles per CTA once M passes
# 152 x 128 rows, both TMEM accumulators in turn); larger K the streaming form
@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (300, 128, 96), (77, 32, 256), (1000, 64, 1024), (5, 32, 64),
                                   (1000, 64, 128), (129, 128, 128), (40000, 128, 128), (40001, 32, 32)])
def test_gemm_plain(Q, M, N, K):
    import torch

    A, B = _bf16((M, K), 1), _bf16((N, K), 2)
    out = torch.full((M, N), np.nan, dtype=torch.float32, device="cuda")
    err = torch.zeros(1, dtype=torch.int32, device="cuda")
    Q.gemm(A.cuda(), B.cuda(), out_f32=out, error=err)
    torch.cuda.synchronize()
    ref = A.double().numpy() @ B.double().numpy().T
    _check(out.cpu().numpy(), ref, K)
    assert err.item() == 0


@pytest.mark.parametrize("M,ldt", [(257, 320), (40000, 40003)])
def test_gemm_epilogues(Q, M, ldt):
    """Bias, ReLU, mask and all three outputs; the transposed copy with a row length that
    is and is not a multiple of 8 (vector and element stores)."""
    import torch

    N, K = 128, 128
    A, B = _bf16((M, K), 3), _bf16((N, K), 4)
    bias = torch.randn(N, generator=torch.Generator().manual_seed(5))
    mask = _bf16((M, N), 6)
    o32 = torch.zeros((M, N), dtype=torch.float32, device="cuda")
    o16 = torch.zeros((M, N), dtype=torch.bfloat16, device="cuda")
    ot = torch.zeros((N, ldt), dtype=torch.bfloat16, device="cuda")
    Q.gemm(A.cuda(), B.cuda(), bias=bias.cuda(), relu=True, mask=mask.cuda(), out_f32=o32, out_bf16=o16, out_bf16_t=ot)
    torch.cuda.synchronize()
    ref = A.double().numpy() @ B.double().numpy().T + bias.double().numpy()[None, :]
    ref = np.maximum(ref, 0.0) * (mask.float().numpy() > 0)
    _check(o32.cpu().numpy(), ref, K)
    assert torch.equal(o16.cpu(), o32.cpu().to(torch.bfloat16))
    assert torch.equal(ot[:, :M].cpu(), o16.cpu().T)
    assert torch.all(ot[:, M:] == 0)


@pytest.mark.parametrize("M,N,K,splits", [(128, 32, 4096, 8), (32, 128, 4096, 8), (128, 128, 65536, 128),
                                           (100, 64, 3000 // 32 * 32, 7)])
def test_gemm_split_k_adds_atomically(Q, M, N, K, splits):
    """The weight-gradient form: K split over CTAs, partial tiles added into out_f32
    (fewer rows than a tile, and slices that do not divide K, included)."""
    import torch

    A, B = _bf16((M, K), 7), _bf16((N, K), 8)
    out = torch.ones((M, N), dtype=torch.float32, device="cuda")
    Q.gemm(A.cuda(), B.cuda(), out_f32=out, k_splits=splits)
    torch.cuda.synchronize()
    ref = 1.0 + A.double().numpy() @ B.double().numpy().T
    _check(out.cpu().numpy(), ref, K)
