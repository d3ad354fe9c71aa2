"""Tensor-core kernels of the learned warm start (GPU required).

References are plain PyTorch CPU computations in FP64 of the same
BF16-rounded inputs; the tensor cores accumulate in FP32, so products agree
to a few FP32 ulps of the accumulated magnitude.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _bf16_pair(M, N, K, seed):
    import torch
    g = torch.Generator().manual_seed(seed)
    A = torch.randn(M, K, generator=g).to(torch.bfloat16)
    B = torch.randn(N, K, generator=g).to(torch.bfloat16)
    ref = A.double() @ B.double().T
    return A, B, ref


def _tol(ref, K):
    return 1e-5 * np.sqrt(K) * max(1.0, float(ref.abs().max()))


def test_gemm_layout_fields():
    """The descriptor's leading offset is the step between core matrices along
    K and the stride offset the step between 8-row groups (the reading of the
    no-swizzle K-major layout used by the kernel)."""
    import torch
    from paper_1406_2686_gb300 import nn
    A, B, ref = _bf16_pair(128, 32, 64, 1)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = {}
    for swap in (0, 1):
        C = nn.gemm(A.cuda(), B.cuda(), layout=(128, 1024, swap), status=st)
        torch.cuda.synchronize()
        out[swap] = float((C.double().cpu() - ref).abs().max())
    assert int(st.item()) == 0
    print("layout errors (lbo field = K step, swapped):", out)
    assert out[0] < _tol(ref, 64)


@pytest.mark.parametrize("M,N,K", [(128, 32, 64), (256, 64, 128), (300, 48, 200), (1000, 128, 4096),
                                   (129, 16, 8), (4096, 100, 432)])
def test_gemm_matches_fp64(M, N, K):
    import torch
    from paper_1406_2686_gb300 import nn
    A, B, ref = _bf16_pair(M, N, K, M + N + K)
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    C = nn.gemm(A.cuda(), B.cuda(), status=st)
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    err = float((C.double().cpu() - ref).abs().max())
    assert err < _tol(ref, K), err


def test_gemm_accumulate_and_strides():
    """C += A B^T into a strided view keeps the old values and the untouched columns."""
    import torch
    from paper_1406_2686_gb300 import nn
    A, B, ref = _bf16_pair(200, 40, 96, 7)
    Cbig = torch.full((200, 64), 2.5, dtype=torch.float32, device="cuda")
    C = Cbig[:, 8:48]
    nn.gemm(A.cuda(), B.cuda(), C=C, accumulate=True)
    torch.cuda.synchronize()
    got = Cbig.double().cpu()
    assert float((got[:, 8:48] - (ref + 2.5)).abs().max()) < _tol(ref, 96)
    assert torch.all(got[:, :8] == 2.5) and torch.all(got[:, 48:] == 2.5)


def test_gemm_rejects_bad_arguments():
    import torch
    from paper_1406_2686_gb300 import nn
    A = torch.zeros(128, 12, dtype=torch.bfloat16, device="cuda")  # K not a multiple of 8
    B = torch.zeros(32, 12, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(nn.NNError):
        nn.gemm(A, B)
    A = torch.zeros(128, 64, dtype=torch.bfloat16, device="cuda")
    B = torch.zeros(32, 64, dtype=torch.bfloat16, device="cuda")
    with pytest.raises(nn.NNError):
        nn.gemm(A, B, layout=(4096, 4096, 0))  # would leave the staged tile
