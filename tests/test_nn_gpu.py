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
                                   (129, 16, 8), (4096, 100, 432), (384, 256, 320), (700, 200, 1000),
                                   (512, 640, 264), (130, 129, 72)])
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


@pytest.mark.parametrize("K,k_split", [(1000, 256), (4096, 1024), (200, 64)])
def test_gemm_splitk_slices_sum_to_product(K, k_split):
    """The split-K form: slice z reduces K in [z k_split, (z + 1) k_split) into
    its own C slice (the last slice ragged, zero-filled beyond K); the slices
    sum to A B^T, and each slice equals the product of its K range."""
    import torch
    from paper_1406_2686_gb300 import nn
    M, N = 260, 96
    A, B, ref = _bf16_pair(M, N, K, K + k_split)
    splits = (K + k_split - 1) // k_split
    parts = torch.full((splits, M, N), 7.0, dtype=torch.float32, device="cuda")
    st = torch.zeros(1, dtype=torch.int32, device="cuda")
    lb = nn.L()
    Ad, Bd = A.cuda(), B.cuda()  # kept alive until the kernel has run
    nn._check(lb.vefd_nn_gemm_bf16_splitk(Ad.data_ptr(), K, Bd.data_ptr(), K, parts.data_ptr(), N, M, N, K, k_split,
                                          M * N, st.data_ptr(), nn._stream()), "splitk")
    torch.cuda.synchronize()
    assert int(st.item()) == 0
    got = parts.double().cpu()
    assert float((got.sum(0) - ref).abs().max()) < _tol(ref, K)
    for z in range(splits):
        k0, k1 = z * k_split, min(K, (z + 1) * k_split)
        sub = A[:, k0:k1].double() @ B[:, k0:k1].double().T
        assert float((got[z] - sub).abs().max()) < _tol(sub, k1 - k0), z


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


# --- convolution layers and the network against PyTorch CPU autograd (FP64) ----

def _torch_weight(lay):
    """Our w[o][((dz*3+dy)*3+dx)*Cin + c] (BF16-rounded) as torch [Cout, Cin, 3, 3, 3]."""
    import torch
    w = lay.w.cpu().to(torch.bfloat16).double()
    return w.view(lay.cout, 3, 3, 3, lay.cin).permute(0, 4, 1, 2, 3).contiguous()


def _ncdhw(x):
    return x.permute(0, 4, 1, 2, 3)


def _rel(a, b):
    import torch
    return float(torch.linalg.norm((a - b).flatten()) / max(1e-30, float(torch.linalg.norm(b.flatten()))))


@pytest.mark.parametrize("cin,cout,stride,relu,shape", [(5, 16, 1, True, (1, 8, 8, 16)), (16, 32, 2, True, (2, 8, 16, 8)),
                                                        (24, 8, 1, False, (1, 16, 8, 8))])
def test_conv_layer_matches_torch(cin, cout, stride, relu, shape):
    """Forward values and the gradients of input, weights and bias of one
    convolution layer agree with FP64 autograd of the same BF16-rounded
    weights (the GEMM operands are BF16: a few 1e-3 relative)."""
    import torch
    import torch.nn.functional as F
    from paper_1406_2686_gb300 import nn
    g = torch.Generator().manual_seed(cin + cout)
    lay = nn.Conv3d(cin, cout, stride, relu, gen=g)
    lay.b.copy_(torch.randn(cout, generator=g).cuda() * 0.1)
    x = torch.randn(*shape, cin, generator=g)
    y = lay.forward(x.cuda().contiguous())
    dy = torch.randn(*y.shape, generator=g)
    dx = lay.backward(dy.cuda())
    torch.cuda.synchronize()
    xr = _ncdhw(x.to(torch.bfloat16).double()).requires_grad_(True)
    wr = _torch_weight(lay).requires_grad_(True)
    br = lay.b.cpu().double().requires_grad_(True)
    yr = F.conv3d(xr, wr, br, stride=stride, padding=1)
    if relu:
        yr = F.relu(yr)
    yr.backward(_ncdhw(dy.double()))
    assert _rel(_ncdhw(y.cpu().double()), yr.detach()) < 1e-2
    assert _rel(_ncdhw(dx.cpu().double()), xr.grad) < 2e-2
    dwr = wr.grad.permute(0, 2, 3, 4, 1).reshape(cout, -1)
    assert _rel(lay.dw.cpu().double(), dwr) < 2e-2
    assert _rel(lay.db.cpu().double(), br.grad) < 1e-3
    assert int(lay.status.item()) == 0


@pytest.mark.parametrize("channels", [(8, 16, 32, 64), (8, 16, 24, 40)])
def test_unet_gradients_match_torch(channels):
    """The whole U-Net (forward, MSE loss, backward through every layer, skip
    and upsampling) against FP64 autograd of the same weights, for the
    doubling channel plan and an uneven one."""
    import torch
    import torch.nn.functional as F
    from paper_1406_2686_gb300 import nn
    net = nn.UNet(5, 8, seed=3, channels=channels)
    g = torch.Generator().manual_seed(5)
    for lay in net.layers:
        lay.b.copy_(torch.randn(lay.cout, generator=g).cuda() * 0.05)
    x = torch.randn(1, 16, 16, 16, 5, generator=g)
    t = torch.randn(1, 16, 16, 16, 8, generator=g)
    out = net.forward(x.cuda().contiguous())
    loss_parts, grad = nn.mse(out, t.cuda().contiguous())
    net.backward(grad)
    torch.cuda.synchronize()
    loss = float(loss_parts.sum()) / out.numel()

    W = {id(l): _torch_weight(l).requires_grad_(True) for l in net.layers}
    Bv = {id(l): l.b.cpu().double().requires_grad_(True) for l in net.layers}

    def run(layers, h):
        for l in layers:
            h = F.conv3d(h, W[id(l)], Bv[id(l)], stride=l.stride, padding=1)
            if l.relu:
                h = F.relu(h)
        return h

    up = lambda h: F.interpolate(h, scale_factor=2, mode="nearest")
    xr = _ncdhw(x.double())
    s0 = run(net.e0, xr)
    s1 = run(net.e1, s0)
    s2 = run(net.e2, s1)
    s3 = run(net.e3, s2)
    u2 = run(net.d2, torch.cat([up(s3), s2], 1))
    u1 = run(net.d1, torch.cat([up(u2), s1], 1))
    o = run(net.d0, torch.cat([up(u1), s0], 1))
    lr = ((o - _ncdhw(t.double())) ** 2).mean()
    lr.backward()
    assert abs(loss / float(lr.detach()) - 1) < 2e-2
    assert _rel(_ncdhw(out.cpu().double()), o.detach()) < 3e-2
    # every GEMM rounds its operands (activations, gradients) to BF16, so the
    # error grows along the backward chain: direction and size are compared
    for l in net.layers:
        dwr = W[id(l)].grad.permute(0, 2, 3, 4, 1).reshape(l.cout, -1)
        for a, r in ((l.dw.cpu().double(), dwr), (l.db.cpu().double(), Bv[id(l)].grad)):
            cos = float((a * r).sum() / (torch.linalg.norm(a) * torch.linalg.norm(r)))
            assert cos > 0.995 and abs(float(torch.linalg.norm(a) / torch.linalg.norm(r)) - 1) < 0.05, (l.cout, cos)
            assert _rel(a, r) < 0.1
    assert net.status() == 0
