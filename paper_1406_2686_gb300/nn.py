"""Binding of the warm-start network's tensor-core kernels (``include/vefd_nn.h``).

Argument marshalling only: the matrix products, convolutions and optimizer
steps run in the CUDA kernels of ``libvefd.so``; torch tensors provide device
memory.  There is no CPU fallback.
"""
import ctypes

from . import vefd

OK, ERR_ARG, ERR_CUDA = 0, -1, -2

NN_EXPORTS = ["vefd_nn_gemm_bf16", "vefd_nn_gemm_bf16_layout"]

_sigs_done = False


def lib():
    global _sigs_done
    L = vefd.load()
    if not _sigs_done:
        vp, cint, cu = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint
        L.vefd_nn_gemm_bf16.argtypes = [vp, cint, vp, cint, vp, cint, cint, cint, cint, cint, vp, vp]
        L.vefd_nn_gemm_bf16_layout.argtypes = [vp, cint, vp, cint, vp, cint, cint, cint, cint, cint, cu, cu, cint, vp,
                                               vp]
        for n in NN_EXPORTS:
            getattr(L, n).restype = cint
        _sigs_done = True
    return L


class NNError(RuntimeError):
    pass


def _check(st, what):
    if st != OK:
        raise NNError("%s failed with status %d" % (what, st))


def _stream():
    import torch
    return torch.cuda.current_stream().cuda_stream


def gemm(A, B, C=None, accumulate=False, status=None, layout=None):
    """C = A @ B.T (or C += A @ B.T) for BF16 A [M, K], B [N, K] (K-major,
    K a multiple of 8) into FP32 C [M, N]; all torch CUDA tensors."""
    import torch
    assert A.dtype == torch.bfloat16 and B.dtype == torch.bfloat16
    M, K = A.shape
    N = B.shape[0]
    if C is None:
        C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    if status is None:
        status = torch.zeros(1, dtype=torch.int32, device=A.device)
    args = (A.data_ptr(), A.stride(0), B.data_ptr(), B.stride(0), C.data_ptr(), C.stride(0), M, N, K,
            int(bool(accumulate)))
    if layout is None:
        _check(lib().vefd_nn_gemm_bf16(*args, status.data_ptr(), _stream()), "gemm")
    else:
        lbo, sbo, swap = layout
        _check(lib().vefd_nn_gemm_bf16_layout(*args, lbo, sbo, swap, status.data_ptr(), _stream()), "gemm")
    return C


# --- remaining kernels of the network ---------------------------------------

_MORE = {
    "vefd_nn_gemm_bf16_splitk": "vp i vp i vp i i i i i ll vp vp",
    "vefd_nn_im2col3d": "vp i i i i i i i vp vp vp",
    "vefd_nn_col2im3d": "vp i i i i i i i vp vp",
    "vefd_nn_bias_act": "vp vp ll i i vp",
    "vefd_nn_act_backward": "vp vp ll i i vp vp vp vp",
    "vefd_nn_colsum": "vp ll i vp vp i vp",
    "vefd_nn_pack_weights": "vp i i i vp vp vp",
    "vefd_nn_splitk_reduce_t": "vp i ll i i i vp i vp",
    "vefd_nn_upsample2": "vp i i i i i vp vp",
    "vefd_nn_upsample2_backward": "vp i i i i i vp i vp",
    "vefd_nn_concat": "vp i vp i ll vp vp",
    "vefd_nn_split": "vp i i ll vp vp i vp",
    "vefd_nn_mse": "vp vp ll vp vp vp",
    "vefd_nn_add": "vp vp ll vp vp",
    "vefd_nn_adam": "vp vp vp vp ll f f f f i vp",
    "vefd_nn_to_fields": "vp vp ll f f f f vp vp vp vp vp",
    "vefd_nn_scale": "vp ll f vp",
}
NN_EXPORTS += list(_MORE) + ["vefd_nn_colsum_scratch"]
_more_done = False


def L():
    global _more_done
    lb = lib()
    if not _more_done:
        m = {"vp": ctypes.c_void_p, "i": ctypes.c_int, "ll": ctypes.c_longlong, "f": ctypes.c_float}
        for name, sig in _MORE.items():
            fn = getattr(lb, name)
            fn.argtypes = [m[t] for t in sig.split()]
            fn.restype = ctypes.c_int
        lb.vefd_nn_colsum_scratch.argtypes = [ctypes.c_longlong, ctypes.c_int]
        lb.vefd_nn_colsum_scratch.restype = ctypes.c_longlong
        _more_done = True
    return lb


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def round8(n):
    return (n + 7) // 8 * 8


class Conv3d:
    """3x3x3 convolution, zero padding 1, stride 1 or 2, on channels-last FP32
    activations [B, D, H, W, C]: im2col, tensor-core GEMM, bias, optional ReLU.
    FP32 master weights w [Cout, 27 Cin] (tap-major columns), BF16 copies for
    the products, Adam moments."""

    def __init__(self, cin, cout, stride=1, relu=True, gen=None):
        import torch
        assert cout % 8 == 0 and stride in (1, 2)
        self.cin, self.cout, self.stride, self.relu = cin, cout, stride, relu
        self.K27 = 27 * cin
        self.Kp = round8(self.K27)
        std = (2.0 / self.K27) ** 0.5
        w = torch.randn(cout, self.K27, generator=gen) * std
        self.w = w.cuda()
        self.b = torch.zeros(cout, device="cuda")
        self.dw = torch.zeros_like(self.w)
        self.db = torch.zeros_like(self.b)
        self.mw, self.vw = torch.zeros_like(self.w), torch.zeros_like(self.w)
        self.mb, self.vb = torch.zeros_like(self.b), torch.zeros_like(self.b)
        self.wb = torch.empty(cout, self.Kp, dtype=torch.bfloat16, device="cuda")
        self.wbT = torch.empty(self.Kp, cout, dtype=torch.bfloat16, device="cuda")
        self.status = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.pack()

    def params(self):
        return [(self.w, self.dw, self.mw, self.vw), (self.b, self.db, self.mb, self.vb)]

    def pack(self):
        _check(L().vefd_nn_pack_weights(_p(self.w), self.cout, self.K27, self.Kp, _p(self.wb), _p(self.wbT),
                                        _stream()), "pack_weights")

    def out_shape(self, shape):
        B, D, H, W, _ = shape
        s = self.stride
        return (B, (D - 1) // s + 1, (H - 1) // s + 1, (W - 1) // s + 1, self.cout)

    def forward(self, x):
        import torch
        B, D, H, W, C = x.shape
        assert C == self.cin and x.is_contiguous()
        oshape = self.out_shape(x.shape)
        V = oshape[0] * oshape[1] * oshape[2] * oshape[3]
        col = torch.empty(V, self.Kp, dtype=torch.bfloat16, device="cuda")
        colT = torch.empty(self.Kp, V, dtype=torch.bfloat16, device="cuda")
        _check(L().vefd_nn_im2col3d(_p(x), B, D, H, W, C, self.stride, self.Kp, _p(col), _p(colT), _stream()),
               "im2col")
        y = torch.empty(V, self.cout, dtype=torch.float32, device="cuda")
        gemm(col, self.wb, C=y, status=self.status)
        _check(L().vefd_nn_bias_act(_p(y), _p(self.b), V, self.cout, int(self.relu), _stream()), "bias_act")
        self._saved = (x.shape, colT, y)
        return y.view(oshape)

    def backward(self, dy, accumulate=False):
        """Gradients of w and b (added when accumulate) and of the input."""
        import torch
        xshape, colT, y = self._saved
        B, D, H, W, C = xshape
        V = y.shape[0]
        dy = dy.reshape(V, self.cout).contiguous()
        g = torch.empty_like(y)
        gb = torch.empty(V, self.cout, dtype=torch.bfloat16, device="cuda")
        gbT = torch.empty(self.cout, V, dtype=torch.bfloat16, device="cuda")
        lb, s = L(), _stream()
        _check(lb.vefd_nn_act_backward(_p(dy), _p(y), V, self.cout, int(self.relu), _p(g), _p(gb), _p(gbT), s),
               "act_backward")
        scratch = torch.empty(lb.vefd_nn_colsum_scratch(V, self.cout), device="cuda")
        _check(lb.vefd_nn_colsum(_p(g), V, self.cout, _p(scratch), _p(self.db), int(accumulate), s), "colsum")
        # dW^T [Kp, Cout] = col^T [Kp, V] . g [V, Cout], split over the voxels
        ksplit = max(64, ((V + 63) // 64 + 127) // 128 * 64)
        splits = (V + ksplit - 1) // ksplit
        parts = torch.empty(splits, self.Kp, self.cout, device="cuda")
        _check(lb.vefd_nn_gemm_bf16_splitk(_p(colT), V, _p(gbT), V, _p(parts), self.cout, self.Kp, self.cout, V,
                                           ksplit, self.Kp * self.cout, _p(self.status), s), "gemm_splitk")
        _check(lb.vefd_nn_splitk_reduce_t(_p(parts), splits, self.Kp * self.cout, self.Kp, self.cout, self.K27,
                                          _p(self.dw), int(accumulate), s), "splitk_reduce")
        # dcol [V, Kp] = g [V, Cout] . W [Cout, Kp]; col2im onto the input
        dcol = gemm(gb, self.wbT, status=self.status)
        dx = torch.empty(B, D, H, W, C, device="cuda")
        _check(lb.vefd_nn_col2im3d(_p(dcol), B, D, H, W, C, self.stride, self.Kp, _p(dx), s), "col2im")
        self._saved = None
        return dx


def upsample2(x):
    import torch
    B, D, H, W, C = x.shape
    y = torch.empty(B, 2 * D, 2 * H, 2 * W, C, device="cuda")
    _check(L().vefd_nn_upsample2(_p(x), B, D, H, W, C, _p(y), _stream()), "upsample2")
    return y


def upsample2_backward(dy, shape):
    import torch
    B, D, H, W, C = shape
    dx = torch.empty(shape, device="cuda")
    _check(L().vefd_nn_upsample2_backward(_p(dy.contiguous()), B, D, H, W, C, _p(dx), 0, _stream()), "upsample2_back")
    return dx


def concat(a, b):
    import torch
    V = a.numel() // a.shape[-1]
    y = torch.empty(*a.shape[:-1], a.shape[-1] + b.shape[-1], device="cuda")
    _check(L().vefd_nn_concat(_p(a), a.shape[-1], _p(b), b.shape[-1], V, _p(y), _stream()), "concat")
    return y


def split_back(dy, ca, cb, da=None, db=None, accumulate=True):
    V = dy.numel() // (ca + cb)
    _check(L().vefd_nn_split(_p(dy.contiguous()), ca, cb, V, _p(da), _p(db), int(accumulate), _stream()), "split")


def add(a, b):
    import torch
    y = torch.empty_like(a)
    _check(L().vefd_nn_add(_p(a), _p(b), a.numel(), _p(y), _stream()), "add")
    return y


def mse(pred, target):
    """(loss as a device scalar tensor, gradient) of the mean squared error."""
    import torch
    n = pred.numel()
    sq = torch.empty_like(pred)
    grad = torch.empty_like(pred)
    _check(L().vefd_nn_mse(_p(pred), _p(target), n, _p(sq), _p(grad), _stream()), "mse")
    # loss = column sum of the squared errors seen as [n / 8, 8], then / n (host side)
    V = n // 8
    out = torch.empty(8, device="cuda")
    scratch = torch.empty(L().vefd_nn_colsum_scratch(V, 8), device="cuda")
    _check(L().vefd_nn_colsum(_p(sq), V, 8, _p(scratch), _p(out), 0, _stream()), "colsum")
    return out, grad


class UNet:
    """3-D convolutional U-Net: four resolution levels (channels c, 2c, 4c, 8c,
    or the per-level plan `channels`, each a multiple of 8), two convolutions
    per level, stride-2 convolutions down, nearest-neighbour upsampling and
    skip concatenation up, a linear 3x3x3 output layer.  Input and output are
    channels-last FP32 [B, D, H, W, C] with D, H, W divisible by 8."""

    def __init__(self, cin, cout, c=16, seed=0, channels=None):
        import torch
        g = torch.Generator().manual_seed(seed)
        c0, c1, c2, c3 = channels if channels is not None else (c, 2 * c, 4 * c, 8 * c)
        self.cout = cout
        self.e0 = [Conv3d(cin, c0, gen=g), Conv3d(c0, c0, gen=g)]
        self.e1 = [Conv3d(c0, c1, 2, gen=g), Conv3d(c1, c1, gen=g)]
        self.e2 = [Conv3d(c1, c2, 2, gen=g), Conv3d(c2, c2, gen=g)]
        self.e3 = [Conv3d(c2, c3, 2, gen=g), Conv3d(c3, c3, gen=g)]
        self.d2 = [Conv3d(c3 + c2, c2, gen=g), Conv3d(c2, c2, gen=g)]
        self.d1 = [Conv3d(c2 + c1, c1, gen=g), Conv3d(c1, c1, gen=g)]
        self.d0 = [Conv3d(c1 + c0, c0, gen=g), Conv3d(c0, cout, relu=False, gen=g)]
        self.layers = self.e0 + self.e1 + self.e2 + self.e3 + self.d2 + self.d1 + self.d0
        self.chan = (c0, c1, c2, c3)
        self.step = 0

    def n_params(self):
        return sum(int(t.numel()) for lay in self.layers for t, _, _, _ in lay.params())

    @staticmethod
    def _run(layers, x):
        for lay in layers:
            x = lay.forward(x)
        return x

    @staticmethod
    def _back(layers, dy, accumulate=False):
        for lay in reversed(layers):
            dy = lay.backward(dy, accumulate)
        return dy

    def forward(self, x):
        s0 = self._run(self.e0, x)
        s1 = self._run(self.e1, s0)
        s2 = self._run(self.e2, s1)
        s3 = self._run(self.e3, s2)
        u2 = self._run(self.d2, concat(upsample2(s3), s2))
        u1 = self._run(self.d1, concat(upsample2(u2), s1))
        out = self._run(self.d0, concat(upsample2(u1), s0))
        self._shapes = (s0.shape, s1.shape, s2.shape, s3.shape, u2.shape, u1.shape)
        return out

    def backward(self, dout, accumulate=False):
        s0s, s1s, s2s, s3s, u2s, u1s = self._shapes
        c0, c1, c2, c3 = self.chan
        import torch
        ds0 = torch.zeros(s0s, device="cuda")
        ds1 = torch.zeros(s1s, device="cuda")
        ds2 = torch.zeros(s2s, device="cuda")
        dcat0 = self._back(self.d0, dout, accumulate)                    # [.., c1 + c0] at level 0
        dup1 = torch.empty(*s0s[:-1], c1, device="cuda")
        split_back(dcat0, c1, c0, dup1, ds0, accumulate=False)
        du1 = upsample2_backward(dup1, u1s)
        dcat1 = self._back(self.d1, du1, accumulate)
        dup2 = torch.empty(*s1s[:-1], c2, device="cuda")
        split_back(dcat1, c2, c1, dup2, ds1, accumulate=False)
        du2 = upsample2_backward(dup2, u2s)
        dcat2 = self._back(self.d2, du2, accumulate)
        dup3 = torch.empty(*s2s[:-1], c3, device="cuda")
        split_back(dcat2, c3, c2, dup3, ds2, accumulate=False)
        ds3 = upsample2_backward(dup3, s3s)
        d = self._back(self.e3, ds3, accumulate)
        d = add(d, ds2)
        d = self._back(self.e2, d, accumulate)
        d = add(d, ds1)
        d = self._back(self.e1, d, accumulate)
        d = add(d, ds0)
        return self._back(self.e0, d, accumulate)

    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.step += 1
        for lay in self.layers:
            for w, g, m, v in lay.params():
                _check(L().vefd_nn_adam(_p(w), _p(g), _p(m), _p(v), w.numel(), lr, beta1, beta2, eps, self.step,
                                        _stream()), "adam")
            lay.pack()

    def status(self):
        return max(int(lay.status.item()) for lay in self.layers)


def to_fields(out, phi0, u_wall, c_scale, rho_tot, L2):
    """Device fields (rho_A, rho_B, u [3, ...], C [6, ...]) for a lattice from a network output [D, H, W, 16]."""
    import torch
    V = phi0.numel()
    rA, rB = torch.empty_like(phi0), torch.empty_like(phi0)
    u = torch.empty(3, *phi0.shape, device="cuda")
    C = torch.empty(6, *phi0.shape, device="cuda")
    _check(L().vefd_nn_to_fields(_p(out.contiguous()), _p(phi0.contiguous()), V, float(u_wall), float(c_scale),
                                 float(rho_tot), float(L2), _p(rA), _p(rB), _p(u), _p(C), _stream()), "to_fields")
    return rA, rB, u, C


def total(x):
    """Sum of all elements of a device FP32 tensor (fixed-order reduction), as a host float."""
    import torch
    n = x.numel()
    assert n % 8 == 0
    out = torch.empty(8, device="cuda")
    scratch = torch.empty(L().vefd_nn_colsum_scratch(n // 8, 8), device="cuda")
    _check(L().vefd_nn_colsum(_p(x.contiguous()), n // 8, 8, _p(scratch), _p(out), 0, _stream()), "colsum")
    return float(sum(out.cpu().tolist()))


def scale(x, factor):
    _check(L().vefd_nn_scale(_p(x), x.numel(), float(factor), _stream()), "scale")
