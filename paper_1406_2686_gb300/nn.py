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
