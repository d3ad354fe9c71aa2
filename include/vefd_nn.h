/*
 * libvefd — tensor-core kernels of the learned warm start (the paper has no
 * counterpart: a convolutional network, trained on fields the method itself
 * produces, predicts near-steady phi, u and C from the set-up parameters so
 * that a run can start close to its steady state; the lattice-Boltzmann /
 * finite-difference step of Sec. 2 then continues and decides the result).
 *
 * Device pointers throughout; work is enqueued on `stream` (NULL = legacy
 * default stream) and the calls do not synchronise.  Errors: VEFD_NN_ERR_ARG
 * for bad sizes, strides, alignment or NULL pointers (nothing is launched),
 * VEFD_NN_ERR_CUDA when a launch fails.  Device-side waits are bounded; a wait
 * that gives up sets bit 1 of *status (device word, caller-owned) and the
 * kernel returns without writing its output.
 */
#ifndef VEFD_NN_H
#define VEFD_NN_H

#ifdef __cplusplus
extern "C" {
#endif

enum { VEFD_NN_OK = 0, VEFD_NN_ERR_ARG = -1, VEFD_NN_ERR_CUDA = -2 };

/* C[M x N] (FP32, row-major, leading dimension ldc) = A[M x K] * B[N x K]^T,
 * or C += A B^T when accumulate != 0.  A and B are BF16, row-major with K
 * contiguous (leading dimensions lda, ldb, multiples of 8 elements; A and B
 * 16-byte aligned); K a multiple of 8, K >= 8.  FP32 accumulation on the
 * tensor cores (tcgen05, accumulator in tensor memory). */
int vefd_nn_gemm_bf16(const void *A, int lda, const void *B, int ldb, float *C, int ldc, int M, int N, int K,
                      int accumulate, unsigned *status, void *stream);
/* The same with an explicit shared-memory operand layout: lbo = byte offset
 * between 8 x 16-byte core matrices along K, sbo = between 8-row groups;
 * desc_swap != 0 encodes them in each other's descriptor field.  For tests of
 * the layout; offsets that would leave a staged tile are rejected. */
int vefd_nn_gemm_bf16_layout(const void *A, int lda, const void *B, int ldb, float *C, int ldc, int M, int N, int K,
                             int accumulate, unsigned lbo, unsigned sbo, int desc_swap, unsigned *status,
                             void *stream);

#ifdef __cplusplus
}
#endif
#endif
