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

/* Split-K form for long reductions: K is cut into slices of k_split (a
 * multiple of 64) and slice z writes C + z * c_split_stride (no accumulate);
 * the slices are summed by vefd_nn_splitk_reduce_t. */
int vefd_nn_gemm_bf16_splitk(const void *A, int lda, const void *B, int ldb, float *C, int ldc, int M, int N, int K,
                             int k_split, long long c_split_stride, unsigned *status, void *stream);

/* ---- convolution layers (3x3x3, zero padding 1, stride 1 or 2) -----------
 * Activations are FP32 channels-last x[v][c], v = ((b D + z) H + y) W + x.
 * Output size per axis n' = (n - 1)/stride + 1, V' voxels.  Column index
 * k = ((dz 3 + dy) 3 + dx) C + c; Kp >= 27 C, a multiple of 8, zero beyond 27 C. */
/* col [V'][Kp] and/or colT [Kp][V'] (BF16; either may be NULL, not both). */
int vefd_nn_im2col3d(const float *x, int B, int D, int H, int W, int C, int stride, int Kp, void *col, void *colT,
                     void *stream);
/* dx[v][c] = sum of dcol over every (output voxel, tap) that read x[v][c] (overwrites dx). */
int vefd_nn_col2im3d(const float *dcol, int B, int D, int H, int W, int C, int stride, int Kp, float *dx, void *stream);
/* y[v][c] += bias[c] (bias may be NULL), then max(y, 0) when relu. */
int vefd_nn_bias_act(float *y, const float *bias, long long V, int C, int relu, void *stream);
/* g = dy, zero where relu and the output y <= 0; gb = BF16 g [V][C], gbT = BF16 g^T [C][V]. */
int vefd_nn_act_backward(const float *dy, const float *y, long long V, int C, int relu, float *g, void *gb, void *gbT,
                         void *stream);
/* out[c] (+)= sum_v a[v][c] in a fixed order; scratch holds vefd_nn_colsum_scratch(V, C) floats; C <= 1024. */
long long vefd_nn_colsum_scratch(long long V, int C);
int vefd_nn_colsum(const float *a, long long V, int C, float *scratch, float *out, int accumulate, void *stream);
/* FP32 weights w[Cout][K27] -> BF16 wb[Cout][Kp] (zero padded) and wbT[Kp][Cout]. */
int vefd_nn_pack_weights(const float *w, int Cout, int K27, int Kp, void *wb, void *wbT, void *stream);
/* dw[o][k] (+)= sum_s parts[s][k][o] for k < K27 (parts: split-K slices of dW^T, stride split_stride). */
int vefd_nn_splitk_reduce_t(const float *parts, int splits, long long split_stride, int Kp, int Cout, int K27,
                            float *dw, int accumulate, void *stream);
/* Nearest-neighbour upsampling by 2 of x [B][D][H][W][C] and its adjoint (sum of the 8 children). */
int vefd_nn_upsample2(const float *x, int B, int D, int H, int W, int C, float *y, void *stream);
int vefd_nn_upsample2_backward(const float *dy, int B, int D, int H, int W, int C, float *dx, int accumulate,
                               void *stream);
/* Channel concatenation y[v] = [a[v], b[v]] and its adjoint (da or db may be NULL). */
int vefd_nn_concat(const float *a, int Ca, const float *b, int Cb, long long V, float *y, void *stream);
int vefd_nn_split(const float *dy, int Ca, int Cb, long long V, float *da, float *db, int accumulate, void *stream);
/* sq = (p - t)^2 and grad = 2 (p - t) / n elementwise (mean-squared-error loss). */
int vefd_nn_mse(const float *p, const float *t, long long n, float *sq, float *grad, void *stream);
/* y = a + b elementwise. */
int vefd_nn_add(const float *a, const float *b, long long n, float *y, void *stream);
/* Warm-start fields of a lattice from a network output out[v][16] (phi - phi0,
 * u / u_wall, (C - I) / c_scale, 6 unused): rho_A, rho_B = rho_tot (1 +- phi)/2
 * with phi clipped to [-0.95, 0.95]; u planes [3][V]; C planes [6][V] (xx xy
 * xz yy yz zz) = I + t c_scale c^ with the largest t in {1, 1/2, ..., 2^-10, 0}
 * giving a symmetric positive definite C with tr C < L2 - 1. */
int vefd_nn_to_fields(const float *out, const float *phi0, long long V, float u_wall, float c_scale, float rho_tot,
                      float L2, float *rhoA, float *rhoB, float *u, float *C, void *stream);
/* x *= factor elementwise. */
int vefd_nn_scale(float *x, long long n, float factor, void *stream);
/* One Adam step (bias-corrected, step >= 1) on w with gradient g and moments m, v. */
int vefd_nn_adam(float *w, const float *g, float *m, float *v, long long n, float lr, float beta1, float beta2,
                 float eps, int step, void *stream);

#ifdef __cplusplus
}
#endif
#endif
