// Memory-bound kernels of the warm-start network around the tensor-core GEMM
// (nn_gemm.cu).  Activations are FP32, channels-last: x[v][c] with voxel
// v = ((b * D + z) * H + y) * W + x.  A 3x3x3 convolution with zero padding 1
// and stride s is col = im2col(x) (BF16, [V'][Kp], tap-major columns
// k = ((dz * 3 + dy) * 3 + dx) * C + c, zero for k >= 27 C), y = col W^T on the
// tensor cores, then bias and ReLU.  Its gradients are dcol = dy W (col2im
// gathers them back onto x) and dW^T = col^T dy (split over voxels, reduced
// here).  Every reduction runs in a fixed order, so results are
// reproducible.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "vefd_nn.h"

namespace {

constexpr int kT = 256;

int grid_for(long long n) {
    long long b = (n + kT - 1) / kT;
    if (b > 152 * 64) b = 152 * 64;
    return (int)(b < 1 ? 1 : b);
}

struct Geo {
    int B, D, H, W, C, s, Do, Ho, Wo;
};

__device__ __forceinline__ float tap_value(const float* __restrict__ x, const Geo& g, long long v, int k) {
    if (k >= 27 * g.C) return 0.0f;
    const int tap = k / g.C, c = k - tap * g.C;
    const int dz = tap / 9, dy = (tap / 3) % 3, dx = tap % 3;
    const int xo = (int)(v % g.Wo);
    long long r = v / g.Wo;
    const int yo = (int)(r % g.Ho);
    r /= g.Ho;
    const int zo = (int)(r % g.Do);
    const int b = (int)(r / g.Do);
    const int zi = zo * g.s + dz - 1, yi = yo * g.s + dy - 1, xi = xo * g.s + dx - 1;
    if (zi < 0 || zi >= g.D || yi < 0 || yi >= g.H || xi < 0 || xi >= g.W) return 0.0f;
    return x[((((long long)b * g.D + zi) * g.H + yi) * g.W + xi) * g.C + c];
}

__global__ void k_im2col(const float* __restrict__ x, Geo g, int Kp, __nv_bfloat16* __restrict__ col) {
    const long long V = (long long)g.B * g.Do * g.Ho * g.Wo, n = V * Kp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        col[e] = __float2bfloat16_rn(tap_value(x, g, e / Kp, (int)(e % Kp)));
}

__global__ void k_im2col_t(const float* __restrict__ x, Geo g, int Kp, __nv_bfloat16* __restrict__ colT) {
    const long long V = (long long)g.B * g.Do * g.Ho * g.Wo, n = V * Kp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        colT[e] = __float2bfloat16_rn(tap_value(x, g, e % V, (int)(e / V)));
}

// dx[v][c] = sum over the taps that read x[v][c] of dcol[v'][tap * C + c]
__global__ void k_col2im(const float* __restrict__ dcol, Geo g, int Kp, float* __restrict__ dx) {
    const long long n = (long long)g.B * g.D * g.H * g.W * g.C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % g.C);
        long long r = e / g.C;
        const int xi = (int)(r % g.W);
        r /= g.W;
        const int yi = (int)(r % g.H);
        r /= g.H;
        const int zi = (int)(r % g.D);
        const int b = (int)(r / g.D);
        float acc = 0.0f;
        for (int dz = 0; dz < 3; ++dz) {
            const int tz = zi - dz + 1;
            if (tz < 0 || tz % g.s) continue;
            const int zo = tz / g.s;
            if (zo >= g.Do) continue;
            for (int dy = 0; dy < 3; ++dy) {
                const int ty = yi - dy + 1;
                if (ty < 0 || ty % g.s) continue;
                const int yo = ty / g.s;
                if (yo >= g.Ho) continue;
                for (int dx = 0; dx < 3; ++dx) {
                    const int tx = xi - dx + 1;
                    if (tx < 0 || tx % g.s) continue;
                    const int xo = tx / g.s;
                    if (xo >= g.Wo) continue;
                    const long long vo = (((long long)b * g.Do + zo) * g.Ho + yo) * g.Wo + xo;
                    acc += dcol[vo * Kp + ((dz * 3 + dy) * 3 + dx) * g.C + c];
                }
            }
        }
        dx[e] = acc;
    }
}

__global__ void k_bias_act(float* __restrict__ y, const float* __restrict__ bias, long long V, int C, int relu) {
    const long long n = V * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        float t = y[e] + (bias ? bias[e % C] : 0.0f);
        if (relu) t = fmaxf(t, 0.0f);
        y[e] = t;
    }
}

// g = dy masked by the ReLU of the output y; BF16 copies in both layouts
__global__ void k_act_back(const float* __restrict__ dy, const float* __restrict__ y, long long V, int C, int relu,
                           float* __restrict__ g, __nv_bfloat16* __restrict__ gb, __nv_bfloat16* __restrict__ gbT) {
    const long long n = V * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float t = (relu && !(y[e] > 0.0f)) ? 0.0f : dy[e];
        g[e] = t;
        gb[e] = __float2bfloat16_rn(t);
        const long long v = e / C;
        const int c = (int)(e - v * C);
        gbT[(long long)c * V + v] = __float2bfloat16_rn(t);
    }
}

// column sums of a [V][C] matrix: partial sums over fixed row ranges, then in order
constexpr int kRowsPerPart = 4096;
__global__ void k_colsum_part(const float* __restrict__ a, long long V, int C, float* __restrict__ part) {
    const int c = threadIdx.x;
    if (c >= C) return;
    const long long r0 = (long long)blockIdx.x * kRowsPerPart;
    const long long r1 = min(V, r0 + kRowsPerPart);
    float acc = 0.0f;
    for (long long r = r0; r < r1; ++r) acc += a[r * C + c];
    part[(long long)blockIdx.x * C + c] = acc;
}

__global__ void k_colsum_final(const float* __restrict__ part, int nparts, int C, float* __restrict__ out,
                               int accumulate) {
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= C) return;
    float acc = 0.0f;
    for (int p = 0; p < nparts; ++p) acc += part[(long long)p * C + c];
    out[c] = accumulate ? out[c] + acc : acc;
}

// FP32 master weights [Cout][27 Cin] -> BF16 [Cout][Kp] (zero padded) and its transpose [Kp][Cout]
__global__ void k_pack_weights(const float* __restrict__ w, int Cout, int K27, int Kp, __nv_bfloat16* __restrict__ wb,
                               __nv_bfloat16* __restrict__ wbT) {
    const long long n = (long long)Cout * Kp;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(e / Kp), k = (int)(e % Kp);
        const __nv_bfloat16 v = __float2bfloat16_rn(k < K27 ? w[(long long)o * K27 + k] : 0.0f);
        wb[e] = v;
        wbT[(long long)k * Cout + o] = v;
    }
}

// dW[o][k] = (accumulate ? dW : 0) + sum over splits of dWT_s[k][o], k < K27
__global__ void k_splitk_reduce_t(const float* __restrict__ parts, int splits, long long split_stride, int Kp, int Cout,
                                  int K27, float* __restrict__ dw, int accumulate) {
    const long long n = (long long)Cout * K27;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int o = (int)(e / K27), k = (int)(e % K27);
        float acc = 0.0f;
        for (int s = 0; s < splits; ++s) acc += parts[s * split_stride + (long long)k * Cout + o];
        dw[e] = accumulate ? dw[e] + acc : acc;
    }
}

__global__ void k_upsample2(const float* __restrict__ x, int B, int D, int H, int W, int C, float* __restrict__ y) {
    const long long n = (long long)B * 8 * D * H * W * C;
    const int D2 = 2 * D, H2 = 2 * H, W2 = 2 * W;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        long long r = e / C;
        const int xx = (int)(r % W2);
        r /= W2;
        const int yy = (int)(r % H2);
        r /= H2;
        const int zz = (int)(r % D2);
        const int b = (int)(r / D2);
        y[e] = x[((((long long)b * D + zz / 2) * H + yy / 2) * W + xx / 2) * C + c];
    }
}

__global__ void k_upsample2_back(const float* __restrict__ dy, int B, int D, int H, int W, int C, float* __restrict__ dx,
                                 int accumulate) {
    const long long n = (long long)B * D * H * W * C;
    const int H2 = 2 * H, W2 = 2 * W;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const int c = (int)(e % C);
        long long r = e / C;
        const int xx = (int)(r % W);
        r /= W;
        const int yy = (int)(r % H);
        r /= H;
        const int zz = (int)(r % D);
        const int b = (int)(r / D);
        float acc = 0.0f;
        for (int q = 0; q < 8; ++q) {
            const int z2 = 2 * zz + (q >> 2), y2 = 2 * yy + ((q >> 1) & 1), x2 = 2 * xx + (q & 1);
            acc += dy[((((long long)b * 2 * D + z2) * H2 + y2) * W2 + x2) * C + c];
        }
        dx[e] = accumulate ? dx[e] + acc : acc;
    }
}

// y[v] = [a[v] (Ca channels), b[v] (Cb channels)]; back: split, optionally accumulating
__global__ void k_concat(const float* __restrict__ a, int Ca, const float* __restrict__ b, int Cb, long long V,
                         float* __restrict__ y) {
    const int C = Ca + Cb;
    const long long n = V * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long v = e / C;
        const int c = (int)(e - v * C);
        y[e] = c < Ca ? a[v * Ca + c] : b[v * Cb + c - Ca];
    }
}

__global__ void k_split(const float* __restrict__ dy, int Ca, int Cb, long long V, float* __restrict__ da,
                        float* __restrict__ db, int accumulate) {
    const int C = Ca + Cb;
    const long long n = V * C;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const long long v = e / C;
        const int c = (int)(e - v * C);
        if (c < Ca ? !da : !db) continue;
        float* dst = c < Ca ? da + v * Ca + c : db + v * Cb + c - Ca;
        *dst = accumulate ? *dst + dy[e] : dy[e];
    }
}

// squared error per element and its gradient 2 (p - t) / n
__global__ void k_mse(const float* __restrict__ p, const float* __restrict__ t, long long n, float* __restrict__ sq,
                      float* __restrict__ grad) {
    const float scale = 2.0f / (float)n;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float d = p[e] - t[e];
        sq[e] = d * d;
        grad[e] = scale * d;
    }
}

__global__ void k_adam(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m, float* __restrict__ v,
                       long long n, float lr, float b1, float b2, float eps, float c1, float c2) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const float ge = g[e];
        const float me = b1 * m[e] + (1.0f - b1) * ge;
        const float ve = b2 * v[e] + (1.0f - b2) * ge * ge;
        m[e] = me;
        v[e] = ve;
        w[e] -= lr * (me / c1) / (sqrtf(ve / c2) + eps);
    }
}

__global__ void k_scale(float* __restrict__ x, long long n, float f) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        x[e] *= f;
}

__global__ void k_add(const float* __restrict__ a, const float* __restrict__ b, long long n, float* __restrict__ y) {
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x)
        y[e] = a[e] + b[e];
}

// Warm-start fields from a network output out[v][16] (channels: phi - phi0,
// u / U, (C - I) / c_scale): rho_A, rho_B = rho_tot (1 +- phi) / 2 with phi
// clipped to [-0.95, 0.95]; u; C = I + t c_scale c^ with the largest t in
// {1, 1/2, ..., 2^-10, 0} for which C is symmetric positive definite
// (leading minors) with tr C < L2 - 3 + 3 (t = 0 gives I).  Layouts as the
// lattice's init_fields: planes of N for u (3) and C (xx xy xz yy yz zz).
__global__ void k_to_fields(const float* __restrict__ out, const float* __restrict__ phi0, long long V, float u_wall,
                            float c_scale, float rho_tot, float L2, float* __restrict__ rhoA, float* __restrict__ rhoB,
                            float* __restrict__ u, float* __restrict__ C) {
    for (long long v = blockIdx.x * (long long)blockDim.x + threadIdx.x; v < V; v += (long long)gridDim.x * blockDim.x) {
        const float* o = out + v * 16;
        const float phi = fminf(fmaxf(phi0[v] + o[0], -0.95f), 0.95f);
        rhoA[v] = 0.5f * rho_tot * (1.0f + phi);
        rhoB[v] = 0.5f * rho_tot * (1.0f - phi);
        for (int k = 0; k < 3; ++k) u[k * V + v] = o[1 + k] * u_wall;
        float c[6];
        for (int k = 0; k < 6; ++k) c[k] = o[4 + k] * c_scale;
        float t = 1.0f;
        for (int it = 0; it <= 11; ++it) {
            if (it == 11) t = 0.0f;
            const float xx = 1.0f + t * c[0], xy = t * c[1], xz = t * c[2], yy = 1.0f + t * c[3], yz = t * c[4],
                        zz = 1.0f + t * c[5];
            const float m2 = xx * yy - xy * xy;
            const float m3 = xx * (yy * zz - yz * yz) - xy * (xy * zz - yz * xz) + xz * (xy * yz - yy * xz);
            if ((xx > 1e-3f && m2 > 1e-6f && m3 > 1e-9f && xx + yy + zz < L2 - 1.0f) || it == 11) break;
            t *= 0.5f;
        }
        const float e[6] = {1.0f, 0.0f, 0.0f, 1.0f, 0.0f, 1.0f};
        for (int k = 0; k < 6; ++k) C[k * V + v] = e[k] + t * c[k];
    }
}

bool bad_geo(int B, int D, int H, int W, int C, int s) {
    return B < 1 || D < 1 || H < 1 || W < 1 || C < 1 || (s != 1 && s != 2);
}

Geo geo_of(int B, int D, int H, int W, int C, int s) {
    Geo g{B, D, H, W, C, s, (D - 1) / s + 1, (H - 1) / s + 1, (W - 1) / s + 1};
    return g;
}

int done() { return cudaGetLastError() == cudaSuccess ? VEFD_NN_OK : VEFD_NN_ERR_CUDA; }

}  // namespace

extern "C" {

int vefd_nn_im2col3d(const float* x, int B, int D, int H, int W, int C, int stride, int Kp, void* col, void* colT,
                     void* stream) {
    if (!x || bad_geo(B, D, H, W, C, stride) || Kp < 27 * C || Kp % 8 != 0 || (!col && !colT)) return VEFD_NN_ERR_ARG;
    const Geo g = geo_of(B, D, H, W, C, stride);
    const long long n = (long long)B * g.Do * g.Ho * g.Wo * Kp;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (col) k_im2col<<<grid_for(n), kT, 0, s>>>(x, g, Kp, (__nv_bfloat16*)col);
    if (colT) k_im2col_t<<<grid_for(n), kT, 0, s>>>(x, g, Kp, (__nv_bfloat16*)colT);
    return done();
}

int vefd_nn_col2im3d(const float* dcol, int B, int D, int H, int W, int C, int stride, int Kp, float* dx, void* stream) {
    if (!dcol || !dx || bad_geo(B, D, H, W, C, stride) || Kp < 27 * C) return VEFD_NN_ERR_ARG;
    const Geo g = geo_of(B, D, H, W, C, stride);
    const long long n = (long long)B * D * H * W * C;
    k_col2im<<<grid_for(n), kT, 0, static_cast<cudaStream_t>(stream)>>>(dcol, g, Kp, dx);
    return done();
}

int vefd_nn_bias_act(float* y, const float* bias, long long V, int C, int relu, void* stream) {
    if (!y || V < 1 || C < 1) return VEFD_NN_ERR_ARG;
    k_bias_act<<<grid_for(V * C), kT, 0, static_cast<cudaStream_t>(stream)>>>(y, bias, V, C, relu);
    return done();
}

int vefd_nn_act_backward(const float* dy, const float* y, long long V, int C, int relu, float* g, void* gb, void* gbT,
                         void* stream) {
    if (!dy || !y || !g || !gb || !gbT || V < 1 || C < 1) return VEFD_NN_ERR_ARG;
    k_act_back<<<grid_for(V * C), kT, 0, static_cast<cudaStream_t>(stream)>>>(dy, y, V, C, relu, g,
                                                                             (__nv_bfloat16*)gb, (__nv_bfloat16*)gbT);
    return done();
}

long long vefd_nn_colsum_scratch(long long V, int C) { return ((V + kRowsPerPart - 1) / kRowsPerPart) * (long long)C; }

int vefd_nn_colsum(const float* a, long long V, int C, float* scratch, float* out, int accumulate, void* stream) {
    if (!a || !scratch || !out || V < 1 || C < 1 || C > 1024) return VEFD_NN_ERR_ARG;
    const int nparts = (int)((V + kRowsPerPart - 1) / kRowsPerPart);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    k_colsum_part<<<nparts, ((C + 31) / 32) * 32, 0, s>>>(a, V, C, scratch);
    k_colsum_final<<<(C + 255) / 256, 256, 0, s>>>(scratch, nparts, C, out, accumulate);
    return done();
}

int vefd_nn_pack_weights(const float* w, int Cout, int K27, int Kp, void* wb, void* wbT, void* stream) {
    if (!w || !wb || !wbT || Cout < 1 || K27 < 1 || Kp < K27 || Kp % 8) return VEFD_NN_ERR_ARG;
    k_pack_weights<<<grid_for((long long)Cout * Kp), kT, 0, static_cast<cudaStream_t>(stream)>>>(
        w, Cout, K27, Kp, (__nv_bfloat16*)wb, (__nv_bfloat16*)wbT);
    return done();
}

int vefd_nn_splitk_reduce_t(const float* parts, int splits, long long split_stride, int Kp, int Cout, int K27,
                            float* dw, int accumulate, void* stream) {
    if (!parts || !dw || splits < 1 || Kp < K27 || Cout < 1 || split_stride < (long long)Kp * Cout) return VEFD_NN_ERR_ARG;
    k_splitk_reduce_t<<<grid_for((long long)Cout * K27), kT, 0, static_cast<cudaStream_t>(stream)>>>(
        parts, splits, split_stride, Kp, Cout, K27, dw, accumulate);
    return done();
}

int vefd_nn_upsample2(const float* x, int B, int D, int H, int W, int C, float* y, void* stream) {
    if (!x || !y || bad_geo(B, D, H, W, C, 1)) return VEFD_NN_ERR_ARG;
    k_upsample2<<<grid_for((long long)B * 8 * D * H * W * C), kT, 0, static_cast<cudaStream_t>(stream)>>>(x, B, D, H, W,
                                                                                                         C, y);
    return done();
}

int vefd_nn_upsample2_backward(const float* dy, int B, int D, int H, int W, int C, float* dx, int accumulate,
                               void* stream) {
    if (!dy || !dx || bad_geo(B, D, H, W, C, 1)) return VEFD_NN_ERR_ARG;
    k_upsample2_back<<<grid_for((long long)B * D * H * W * C), kT, 0, static_cast<cudaStream_t>(stream)>>>(
        dy, B, D, H, W, C, dx, accumulate);
    return done();
}

int vefd_nn_concat(const float* a, int Ca, const float* b, int Cb, long long V, float* y, void* stream) {
    if (!a || !b || !y || Ca < 1 || Cb < 1 || V < 1) return VEFD_NN_ERR_ARG;
    k_concat<<<grid_for(V * (Ca + Cb)), kT, 0, static_cast<cudaStream_t>(stream)>>>(a, Ca, b, Cb, V, y);
    return done();
}

int vefd_nn_split(const float* dy, int Ca, int Cb, long long V, float* da, float* db, int accumulate, void* stream) {
    if (!dy || Ca < 1 || Cb < 1 || V < 1 || (!da && !db)) return VEFD_NN_ERR_ARG;
    k_split<<<grid_for(V * (Ca + Cb)), kT, 0, static_cast<cudaStream_t>(stream)>>>(dy, Ca, Cb, V, da, db, accumulate);
    return done();
}

int vefd_nn_mse(const float* p, const float* t, long long n, float* sq, float* grad, void* stream) {
    if (!p || !t || !sq || !grad || n < 1) return VEFD_NN_ERR_ARG;
    k_mse<<<grid_for(n), kT, 0, static_cast<cudaStream_t>(stream)>>>(p, t, n, sq, grad);
    return done();
}

int vefd_nn_add(const float* a, const float* b, long long n, float* y, void* stream) {
    if (!a || !b || !y || n < 1) return VEFD_NN_ERR_ARG;
    k_add<<<grid_for(n), kT, 0, static_cast<cudaStream_t>(stream)>>>(a, b, n, y);
    return done();
}

int vefd_nn_to_fields(const float* out, const float* phi0, long long V, float u_wall, float c_scale, float rho_tot,
                      float L2, float* rhoA, float* rhoB, float* u, float* C, void* stream) {
    if (!out || !phi0 || !rhoA || !rhoB || !u || !C || V < 1 || !(L2 > 3.0f)) return VEFD_NN_ERR_ARG;
    k_to_fields<<<grid_for(V), kT, 0, static_cast<cudaStream_t>(stream)>>>(out, phi0, V, u_wall, c_scale, rho_tot, L2,
                                                                         rhoA, rhoB, u, C);
    return done();
}

int vefd_nn_scale(float* x, long long n, float factor, void* stream) {
    if (!x || n < 1) return VEFD_NN_ERR_ARG;
    k_scale<<<grid_for(n), kT, 0, static_cast<cudaStream_t>(stream)>>>(x, n, factor);
    return done();
}

int vefd_nn_adam(float* w, const float* g, float* m, float* v, long long n, float lr, float beta1, float beta2,
                 float eps, int step, void* stream) {
    if (!w || !g || !m || !v || n < 1 || step < 1 || !(lr > 0.0f)) return VEFD_NN_ERR_ARG;
    const float c1 = 1.0f - powf(beta1, (float)step), c2 = 1.0f - powf(beta2, (float)step);
    k_adam<<<grid_for(n), kT, 0, static_cast<cudaStream_t>(stream)>>>(w, g, m, v, n, lr, beta1, beta2, eps, c1, c2);
    return done();
}

}  // extern "C"
