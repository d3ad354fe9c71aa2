// Derived fields and FP64 diagnostics of the current state.
//
// Diagnostics (Sec. 4.1 measures of Gupta, Sbragaglia & Scagliarini and the
// conservation checks): each block reduces its grid-stride share of nodes in
// FP64 with warp shuffles, writes one row of partials, and a single block
// sums the rows in a fixed order, so the result does not depend on block
// scheduling.  Sums: density deviations per component, momentum rho u,
// sigma_P,xy, sigma_P,xx - sigma_P,yy, tr sigma_P - 3, droplet volume, and the
// zeroth to second moments of the indicator phi > 0 in the plane z = NZ/2
// (semi-axes and orientation follow on the host); maxima: tr C / L^2 and |u|.
#include <cmath>

#include "vefd_internal.cuh"

namespace vefd {

namespace {

int grid_1d(long long n) {
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

template <int NC>
__global__ void k_derived(int which, int ncomp, const float* __restrict__ drho, const float* __restrict__ Ct,
                          float* __restrict__ dst, StepParams p) {
    const long long N = p.N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        if (which == 0) {
            dst[i] = p.rho_ref[0] + drho[i * ncomp];
        } else if (which == 1) {
            dst[i] = ncomp == 2 ? p.rho_ref[1] + drho[2 * i + 1] : 0.0f;
        } else if (which == 2) {
            if (ncomp == 2) {
                const float a = p.rho_ref[0] + drho[2 * i], b = p.rho_ref[1] + drho[2 * i + 1];
                dst[i] = (a - b) / (a + b);
            } else {
                dst[i] = 1.0f;
            }
        } else if (which == 4 || which == 5) {
            float c[NC];
#pragma unroll
            for (int k = 0; k < NC; ++k) c[k] = Ct[k * N + i];
            const float tr = NC == 6 ? c[0] + c[3] + c[5] : c[0] + c[2] + c[3];
            const float fm1 = which == 5 ? tr / (p.L2m3 - tr) : 0.0f;
            const float f = 1.0f + fm1;
#pragma unroll
            for (int k = 0; k < NC; ++k) {
                const bool diag = NC == 6 ? (k == 0 || k == 3 || k == 5) : (k == 0 || k == 2 || k == 3);
                // f C = f Ct + f I
                dst[k * N + i] = f * c[k] + (diag ? f : 0.0f);
            }
        }
    }
}

template <int NC>
__global__ void k_tensor_shift(const float* __restrict__ src, float* __restrict__ dst, long long N, float sign) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const bool diag = NC == 6 ? (k == 0 || k == 3 || k == 5) : (k == 0 || k == 2 || k == 3);
            dst[k * N + i] = src[k * N + i] + (diag ? sign : 0.0f);
        }
    }
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Exactly (n / d > 0) without the division, for the doubles the indicator
// compares (differences of FP32 values, so the quotient never underflows):
// a finite nonzero d keeps or flips the sign of n; d = +-0 gives +-inf of the
// sign n and d share (NaN for n = 0 or NaN); an infinite or NaN d gives a
// zero or NaN quotient.
__device__ __forceinline__ bool ratio_positive(double n, double d) {
    if (d != 0.0 && isfinite(d)) return d > 0.0 ? n > 0.0 : n < 0.0;
    if (d == 0.0) return n != 0.0 && !isnan(n) && signbit(n) == signbit(d);
    return false;
}

__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

template <int D, int NC>
__global__ void __launch_bounds__(256) k_diag_partial(const float* __restrict__ drho, const float* __restrict__ u,
                                                      const float* __restrict__ Ct, int ncomp,
                                                      double* __restrict__ partial, StepParams p) {
    const long long N = p.N;
    const int zc = p.nz / 2;
    double acc[kDiagVals];
#pragma unroll
    for (int k = 0; k < kDiagVals; ++k) acc[k] = 0.0;
    // the maxima are kept of tr(C - I) and |u|^2; the host maps them to
    // max tr C / L^2 and max |u| (both maps are monotone, so the result is the
    // same as mapping every node)
    acc[15] = -INFINITY;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        // a lattice has fewer than 2^31 nodes (checked at creation)
        const int ii = (int)i;
        const int x = ii % p.nx;
        const int r = ii / p.nx;
        const int y = r % p.ny;
        const int z = r / p.ny;
        const double dA = drho[i * ncomp];
        const double dB = ncomp == 2 ? (double)drho[2 * i + 1] : 0.0;
        const double rA = (double)p.rho_ref[0] + dA;
        const double rB = ncomp == 2 ? (double)p.rho_ref[1] + dB : 0.0;
        const double rho = rA + rB;
        acc[0] += dA;
        acc[1] += dB;
        double u2 = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const double uk = u[k * N + i];
            acc[2 + k] += rho * uk;
            u2 += uk * uk;
        }
        double c[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) c[k] = Ct[k * N + i];
        const double trt = NC == 6 ? c[0] + c[3] + c[5] : c[0] + c[2] + c[3];
        const double fm1 = trt / ((double)p.L2m3 - trt);
        const double f = 1.0 + fm1;
        const double cxx = c[0], cxy = c[1], cyy = NC == 6 ? c[3] : c[2];
        acc[5] += f * cxy;
        acc[6] += f * (cxx - cyy);
        acc[7] += f * trt + 3.0 * fm1;
        const bool ind = ncomp == 2 ? ratio_positive(rA - rB, rho) : true;
        if (ind) {
            acc[8] += 1.0;
            if (z == zc) {
                acc[9] += 1.0;
                acc[10] += x;
                acc[11] += y;
                acc[12] += (double)x * x;
                acc[13] += (double)x * y;
                acc[14] += (double)y * y;
            }
        }
        acc[15] = fmax(acc[15], trt);
        acc[16] = fmax(acc[16], u2);
    }
    __shared__ double sh[kDiagVals][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kDiagVals; ++k) {
        const double v = k < kDiagSums ? warp_sum(acc[k]) : warp_max(acc[k]);
        if (lane == 0) sh[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < kDiagVals) {
        const int k = threadIdx.x;
        double v = sh[k][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v = k < kDiagSums ? v + sh[k][w] : fmax(v, sh[k][w]);
        partial[blockIdx.x * kDiagVals + k] = v;
    }
}

// One warp per value: lane l combines rows l, l + 32, l + 64, ... in index
// order, then the lanes are combined by a fixed shuffle tree, so the result
// does not depend on scheduling.
__global__ void k_diag_final(const double* __restrict__ partial, int nrows, double* __restrict__ out) {
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= kDiagVals) return;
    const bool sum = k < kDiagSums;
    double v = sum ? 0.0 : -INFINITY;
    for (int r = lane; r < nrows; r += 32) {
        const double t = partial[r * kDiagVals + k];
        v = sum ? v + t : fmax(v, t);
    }
    v = sum ? warp_sum(v) : warp_max(v);
    if (lane == 0) out[k] = v;
}

// Initial densities: FP64 sums of rho_A and rho_B and the count of values
// that are not finite or are negative, per block over a grid-stride share,
// then summed over the rows in index order (one thread per value).
__global__ void __launch_bounds__(256) k_density_sums(const float* __restrict__ a, const float* __restrict__ b,
                                                      long long N, double* __restrict__ partial) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const float va = a[i];
        acc[0] += va;
        acc[2] += (isfinite(va) && va >= 0.0f) ? 0.0 : 1.0;
        if (b) {
            const float vb = b[i];
            acc[1] += vb;
            acc[2] += (isfinite(vb) && vb >= 0.0f) ? 0.0 : 1.0;
        }
    }
    __shared__ double sh[3][8];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double v = warp_sum(acc[k]);
        if (lane == 0) sh[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
        double v = sh[threadIdx.x][0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) v += sh[threadIdx.x][w];
        partial[blockIdx.x * 3 + threadIdx.x] = v;
    }
}

// One warp per value, as k_diag_final.
__global__ void k_density_final(const double* __restrict__ partial, int nrows, double* __restrict__ out) {
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= 3) return;
    double v = 0.0;
    for (int r = lane; r < nrows; r += 32) v += partial[r * 3 + k];
    v = warp_sum(v);
    if (lane == 0) out[k] = v;
}

}  // namespace

cudaError_t launch_density_sums(const float* rho_A, const float* rho_B, long long N, double* partial, double* out,
                                cudaStream_t s) {
    long long blocks = (N + 255) / 256;
    if (blocks > kDiagBlocks) blocks = kDiagBlocks;
    if (blocks < 1) blocks = 1;
    k_density_sums<<<(int)blocks, 256, 0, s>>>(rho_A, rho_B, N, partial);
    k_density_final<<<1, 3 * 32, 0, s>>>(partial, (int)blocks, out);
    return cudaGetLastError();
}

cudaError_t launch_derived(int lattice, int ncomp, int which, const StepParams& p, const float* drho,
                           const float* Ct, float* dst, cudaStream_t s) {
    const int g = grid_1d(p.N);
    if (lattice == 1) k_derived<6><<<g, 256, 0, s>>>(which, ncomp, drho, Ct, dst, p);
    else k_derived<4><<<g, 256, 0, s>>>(which, ncomp, drho, Ct, dst, p);
    return cudaGetLastError();
}

cudaError_t launch_tensor_shift(int lattice, const float* src, float* dst, long long N, float sign, cudaStream_t s) {
    const int g = grid_1d(N);
    if (lattice == 1) k_tensor_shift<6><<<g, 256, 0, s>>>(src, dst, N, sign);
    else k_tensor_shift<4><<<g, 256, 0, s>>>(src, dst, N, sign);
    return cudaGetLastError();
}

cudaError_t launch_diagnostics(int lattice, int ncomp, const StepParams& p, const float* drho, const float* u,
                               const float* Ct, double* partial, double* out, cudaStream_t s) {
    long long blocks = (p.N + 255) / 256;
    if (blocks > kDiagBlocks) blocks = kDiagBlocks;
    if (blocks < 1) blocks = 1;
    if (lattice == 1) k_diag_partial<3, 6><<<(int)blocks, 256, 0, s>>>(drho, u, Ct, ncomp, partial, p);
    else k_diag_partial<2, 4><<<(int)blocks, 256, 0, s>>>(drho, u, Ct, ncomp, partial, p);
    k_diag_final<<<1, kDiagVals * 32, 0, s>>>(partial, (int)blocks, out);
    return cudaGetLastError();
}

}  // namespace vefd
