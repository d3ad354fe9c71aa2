// Finite-difference FENE-P update of the conformation tensor (Eq. FENE of
// Gupta, Sbragaglia & Scagliarini, with the artificial diffusivity and the
// time integration described at the end of Sec. 2):
//   R = -(u.grad)C + C.grad u + (grad u)^T.C - (f(r_P) C - I)/tau_P + kappa lap C,
//   (grad u)_ij = d_i u_j, f(r_P) = (L^2 - 3)/(L^2 - tr C),
//   C^{n+1} = C^n + 3/2 R^n - 1/2 R^{n-1}   (forward Euler without history).
// Second-order central differences, periodic in x and z; at walls the ghost
// row is the linear extrapolation v(-1) = 2 v(0) - v(1), which makes the
// first derivative one-sided and the second derivative vanish.
// Stored variable: Ct = C - I, so (f C - I) = f Ct + (f - 1) I with
// f - 1 = tr Ct / (L^2 - 3 - tr Ct), evaluated without cancellation.
// The update runs in the same pass as the densities of the new populations
// (k_post), since both only wait for the lattice kernel.
#include <cuda.h>

#include "vefd_internal.cuh"

namespace vefd {

namespace {

__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

template <int NC>
__device__ __forceinline__ constexpr int tidx(int i, int j) {
    // stored component of (i, j), -1 when identically zero (D2Q9 xz, yz)
    if (NC == 6) {
        return (i == 0) ? j : (i == 1 ? (j == 0 ? 1 : (j == 1 ? 3 : 4)) : (j == 0 ? 2 : (j == 1 ? 4 : 5)));
    } else {
        return (i == 0) ? (j == 0 ? 0 : (j == 1 ? 1 : -1))
             : (i == 1 ? (j == 0 ? 1 : (j == 1 ? 2 : -1)) : (j == 2 ? 3 : -1));
    }
}

template <int NC>
__device__ __forceinline__ constexpr bool is_diag(int k) {
    return NC == 6 ? (k == 0 || k == 3 || k == 5) : (k == 0 || k == 2 || k == 3);
}

template <int NC>
__device__ __forceinline__ constexpr int row_of(int k) {
    return NC == 6 ? (k <= 2 ? 0 : (k <= 4 ? 1 : 2)) : (k <= 1 ? 0 : (k == 2 ? 1 : 2));
}

template <int NC>
__device__ __forceinline__ constexpr int col_of(int k) {
    return NC == 6 ? (k == 0 ? 0 : (k == 1 ? 1 : (k == 2 ? 2 : (k == 3 ? 1 : 2)))) : (k == 0 ? 0 : (k <= 2 ? 1 : 2));
}

// One FENE-P update at node (x, y, z): reads C - I and u with their stencil
// neighbours and the AB2 history, writes C - I of the next time level and the
// new history, and sets the guard bits.
template <int D, int NC>
__device__ __forceinline__ void fenep_node(const float* __restrict__ Ct, float* __restrict__ Cout,
                                           float* __restrict__ R, const float* __restrict__ u,
                                           unsigned* __restrict__ status, const StepParams& p, int x, int y, int z,
                                           float cnew[NC]) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const long long N = p.N;
    const long long i = ((long long)z * ny + y) * nx + x;
    const long long ixm = i - x + wrap1(x - 1, nx), ixp = i - x + wrap1(x + 1, nx);
    // y neighbours and the stencil weights of the first and second derivative
    long long iym, iyp;
    float hy1 = 0.5f, hy2 = 1.0f;  // d_y v = hy1 (v+ - v-); d_yy v = hy2 (v+ - 2 v + v-)
    if (p.walls && y == 0) {
        iym = i;
        iyp = i + nx;
        hy1 = 1.0f;
        hy2 = 0.0f;
    } else if (p.walls && y == ny - 1) {
        iym = i - nx;
        iyp = i;
        hy1 = 1.0f;
        hy2 = 0.0f;
    } else {
        iym = ((long long)z * ny + wrap1(y - 1, ny)) * nx + x;
        iyp = ((long long)z * ny + wrap1(y + 1, ny)) * nx + x;
    }
    long long izm = i, izp = i;
    if (D == 3) {
        izm = ((long long)wrap1(z - 1, nz) * ny + y) * nx + x;
        izp = ((long long)wrap1(z + 1, nz) * ny + y) * nx + x;
    }

    // velocity gradient Gu[a][b] = d_a u_b and the local velocity
    float Gu[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float uu[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int b = 0; b < D; ++b) {
        const float* ub = u + b * N;
        uu[b] = __ldg(ub + i);
        Gu[0][b] = 0.5f * (__ldg(ub + ixp) - __ldg(ub + ixm));
        Gu[1][b] = hy1 * (__ldg(ub + iyp) - __ldg(ub + iym));
        if (D == 3) Gu[2][b] = 0.5f * (__ldg(ub + izp) - __ldg(ub + izm));
    }

    float c[NC], adv[NC], lap[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const float* ck = Ct + k * N;
        const float c0 = __ldg(ck + i);
        const float cxm = __ldg(ck + ixm), cxp = __ldg(ck + ixp);
        const float cym = __ldg(ck + iym), cyp = __ldg(ck + iyp);
        c[k] = c0;
        float a = uu[0] * 0.5f * (cxp - cxm) + uu[1] * hy1 * (cyp - cym);
        float l = (cxp - 2.0f * c0 + cxm) + hy2 * (cyp - 2.0f * c0 + cym);
        if (D == 3) {
            const float czm = __ldg(ck + izm), czp = __ldg(ck + izp);
            a += uu[2] * 0.5f * (czp - czm);
            l += czp - 2.0f * c0 + czm;
        }
        adv[k] = a;
        lap[k] = l;
    }
    float tr = NC == 6 ? c[0] + c[3] + c[5] : c[0] + c[2] + c[3];
    const float fm1 = tr / (p.L2m3 - tr);
    const float f = 1.0f + fm1;

    // full C = Ct + I as a 3x3 matrix
    float Cm[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int k = tidx<NC>(a, b);
            Cm[a][b] = (k < 0 ? 0.0f : c[k]) + (a == b ? 1.0f : 0.0f);
        }

    float trn = 0.0f;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const int a = row_of<NC>(k), b = col_of<NC>(k);
        float up = 0.0f;
#pragma unroll
        for (int e = 0; e < D; ++e) up += Cm[a][e] * Gu[e][b] + Gu[e][a] * Cm[e][b];
        const float relax = (f * c[k] + (is_diag<NC>(k) ? fm1 : 0.0f)) * p.inv_tau_p;
        const float Rk = -adv[k] + up - relax + p.kappa * lap[k];
        const float inc = p.have_prev ? 1.5f * Rk - 0.5f * R[k * N + i] : Rk;
        const float cn = c[k] + inc;
        cnew[k] = cn;
        Cout[k * N + i] = cn;
        R[k * N + i] = Rk;
        if (is_diag<NC>(k)) trn += cn;
        bad |= isnan(cn);
    }
    if (bad || isnan(tr)) atomicOr(status, kStNan);
    else if (trn >= p.L2m3 || tr >= p.L2m3) atomicOr(status, kStTrace);
}

// Feedback stress at one node, Q = (f C - I) m(phi) = (f Ct + (f - 1) I) m(phi)
// with f - 1 = tr Ct / (L^2 - 3 - tr Ct) and m = 1, f_+(phi) or f_-(phi)
// (Eq. NS and the last equation of Sec. 2); stored as the NQ components
// xx xy xz yy yz zz (3D) or xx xy yy (2D) that the divergence needs.
template <class L, int NCOMP>
__device__ __forceinline__ void store_feedback(const float c[L::NC], const float d[NCOMP], const StepParams& p,
                                               float* __restrict__ Q, long long N, long long i) {
    const float tr = L::NC == 6 ? c[0] + c[3] + c[5] : c[0] + c[2] + c[3];
    const float fm1 = tr / (p.L2m3 - tr);
    const float f = 1.0f + fm1;
    float m = 1.0f;
    if (p.phase != 0) {
        float phi = 1.0f;  // one component: phi = 1 everywhere
        if (NCOMP == 2) {
            const float ra = p.rho_ref[0] + d[0], rb = p.rho_ref[1] + d[NCOMP - 1];
            phi = (ra - rb) / (ra + rb);
        }
        const float t = tanhf(phi * p.inv_delta);
        m = p.phase > 0 ? 0.5f * (1.0f + t) : 0.5f * (1.0f - t);
    }
    if (L::NC == 6) {
#pragma unroll
        for (int k = 0; k < 6; ++k) Q[k * N + i] = (f * c[k] + (is_diag<6>(k) ? fm1 : 0.0f)) * m;
    } else {
        Q[i] = (f * c[0] + fm1) * m;          // xx
        Q[N + i] = (f * c[1]) * m;            // xy
        Q[2 * N + i] = (f * c[2] + fm1) * m;  // yy
    }
}

// After the lattice kernel of step n: densities of the new populations
// (same summation order as the moments kernel), the FENE-P update of C from
// time n to n+1 when the polymer is evolved, and the feedback stress of time
// n+1 for the next lattice step.  All of it only reads data the lattice kernel
// has finished writing, so one pass over the lattice does it.
template <class L, int NCOMP, bool FD>
__global__ void __launch_bounds__(128) k_post(const float* __restrict__ fnew, float* __restrict__ drho,
                                              const float* __restrict__ Ct, float* __restrict__ Cout,
                                              float* __restrict__ R, const float* __restrict__ u,
                                              float* __restrict__ Q, unsigned* __restrict__ status, StepParams p,
                                              int rev) {
    const int bxi = rev ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x;
    const int byi = rev ? (int)(gridDim.y - 1 - blockIdx.y) : (int)blockIdx.y;
    const int x = bxi * blockDim.x + threadIdx.x;
    const int y = byi * blockDim.y + threadIdx.y;
    const int z = rev ? (int)(gridDim.z - 1 - blockIdx.z) : (int)blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long N = p.N;
    const long long i = ((long long)z * p.ny + y) * p.nx + x;
    float d[NCOMP];
#pragma unroll
    for (int s = 0; s < NCOMP; ++s) {
        d[s] = 0.0f;
#pragma unroll
        for (int a = 0; a < L::Q; ++a) d[s] += __ldg(fnew + (s * L::Q + a) * N + i);
    }
    float c[L::NC];
    if (FD) {
        fenep_node<L::D, L::NC>(Ct, Cout, R, u, status, p, x, y, z, c);
    } else {
#pragma unroll
        for (int k = 0; k < L::NC; ++k) c[k] = __ldg(Ct + k * N + i);
    }
#pragma unroll
    for (int s = 0; s < NCOMP; ++s) drho[s * N + i] = d[s];
    if (p.feedback != 0.0f) store_feedback<L, NCOMP>(c, d, p, Q, N, i);
}

// The same pass with the tile's new populations staged in shared memory by
// one bulk tensor copy, issued before the stencil loads so that both are in
// flight together; the densities are summed from shared memory afterwards in
// the same order.
template <class L, int NCOMP, bool FD, int BX, int BY, int BZ>
__global__ void __launch_bounds__(BX * BY * BZ) k_post_tma(const __grid_constant__ CUtensorMap tm_fnew,
                                                           float* __restrict__ drho, const float* __restrict__ Ct,
                                                           float* __restrict__ Cout, float* __restrict__ R,
                                                           const float* __restrict__ u, float* __restrict__ Q,
                                                           unsigned* __restrict__ status, StepParams p, int rev) {
    constexpr int P = NCOMP * L::Q;
    constexpr int T = BX * BY * BZ;
    constexpr unsigned kBytes = (unsigned)(P * T * sizeof(float));
    extern __shared__ __align__(128) float sf[];  // [P][BZ][BY][BX]
    __shared__ __align__(8) unsigned long long bar;
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const int x0 = (rev ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x) * BX;
    const int y0 = (rev ? (int)(gridDim.y - 1 - blockIdx.y) : (int)blockIdx.y) * BY;
    const int z0 = (rev ? (int)(gridDim.z - 1 - blockIdx.z) : (int)blockIdx.z) * BZ;
    const bool leader = (tx | ty | tz) == 0;
    const unsigned bar_a = smem_u32(&bar);
    if (leader) mbar_init(bar_a);
    __syncthreads();
    if (leader) tma_load_4d(smem_u32(sf), &tm_fnew, x0, y0, z0, 0, bar_a, kBytes);
    const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
    const bool active = x < p.nx && y < p.ny && z < p.nz;
    const long long N = p.N;
    const long long i = active ? ((long long)z * p.ny + y) * p.nx + x : 0;
    float c[L::NC];
    if (active) {
        if (FD) {
            fenep_node<L::D, L::NC>(Ct, Cout, R, u, status, p, x, y, z, c);
        } else {
#pragma unroll
            for (int k = 0; k < L::NC; ++k) c[k] = __ldg(Ct + k * N + i);
        }
    }
    if (!mbar_wait_bounded(bar_a)) {
        if (leader) atomicOr(status, kStTimeout);
        return;
    }
    if (!active) return;
    const int t = (tz * BY + ty) * BX + tx;
    float d[NCOMP];
#pragma unroll
    for (int s = 0; s < NCOMP; ++s) {
        d[s] = 0.0f;
#pragma unroll
        for (int a = 0; a < L::Q; ++a) d[s] += sf[(s * L::Q + a) * T + t];
        drho[s * N + i] = d[s];
    }
    if (p.feedback != 0.0f) store_feedback<L, NCOMP>(c, d, p, Q, N, i);
}

// Densities and feedback stress of a given state (no time step).
template <class L, int NCOMP>
__global__ void __launch_bounds__(128) k_pre(const float* __restrict__ f, float* __restrict__ drho,
                                             const float* __restrict__ Ct, float* __restrict__ Q, StepParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long N = p.N;
    const long long i = ((long long)z * p.ny + y) * p.nx + x;
    float d[NCOMP];
#pragma unroll
    for (int s = 0; s < NCOMP; ++s) {
        d[s] = 0.0f;
#pragma unroll
        for (int a = 0; a < L::Q; ++a) d[s] += __ldg(f + (s * L::Q + a) * N + i);
        drho[s * N + i] = d[s];
    }
    float c[L::NC];
#pragma unroll
    for (int k = 0; k < L::NC; ++k) c[k] = __ldg(Ct + k * N + i);
    if (p.feedback != 0.0f) store_feedback<L, NCOMP>(c, d, p, Q, N, i);
}

}  // namespace

cudaError_t launch_post(int lattice, int ncomp, bool fd, const StepParams& p, const StepBufs& b,
                        const float* fnew, cudaStream_t s, int rev) {
    dim3 blk(32, 4, 1), grd((p.nx + 31) / 32, (p.ny + 3) / 4, p.nz);
#define VEFD_POST(LT, NCP)                                                                                        \
    do {                                                                                                          \
        if (fd)                                                                                                   \
            k_post<LT, NCP, true><<<grd, blk, 0, s>>>(fnew, b.drho, b.Cin, b.Cout, b.R, b.u, b.Q, b.status, p, rev);  \
        else                                                                                                      \
            k_post<LT, NCP, false><<<grd, blk, 0, s>>>(fnew, b.drho, b.Cin, b.Cout, b.R, b.u, b.Q, b.status, p, rev); \
    } while (0)
    if (lattice == 1) {
        if (ncomp == 2) VEFD_POST(D3Q19, 2);
        else VEFD_POST(D3Q19, 1);
    } else {
        if (ncomp == 2) VEFD_POST(D2Q9, 2);
        else VEFD_POST(D2Q9, 1);
    }
#undef VEFD_POST
    return cudaGetLastError();
}

namespace {
template <class L, int NCOMP, int BX, int BY, int BZ>
cudaError_t post_tma(bool fd, const CUtensorMap* tm, const StepParams& p, const StepBufs& b, cudaStream_t s, int rev) {
    constexpr int smem = NCOMP * L::Q * BX * BY * BZ * (int)sizeof(float);
    dim3 blk(BX, BY, BZ), grd((p.nx + BX - 1) / BX, (p.ny + BY - 1) / BY, (p.nz + BZ - 1) / BZ);
    if (fd)
        k_post_tma<L, NCOMP, true, BX, BY, BZ><<<grd, blk, smem, s>>>(*tm, b.drho, b.Cin, b.Cout, b.R, b.u, b.Q,
                                                                       b.status, p, rev);
    else
        k_post_tma<L, NCOMP, false, BX, BY, BZ><<<grd, blk, smem, s>>>(*tm, b.drho, b.Cin, b.Cout, b.R, b.u, b.Q,
                                                                        b.status, p, rev);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_post_tma(int lattice, int ncomp, bool fd, const StepParams& p, const StepBufs& b,
                            const void* tensor_map_fnew, cudaStream_t s, int rev) {
    const CUtensorMap* tm = static_cast<const CUtensorMap*>(tensor_map_fnew);
    if (lattice == 1)
        return ncomp == 2 ? post_tma<D3Q19, 2, 32, 4, 2>(fd, tm, p, b, s, rev) : post_tma<D3Q19, 1, 32, 4, 2>(fd, tm, p, b, s, rev);
    return ncomp == 2 ? post_tma<D2Q9, 2, 32, 8, 1>(fd, tm, p, b, s, rev) : post_tma<D2Q9, 1, 32, 8, 1>(fd, tm, p, b, s, rev);
}

cudaError_t launch_pre(int lattice, int ncomp, const StepParams& p, const StepBufs& b, cudaStream_t s) {
    dim3 blk(32, 4, 1), grd((p.nx + 31) / 32, (p.ny + 3) / 4, p.nz);
    if (lattice == 1) {
        if (ncomp == 2) k_pre<D3Q19, 2><<<grd, blk, 0, s>>>(b.fin, b.drho, b.Cin, b.Q, p);
        else k_pre<D3Q19, 1><<<grd, blk, 0, s>>>(b.fin, b.drho, b.Cin, b.Q, p);
    } else {
        if (ncomp == 2) k_pre<D2Q9, 2><<<grd, blk, 0, s>>>(b.fin, b.drho, b.Cin, b.Q, p);
        else k_pre<D2Q9, 1><<<grd, blk, 0, s>>>(b.fin, b.drho, b.Cin, b.Q, p);
    }
    return cudaGetLastError();
}

}  // namespace vefd
