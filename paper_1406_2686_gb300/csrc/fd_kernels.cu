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
// Optionally (StepParams::chol) the AB2 step advances the log-Cholesky factor
// of sigma_P = f C instead of C (the Cholesky scheme of Sec. 2).
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

// Cholesky scheme (Sec. 2): sigma_P = f(r_P) C = L L^T with L lower
// triangular.  For the right-hand side dC/dt of the direct scheme,
//   d sigma_P/dt = f dC/dt + sigma_P f tr(dC/dt) / (L^2 - 3),
//   dL/dt = L Phi(L^-1 (d sigma_P/dt) L^-T),  Phi = lower triangle, diagonal halved,
// and AB2 advances lambda = (ln l_ii, l_ij for i > j) with the history of its
// rates.  The new C = L L^T / f with f = (L^2 - 3 + tr L L^T)/L^2 is SPD with
// tr C < L^2 whenever lambda is finite.  c and cnew hold C - I; Rk is dC/dt;
// Rprev and Rnew the lambda rates, in the stored component slots.
template <int NC>
__device__ __forceinline__ void chol_step(const float c[NC], const float Rk[NC], const float Rprev[NC], int have_prev,
                                          float L2m3, float cnew[NC], float Rnew[NC]) {
    float C[3][3], Cd[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            const int k = tidx<NC>(a, b);
            C[a][b] = (k < 0 ? 0.0f : c[k]) + (a == b ? 1.0f : 0.0f);
            Cd[a][b] = k < 0 ? 0.0f : Rk[k];
        }
    const float trt = NC == 6 ? c[0] + c[3] + c[5] : c[0] + c[2] + c[3];
    const float f = L2m3 / (L2m3 - trt);
    const float trd = Cd[0][0] + Cd[1][1] + Cd[2][2];
    const float g = f * trd / L2m3;
    float S[3][3], Sd[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            S[a][b] = f * C[a][b];
            Sd[a][b] = f * Cd[a][b] + S[a][b] * g;
        }
    // S = L L^T and the inverse of L
    float L[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j <= i; ++j) {
            float v = S[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
            L[i][j] = (i == j) ? sqrtf(v) : v / L[j][j];
        }
    float Li[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        Li[j][j] = 1.0f / L[j][j];
#pragma unroll
        for (int i = j + 1; i < 3; ++i) {
            float v = 0.0f;
#pragma unroll
            for (int k = j; k < i; ++k) v -= L[i][k] * Li[k][j];
            Li[i][j] = v / L[i][i];
        }
    }
    // A = L^-1 Sd L^-T (symmetric; lower triangle), Phi(A), dL/dt = L Phi(A)
    float T[3][3], P[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float v = 0.0f;
#pragma unroll
            for (int k = 0; k <= i; ++k) v += Li[i][k] * Sd[k][j];
            T[i][j] = v;
        }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            float v = 0.0f;
            if (j <= i) {
#pragma unroll
                for (int k = 0; k <= j; ++k) v += T[i][k] * Li[j][k];
                if (i == j) v *= 0.5f;
            }
            P[i][j] = v;
        }
    float Ln[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const int i = col_of<NC>(k), j = row_of<NC>(k);  // lower-triangle entry (i >= j)
        float ld = 0.0f;
#pragma unroll
        for (int q = 0; q < 3; ++q)
            if (q >= j && q <= i) ld += L[i][q] * P[q][j];
        const float lam = (i == j) ? logf(L[i][i]) : L[i][j];
        const float rl = (i == j) ? ld / L[i][i] : ld;
        const float lamn = lam + (have_prev ? 1.5f * rl - 0.5f * Rprev[k] : rl);
        Ln[i][j] = (i == j) ? expf(lamn) : lamn;
        Rnew[k] = rl;
    }
    float Sn[3][3];
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            float v = 0.0f;
#pragma unroll
            for (int q = 0; q < 3; ++q) v += Ln[a][q] * Ln[b][q];
            Sn[a][b] = v;
        }
    const float inv_fn = (L2m3 + 3.0f) / (L2m3 + Sn[0][0] + Sn[1][1] + Sn[2][2]);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const int a = row_of<NC>(k), b = col_of<NC>(k);
        cnew[k] = Sn[a][b] * inv_fn - (a == b ? 1.0f : 0.0f);
    }
}

// FENE-P update at one node from its gathered stencil.  v(k, d) returns field
// k (0..NC-1: C - I components, NC..NC+D-1: velocity components) at stencil
// point d (0 centre, 1 -x, 2 +x, 3 -y, 4 +y, 5 -z, 6 +z); hy1 and hy2 are the
// y weights of the first and second differences (1/2 and 1 inside, 1 and 0
// at a wall row, where the -y or +y point is the node itself).  Writes the new
// C - I to cnew, the right-hand side to Rnew, and returns the guard bits.
template <int D, int NC, class V>
__device__ __forceinline__ unsigned fenep_compute(V v, float hy1, float hy2, const float Rprev[NC], const StepParams& p,
                                                  float cnew[NC], float Rnew[NC]) {
    // velocity gradient Gu[a][b] = d_a u_b and the local velocity
    float Gu[3][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
    float uu[3] = {0.f, 0.f, 0.f};
#pragma unroll
    for (int b = 0; b < D; ++b) {
        uu[b] = v(NC + b, 0);
        Gu[0][b] = 0.5f * (v(NC + b, 2) - v(NC + b, 1));
        Gu[1][b] = hy1 * (v(NC + b, 4) - v(NC + b, 3));
        if (D == 3) Gu[2][b] = 0.5f * (v(NC + b, 6) - v(NC + b, 5));
    }
    float c[NC], adv[NC], lap[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const float c0 = v(k, 0);
        const float cxm = v(k, 1), cxp = v(k, 2), cym = v(k, 3), cyp = v(k, 4);
        c[k] = c0;
        float a = uu[0] * 0.5f * (cxp - cxm) + uu[1] * hy1 * (cyp - cym);
        float l = (cxp - 2.0f * c0 + cxm) + hy2 * (cyp - 2.0f * c0 + cym);
        if (D == 3) {
            const float czm = v(k, 5), czp = v(k, 6);
            a += uu[2] * 0.5f * (czp - czm);
            l += czp - 2.0f * c0 + czm;
        }
        adv[k] = a;
        lap[k] = l;
    }
    const float tr = NC == 6 ? c[0] + c[3] + c[5] : c[0] + c[2] + c[3];
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
    float Rc[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        const int a = row_of<NC>(k), b = col_of<NC>(k);
        float up = 0.0f;
#pragma unroll
        for (int e = 0; e < D; ++e) up += Cm[a][e] * Gu[e][b] + Gu[e][a] * Cm[e][b];
        const float relax = (f * c[k] + (is_diag<NC>(k) ? fm1 : 0.0f)) * p.inv_tau_p;
        Rc[k] = -adv[k] + up - relax + p.kappa * lap[k];
    }
    if (p.chol) {
        chol_step<NC>(c, Rc, Rprev, p.have_prev, p.L2m3, cnew, Rnew);
    } else {
        // Compensated AB2: the sum c + inc is rounded to FP32, and its exact
        // rounding error e (Knuth's TwoSum) is carried into the next step's
        // increment through the stored history, R~ = R - 2e, so that
        // 3/2 R' - 1/2 R~ = 3/2 R' - 1/2 R + e.  Near steady state the increment
        // falls below half an ulp of C - I; without the carry it would be lost
        // and C would stall up to (tau_P / f) ulp short of the fixed point.
        // The history then stays within FP32 rounding of max(|R|, |e|).
#pragma unroll
        for (int k = 0; k < NC; ++k) {
            const float inc = p.have_prev ? 1.5f * Rc[k] - 0.5f * Rprev[k] : Rc[k];
            const float sum = c[k] + inc;
            const float inc_kept = sum - c[k];
            const float err = (c[k] - (sum - inc_kept)) + (inc - inc_kept);
            cnew[k] = sum;
            Rnew[k] = fmaf(-2.0f, err, Rc[k]);
        }
    }
    float trn = 0.0f;
    bool bad = false;
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        if (is_diag<NC>(k)) trn += cnew[k];
        bad |= isnan(cnew[k]);
    }
    if (bad || isnan(tr)) return kStNan;
    if (trn >= p.L2m3 || tr >= p.L2m3) return kStTrace;
    return 0u;
}

// One FENE-P update at node (x, y, z) with its stencil read from global
// memory; writes C - I of the next time level and the new history.
template <int D, int NC>
__device__ __forceinline__ void fenep_node(const float* __restrict__ Ct, float* __restrict__ Cout,
                                           float* __restrict__ R, const float* __restrict__ u,
                                           unsigned* __restrict__ status, const StepParams& p, int x, int y, int z,
                                           float cnew[NC]) {
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const long long N = p.N;
    const long long i = ((long long)z * ny + y) * nx + x;
    long long idx[7];
    idx[0] = i;
    idx[1] = i - x + wrap1(x - 1, nx);
    idx[2] = i - x + wrap1(x + 1, nx);
    float hy1 = 0.5f, hy2 = 1.0f;
    if (p.walls && y == 0) {
        idx[3] = i;
        idx[4] = i + nx;
        hy1 = 1.0f;
        hy2 = 0.0f;
    } else if (p.walls && y == ny - 1) {
        idx[3] = i - nx;
        idx[4] = i;
        hy1 = 1.0f;
        hy2 = 0.0f;
    } else {
        idx[3] = ((long long)z * ny + wrap1(y - 1, ny)) * nx + x;
        idx[4] = ((long long)z * ny + wrap1(y + 1, ny)) * nx + x;
    }
    idx[5] = idx[6] = i;
    if (D == 3) {
        idx[5] = ((long long)wrap1(z - 1, nz) * ny + y) * nx + x;
        idx[6] = ((long long)wrap1(z + 1, nz) * ny + y) * nx + x;
    }
    auto v = [&](int k, int d) -> float {
        const float* base = k < NC ? Ct + k * N : u + (k - NC) * N;
        return idx_ok(idx[d], N, status) ? __ldg(base + idx[d]) : 0.0f;
    };
    float Rprev[NC], Rnew[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) Rprev[k] = p.have_prev ? R[k * N + i] : 0.0f;
    const unsigned bits = fenep_compute<D, NC>(v, hy1, hy2, Rprev, p, cnew, Rnew);
#pragma unroll
    for (int k = 0; k < NC; ++k) {
        Cout[k * N + i] = cnew[k];
        R[k * N + i] = Rnew[k];
    }
    if (bits) atomicOr(status, bits);
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
template <class PT, class L, int NCOMP, bool FD>
__global__ void __launch_bounds__(128) k_post(const PT* __restrict__ fnew, const float* __restrict__ frest,
                                              float* __restrict__ drho,
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
        d[s] = __ldg(frest + s * N + i);
#pragma unroll
        for (int a = 1; a < L::Q; ++a) d[s] += pop_load(fnew + (s * (L::Q - 1) + a - 1) * N + i);
    }
    float c[L::NC];
    if (FD) {
        fenep_node<L::D, L::NC>(Ct, Cout, R, u, status, p, x, y, z, c);
    } else {
#pragma unroll
        for (int k = 0; k < L::NC; ++k) c[k] = __ldg(Ct + k * N + i);
    }
    dens_store<NCOMP>(drho, i, d);
    if (p.feedback != 0.0f) store_feedback<L, NCOMP>(c, d, p, Q, N, i);
}

// The same pass with the tile's new populations staged in shared memory by
// one bulk tensor copy, issued before the stencil loads so that both are in
// flight together; the densities are summed from shared memory afterwards in
// the same order.
template <class PT, class L, int NCOMP, bool FD, int BX, int BY, int BZ>
__global__ void __launch_bounds__(BX * BY * BZ) k_post_tma(const __grid_constant__ CUtensorMap tm_fnew,
                                                           const float* __restrict__ frest,
                                                           float* __restrict__ drho, const float* __restrict__ Ct,
                                                           float* __restrict__ Cout, float* __restrict__ R,
                                                           const float* __restrict__ u, float* __restrict__ Q,
                                                           unsigned* __restrict__ status, StepParams p, int rev) {
    constexpr int P = NCOMP * (L::Q - 1);  // moving populations
    constexpr int T = BX * BY * BZ;
    constexpr unsigned kBytes = (unsigned)(P * T * sizeof(PT));
    extern __shared__ __align__(128) unsigned char sraw[];
    PT* sf = reinterpret_cast<PT*>(sraw);  // [P][BZ][BY][BX]
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
    float rest[NCOMP];
    if (active) {
#pragma unroll
        for (int s = 0; s < NCOMP; ++s) rest[s] = __ldg(frest + s * N + i);
        if (FD) {
            fenep_node<L::D, L::NC>(Ct, Cout, R, u, status, p, x, y, z, c);
        } else {
#pragma unroll
            for (int k = 0; k < L::NC; ++k) c[k] = __ldg(Ct + k * N + i);
        }
    }
    if (!mbar_wait_bounded(bar_a)) {
        if (leader) {
            atomicOr(status, kStTimeout);
            mbar_wait_bounded(bar_a);  // bounded: let the copy land before leaving
        }
        return;
    }
    if (!active) return;
    const int t = (tz * BY + ty) * BX + tx;
    float d[NCOMP];
#pragma unroll
    for (int s = 0; s < NCOMP; ++s) {
        d[s] = rest[s];
#pragma unroll
        for (int a = 1; a < L::Q; ++a) d[s] += pop_get(sf[(s * (L::Q - 1) + a - 1) * T + t]);
    }
    dens_store<NCOMP>(drho, i, d);
    if (p.feedback != 0.0f) store_feedback<L, NCOMP>(c, d, p, Q, N, i);
}

// D3Q19 variant of the pass that marches along z through a column of
// 32 x 8 nodes.  C - I and u of four consecutive planes (with a one-node halo
// in x and y) live in a shared-memory ring, so every stencil value is read
// from global memory about 1.3 times instead of 7; each plane's new
// populations arrive by one bulk tensor copy (box 32 x 8 x 1 x P) that
// overlaps the stencil arithmetic.  Needs NX % 32 == 0 and NY % 8 == 0.
constexpr int kZmBX = 32, kZmBY = 8, kZmHX = kZmBX + 2, kZmHY = kZmBY + 2, kZmNF = 9;
constexpr int kZmPlane = kZmNF * kZmHY * kZmHX;  // floats per ring plane

template <class PT, int NCOMP>
constexpr int zm_smem_bytes() {
    return NCOMP * 18 * kZmBX * kZmBY * (int)sizeof(PT) + 4 * kZmPlane * (int)sizeof(float);
}

// MODE 0: the densities of the new populations, staged plane by plane.
// MODE 1 (FUSED): after the column-marching lattice kernel.  drho then holds
// each node's partial density (the rest population and every population that
// arrived from inside its 32 x 8 column and lattice-kernel z-segment of
// length zl); the pass adds, from fnew, the populations that crossed a column
// side or a segment end, in direction order, and needs no population copy.
// MODE 2 (PARTS): after the staged lattice kernel with partial densities
// (tile_partials): each node's density is its slot-0 sum plus, in slot
// order, the slots its position in its lattice tile (32 x part_by x part_bz)
// implies; no population is read.
// One 32 x 8 column (origin x0, y0) over the planes [z0, z0 + zs) of the
// pass; tm_fnew is the tensor map of the new populations (box 32 x 8 x 1 x P).
template <class PT, int NCOMP, bool FD, int MODE>
__device__ __forceinline__ void post_column(const CUtensorMap* tm_fnew, const float* __restrict__ frest,
                                            float* __restrict__ drho, const float* __restrict__ Ct,
                                            float* __restrict__ Cout, float* __restrict__ R,
                                            const float* __restrict__ u, float* __restrict__ Q,
                                            unsigned* __restrict__ status, const StepParams& p, int x0, int y0, int z0,
                                            int zs, const PT* __restrict__ fnew, int zl,
                                            const float* __restrict__ part = nullptr, int part_by = 1,
                                            int part_bz = 1) {
    constexpr bool FUSED = MODE == 1, PARTS = MODE == 2;
    using L = D3Q19;
    constexpr int P = NCOMP * (L::Q - 1);  // moving populations
    constexpr int T = kZmBX * kZmBY;
    constexpr unsigned kBytes = (unsigned)(P * T * sizeof(PT));
    extern __shared__ __align__(128) unsigned char sraw[];
    PT* sP = reinterpret_cast<PT*>(sraw);  // [P][BY][BX] populations of the current plane (MODE 0)
    float* ring = reinterpret_cast<float*>(sraw + (MODE != 0 ? 0 : P * T * sizeof(PT)));  // [4][NF][HY][HX]
    __shared__ __align__(8) unsigned long long bar;
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const int N = (int)p.N, plane = nx * ny;
    const int z1 = min(z0 + zs, nz);
    const int x = x0 + tx, y = y0 + ty;
    const bool leader = (tx | ty) == 0;
    const unsigned bar_a = smem_u32(&bar);
    if (leader) mbar_init(bar_a);
    // everything below reads or overwrites data of the preceding lattice kernel
    pdl_wait();

    // which ring cells this thread stages: its own (interior) cell and, for
    // some warps, one halo cell (rows y0-1 / y0+8, columns x0-1 / x0+32)
    int hr = -1, hc = -1;
    if (ty == 0) {
        hr = 0;
        hc = tx + 1;
    } else if (ty == kZmBY - 1) {
        hr = kZmHY - 1;
        hc = tx + 1;
    } else if (ty == 1 && tx < 2 * kZmHY) {
        hr = tx % kZmHY;
        hc = tx < kZmHY ? 0 : kZmHX - 1;
    }
    int hx = 0, hyg = 0;
    bool hvalid = false;
    if (hr >= 0) {
        hx = wrap1(x0 - 1 + hc, nx);
        const int yy = y0 - 1 + hr;
        if (p.walls) {
            hvalid = yy >= 0 && yy < ny;  // ghost rows beyond walls are never read
            hyg = yy;
        } else {
            hvalid = true;
            hyg = wrap1(yy, ny);
        }
    }
    auto load_plane = [&](int zp, float v_in[kZmNF], float v_h[kZmNF]) {
        const int zz = wrap1(zp, nz);
        const int gi = zz * plane + y * nx + x;
        const int gh = zz * plane + hyg * nx + hx;
#pragma unroll
        const bool ok_i = idx_ok(gi, N, status), ok_h = hvalid && idx_ok(gh, N, status);
        for (int k = 0; k < kZmNF; ++k) {
            const float* base = k < 6 ? Ct + k * N : u + (k - 6) * N;
            v_in[k] = ok_i ? __ldg(base + gi) : 0.0f;
            if (hvalid) v_h[k] = ok_h ? __ldg(base + gh) : 0.0f;
        }
    };
    auto store_plane = [&](int slot, const float v_in[kZmNF], const float v_h[kZmNF]) {
        float* rp = ring + slot * kZmPlane;
#pragma unroll
        for (int k = 0; k < kZmNF; ++k) {
            rp[(k * kZmHY + ty + 1) * kZmHX + tx + 1] = v_in[k];
            if (hvalid) rp[(k * kZmHY + hr) * kZmHX + hc] = v_h[k];
        }
    };
    float vi[kZmNF], vh[kZmNF];
    // prologue: planes z0-1, z0, z0+1 into slots 0, 1, 2
    for (int q = 0; q < 3; ++q) {
        load_plane(z0 - 1 + q, vi, vh);
        store_plane(q, vi, vh);
    }
    __syncthreads();

    const bool wall_lo = p.walls && y == 0, wall_hi = p.walls && y == ny - 1;
    const float hy1 = (wall_lo || wall_hi) ? 1.0f : 0.5f;
    const float hy2 = (wall_lo || wall_hi) ? 0.0f : 1.0f;
    const int ry = ty + 1, rc = tx + 1;
    const int rym = wall_lo ? ry : ry - 1, ryp = wall_hi ? ry : ry + 1;
    const int t = ty * kZmBX + tx;

    const ColumnTopo topo{nx == 32, ny == 8 && !p.walls, nz == 1};
    for (int k = 0; k < z1 - z0; ++k) {
        const int z = z0 + k;
        // the next step's lattice kernel may be scheduled once every block is on its last plane
        if (k == z1 - z0 - 1) pdl_trigger();
        // new populations of this plane: one bulk copy (the buffer was released
        // by every thread at the barrier ending the previous iteration)
        if (MODE == 0 && leader) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tma_load_4d(smem_u32(sP), tm_fnew, x0, y0, z, 0, bar_a, kBytes);
        }
        // stage plane z+2 while this plane is computed
        const bool more = z + 2 <= z1;
        if (more) load_plane(z + 2, vi, vh);
        const int i = z * plane + y * nx + x;
        float rest[NCOMP];
        if (FUSED) {
            // partial density plus what crossed a column side or a segment end
            const bool wlo = p.walls && y == 0, whi = p.walls && y == ny - 1;
            const int zs_lo = (z / zl) * zl, zs_hi = min(zs_lo + zl, nz);  // this plane's lattice-kernel segment
            float part[NCOMP];
            dens_get<NCOMP>(drho, i, part);
#pragma unroll
            for (int s = 0; s < NCOMP; ++s) {
                float d = part[s];
#pragma unroll
                for (int a = 1; a < L::Q; ++a) {
                    const int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
                    if ((cy > 0 && wlo) || (cy < 0 && whi)) continue;  // bounce-back: counted in the partial
                    const int zsrc = z - cz;
                    const bool same_seg = topo.nz1 || (zsrc >= zs_lo && zsrc < zs_hi);
                    const bool same_col = (topo.nx32 || (unsigned)(tx - cx) < 32u) && (topo.ny8p || (unsigned)(ty - cy) < 8u);
                    if (same_seg && same_col) continue;
                    d += pop_get(fnew[(s * (L::Q - 1) + a - 1) * N + i]);
                }
                rest[s] = d;
            }
        } else if (PARTS) {
            // slot 0, then the neighbouring tiles' pushes (x, y, z, xy, xz, yz)
            const int ly = y % part_by, lz = z % part_bz;
            const bool xe = tx == 0 || tx == kZmBX - 1;
            const bool ye = (ly == 0 && (y > 0 || !p.walls)) || (ly == part_by - 1 && (y < ny - 1 || !p.walls));
            const bool ze = lz == 0 || lz == part_bz - 1;
            const bool use[7] = {true, xe, ye, ze, xe && ye, xe && ze, ye && ze};
#pragma unroll
            for (int s = 0; s < NCOMP; ++s) rest[s] = 0.0f;
#pragma unroll
            for (int q = 0; q < 7; ++q) {
                if (!use[q]) continue;
                float w[NCOMP] = {};
                if (idx_ok(i, N, status)) dens_ldg<NCOMP>(part + (long long)q * N * NCOMP, i, w);
#pragma unroll
                for (int s = 0; s < NCOMP; ++s) rest[s] = q == 0 ? w[s] : rest[s] + w[s];
            }
        } else {
#pragma unroll
            for (int s = 0; s < NCOMP; ++s) rest[s] = __ldg(frest + s * N + i);
        }
        float c[6];
        if (FD) {
            const float* pm = ring + (k % 4) * kZmPlane;
            const float* pc = ring + ((k + 1) % 4) * kZmPlane;
            const float* pp = ring + ((k + 2) % 4) * kZmPlane;
            auto v = [&](int f, int d) -> float {
                const int o = f * kZmHY * kZmHX;
                switch (d) {
                case 0: return pc[o + ry * kZmHX + rc];
                case 1: return pc[o + ry * kZmHX + rc - 1];
                case 2: return pc[o + ry * kZmHX + rc + 1];
                case 3: return pc[o + rym * kZmHX + rc];
                case 4: return pc[o + ryp * kZmHX + rc];
                case 5: return pm[o + ry * kZmHX + rc];
                default: return pp[o + ry * kZmHX + rc];
                }
            };
            float Rprev[6], Rnew[6];
#pragma unroll
            for (int q = 0; q < 6; ++q) Rprev[q] = p.have_prev ? R[q * N + i] : 0.0f;
            const unsigned bits = fenep_compute<3, 6>(v, hy1, hy2, Rprev, p, c, Rnew);
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                Cout[q * N + i] = c[q];
                R[q * N + i] = Rnew[q];
            }
            if (bits) atomicOr(status, bits);
        } else {
            const float* pc = ring + ((k + 1) % 4) * kZmPlane;
#pragma unroll
            for (int q = 0; q < 6; ++q) c[q] = pc[(q * kZmHY + ry) * kZmHX + rc];
        }
        // densities of the new populations (same summation order as elsewhere)
        float d[NCOMP];
        if (FUSED || PARTS) {
#pragma unroll
            for (int s = 0; s < NCOMP; ++s) d[s] = rest[s];
            dens_store<NCOMP>(drho, i, d);
        } else {
            const bool ok = mbar_wait_bounded_parity(bar_a, (unsigned)(k & 1));
            if (__syncthreads_or(!ok)) {
                if (leader) {
                    atomicOr(status, kStTimeout);
                    mbar_wait_bounded_parity(bar_a, (unsigned)(k & 1));  // bounded: let the copy land
                }
                return;
            }
#pragma unroll
            for (int s = 0; s < NCOMP; ++s) {
                d[s] = rest[s];
#pragma unroll
                for (int a = 1; a < L::Q; ++a) d[s] += pop_get(sP[(s * (L::Q - 1) + a - 1) * T + t]);
            }
            dens_store<NCOMP>(drho, i, d);
        }
        if (p.feedback != 0.0f) store_feedback<L, NCOMP>(c, d, p, Q, N, i);
        if (more) store_plane((k + 3) % 4, vi, vh);
        __syncthreads();
    }
}

template <class PT, int NCOMP, bool FD, int MODE>
__global__ void __launch_bounds__(kZmBX * kZmBY, 2) k_post_zm(const __grid_constant__ CUtensorMap tm_fnew,
                                                               const float* __restrict__ frest,
                                                               float* __restrict__ drho, const float* __restrict__ Ct,
                                                               float* __restrict__ Cout, float* __restrict__ R,
                                                               const float* __restrict__ u, float* __restrict__ Q,
                                                               unsigned* __restrict__ status, StepParams p, int zs,
                                                               int rev, const PT* __restrict__ fnew, int zl,
                                                               const float* __restrict__ part, int part_by,
                                                               int part_bz) {
    const int x0 = (rev ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x) * kZmBX;
    const int y0 = p.ylo + (rev ? (int)(gridDim.y - 1 - blockIdx.y) : (int)blockIdx.y) * kZmBY;
    const int z0 = (rev ? (int)(gridDim.z - 1 - blockIdx.z) : (int)blockIdx.z) * zs;
    post_column<PT, NCOMP, FD, MODE>(&tm_fnew, frest, drho, Ct, Cout, R, u, Q, status, p, x0, y0, z0, zs, fnew, zl,
                                     part, part_by, part_bz);
}

// Batched ensemble form: block i (taken in reverse order, so the pass starts on
// the tiles the lattice kernel touched last) runs column item i - start[m] of
// member m: columns x-fastest, then y, then z-segments of the member's zs planes.
template <class PT, int NCOMP, bool FD>
__global__ void __launch_bounds__(kZmBX * kZmBY, 2)
    k_post_batch(const EnsMember* __restrict__ members, const int* __restrict__ start, int nm, int parity) {
    const int item = (int)(gridDim.x - 1 - blockIdx.x);
    const int m = batch_member(start, nm, item);
    const EnsMember& M = members[m];
    const int t = item - start[m];
    const StepParams p = M.p;
    const StepBufs b = M.b[parity];
    const int r = t / M.ncx;
    const CUtensorMap* tm = &M.tm_post[1 - (M.cur0 ^ parity)];      // the populations just written
    if ((threadIdx.x | threadIdx.y) == 0) tensormap_acquire(tm);  // the thread that issues the copies
    post_column<PT, NCOMP, FD, 0>(tm, b.frest, b.drho, b.Cin, b.Cout, b.R, b.u, b.Q, b.status, p,
                                      (t % M.ncx) * kZmBX, (r % M.ncy) * kZmBY, (r / M.ncy) * M.zs, M.zs,
                                      static_cast<const PT*>(b.fout), 1);
}

// Densities and feedback stress of a given state (no time step).
template <class PT, class L, int NCOMP>
__global__ void __launch_bounds__(128) k_pre(const PT* __restrict__ f, const float* __restrict__ frest,
                                             float* __restrict__ drho,
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
        d[s] = __ldg(frest + s * N + i);
#pragma unroll
        for (int a = 1; a < L::Q; ++a) d[s] += pop_load(f + (s * (L::Q - 1) + a - 1) * N + i);
    }
    dens_store<NCOMP>(drho, i, d);
    float c[L::NC];
#pragma unroll
    for (int k = 0; k < L::NC; ++k) c[k] = __ldg(Ct + k * N + i);
    if (p.feedback != 0.0f) store_feedback<L, NCOMP>(c, d, p, Q, N, i);
}

}  // namespace

cudaError_t launch_post(int lattice, int ncomp, bool fd, const StepParams& p, const StepBufs& b,
                        const void* fnew, cudaStream_t s, int rev) {
    dim3 blk(32, 4, 1), grd((p.nx + 31) / 32, (p.ny + 3) / 4, p.nz);
#define VEFD_POST(LT, NCP)                                                                                  \
    do {                                                                                                    \
        const PT* fn = static_cast<const PT*>(fnew);                                                        \
        if (fd)                                                                                             \
            k_post<PT, LT, NCP, true><<<grd, blk, 0, s>>>(fn, b.frest, b.drho, b.Cin, b.Cout, b.R, b.u, b.Q, b.status, p,  \
                                                          rev);                                             \
        else                                                                                                \
            k_post<PT, LT, NCP, false><<<grd, blk, 0, s>>>(fn, b.frest, b.drho, b.Cin, b.Cout, b.R, b.u, b.Q, b.status, p, \
                                                           rev);                                            \
    } while (0)
    VEFD_WITH_PT(p.prec, {
        if (lattice == 1) {
            if (ncomp == 2) VEFD_POST(D3Q19, 2);
            else VEFD_POST(D3Q19, 1);
        } else {
            if (ncomp == 2) VEFD_POST(D2Q9, 2);
            else VEFD_POST(D2Q9, 1);
        }
    });
#undef VEFD_POST
    return cudaGetLastError();
}

namespace {
template <class PT, class L, int NCOMP, int BX, int BY, int BZ>
cudaError_t post_tma(bool fd, const CUtensorMap* tm, const StepParams& p, const StepBufs& b, cudaStream_t s, int rev) {
    constexpr int smem = NCOMP * (L::Q - 1) * BX * BY * BZ * (int)sizeof(PT);
    dim3 blk(BX, BY, BZ), grd((p.nx + BX - 1) / BX, (p.ny + BY - 1) / BY, (p.nz + BZ - 1) / BZ);
    if (fd)
        k_post_tma<PT, L, NCOMP, true, BX, BY, BZ><<<grd, blk, smem, s>>>(*tm, b.frest, b.drho, b.Cin, b.Cout, b.R, b.u, b.Q,
                                                                           b.status, p, rev);
    else
        k_post_tma<PT, L, NCOMP, false, BX, BY, BZ><<<grd, blk, smem, s>>>(*tm, b.frest, b.drho, b.Cin, b.Cout, b.R, b.u, b.Q,
                                                                            b.status, p, rev);
    return cudaGetLastError();
}
}  // namespace

cudaError_t launch_post_tma(int lattice, int ncomp, bool fd, const StepParams& p, const StepBufs& b,
                            const void* tensor_map_fnew, cudaStream_t s, int rev) {
    const CUtensorMap* tm = static_cast<const CUtensorMap*>(tensor_map_fnew);
    cudaError_t e = cudaSuccess;
    VEFD_WITH_PT(p.prec, {
        if (lattice == 1)
            e = ncomp == 2 ? post_tma<PT, D3Q19, 2, 32, 4, 2>(fd, tm, p, b, s, rev)
                           : post_tma<PT, D3Q19, 1, 32, 4, 2>(fd, tm, p, b, s, rev);
        else
            e = ncomp == 2 ? post_tma<PT, D2Q9, 2, 32, 8, 1>(fd, tm, p, b, s, rev)
                           : post_tma<PT, D2Q9, 1, 32, 8, 1>(fd, tm, p, b, s, rev);
    });
    return e;
}

bool post_zm_eligible(int lattice, int nx, int ny) { return lattice == 1 && nx % kZmBX == 0 && ny % kZmBY == 0; }

namespace {
int g_sm_count = 0;

template <class PT, int NCOMP, bool FD, int MODE>
cudaError_t post_zm(const CUtensorMap* tm, const StepParams& p, const StepBufs& b, cudaStream_t s, int rev, int zl,
                    Parts parts = Parts{}) {
    constexpr bool FUSED = MODE == 1;
    constexpr int smem = MODE != 0 ? 4 * kZmPlane * (int)sizeof(float) : zm_smem_bytes<PT, NCOMP>();
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e =
            cudaFuncSetAttribute(k_post_zm<PT, NCOMP, FD, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    if (!g_sm_count) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) g_sm_count = 152;
    }
    // one wave: split z so that the columns x z-segments fill two blocks per SM
    const int bxy = (p.nx / kZmBX) * (p.ny / kZmBY);
    int nzb = (2 * g_sm_count) / bxy;
    if (nzb < 1) nzb = 1;
    if (nzb > p.nz) nzb = p.nz;
    const int zs = p.post_zs > 0 ? (p.post_zs < p.nz ? p.post_zs : p.nz) : (p.nz + nzb - 1) / nzb;
    nzb = (p.nz + zs - 1) / zs;
    dim3 blk(kZmBX, kZmBY, 1), grd(p.nx / kZmBX, (p.yhi - p.ylo) / kZmBY, nzb);
    // FUSED reads the partial densities of the new time level and completes them in place
    float* dens = FUSED ? b.drho_next : b.drho;
    const CUtensorMap dummy{};
    return launch_pdl(p.pdl != 0, k_post_zm<PT, NCOMP, FD, MODE>, grd, blk, smem, s, MODE != 0 ? dummy : *tm,
                      (const float*)b.frest, dens, (const float*)b.Cin, b.Cout, b.R, (const float*)b.u, b.Q, b.status,
                      p, zs, rev, static_cast<const PT*>(b.fout), zl, (const float*)parts.part, parts.by, parts.bz);
}
}  // namespace

cudaError_t launch_post_zm(int ncomp, bool fd, const StepParams& p, const StepBufs& b, const void* tensor_map_fnew,
                           cudaStream_t s, int rev, Parts parts) {
    const CUtensorMap* tm = static_cast<const CUtensorMap*>(tensor_map_fnew);
    cudaError_t e = cudaSuccess;
    if (parts.part && (parts.by < 2 || parts.bz < 2)) return cudaErrorInvalidValue;
    VEFD_WITH_PT(p.prec, {
        if (parts.part) {
            if (ncomp == 2)
                e = fd ? post_zm<PT, 2, true, 2>(tm, p, b, s, rev, 1, parts)
                       : post_zm<PT, 2, false, 2>(tm, p, b, s, rev, 1, parts);
            else
                e = fd ? post_zm<PT, 1, true, 2>(tm, p, b, s, rev, 1, parts)
                       : post_zm<PT, 1, false, 2>(tm, p, b, s, rev, 1, parts);
        } else if (ncomp == 2) {
            e = fd ? post_zm<PT, 2, true, 0>(tm, p, b, s, rev, 1) : post_zm<PT, 2, false, 0>(tm, p, b, s, rev, 1);
        } else {
            e = fd ? post_zm<PT, 1, true, 0>(tm, p, b, s, rev, 1) : post_zm<PT, 1, false, 0>(tm, p, b, s, rev, 1);
        }
    });
    return e;
}

cudaError_t launch_post_zm_fused(int ncomp, bool fd, const StepParams& p, const StepBufs& b, cudaStream_t s, int zs,
                                 int rev) {
    cudaError_t e = cudaSuccess;
    VEFD_WITH_PT(p.prec, {
        if (ncomp == 2)
            e = fd ? post_zm<PT, 2, true, 1>(nullptr, p, b, s, rev, zs) : post_zm<PT, 2, false, 1>(nullptr, p, b, s, rev, zs);
        else
            e = fd ? post_zm<PT, 1, true, 1>(nullptr, p, b, s, rev, zs) : post_zm<PT, 1, false, 1>(nullptr, p, b, s, rev, zs);
    });
    return e;
}

namespace {
template <class PT, int NCOMP, bool FD>
cudaError_t post_batch(const EnsMember* members, const int* start, int nm, int items, int parity, bool pdl,
                       cudaStream_t s) {
    constexpr int smem = zm_smem_bytes<PT, NCOMP>();
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_post_batch<PT, NCOMP, FD>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    return launch_pdl(pdl, k_post_batch<PT, NCOMP, FD>, dim3(items), dim3(kZmBX, kZmBY, 1), smem, s, members, start,
                      nm, parity);
}
}  // namespace

cudaError_t launch_post_batch(int ncomp, int prec, bool fd, const EnsMember* members, const int* start, int nm,
                              int items, int parity, bool pdl, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    VEFD_WITH_PT(prec, {
        if (ncomp == 2)
            e = fd ? post_batch<PT, 2, true>(members, start, nm, items, parity, pdl, s)
                   : post_batch<PT, 2, false>(members, start, nm, items, parity, pdl, s);
        else
            e = fd ? post_batch<PT, 1, true>(members, start, nm, items, parity, pdl, s)
                   : post_batch<PT, 1, false>(members, start, nm, items, parity, pdl, s);
    });
    return e;
}

cudaError_t launch_pre(int lattice, int ncomp, const StepParams& p, const StepBufs& b, cudaStream_t s) {
    dim3 blk(32, 4, 1), grd((p.nx + 31) / 32, (p.ny + 3) / 4, p.nz);
    VEFD_WITH_PT(p.prec, {
        const PT* f = static_cast<const PT*>(b.fin);
        if (lattice == 1) {
            if (ncomp == 2) k_pre<PT, D3Q19, 2><<<grd, blk, 0, s>>>(f, b.frest, b.drho, b.Cin, b.Q, p);
            else k_pre<PT, D3Q19, 1><<<grd, blk, 0, s>>>(f, b.frest, b.drho, b.Cin, b.Q, p);
        } else {
            if (ncomp == 2) k_pre<PT, D2Q9, 2><<<grd, blk, 0, s>>>(f, b.frest, b.drho, b.Cin, b.Q, p);
            else k_pre<PT, D2Q9, 1><<<grd, blk, 0, s>>>(f, b.frest, b.drho, b.Cin, b.Q, p);
        }
    });
    return cudaGetLastError();
}

}  // namespace vefd
