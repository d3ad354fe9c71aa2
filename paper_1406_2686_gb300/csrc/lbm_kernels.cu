// Lattice-Boltzmann kernels of the hybrid step (Sec. 2 of Gupta,
// Sbragaglia & Scagliarini):
//   k_moments  : rho_s - rho_ref_s = sum_a fd_a^s                     (Sec. 2, moments)
//   k_lattice  : per node, in registers: moments, Shan-Chen force (Eq. SCforce),
//                polymer feedback (eta_P/tau_P) div[(f C - I) m(phi)] (Eq. NS,
//                last equation of Sec. 2), velocity (Eq. equilibrium:vel),
//                viscosity (Eq. smoothingvisco), forced BGK collision (Eq. LB)
//                and push streaming with half-way bounce-back on moving walls.
// One thread per node; a warp covers 32 consecutive x, so every population
// plane is read and written as contiguous 128-byte rows (writes of moving
// populations are shifted by one element in x).
#include "vefd_internal.cuh"

namespace vefd {

namespace {

__device__ __forceinline__ int wrap1(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Row index of a neighbour in y: periodic, or clamped to the wall row (the
// Shan-Chen density across a wall equals the adjacent fluid row).
__device__ __forceinline__ int y_clamped(int y, int ny, int walls) {
    if (walls) return y < 0 ? 0 : (y >= ny ? ny - 1 : y);
    return wrap1(y, ny);
}

template <class L, int NCOMP>
__global__ void __launch_bounds__(128) k_moments(const float* __restrict__ fd, float* __restrict__ drho,
                                                 StepParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const long long N = p.N;
    const long long i = ((long long)z * p.ny + y) * p.nx + x;
#pragma unroll
    for (int s = 0; s < NCOMP; ++s) {
        float d = 0.0f;
#pragma unroll
        for (int a = 0; a < L::Q; ++a) d += __ldg(fd + (s * L::Q + a) * N + i);
        drho[s * N + i] = d;
    }
}

// Feedback stress components needed for the divergence at one neighbour:
// Q = (f C - I) m(phi) = (f Ct + (f - 1) I) m(phi), with f - 1 = tr Ct / (L^2 - 3 - tr Ct).
template <class L>
struct QTensor {
    float q[L::NC];
};

template <class L, int NCOMP>
__device__ __forceinline__ QTensor<L> feedback_stress(const float* __restrict__ Ct, long long N, long long j,
                                                      float drA, float drB, const StepParams& p) {
    QTensor<L> r;
    float c[L::NC];
#pragma unroll
    for (int k = 0; k < L::NC; ++k) c[k] = __ldg(Ct + k * N + j);
    float tr;
    if (L::NC == 6) tr = c[0] + c[3] + c[5];
    else tr = c[0] + c[2] + c[3];
    const float fm1 = tr / (p.L2m3 - tr);
    const float f = 1.0f + fm1;
    float m = 1.0f;
    if (p.phase != 0) {
        // one component: phi = 1 everywhere
        float phi = 1.0f;
        if (NCOMP == 2) {
            const float ra = p.rho_ref[0] + drA, rb = p.rho_ref[1] + drB;
            phi = (ra - rb) / (ra + rb);
        }
        const float t = tanhf(phi * p.inv_delta);
        m = p.phase > 0 ? 0.5f * (1.0f + t) : 0.5f * (1.0f - t);
    }
#pragma unroll
    for (int k = 0; k < L::NC; ++k) {
        bool diag = (L::NC == 6) ? (k == 0 || k == 3 || k == 5) : (k == 0 || k == 2 || k == 3);
        r.q[k] = (f * c[k] + (diag ? fm1 : 0.0f)) * m;
    }
    return r;
}

// index of tensor component (i, j) in the stored order
template <class L>
__device__ __forceinline__ constexpr int sym(int i, int j) {
    if (L::NC == 6) {
        return (i == 0) ? j : (i == 1 ? (j == 0 ? 1 : (j == 1 ? 3 : 4)) : (j == 0 ? 2 : (j == 1 ? 4 : 5)));
    } else {  // xx xy yy zz
        return (i == 0) ? (j == 0 ? 0 : (j == 1 ? 1 : -1))
             : (i == 1 ? (j == 0 ? 1 : (j == 1 ? 2 : -1)) : (j == 2 ? 3 : -1));
    }
}

template <class L, int NCOMP, bool STREAM>
__global__ void __launch_bounds__(128) k_lattice(StepBufs b, StepParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= p.nx || y >= p.ny) return;
    const int nx = p.nx, ny = p.ny, nz = p.nz;
    const long long N = p.N;
    const long long i = ((long long)z * ny + y) * nx + x;

    // --- moments (same summation order as k_moments) -----------------------
    float f[NCOMP][L::Q];
    float dr[NCOMP];
    float jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
    for (int s = 0; s < NCOMP; ++s) {
        dr[s] = 0.0f;
#pragma unroll
        for (int a = 0; a < L::Q; ++a) {
            f[s][a] = __ldg(b.fin + (s * L::Q + a) * N + i);
            dr[s] += f[s][a];
        }
    }
#pragma unroll
    for (int s = 0; s < NCOMP; ++s)
#pragma unroll
        for (int a = 1; a < L::Q; ++a) {
            if (L::cx(a)) jx += L::cx(a) * f[s][a];
            if (L::cy(a)) jy += L::cy(a) * f[s][a];
            if (L::cz(a)) jz += L::cz(a) * f[s][a];
        }
    float rs[NCOMP];
    float rho = 0.0f;
#pragma unroll
    for (int s = 0; s < NCOMP; ++s) {
        rs[s] = p.rho_ref[s] + dr[s];
        rho += rs[s];
    }
    const float inv_rho = 1.0f / rho;

    // neighbour coordinates
    const int xm = wrap1(x - 1, nx), xp = wrap1(x + 1, nx);
    const int zm = wrap1(z - 1, nz), zp = wrap1(z + 1, nz);
    const int ymc = y_clamped(y - 1, ny, p.walls), ypc = y_clamped(y + 1, ny, p.walls);
    auto nbr = [&](int dx, int dy, int dz) -> long long {
        const int xx = dx < 0 ? xm : (dx > 0 ? xp : x);
        const int yy = dy < 0 ? ymc : (dy > 0 ? ypc : y);
        const int zz = dz < 0 ? zm : (dz > 0 ? zp : z);
        return ((long long)zz * ny + yy) * nx + xx;
    };

    // --- Shan-Chen force: g_s = -G rho_s sum_a w_a rho_s'(x + c_a) c_a ---------
    // The sum uses density deviations: sum_a w_a c_a rho_ref = 0.
    float g[NCOMP][3];
    float axis_dr[NCOMP][6];  // deviations at -x +x -y +y -z +z (for phi of the feedback)
#pragma unroll
    for (int s = 0; s < NCOMP; ++s) g[s][0] = g[s][1] = g[s][2] = 0.0f;
    if (NCOMP == 2) {
        float acc[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
        for (int a = 1; a < L::Q; ++a) {
            const long long j = nbr(L::cx(a), L::cy(a), L::cz(a));
            const float wa = L::w(a);
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const float dn = __ldg(b.drho + s * N + j);
                // axis neighbours are remembered for the order parameter
                if (L::cy(a) == 0 && L::cz(a) == 0) axis_dr[s][L::cx(a) < 0 ? 0 : 1] = dn;
                if (L::cx(a) == 0 && L::cz(a) == 0) axis_dr[s][L::cy(a) < 0 ? 2 : 3] = dn;
                if (L::cx(a) == 0 && L::cy(a) == 0) axis_dr[s][L::cz(a) < 0 ? 4 : 5] = dn;
                const float t = wa * dn;
                if (L::cx(a)) acc[s][0] += L::cx(a) * t;
                if (L::cy(a)) acc[s][1] += L::cy(a) * t;
                if (L::cz(a)) acc[s][2] += L::cz(a) * t;
            }
        }
        // force on A from B's neighbourhood and on B from A's
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            g[0][k] = -p.G * rs[0] * acc[1][k];
            g[1 % NCOMP][k] = -p.G * rs[NCOMP - 1] * acc[0][k];
        }
    } else {
#pragma unroll
        for (int q = 0; q < 6; ++q) axis_dr[0][q] = 0.0f;
    }

    // --- polymer feedback force F_p = (eta_P/tau_P) div Q ----------------------
    float Fp[3] = {0.0f, 0.0f, 0.0f};
    if (p.feedback != 0.0f) {
        const float drA0 = dr[0], drB0 = NCOMP == 2 ? dr[NCOMP - 1] : 0.0f;
        auto q_at = [&](long long j, int axis_slot) -> QTensor<L> {
            float dA = 0.f, dB = 0.f;
            if (NCOMP == 2) {
                if (axis_slot < 0) {
                    dA = drA0;
                    dB = drB0;
                } else {
                    dA = axis_dr[0][axis_slot];
                    dB = axis_dr[NCOMP - 1][axis_slot];
                }
            }
            return feedback_stress<L, NCOMP>(b.Cin, N, j, dA, dB, p);
        };
        float div[3] = {0.f, 0.f, 0.f};
        // x: periodic central difference of Q_x.
        {
            QTensor<L> qm = q_at(nbr(-1, 0, 0), 0), qp = q_at(nbr(1, 0, 0), 1);
#pragma unroll
            for (int jj = 0; jj < L::D; ++jj) div[jj] += 0.5f * (qp.q[sym<L>(0, jj)] - qm.q[sym<L>(0, jj)]);
        }
        // y: central difference, or one-sided at walls (linear-extrapolation ghost).
        {
            QTensor<L> qm, qp;
            float h = 0.5f;
            if (p.walls && y == 0) {
                qm = q_at(i, -1);
                qp = q_at(nbr(0, 1, 0), 3);
                h = 1.0f;
            } else if (p.walls && y == ny - 1) {
                qm = q_at(nbr(0, -1, 0), 2);
                qp = q_at(i, -1);
                h = 1.0f;
            } else {
                qm = q_at(nbr(0, -1, 0), 2);
                qp = q_at(nbr(0, 1, 0), 3);
            }
#pragma unroll
            for (int jj = 0; jj < L::D; ++jj) div[jj] += h * (qp.q[sym<L>(1, jj)] - qm.q[sym<L>(1, jj)]);
        }
        if (L::D == 3) {
            QTensor<L> qm = q_at(nbr(0, 0, -1), 4), qp = q_at(nbr(0, 0, 1), 5);
#pragma unroll
            for (int jj = 0; jj < 3; ++jj) div[jj] += 0.5f * (qp.q[sym<L>(2, jj)] - qm.q[sym<L>(2, jj)]);
        }
#pragma unroll
        for (int k = 0; k < 3; ++k) Fp[k] = p.feedback * div[k];
    }

    // --- velocity with half the total force (Eq. equilibrium:vel) --------------
    float Fb[3];  // polymer + external, shared by rho_s / rho
#pragma unroll
    for (int k = 0; k < 3; ++k) Fb[k] = Fp[k] + p.fext[k];
    float Ftot[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        Ftot[k] = Fb[k];
#pragma unroll
        for (int s = 0; s < NCOMP; ++s) Ftot[k] += g[s][k];
    }
    const float ux = (jx + 0.5f * Ftot[0]) * inv_rho;
    const float uy = (jy + 0.5f * Ftot[1]) * inv_rho;
    const float uz = L::D == 3 ? (jz + 0.5f * Ftot[2]) * inv_rho : 0.0f;
    const float usq = ux * ux + uy * uy + uz * uz;

    // --- relaxation time: rho c_s^2 (tau - 1/2) = eta_A f_+ + eta_B f_- --------
    float eta;
    if (NCOMP == 2) {
        const float phi = (rs[0] - rs[NCOMP - 1]) * inv_rho;
        const float t = tanhf(phi * p.inv_delta);
        eta = p.eta_A * 0.5f * (1.0f + t) + p.eta_B * 0.5f * (1.0f - t);
    } else {
        eta = p.eta_A * 0.5f * (1.0f + tanhf(p.inv_delta));
        eta += p.eta_B * 0.5f * (1.0f - tanhf(p.inv_delta));
    }
    const float tau = 0.5f + eta * 3.0f * inv_rho;
    const float omega = 1.0f / tau;
    const float src_w = 1.0f - 0.5f * omega;

    // --- guards -----------------------------------------------------------------
    {
        unsigned bits = 0;
        if (isnan(usq) || isnan(rho)) bits |= kStNan;
        else if (usq > 0.09f) bits |= kStMach;
        if (!(rho > 0.0f) && !isnan(rho)) bits |= kStRho;
        if (bits) atomicOr(b.status, bits);
    }

    if (!STREAM) {
        b.u[i] = ux;
        b.u[N + i] = uy;
        if (L::D == 3) b.u[2 * N + i] = uz;
        if (b.dbg) {
            for (int k = 0; k < 3; ++k) {
                b.dbg[k * N + i] = g[0][k];
                b.dbg[(3 + k) * N + i] = NCOMP == 2 ? g[NCOMP - 1][k] : 0.0f;
                b.dbg[(6 + k) * N + i] = Fp[k];
            }
            b.dbg[9 * N + i] = tau;
        }
        return;
    }
    b.u[i] = ux;
    b.u[N + i] = uy;
    if (L::D == 3) b.u[2 * N + i] = uz;

    // --- collision and streaming per component --------------------------------
    const float uw3 = 3.0f * p.u_wall;
#pragma unroll
    for (int s = 0; s < NCOMP; ++s) {
        const float share = rs[s] * inv_rho;
        const float Fx = g[s][0] + share * Fb[0];
        const float Fy = g[s][1] + share * Fb[1];
        const float Fz = g[s][2] + share * Fb[2];
        const float uF = ux * Fx + uy * Fy + uz * Fz;
        const float rsv = rs[s];
        const float drs = dr[s];
        // The collision conserves mass exactly: sum_a f*_a = sum_a f_a.  The rest
        // population is therefore taken as that remainder after the moving ones,
        // so that the FP32 lattice weights (whose sum is 1 + 1.5e-8) leave no
        // systematic mass bias; what remains is unbiased rounding.
        float moved = 0.0f;
#pragma unroll
        for (int a = 1; a <= L::Q; ++a) {
            const int ai = a == L::Q ? 0 : a;  // rest population last
            const int cx = L::cx(ai), cy = L::cy(ai), cz = L::cz(ai);
            const float wa = L::w(ai);
            const float cu = cx * ux + cy * uy + cz * uz;
            const float cF = cx * Fx + cy * Fy + cz * Fz;
            // deviation equilibrium: E_a - w_a rho_ref = w_a [drho + rho (3 cu + 4.5 cu^2 - 1.5 u^2)]
            const float Ed = wa * (drs + rsv * (3.0f * cu + 4.5f * cu * cu - 1.5f * usq));
            const float S = wa * (3.0f * (cF - uF) + 9.0f * cu * cF);
            float fpost;
            if (ai == 0) {
                fpost = drs - moved;
            } else {
                fpost = f[s][ai] + omega * (Ed - f[s][ai]) + src_w * S;
                moved += fpost;
            }
            int yt = y + cy;
            if (p.walls && (yt < 0 || yt >= ny)) {
                // half-way bounce-back into the opposite direction at this node,
                // moving wall +U (lower) / -U (upper): -2 w rho_s (c.U)/c_s^2
                const float Uw = yt < 0 ? uw3 : -uw3;
                b.fout[(s * L::Q + opposite(ai)) * N + i] = fpost - 2.0f * wa * rsv * (float)cx * Uw;
            } else {
                yt = wrap1(yt, ny);
                const int xt = cx < 0 ? xm : (cx > 0 ? xp : x);
                const int zt = cz < 0 ? zm : (cz > 0 ? zp : z);
                b.fout[(s * L::Q + ai) * N + ((long long)zt * ny + yt) * nx + xt] = fpost;
            }
        }
    }
}

template <class L, int NCOMP>
__global__ void k_init_eq(const float* __restrict__ rhoA, const float* __restrict__ rhoB,
                          const float* __restrict__ u, float* __restrict__ fd, StepParams p) {
    const long long N = p.N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
        const float ux = u ? u[i] : 0.0f, uy = u ? u[N + i] : 0.0f;
        const float uz = (u && L::D == 3) ? u[2 * N + i] : 0.0f;
        const float usq = ux * ux + uy * uy + uz * uz;
#pragma unroll
        for (int s = 0; s < NCOMP; ++s) {
            const float r = s == 0 ? rhoA[i] : rhoB[i];
            const float d = r - p.rho_ref[s];
            // moving populations first; the rest population carries the remainder
            // so that the stored deviations sum to rho - rho_ref
            float moved = 0.0f;
#pragma unroll
            for (int a = 1; a < L::Q; ++a) {
                const float cu = L::cx(a) * ux + L::cy(a) * uy + L::cz(a) * uz;
                const float e = L::w(a) * (d + r * (3.0f * cu + 4.5f * cu * cu - 1.5f * usq));
                fd[(s * L::Q + a) * N + i] = e;
                moved += e;
            }
            fd[(s * L::Q) * N + i] = d - moved;
        }
    }
}

template <class L, int NCOMP>
__global__ void k_pops_convert(const float* __restrict__ src, float* __restrict__ dst, int to_abs, StepParams p) {
    const long long N = p.N;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < N; i += (long long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int s = 0; s < NCOMP; ++s)
#pragma unroll
            for (int a = 0; a < L::Q; ++a) {
                const float sh = L::w(a) * p.rho_ref[s];
                const long long k = (s * L::Q + a) * N + i;
                dst[k] = to_abs ? src[k] + sh : src[k] - sh;
            }
    }
}

int grid_1d(long long n) {
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

dim3 node_grid(const StepParams& p) { return dim3((p.nx + 31) / 32, (p.ny + 3) / 4, p.nz); }

}  // namespace

cudaError_t launch_moments(int lattice, int ncomp, const StepParams& p, const StepBufs& b, cudaStream_t s) {
    dim3 blk(32, 4, 1), grd = node_grid(p);
    if (lattice == 1) {
        if (ncomp == 2) k_moments<D3Q19, 2><<<grd, blk, 0, s>>>(b.fin, b.drho, p);
        else k_moments<D3Q19, 1><<<grd, blk, 0, s>>>(b.fin, b.drho, p);
    } else {
        if (ncomp == 2) k_moments<D2Q9, 2><<<grd, blk, 0, s>>>(b.fin, b.drho, p);
        else k_moments<D2Q9, 1><<<grd, blk, 0, s>>>(b.fin, b.drho, p);
    }
    return cudaGetLastError();
}

cudaError_t launch_lattice(int lattice, int ncomp, bool stream_pops, const StepParams& p, const StepBufs& b,
                           cudaStream_t s) {
    dim3 blk(32, 4, 1), grd = node_grid(p);
#define VEFD_LAT(LT, NCP)                                                         \
    do {                                                                          \
        if (stream_pops) k_lattice<LT, NCP, true><<<grd, blk, 0, s>>>(b, p);      \
        else k_lattice<LT, NCP, false><<<grd, blk, 0, s>>>(b, p);                 \
    } while (0)
    if (lattice == 1) {
        if (ncomp == 2) VEFD_LAT(D3Q19, 2);
        else VEFD_LAT(D3Q19, 1);
    } else {
        if (ncomp == 2) VEFD_LAT(D2Q9, 2);
        else VEFD_LAT(D2Q9, 1);
    }
#undef VEFD_LAT
    return cudaGetLastError();
}

cudaError_t launch_init_equilibrium(int lattice, int ncomp, const StepParams& p, const float* rhoA,
                                    const float* rhoB, const float* u, float* fd, cudaStream_t s) {
    const int g = grid_1d(p.N);
    if (lattice == 1) {
        if (ncomp == 2) k_init_eq<D3Q19, 2><<<g, 256, 0, s>>>(rhoA, rhoB, u, fd, p);
        else k_init_eq<D3Q19, 1><<<g, 256, 0, s>>>(rhoA, rhoB, u, fd, p);
    } else {
        if (ncomp == 2) k_init_eq<D2Q9, 2><<<g, 256, 0, s>>>(rhoA, rhoB, u, fd, p);
        else k_init_eq<D2Q9, 1><<<g, 256, 0, s>>>(rhoA, rhoB, u, fd, p);
    }
    return cudaGetLastError();
}

cudaError_t launch_pops_convert(int lattice, int ncomp, const StepParams& p, const float* src, float* dst,
                                int to_absolute, cudaStream_t s) {
    const int g = grid_1d(p.N);
    if (lattice == 1) {
        if (ncomp == 2) k_pops_convert<D3Q19, 2><<<g, 256, 0, s>>>(src, dst, to_absolute, p);
        else k_pops_convert<D3Q19, 1><<<g, 256, 0, s>>>(src, dst, to_absolute, p);
    } else {
        if (ncomp == 2) k_pops_convert<D2Q9, 2><<<g, 256, 0, s>>>(src, dst, to_absolute, p);
        else k_pops_convert<D2Q9, 1><<<g, 256, 0, s>>>(src, dst, to_absolute, p);
    }
    return cudaGetLastError();
}

}  // namespace vefd
