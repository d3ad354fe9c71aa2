#pragma once
// Lattice-Boltzmann kernel templates of the hybrid step (Sec. 2 of Gupta,
// Sbragaglia & Scagliarini), instantiated by lbm_kernels.cu (single
// relaxation time) and lbm_mrt.cu (relaxation in moment space):
//   k_moments     rho_s - rho_ref_s = sum_a fd_a^s                    (Sec. 2, moments)
//   k_lattice     per node: moments, Shan-Chen force (Eq. SCforce), polymer
//                 feedback (eta_P/tau_P) div[(f C - I) m(phi)] (Eq. NS and the
//                 last equation of Sec. 2) from the per-node stress written by
//                 the densities/FD pass, velocity (Eq. equilibrium:vel),
//                 viscosity (Eq. smoothingvisco), forced collision (Eq. LB)
//                 and push streaming with half-way bounce-back on moving walls.
//                 Populations held in registers; used for any lattice size and
//                 for the macroscopic (non-streaming) passes.
//   k_lattice_tma the same step for lattices whose rows are 16-byte multiples:
//                 one TMA copy stages the block's populations (all components
//                 and directions of a 32 x BY x BZ tile) in shared memory while
//                 the threads gather the neighbour densities and the feedback
//                 stress; the collision then reads its populations from shared
//                 memory, which keeps register use low and the memory system busy.
//   k_lattice_pers persistent form of k_lattice_tma with two staging buffers.
// The collision (template COLL) is the single-relaxation-time form of
// Eq. (LB) (0) or its moment-space form with the paper's relaxation times (1).
// One thread per node; a warp covers 32 consecutive x, so every population
// plane is read and written as contiguous 128-byte rows (writes of moving
// populations are shifted by one element in x).
#include <cuda.h>

#include <algorithm>

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

// Tile coordinate along one grid axis, optionally traversed backwards.
__device__ __forceinline__ int tile_index(unsigned b, unsigned n, int rev) { return rev ? (int)(n - 1 - b) : (int)b; }

template <class PT, class L, int NCOMP>
__global__ void __launch_bounds__(128) k_moments(const PT* __restrict__ fd, const float* __restrict__ frest,
                                                 float* __restrict__ drho, StepParams p, int rev) {
    const int x = tile_index(blockIdx.x, gridDim.x, rev) * blockDim.x + threadIdx.x;
    const int y = tile_index(blockIdx.y, gridDim.y, rev) * blockDim.y + threadIdx.y;
    const int z = tile_index(blockIdx.z, gridDim.z, rev);
    if (x >= p.nx || y >= p.ny) return;
    const long long N = p.N;
    const long long i = ((long long)z * p.ny + y) * p.nx + x;
    float d[NCOMP];
#pragma unroll
    for (int s = 0; s < NCOMP; ++s) {
        d[s] = __ldg(frest + s * N + i);
#pragma unroll
        for (int a = 1; a < L::Q; ++a) d[s] += pop_load(fd + (s * (L::Q - 1) + a - 1) * N + i);
    }
    dens_store<NCOMP>(drho, i, d);
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

// index of feedback-stress component (i, j), i, j < D, in the stored order
template <class L>
__device__ __forceinline__ constexpr int qidx(int i, int j) {
    return L::D == 3 ? sym<L>(i, j) : (i + j);  // 2D: xx 0, xy 1, yy 2
}

// Neighbour offsets of one node (periodic images and wall clamping folded in),
// as 32-bit node-index differences: lattices are limited to fewer than 2^31
// population entries, so every plane offset fits.
struct Nbr {
    int x, y, z, ny, i;
    int ox[3], oy[3], oz[3];  // for d = -1, 0, +1 along x, y (clamped at walls), z
    __device__ __forceinline__ int at(int dx, int dy, int dz) const { return i + ox[dx + 1] + oy[dy + 1] + oz[dz + 1]; }
};

__device__ __forceinline__ Nbr make_nbr(int x, int y, int z, const StepParams& p) {
    Nbr n;
    n.x = x;
    n.y = y;
    n.z = z;
    n.ny = p.ny;
    const int nx = p.nx, plane = p.nx * p.ny;
    n.i = (z * p.ny + y) * nx + x;
    n.ox[0] = wrap1(x - 1, nx) - x;
    n.ox[1] = 0;
    n.ox[2] = wrap1(x + 1, nx) - x;
    n.oy[0] = (y_clamped(y - 1, p.ny, p.walls) - y) * nx;
    n.oy[1] = 0;
    n.oy[2] = (y_clamped(y + 1, p.ny, p.walls) - y) * nx;
    n.oz[0] = (wrap1(z - 1, p.nz) - z) * plane;
    n.oz[1] = 0;
    n.oz[2] = (wrap1(z + 1, p.nz) - z) * plane;
    return n;
}

// Neighbour part of the forces at one node:
//   acc[s] = sum_{a>0} w_a (rho_s(x + c_a) - rho_ref_s) c_a   (Shan-Chen lattice sum;
//            sum_a w_a c_a rho_ref = 0 so deviations suffice)
//   Fp     = (eta_P / tau_P) div Q, Q = (f C - I) m(phi) precomputed per node,
//            central differences, one-sided at walls (the linear-extrapolation
//            ghost row v(-1) = 2 v(0) - v(1)).
template <class L, int NCOMP>
__device__ __forceinline__ void neighbour_forces(const StepBufs& b, const StepParams& p, const Nbr& nb,
                                                 float acc[2][3], float Fp[3], float qloc[L::NQ]) {
    const int N = (int)p.N;
    const int i = nb.i;
#pragma unroll
    for (int s = 0; s < 2; ++s) acc[s][0] = acc[s][1] = acc[s][2] = 0.0f;
    if (NCOMP == 2) {
        // sums per weight class (axis, face diagonal), weighted once at the end
        float sa[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}}, sd[2][3] = {{0.f, 0.f, 0.f}, {0.f, 0.f, 0.f}};
#pragma unroll
        for (int a = 1; a < L::Q; ++a) {
            const int j = nb.at(L::cx(a), L::cy(a), L::cz(a));
            const bool axis = L::w(a) == L::w(1);
            float dj[2] = {0.0f, 0.0f};
            if (idx_ok(j, N, b.status)) dens_ldg<2>(b.drho, j, dj);
#pragma unroll
            for (int s = 0; s < 2; ++s) {
                const float t = dj[s];
                float* acc_s = axis ? sa[s] : sd[s];
                if (L::cx(a)) acc_s[0] += L::cx(a) * t;
                if (L::cy(a)) acc_s[1] += L::cy(a) * t;
                if (L::cz(a)) acc_s[2] += L::cz(a) * t;
            }
        }
#pragma unroll
        for (int s = 0; s < 2; ++s)
#pragma unroll
            for (int k = 0; k < 3; ++k) acc[s][k] = L::w(1) * sa[s][k] + L::w(L::Q - 1) * sd[s][k];
    }
    Fp[0] = Fp[1] = Fp[2] = 0.0f;
#pragma unroll
    for (int k = 0; k < L::NQ; ++k) qloc[k] = 0.0f;
    if (p.feedback == 0.0f) return;
    const float* Q = b.Q;
    if (p.coupling == 1) {
        // the stress enters this node's equilibrium instead (Eq. MODEtransformation)
#pragma unroll
        for (int k = 0; k < L::NQ; ++k) qloc[k] = __ldg(Q + k * N + i);
        return;
    }
    float div[3] = {0.f, 0.f, 0.f};
    auto qget = [&](int k, int j) -> float { return idx_ok(j, N, b.status) ? __ldg(Q + k * N + j) : 0.0f; };
    {
        const int jm = nb.at(-1, 0, 0), jp = nb.at(1, 0, 0);
#pragma unroll
        for (int jj = 0; jj < L::D; ++jj) {
            const int k = qidx<L>(0, jj);
            div[jj] += 0.5f * (qget(k, jp) - qget(k, jm));
        }
    }
    {
        int jm = nb.at(0, -1, 0), jp = nb.at(0, 1, 0);
        float h = 0.5f;
        if (p.walls && nb.y == 0) {
            jm = i;
            h = 1.0f;
        } else if (p.walls && nb.y == nb.ny - 1) {
            jp = i;
            h = 1.0f;
        }
#pragma unroll
        for (int jj = 0; jj < L::D; ++jj) {
            const int k = qidx<L>(1, jj);
            div[jj] += h * (qget(k, jp) - qget(k, jm));
        }
    }
    if (L::D == 3) {
        const int jm = nb.at(0, 0, -1), jp = nb.at(0, 0, 1);
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
            const int k = qidx<L>(2, jj);
            div[jj] += 0.5f * (qget(k, jp) - qget(k, jm));
        }
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) Fp[k] = p.feedback * div[k];
}

// Local state after the forces: velocity, relaxation, per-component force and,
// for the equilibrium coupling, the component's share of the polymer stress
// T_s = tq[s] Q with tq[s] = -(rho_s/rho)(eta_P/tau_P).
template <int NCOMP>
struct Local {
    float rs[NCOMP], dr[NCOMP];
    float inv_rho, ux, uy, uz, usq, omega, src_w;
    float F[NCOMP][3];
    float tq[NCOMP];
};

template <class L, int NCOMP>
__device__ __forceinline__ void local_state(const StepParams& p, const float dr[NCOMP], float jx, float jy, float jz,
                                            const float acc[2][3], const float Fp[3], Local<NCOMP>& st,
                                            unsigned* status) {
    float rho = 0.0f;
#pragma unroll
    for (int s = 0; s < NCOMP; ++s) {
        st.dr[s] = dr[s];
        st.rs[s] = p.rho_ref[s] + dr[s];
        rho += st.rs[s];
    }
    st.inv_rho = 1.0f / rho;
    // Shan-Chen: force on A from B's neighbourhood and on B from A's
    float g[NCOMP][3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (NCOMP == 2) {
            g[0][k] = -p.G * st.rs[0] * acc[1][k];
            g[NCOMP - 1][k] = -p.G * st.rs[NCOMP - 1] * acc[0][k];
        } else {
            g[0][k] = 0.0f;
        }
    }
    float Fb[3], Ftot[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        Fb[k] = Fp[k] + p.fext[k];
        Ftot[k] = Fb[k];
#pragma unroll
        for (int s = 0; s < NCOMP; ++s) Ftot[k] += g[s][k];
    }
    // velocity with half the total force (Eq. equilibrium:vel)
    st.ux = (jx + 0.5f * Ftot[0]) * st.inv_rho;
    st.uy = (jy + 0.5f * Ftot[1]) * st.inv_rho;
    st.uz = L::D == 3 ? (jz + 0.5f * Ftot[2]) * st.inv_rho : 0.0f;
    st.usq = st.ux * st.ux + st.uy * st.uy + st.uz * st.uz;
    // rho c_s^2 (tau - 1/2) = eta_A f_+(phi) + eta_B f_-(phi); one component: phi = 1
    const float phi = NCOMP == 2 ? (st.rs[0] - st.rs[NCOMP - 1]) * st.inv_rho : 1.0f;
    const float t = tanhf(phi * p.inv_delta);
    const float eta = p.eta_A * 0.5f * (1.0f + t) + p.eta_B * 0.5f * (1.0f - t);
    const float tau = 0.5f + eta * 3.0f * st.inv_rho;
    st.omega = 1.0f / tau;
    st.src_w = 1.0f - 0.5f * st.omega;
#pragma unroll
    for (int s = 0; s < NCOMP; ++s) {
        const float share = st.rs[s] * st.inv_rho;
#pragma unroll
        for (int k = 0; k < 3; ++k) st.F[s][k] = g[s][k] + share * Fb[k];
        st.tq[s] = p.coupling == 1 ? -share * p.feedback : 0.0f;
    }
    unsigned bits = 0;
    if (isnan(st.usq) || isnan(rho)) bits |= kStNan;
    else if (st.usq > 0.09f) bits |= kStMach;
    if (!(rho > 0.0f) && !isnan(rho)) bits |= kStRho;
    if (bits) atomicOr(status, bits);
}

// Second moments Pi_ij = sum_a c_ai c_aj f_a of stored deviations, in the
// order xx xy xz yy yz zz (2D: xz = yz = zz = 0); the moment-space collision
// needs them per component.
template <class L>
__device__ __forceinline__ void pi_add(float pi[6], int a, float fa) {
    const int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
    if (cx) pi[0] += fa;
    if (cx * cy) pi[1] += (float)(cx * cy) * fa;
    if (cx * cz) pi[2] += (float)(cx * cz) * fa;
    if (cy) pi[3] += fa;
    if (cy * cz) pi[4] += (float)(cy * cz) * fa;
    if (cz) pi[5] += fa;
}

// Collision of every population of every component and push streaming.
// fget(s, a) returns the stored deviation f_a^s of this node; pif[s] the
// second moments of component s's stored deviations (moment-space collision).
//
// Single relaxation time (collision 0).  Opposite directions a and a'
// (c_a' = -c_a) share c.u and c.F up to sign, so each pair is relaxed
// together.  For the deviation equilibrium and the source of Sec. 2
// (Eqs. LB and equilibrium),
//   omega E_a + (1 - omega/2) S_a = w_a [K0 + (c.u)(c.R)] + w_a c.P
// with, per component, K0 = omega (drho - 1.5 rho u.u) - 3 (1 - omega/2) u.F,
// R = 4.5 omega rho u + 9 (1 - omega/2) F and P = 3 omega rho u +
// 3 (1 - omega/2) F; the bracket is even in c and c.P odd, so
//   f*_a  = (1 - omega) f_a  + w_a [K0 + (c.u)(c.R)] + w_a c.P
//   f*_a' = (1 - omega) f_a' + w_a [K0 + (c.u)(c.R)] - w_a c.P.
// The weight is folded into K0, R and P once per weight class.
//
// Moment space (collision 1) with the paper's rates: momentum and
// non-hydrodynamic moments at unit relaxation time, shear and bulk moments at
// omega = 1/tau (tau_b = tau_s).  Writing Eq. (LB) as
// f* = E + S/2 + sum_k (1 - s_k) M_k (m_k - m_k^eq + S^_k/2)/|M_k|^2, only the
// bulk and shear rows survive, and their projections depend on
// g = f - E + S/2 only through its second moment
//   Pi^neq = Pi(f) - rho c_s^2 I - rho u u - T + (u F + F u)/2,
// so
//   f*_a = E_a + S_a/2 + (1 - omega) [h0 + c_a.H.c_a]
// with D3Q19 h0 = -(5/21) tr Pi^neq, H_ii = Pi^neq_ii/6 + (2/21) tr Pi^neq,
// H_ij = Pi^neq_ij/8 (the rows 19c^2 - 30, 3c_x^2 - c^2, c_y^2 - c_z^2,
// c_x c_y, c_y c_z, c_x c_z with squared norms 2394, 36, 12, 4, 4, 4), and
// D2Q9 h0 = -tr Pi^neq/3, H_ii = Pi^neq_ii/2, H_xy = Pi^neq_xy/8 (rows
// 3c^2 - 4, c_x^2 - c_y^2, c_x c_y with norms 36, 4, 4).  The bracket is even
// in c, so pairs are again relaxed together and the populations enter only
// through Pi(f).
//
// collide_emit computes every pair's post-collision values, applies the
// moving-wall term to a population that leaves through a wall (it returns to
// this node in the opposite direction), rounds to the storage type and hands
// the stored values to emit(s, a, va, vb, bounced_a, bounced_b) for a and its
// opposite a + 1; rest[s] receives the component's rest population.
template <class PT, class L, int NCOMP, int COLL, class FGet, class Emit>
__device__ __forceinline__ void collide_emit(const StepParams& p, const Local<NCOMP>& st, const float qloc[L::NQ],
                                             const float (*pif)[6], bool wall_lo, bool wall_hi, FGet fget, Emit emit,
                                             float rest[NCOMP]) {
    const float uw6 = 6.0f * p.u_wall;  // 2 (c.U) / c_s^2 with U = +-u_wall along x
    const float keep = 1.0f - st.omega;
    constexpr bool mrt = COLL == 1;
    // trace of the local feedback stress over the lattice dimensions (equilibrium coupling)
    const float trq = L::NQ == 6 ? qloc[0] + qloc[3] + qloc[5] : qloc[0] + qloc[2];
    constexpr float w_axis = L::w(1), w_diag = L::w(L::Q - 1);
#pragma unroll
    for (int s = 0; s < NCOMP; ++s) {
        const float Fx = st.F[s][0], Fy = st.F[s][1], Fz = st.F[s][2];
        const float uF = st.ux * Fx + st.uy * Fy + st.uz * Fz;
        const float rsv = st.rs[s], drs = st.dr[s];
        // per-component coefficients of the even and odd parts (see above)
        float K0, Rx, Ry, Rz, Px, Py, Pz, tqo;
        // moment-space part (1 - omega)[h0 + c.H.c]
        float kh0 = 0.0f, kH[3] = {0.f, 0.f, 0.f}, kX[3] = {0.f, 0.f, 0.f};  // kX: 2 H_xy, 2 H_yz, 2 H_xz
        if (mrt) {
            K0 = drs - 1.5f * rsv * st.usq - 1.5f * uF;
            const float r45 = 4.5f * rsv;
            Rx = r45 * st.ux + 4.5f * Fx;
            Ry = r45 * st.uy + 4.5f * Fy;
            Rz = r45 * st.uz + 4.5f * Fz;
            const float r3 = 3.0f * rsv;
            Px = r3 * st.ux + 1.5f * Fx;
            Py = r3 * st.uy + 1.5f * Fy;
            Pz = r3 * st.uz + 1.5f * Fz;
            tqo = 4.5f * st.tq[s];
            // Pi^neq of this component (T = tq Q for the equilibrium coupling)
            const float tq = st.tq[s];
            const float dcs = drs * (1.0f / 3.0f);
            float pxx = pif[s][0] - dcs - rsv * st.ux * st.ux + st.ux * Fx;
            float pxy = pif[s][1] - rsv * st.ux * st.uy + 0.5f * (st.ux * Fy + st.uy * Fx);
            float pyy = pif[s][3] - dcs - rsv * st.uy * st.uy + st.uy * Fy;
            float pxz = 0.0f, pyz = 0.0f, pzz = 0.0f;
            if (L::D == 3) {
                pxz = pif[s][2] - rsv * st.ux * st.uz + 0.5f * (st.ux * Fz + st.uz * Fx);
                pyz = pif[s][4] - rsv * st.uy * st.uz + 0.5f * (st.uy * Fz + st.uz * Fy);
                pzz = pif[s][5] - dcs - rsv * st.uz * st.uz + st.uz * Fz;
            }
            if (p.coupling == 1) {
                if (L::NQ == 6) {
                    pxx -= tq * qloc[0];
                    pxy -= tq * qloc[1];
                    pxz -= tq * qloc[2];
                    pyy -= tq * qloc[3];
                    pyz -= tq * qloc[4];
                    pzz -= tq * qloc[5];
                } else {
                    pxx -= tq * qloc[0];
                    pxy -= tq * qloc[1];
                    pyy -= tq * qloc[2];
                }
            }
            if (L::D == 3) {
                const float tr = pxx + pyy + pzz;
                kh0 = keep * (-5.0f / 21.0f) * tr;
                const float t2 = (2.0f / 21.0f) * tr;
                kH[0] = keep * (pxx * (1.0f / 6.0f) + t2);
                kH[1] = keep * (pyy * (1.0f / 6.0f) + t2);
                kH[2] = keep * (pzz * (1.0f / 6.0f) + t2);
                kX[0] = keep * 0.25f * pxy;
                kX[1] = keep * 0.25f * pyz;
                kX[2] = keep * 0.25f * pxz;
            } else {
                kh0 = keep * (-1.0f / 3.0f) * (pxx + pyy);
                kH[0] = keep * 0.5f * pxx;
                kH[1] = keep * 0.5f * pyy;
                kX[0] = keep * 0.25f * pxy;
            }
        } else {
            K0 = st.omega * (drs - 1.5f * rsv * st.usq) - 3.0f * st.src_w * uF;
            const float orho = st.omega * rsv;
            const float r45 = 4.5f * orho, s9 = 9.0f * st.src_w, r3 = 3.0f * orho, s3 = 3.0f * st.src_w;
            Rx = r45 * st.ux + s9 * Fx;
            Ry = r45 * st.uy + s9 * Fy;
            Rz = r45 * st.uz + s9 * Fz;
            Px = r3 * st.ux + s3 * Fx;
            Py = r3 * st.uy + s3 * Fy;
            Pz = r3 * st.uz + s3 * Fz;
            // w (c c - c_s^2 I):T / (2 c_s^4) = 4.5 w (c.T.c - tr T / 3), relaxed with omega
            tqo = 4.5f * st.tq[s] * st.omega;
        }
        // The collision and the wall exchange conserve mass exactly (the source
        // has no zeroth moment; the moving-wall terms of a node sum to zero), so
        // the rest population is taken as the remainder after the moving ones
        // as they are stored (after rounding to the storage type).  Kept in
        // FP32, it carries the node's mass exactly: neither the FP32 weights
        // (sum 1 + 1.5e-8) nor 16-bit rounding of the moving populations leave
        // a systematic mass drift.
        float moved = 0.0f;
#pragma unroll
        for (int wc = 0; wc < 2; ++wc) {
            // weight class: axis directions, then face diagonals
            const float wa = wc == 0 ? w_axis : w_diag;
            const float k0 = wa * K0;
            const float rx = wa * Rx, ry = wa * Ry, rz = wa * Rz;
            const float px = wa * Px, py = wa * Py, pz = wa * Pz;
            const float wrs = wa * rsv, tqw = wa * tqo;
#pragma unroll
            for (int a = 1; a < L::Q; a += 2) {
                if ((L::w(a) == w_axis) != (wc == 0)) continue;
                const int ab = a + 1;  // opposite of a
                const int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
                const float cu = cx * st.ux + cy * st.uy + cz * st.uz;
                const float cr = cx * rx + cy * ry + cz * rz;
                const float cp = cx * px + cy * py + cz * pz;
                float even = fmaf(cu, cr, k0);
                if (p.coupling == 1) {
                    float cqc;
                    if (L::NQ == 6)
                        cqc = cx * cx * qloc[0] + cy * cy * qloc[3] + cz * cz * qloc[5] +
                              2.0f * (cx * cy * qloc[1] + cx * cz * qloc[2] + cy * cz * qloc[4]);
                    else
                        cqc = cx * cx * qloc[0] + cy * cy * qloc[2] + 2.0f * cx * cy * qloc[1];
                    even += tqw * (cqc - trq * (1.0f / 3.0f));
                }
                float fa, fb;
                if (mrt) {
                    const float quad = kh0 + (cx ? kH[0] : 0.0f) + (cy ? kH[1] : 0.0f) + (cz ? kH[2] : 0.0f) +
                                       (float)(cx * cy) * kX[0] + (float)(cy * cz) * kX[1] + (float)(cx * cz) * kX[2];
                    even += quad;
                    fa = even + cp;
                    fb = even - cp;
                } else {
                    fa = fmaf(keep, fget(s, a), even + cp);
                    fb = fmaf(keep, fget(s, ab), even - cp);
                }
                // a streams to x + c, its opposite to x - c; a population leaving
                // through a wall returns to this node in the opposite direction with
                // the moving-wall term -2 w rho_s (c.U)/c_s^2 (+U lower, -U upper)
                const bool ba = (cy > 0 && wall_hi) || (cy < 0 && wall_lo);
                const bool bb = (cy < 0 && wall_hi) || (cy > 0 && wall_lo);
                const PT va = pop_put<PT>(ba ? fa - wrs * (float)cx * (cy < 0 ? uw6 : -uw6) : fa);
                moved += pop_get(va);
                const PT vb = pop_put<PT>(bb ? fb + wrs * (float)cx * (cy > 0 ? uw6 : -uw6) : fb);
                moved += pop_get(vb);
                emit(s, a, va, vb, ba, bb);
            }
        }
        rest[s] = drs - moved;
    }
}

// Collision and push streaming: each stored value goes to its destination
// node (periodic offsets in x, y, z), a bounced one to this node's opposite
// direction; the rest population is updated in place.  EDGE = false is for
// nodes known to have y-neighbours inside the lattice (no wall row, no
// periodic wrap in y), which skips the bounce-back and wrap logic.  PARTS:
// every value this node emits in direction a (as stored, bounced or not) is
// also written to its staging slot a (own[(s (Q-1) + a - 1) T]), whose
// pre-collision content has just been read, and the new rest populations are
// returned in rest_out.
template <class PT, class L, int NCOMP, int COLL, bool EDGE = true, bool PARTS = false, class FGet>
__device__ __forceinline__ void collide_stream(const StepBufs& b, const StepParams& p, const Nbr& nb,
                                               const Local<NCOMP>& st, const float qloc[L::NQ],
                                               const float (*pif)[6], FGet fget, PT* own = nullptr, int T = 0,
                                               float* rest_out = nullptr) {
    const int N = (int)p.N;
    const int node = nb.i;
    const int* ox = nb.ox;
    const int* oz = nb.oz;
    // streaming offsets in y are periodic (walls are handled by bounce-back)
    const int nx = p.nx;
    int oy[3];
    const bool wall_lo = EDGE && p.walls && nb.y == 0, wall_hi = EDGE && p.walls && nb.y == nb.ny - 1;
    oy[0] = (EDGE && nb.y == 0 ? nb.ny - 1 : -1) * nx;
    oy[1] = 0;
    oy[2] = (EDGE && nb.y == nb.ny - 1 ? 1 - nb.ny : 1) * nx;
    float rest[NCOMP];
    collide_emit<PT, L, NCOMP, COLL>(
        p, st, qloc, pif, wall_lo, wall_hi, fget,
        [&](int s, int a, PT va, PT vb, bool ba, bool bb) {
            // moving populations: plane a - 1 of component s
            PT* out = static_cast<PT*>(b.fout) + (long long)s * (L::Q - 1) * N - N;
            const int ab = a + 1;
            const int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
            if (ba) out[ab * N + node] = va;
            else if (idx_ok(node + ox[cx + 1] + oy[cy + 1] + oz[cz + 1], N, b.status))
                out[a * N + node + ox[cx + 1] + oy[cy + 1] + oz[cz + 1]] = va;
            if (bb) out[a * N + node] = vb;
            else if (idx_ok(node + ox[1 - cx] + oy[1 - cy] + oz[1 - cz], N, b.status))
                out[ab * N + node + ox[1 - cx] + oy[1 - cy] + oz[1 - cz]] = vb;
            if constexpr (PARTS) {
                own[(s * (L::Q - 1) + a - 1) * T] = va;
                own[(s * (L::Q - 1) + ab - 1) * T] = vb;
            }
        },
        rest);
    // the rest population stays at the node, in FP32, and is updated in place
#pragma unroll
    for (int s = 0; s < NCOMP; ++s) b.frest[s * N + node] = rest[s];
    if constexpr (PARTS) {
#pragma unroll
        for (int s = 0; s < NCOMP; ++s) rest_out[s] = rest[s];
    }
}

template <class PT, class L, int NCOMP, bool STREAM, int COLL>
__global__ void __launch_bounds__(128) k_lattice(StepBufs b, StepParams p, int rev) {
    const int x = tile_index(blockIdx.x, gridDim.x, rev) * blockDim.x + threadIdx.x;
    const int y = tile_index(blockIdx.y, gridDim.y, rev) * blockDim.y + threadIdx.y;
    const int z = tile_index(blockIdx.z, gridDim.z, rev);
    if (x >= p.nx || y >= p.ny) return;
    const long long N = p.N;
    const long long i = ((long long)z * p.ny + y) * p.nx + x;

    // moments (same summation order as k_moments)
    float f[NCOMP][L::Q];
    float dr[NCOMP];
    float jx = 0.0f, jy = 0.0f, jz = 0.0f;
#pragma unroll
    for (int s = 0; s < NCOMP; ++s) {
        dr[s] = 0.0f;
#pragma unroll
        for (int a = 0; a < L::Q; ++a) {
            f[s][a] = a == 0 ? b.frest[s * N + i]
                             : pop_load(static_cast<const PT*>(b.fin) + (s * (L::Q - 1) + a - 1) * N + i);
            dr[s] += f[s][a];
        }
    }
    float pif[NCOMP][6];
#pragma unroll
    for (int s = 0; s < NCOMP; ++s) {
#pragma unroll
        for (int k = 0; k < 6; ++k) pif[s][k] = 0.0f;
#pragma unroll
        for (int a = 1; a < L::Q; ++a) {
            if (L::cx(a)) jx += L::cx(a) * f[s][a];
            if (L::cy(a)) jy += L::cy(a) * f[s][a];
            if (L::cz(a)) jz += L::cz(a) * f[s][a];
            if (COLL == 1) pi_add<L>(pif[s], a, f[s][a]);
        }
    }
    const Nbr nb = make_nbr(x, y, z, p);
    float acc[2][3], Fp[3], qloc[L::NQ];
    neighbour_forces<L, NCOMP>(b, p, nb, acc, Fp, qloc);
    Local<NCOMP> st;
    local_state<L, NCOMP>(p, dr, jx, jy, jz, acc, Fp, st, b.status);
    b.u[i] = st.ux;
    b.u[N + i] = st.uy;
    if (L::D == 3) b.u[2 * N + i] = st.uz;
    if (!STREAM) {
        if (b.dbg) {
            // g_s from the lattice sums; F_p; tau
            for (int k = 0; k < 3; ++k) {
                b.dbg[k * N + i] = NCOMP == 2 ? -p.G * st.rs[0] * acc[1][k] : 0.0f;
                b.dbg[(3 + k) * N + i] = NCOMP == 2 ? -p.G * st.rs[NCOMP - 1] * acc[0][k] : 0.0f;
                b.dbg[(6 + k) * N + i] = Fp[k];
            }
            b.dbg[9 * N + i] = 1.0f / st.omega;
        }
        return;
    }
    collide_stream<PT, L, NCOMP, COLL>(b, p, nb, st, qloc, pif, [&](int s, int a) { return f[s][a]; });
}

// --- TMA-staged variant --------------------------------------------------------

// Threads per SM the register budget of the staged lattice kernel is sized
// for (1024: 64 registers per thread).
#ifndef VEFD_LATTICE_THREADS_PER_SM
#define VEFD_LATTICE_THREADS_PER_SM 1024
#endif

// Node work of the staged kernels, split around the wait for the staged
// populations: gather (neighbour densities and feedback stress, overlapping
// the copy), then moments, local state and collision from shared memory.
template <class L, int NCOMP>
struct NodeGather {
    float dr[NCOMP];
    float acc[2][3], Fp[3], qloc[L::NQ];
    Nbr nb;
};

template <class L, int NCOMP>
__device__ __forceinline__ void node_gather(const StepBufs& b, const StepParams& p, int x, int y, int z, bool active,
                                            NodeGather<L, NCOMP>& g) {
    g.nb = make_nbr(active ? x : 0, active ? y : 0, active ? z : 0, p);
    if (!active) return;
    // the node's own deviations come from the density buffer (bit-identical to
    // the sum of the staged populations)
    dens_ldg<NCOMP>(b.drho, g.nb.i, g.dr);
    neighbour_forces<L, NCOMP>(b, p, g.nb, g.acc, g.Fp, g.qloc);
}

template <class PT, class L, int NCOMP, int T, int COLL, bool EDGE = true, bool PARTS = false>
__device__ __forceinline__ void node_collide(const StepBufs& b, const StepParams& p, const PT* sf, int t,
                                             const NodeGather<L, NCOMP>& g, PT* own = nullptr,
                                             float* rest_out = nullptr) {
    const long long N = p.N;
    const int i = g.nb.i;
    float jx = 0.0f, jy = 0.0f, jz = 0.0f;
    float pif[NCOMP][6];
#pragma unroll
    for (int s = 0; s < NCOMP; ++s) {
#pragma unroll
        for (int k = 0; k < 6; ++k) pif[s][k] = 0.0f;
#pragma unroll
        for (int a = 1; a < L::Q; ++a) {
            const float fa = pop_get(sf[(s * (L::Q - 1) + a - 1) * T + t]);
            if (L::cx(a)) jx += L::cx(a) * fa;
            if (L::cy(a)) jy += L::cy(a) * fa;
            if (L::cz(a)) jz += L::cz(a) * fa;
            if (COLL == 1) pi_add<L>(pif[s], a, fa);
        }
    }
    Local<NCOMP> st;
    local_state<L, NCOMP>(p, g.dr, jx, jy, jz, g.acc, g.Fp, st, b.status);
    b.u[i] = st.ux;
    b.u[N + i] = st.uy;
    if (L::D == 3) b.u[2 * N + i] = st.uz;
    // volatile reads keep the populations in shared memory instead of registers
    collide_stream<PT, L, NCOMP, COLL, EDGE, PARTS>(
        b, p, g.nb, st, g.qloc, pif, [&](int s, int a) { return pop_smem(sf, (s * (L::Q - 1) + a - 1) * T + t); },
        own, T, rest_out);
}

// Partial densities of time n+1 from one staged D3Q19 tile (BX, BY, BZ >= 2),
// after every thread has written what its node emitted into its own slots
// of sf.  Slot 0 of b.part gets, for each node d of the tile, its new rest
// population plus, in direction order, each population that reached d from
// inside the tile or came back to d from a wall.  Slots 1-6 get, for each node
// e just outside the tile (in the neighbouring tile across x, y, z, xy, xz or
// yz), the sum in direction order of the populations this tile pushed into e.
// A node lies on at most one face of its tile per axis, so for every node and
// slot at most one tile writes, and the densities pass reads exactly the
// slots its node's position in its tile implies (slot 0 always; a slot across
// y only when that side is not a wall).  Positions beyond a wall receive
// nothing (those populations bounced back into slot 0 of their source).
template <class PT, int NCOMP, int BX, int BY, int BZ>
__device__ __forceinline__ void tile_partials(const PT* sf, const StepBufs& b, const StepParams& p, float* part,
                                              int x0, int y0, int z0, int t, const float rest[NCOMP], bool active) {
    using L = D3Q19;
    static_assert(BX >= 2 && BY >= 2 && BZ >= 2, "a node must lie on at most one face per axis");
    constexpr int T = BX * BY * BZ;
    const int N = (int)p.N, nx = p.nx, ny = p.ny, nz = p.nz;
    const int tx = t % BX, ty = (t / BX) % BY, tz = t / (BX * BY);
    auto val = [&](int s, int a, int src) -> float { return pop_get(sf[(s * (L::Q - 1) + a - 1) * T + src]); };
    if (active) {
        const int y = y0 + ty;
        float v[NCOMP];
#pragma unroll
        for (int s = 0; s < NCOMP; ++s) v[s] = rest[s];
#pragma unroll
        for (int a = 1; a < L::Q; ++a) {
            const int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
            const int gy = y - cy;
            if (p.walls && (gy < 0 || gy >= ny)) {
                // from beyond a wall: this node's own value in the opposite direction, bounced
                const int ao = (a & 1) ? a + 1 : a - 1;
#pragma unroll
                for (int s = 0; s < NCOMP; ++s) v[s] += val(s, ao, t);
            } else if ((unsigned)(tx - cx) < (unsigned)BX && (unsigned)(ty - cy) < (unsigned)BY &&
                       (unsigned)(tz - cz) < (unsigned)BZ) {
                const int src = t - ((cz * BY + cy) * BX + cx);
#pragma unroll
                for (int s = 0; s < NCOMP; ++s) v[s] += val(s, a, src);
            }
        }
        const int i = ((z0 + tz) * ny + y) * nx + x0 + tx;
        if (idx_ok(i, N, b.status)) dens_store<NCOMP>(part, i, v);
    }
    // the shell: z faces, y faces, yz edges, x faces, xy edges, xz edges
    constexpr int nZ = 2 * BX * BY, nY = 2 * BX * BZ, nYZ = 4 * BX, nX = 2 * BY * BZ, nXY = 4 * BZ, nXZ = 4 * BY;
    constexpr int total = nZ + nY + nYZ + nX + nXY + nXZ;
    for (int w = t; w < total; w += T) {
        int ex, ey, ez, slot, q = w;
        if (q < nZ) {
            slot = 3;
            ez = q >= BX * BY ? BZ : -1;
            q %= BX * BY;
            ex = q % BX;
            ey = q / BX;
        } else if ((q -= nZ) < nY) {
            slot = 2;
            ey = q >= BX * BZ ? BY : -1;
            q %= BX * BZ;
            ex = q % BX;
            ez = q / BX;
        } else if ((q -= nY) < nYZ) {
            slot = 6;
            ey = (q & 1) ? BY : -1;
            ez = (q & 2) ? BZ : -1;
            ex = q >> 2;
        } else if ((q -= nYZ) < nX) {
            slot = 1;
            ex = q >= BY * BZ ? BX : -1;
            q %= BY * BZ;
            ey = q % BY;
            ez = q / BY;
        } else if ((q -= nX) < nXY) {
            slot = 4;
            ex = (q & 1) ? BX : -1;
            ey = (q & 2) ? BY : -1;
            ez = q >> 2;
        } else {
            q -= nXY;
            slot = 5;
            ex = (q & 1) ? BX : -1;
            ez = (q & 2) ? BZ : -1;
            ey = q >> 2;
        }
        const int gy = y0 + ey;
        if (p.walls && (gy < 0 || gy >= ny)) continue;
        float v[NCOMP];
#pragma unroll
        for (int s = 0; s < NCOMP; ++s) v[s] = 0.0f;
#pragma unroll
        for (int a = 1; a < L::Q; ++a) {
            const int sx = ex - L::cx(a), sy = ey - L::cy(a), sz = ez - L::cz(a);
            if ((unsigned)sx < (unsigned)BX && (unsigned)sy < (unsigned)BY && (unsigned)sz < (unsigned)BZ) {
                const int src = (sz * BY + sy) * BX + sx;
#pragma unroll
                for (int s = 0; s < NCOMP; ++s) v[s] += val(s, a, src);
            }
        }
        const int gx = wrap1(x0 + ex, nx), gz = wrap1(z0 + ez, nz), gyy = p.walls ? gy : wrap1(gy, ny);
        const int i = (gz * ny + gyy) * nx + gx;
        if (idx_ok(i, N, b.status)) dens_store<NCOMP>(part + (long long)slot * N * NCOMP, i, v);
    }
}

// One staged tile (origin x0, y0, z0) of the lattice kernel; tm_fin is the
// tensor map of b.fin with box BX x BY x BZ x P.  PARTS (D3Q19): the
// post-collision values also stay in the staging slots, and the tile writes
// the partial densities of time n+1 to `part` (tile_partials).
template <class PT, class L, int NCOMP, int BX, int BY, int BZ, int COLL, bool PARTS = false>
__device__ __forceinline__ void lattice_tile(const CUtensorMap* tm_fin, const StepBufs& b, const StepParams& p, int x0,
                                             int y0, int z0, float* part = nullptr) {
    constexpr int P = NCOMP * (L::Q - 1);  // moving populations
    constexpr int T = BX * BY * BZ;
    constexpr unsigned kBytes = (unsigned)(P * T * sizeof(PT));
    extern __shared__ __align__(128) unsigned char sraw[];
    PT* sf = reinterpret_cast<PT*>(sraw);  // [P][BZ][BY][BX], the TMA box layout
    __shared__ __align__(8) unsigned long long bar;
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const bool leader = (tx | ty | tz) == 0;
    const unsigned bar_a = smem_u32(&bar);
    if (leader) mbar_init(bar_a);
    __syncthreads();
    // the populations of time n are complete before this kernel can start
    if (leader) tma_load_4d(smem_u32(sf), tm_fin, x0, y0, z0, 0, bar_a, kBytes);
    const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
    const bool active = x < p.nx && y < p.ny && z < p.nz;
    // densities, feedback stress, velocity and rest populations are shared with
    // the preceding densities/FENE-P pass
    pdl_wait();
    NodeGather<L, NCOMP> g;
    node_gather<L, NCOMP>(b, p, x, y, z, active, g);
    if constexpr (PARTS) {
        const int t = (tz * BY + ty) * BX + tx;
        // the tile's threads meet at a barrier below: take the timeout
        // decision together
        const bool ok = mbar_wait_bounded(bar_a);
        if (__syncthreads_or(!ok)) {
            if (leader) {
                atomicOr(b.status, kStTimeout);
                mbar_wait_bounded(bar_a);  // bounded: let the copy land before leaving
            }
            return;
        }
        pdl_trigger();
        float rest[NCOMP];
#pragma unroll
        for (int s = 0; s < NCOMP; ++s) rest[s] = 0.0f;
        if (active) {
            if (y0 > 0 && y0 + BY < p.ny)
                node_collide<PT, L, NCOMP, T, COLL, false, true>(b, p, sf, t, g, sf + t, rest);
            else
                node_collide<PT, L, NCOMP, T, COLL, true, true>(b, p, sf, t, g, sf + t, rest);
        }
        __syncthreads();
        tile_partials<PT, NCOMP, BX, BY, BZ>(sf, b, p, part, x0, y0, z0, t, rest, active);
        return;
    }
    // bounded wait for the staged populations; on timeout report and leave
    if (!mbar_wait_bounded(bar_a)) {
        if (leader) {
            atomicOr(b.status, kStTimeout);
            mbar_wait_bounded(bar_a);  // bounded: let the copy land before leaving
        }
        return;
    }
    pdl_trigger();
    if (!active) return;
    // tiles whose rows all have both y-neighbours inside the lattice take the
    // path without bounce-back and y-wrap logic (block-uniform branch)
    if (y0 > 0 && y0 + BY < p.ny)
        node_collide<PT, L, NCOMP, T, COLL, false>(b, p, sf, (tz * BY + ty) * BX + tx, g);
    else
        node_collide<PT, L, NCOMP, T, COLL, true>(b, p, sf, (tz * BY + ty) * BX + tx, g);
}

template <class PT, class L, int NCOMP, int BX, int BY, int BZ, int COLL>
__global__ void __launch_bounds__(BX * BY * BZ, VEFD_LATTICE_THREADS_PER_SM / (BX * BY * BZ))
    k_lattice_tma(const __grid_constant__ CUtensorMap tm_fin, StepBufs b, StepParams p, int rev) {
    lattice_tile<PT, L, NCOMP, BX, BY, BZ, COLL>(&tm_fin, b, p, tile_index(blockIdx.x, gridDim.x, rev) * BX,
                                                 p.ylo + tile_index(blockIdx.y, gridDim.y, rev) * BY,
                                                 tile_index(blockIdx.z, gridDim.z, rev) * BZ);
}

// The same tile that also writes the partial densities of time n+1 (post mode 3).
template <class PT, class L, int NCOMP, int BX, int BY, int BZ, int COLL>
__global__ void __launch_bounds__(BX * BY * BZ, VEFD_LATTICE_THREADS_PER_SM / (BX * BY * BZ))
    k_lattice_tma_parts(const __grid_constant__ CUtensorMap tm_fin, StepBufs b, StepParams p, int rev, float* part) {
    lattice_tile<PT, L, NCOMP, BX, BY, BZ, COLL, true>(&tm_fin, b, p, tile_index(blockIdx.x, gridDim.x, rev) * BX,
                                                       p.ylo + tile_index(blockIdx.y, gridDim.y, rev) * BY,
                                                       tile_index(blockIdx.z, gridDim.z, rev) * BZ, part);
}

// Batched ensemble form: block i runs tile i - start[m] of member m with that
// member's parameters, buffers and tensor map (parity selects the ping-pong
// state).  Tiles are 32 x BY x BZ (32 x 4 x 2 or 32 x 8 x 1, the ensemble's
// tile choice; the member table's tile counts and tensor maps follow it).
template <class PT, int NCOMP, int COLL, int BY, int BZ>
__global__ void __launch_bounds__(256, VEFD_LATTICE_THREADS_PER_SM / 256)
    k_lattice_batch(const EnsMember* __restrict__ members, const int* __restrict__ start, int nm, int parity) {
    static_assert(BY * BZ == 8, "256-thread tiles");
    const int m = batch_member(start, nm, (int)blockIdx.x);
    const EnsMember& M = members[m];
    const int t = (int)blockIdx.x - start[m];
    // the member's parameters and buffers, read from shared memory by the node code
    __shared__ StepParams sp;
    __shared__ StepBufs sb;
    const int lt = (threadIdx.z * BY + threadIdx.y) * 32 + threadIdx.x;
    static_assert(sizeof(StepParams) % 4 == 0 && sizeof(StepBufs) % 4 == 0, "word copies");
    if (lt < (int)(sizeof(StepParams) / 4))
        reinterpret_cast<int*>(&sp)[lt] = reinterpret_cast<const int*>(&M.p)[lt];
    else if (lt - (int)(sizeof(StepParams) / 4) < (int)(sizeof(StepBufs) / 4))
        reinterpret_cast<int*>(&sb)[lt - sizeof(StepParams) / 4] =
            reinterpret_cast<const int*>(&M.b[parity])[lt - sizeof(StepParams) / 4];
    const int r = t / M.ntx;
    const int x0 = (t % M.ntx) * 32, y0 = (r % M.nty) * BY, z0 = (r / M.nty) * BZ;
    const CUtensorMap* tm = &M.tm_lat[M.cur0 ^ parity];  // the populations read
    if (lt == 0) tensormap_acquire(tm);                   // the thread that issues the copy
    __syncthreads();
    lattice_tile<PT, D3Q19, NCOMP, 32, BY, BZ, COLL>(tm, sb, sp, x0, y0, z0);
}

template <int COLL, int BY, int BZ>
cudaError_t launch_lattice_batch_tile(int ncomp, int prec, const EnsMember* members, const int* start, int nm,
                                      int items, int parity, bool pdl, cudaStream_t s) {
    cudaError_t e = cudaSuccess;
    VEFD_WITH_PT(prec, {
        constexpr int smem_unit = 18 * 256 * (int)sizeof(PT);
        if (ncomp == 2)
            e = launch_pdl(pdl, k_lattice_batch<PT, 2, COLL, BY, BZ>, dim3(items), dim3(32, BY, BZ), 2 * smem_unit, s,
                           members, start, nm, parity);
        else
            e = launch_pdl(pdl, k_lattice_batch<PT, 1, COLL, BY, BZ>, dim3(items), dim3(32, BY, BZ), smem_unit, s,
                           members, start, nm, parity);
    });
    return e;
}

// tile 0: 32 x 4 x 2, tile 1: 32 x 8 x 1
template <int COLL>
cudaError_t launch_lattice_batch_coll(int ncomp, int prec, int tile, const EnsMember* members, const int* start,
                                      int nm, int items, int parity, bool pdl, cudaStream_t s) {
    return tile == 1 ? launch_lattice_batch_tile<COLL, 8, 1>(ncomp, prec, members, start, nm, items, parity, pdl, s)
                     : launch_lattice_batch_tile<COLL, 4, 2>(ncomp, prec, members, start, nm, items, parity, pdl, s);
}

// Persistent form (single-relaxation-time collision): a grid of (SMs x
// resident blocks) walks the tiles in order
// (tile = block + k * grid, backwards when rev is set) with two staging
// buffers, so the copy of a block's next tile is in flight while it computes
// the current one and the copy engine never idles between tiles.
// Resident blocks per SM the persistent kernel's registers are budgeted for:
// as many as the two staging buffers leave room for in 227 KB of shared
// memory (1 KB reserved per block), at most the 64-register budget.
template <class PT, class L, int NCOMP, int T>
constexpr int pers_blocks() {
    constexpr int smem = 2 * NCOMP * (L::Q - 1) * T * (int)sizeof(PT) + 1024 + 128;
    constexpr int by_smem = (227 * 1024) / smem;
    constexpr int by_regs = VEFD_LATTICE_THREADS_PER_SM / T;
    return by_smem < 1 ? 1 : (by_smem < by_regs ? by_smem : by_regs);
}

template <class PT, class L, int NCOMP, int BX, int BY, int BZ>
__global__ void __launch_bounds__(BX * BY * BZ, (pers_blocks<PT, L, NCOMP, BX * BY * BZ>())) k_lattice_pers(const __grid_constant__ CUtensorMap tm_fin, StepBufs b,
                                                               StepParams p, int rev, int ntx, int nty, int ntiles) {
    constexpr int P = NCOMP * (L::Q - 1);
    constexpr int T = BX * BY * BZ;
    constexpr unsigned kBytes = (unsigned)(P * T * sizeof(PT));
    extern __shared__ __align__(128) unsigned char sraw[];
    PT* sbuf = reinterpret_cast<PT*>(sraw);  // two buffers of [P][BZ][BY][BX]
    __shared__ __align__(8) unsigned long long bars[2];
    const int tx = threadIdx.x, ty = threadIdx.y, tz = threadIdx.z;
    const bool leader = (tx | ty | tz) == 0;
    const unsigned bar0 = smem_u32(&bars[0]), bar1 = smem_u32(&bars[1]);
    auto origin = [&](int tile, int& x0, int& y0, int& z0) {
        const int q = rev ? ntiles - 1 - tile : tile;
        x0 = (q % ntx) * BX;
        const int r = q / ntx;
        y0 = (r % nty) * BY;
        z0 = (r / nty) * BZ;
    };
    auto issue = [&](int tile, int slot) {
        int x0, y0, z0;
        origin(tile, x0, y0, z0);
        tma_load_4d(smem_u32(sbuf + slot * P * T), &tm_fin, x0, y0, z0, 0, slot ? bar1 : bar0, kBytes);
    };
    if (leader) {
        mbar_init(bar0);
        mbar_init(bar1);
    }
    __syncthreads();
    const int stride = gridDim.x;
    if (leader) {
        if ((int)blockIdx.x < ntiles) issue(blockIdx.x, 0);
        if ((int)blockIdx.x + stride < ntiles) issue(blockIdx.x + stride, 1);
    }
    const int t = (tz * BY + ty) * BX + tx;
    for (int k = 0;; ++k) {
        const int tile = (int)blockIdx.x + k * stride;
        if (tile >= ntiles) break;
        const int slot = k & 1;
        int x0, y0, z0;
        origin(tile, x0, y0, z0);
        const int x = x0 + tx, y = y0 + ty, z = z0 + tz;
        const bool active = x < p.nx && y < p.ny && z < p.nz;
        NodeGather<L, NCOMP> g;
        node_gather<L, NCOMP>(b, p, x, y, z, active, g);
        const bool ok = mbar_wait_bounded_parity(slot ? bar1 : bar0, (unsigned)((k >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            if (leader) {
                atomicOr(b.status, kStTimeout);
                // let the copies this block still has in flight land (bounded) before leaving
                mbar_wait_bounded_parity(slot ? bar1 : bar0, (unsigned)((k >> 1) & 1));
                if (tile + stride < ntiles)
                    mbar_wait_bounded_parity(slot ? bar0 : bar1, (unsigned)(((k + 1) >> 1) & 1));
            }
            return;
        }
        if (active) node_collide<PT, L, NCOMP, T, 0>(b, p, sbuf + slot * P * T, t, g);
        // every thread is done with this buffer: refill it with the tile after next
        __syncthreads();
        if (leader && tile + 2 * stride < ntiles) {
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            issue(tile + 2 * stride, slot);
        }
    }
}

dim3 node_grid(const StepParams& p) { return dim3((p.nx + 31) / 32, (p.ny + 3) / 4, p.nz); }

template <class PT, class L, int NCOMP, int BX, int BY, int BZ, int COLL>
cudaError_t launch_tma_tile(const CUtensorMap* tm, const StepParams& p, const StepBufs& b, int rev, cudaStream_t s) {
    constexpr int smem = NCOMP * (L::Q - 1) * BX * BY * BZ * (int)sizeof(PT);
    static_assert(smem <= 48 * 1024, "staged tile must fit the default shared-memory limit");
    dim3 blk(BX, BY, BZ), grd((p.nx + BX - 1) / BX, (p.yhi - p.ylo + BY - 1) / BY, (p.nz + BZ - 1) / BZ);
    return launch_pdl(p.pdl != 0, k_lattice_tma<PT, L, NCOMP, BX, BY, BZ, COLL>, grd, blk, smem, s, *tm, b, p, rev);
}

template <class PT, class L, int NCOMP, int BX, int BY, int BZ, int COLL>
cudaError_t launch_tma_tile_parts(const CUtensorMap* tm, const StepParams& p, const StepBufs& b, int rev,
                                  cudaStream_t s, float* part) {
    constexpr int smem = NCOMP * (L::Q - 1) * BX * BY * BZ * (int)sizeof(PT);
    static_assert(smem <= 48 * 1024, "staged tile must fit the default shared-memory limit");
    dim3 blk(BX, BY, BZ), grd((p.nx + BX - 1) / BX, (p.yhi - p.ylo + BY - 1) / BY, (p.nz + BZ - 1) / BZ);
    return launch_pdl(p.pdl != 0, k_lattice_tma_parts<PT, L, NCOMP, BX, BY, BZ, COLL>, grd, blk, smem, s, *tm, b, p,
                      rev, part);
}

// Column-marching form (D3Q19, NX % 32 == 0, NY % 8 == 0) that also yields
// partial densities of the new populations, so that the densities pass reads
// back only the populations that crossed a column side or a segment end.  A
// block owns a 32 x 8 column and walks the planes [z0, z1) of its z-segment;
// per plane:
//   1. the plane's moving populations f^n arrive by one bulk tensor copy (box
//      32 x 8 x 1 x P) into one of two staging buffers; the copy of the next
//      plane is issued at the start of the iteration, so it overlaps this
//      plane's work;
//   2. each thread gathers neighbour densities and feedback stress, collides
//      its node and pushes every value to its destination in global memory
//      exactly as the tiled kernel does (bounced ones to its own node), and
//      also writes each value into its own staging slot, whose pre-collision
//      content it has consumed;
//   3. after a barrier each thread adds, in a fixed direction order, the
//      values arriving at its (x, y) from inside the column (from the slots of
//      their source threads; bounced ones from its own slots) to partial
//      densities of planes z - 1, z, z + 1 when that plane lies in the segment;
//   4. plane z - 1 has then received everything from inside the column and
//      segment, and its partial density goes to b.drho_next.
// The densities pass adds the populations that crossed a column side or a
// segment end, reading them from the new population buffer.
template <class PT, int NCOMP, int COLL, bool EDGE>
__device__ __forceinline__ void lattice_column(const CUtensorMap* tm_fin, const StepBufs& b, const StepParams& p,
                                               int x0, int y0, int z0, int z1) {
    using L = D3Q19;
    constexpr int P = NCOMP * (L::Q - 1);
    constexpr int T = 256;
    constexpr unsigned kBytes = (unsigned)(P * T * sizeof(PT));
    extern __shared__ __align__(128) unsigned char sraw[];
    PT* sbuf = reinterpret_cast<PT*>(sraw);  // two buffers of [P][8][32]
    __shared__ __align__(8) unsigned long long bars[2];
    const int tx = threadIdx.x, ty = threadIdx.y, t = ty * 32 + tx;
    const int nx = p.nx, ny = p.ny, nz = p.nz, N = (int)p.N, plane = nx * ny;
    const int x = x0 + tx, y = y0 + ty;
    const bool leader = t == 0;
    const unsigned bar0 = smem_u32(&bars[0]), bar1 = smem_u32(&bars[1]);
    if (leader) {
        mbar_init(bar0);
        mbar_init(bar1);
    }
    __syncthreads();
    const int nplanes = z1 - z0;
    if (leader && nplanes > 0) tma_load_4d(smem_u32(sbuf), tm_fin, x0, y0, z0, 0, bar0, kBytes);
    const ColumnTopo topo{nx == 32, ny == 8 && !p.walls, nz == 1};
    const bool wall_lo = EDGE && p.walls && y == 0, wall_hi = EDGE && p.walls && y == ny - 1;
    // streaming offsets in y are periodic (walls are handled by bounce-back)
    int oy[3];
    oy[0] = (EDGE && y == 0 ? ny - 1 : -1) * nx;
    oy[1] = 0;
    oy[2] = (EDGE && y == ny - 1 ? 1 - ny : 1) * nx;
    PT* const fout = static_cast<PT*>(b.fout);
    float pm[NCOMP], pc[NCOMP], pn[NCOMP];  // partial densities of planes z - 1, z, z + 1
#pragma unroll
    for (int s = 0; s < NCOMP; ++s) pm[s] = pc[s] = pn[s] = 0.0f;
    for (int k = 0; k < nplanes; ++k) {
        const int z = z0 + k, slot = k & 1;
        PT* const sP = sbuf + slot * P * T;
        if (leader && k + 1 < nplanes) {
            // the other buffer was released by every thread at the barrier ending the previous plane
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            tma_load_4d(smem_u32(sbuf + (slot ^ 1) * P * T), tm_fin, x0, y0, z + 1, 0, slot ? bar0 : bar1, kBytes);
        }
        NodeGather<L, NCOMP> g;
        node_gather<L, NCOMP>(b, p, x, y, z, true, g);
        const bool ok = mbar_wait_bounded_parity(slot ? bar1 : bar0, (unsigned)((k >> 1) & 1));
        if (__syncthreads_or(!ok)) {
            if (leader) {
                atomicOr(b.status, kStTimeout);
                // let the copies this block still has in flight land (bounded) before leaving
                mbar_wait_bounded_parity(slot ? bar1 : bar0, (unsigned)((k >> 1) & 1));
                if (k + 1 < nplanes) mbar_wait_bounded_parity(slot ? bar0 : bar1, (unsigned)(((k + 1) >> 1) & 1));
            }
            return;
        }
        const int node = g.nb.i;
        float jx = 0.0f, jy = 0.0f, jz = 0.0f;
        float pif[NCOMP][6];
#pragma unroll
        for (int s = 0; s < NCOMP; ++s) {
#pragma unroll
            for (int q = 0; q < 6; ++q) pif[s][q] = 0.0f;
#pragma unroll
            for (int a = 1; a < L::Q; ++a) {
                const float fa = pop_get(sP[(s * (L::Q - 1) + a - 1) * T + t]);
                if (L::cx(a)) jx += L::cx(a) * fa;
                if (L::cy(a)) jy += L::cy(a) * fa;
                if (L::cz(a)) jz += L::cz(a) * fa;
                if (COLL == 1) pi_add<L>(pif[s], a, fa);
            }
        }
        Local<NCOMP> st;
        local_state<L, NCOMP>(p, g.dr, jx, jy, jz, g.acc, g.Fp, st, b.status);
        b.u[node] = st.ux;
        b.u[N + node] = st.uy;
        b.u[2 * N + node] = st.uz;
        const int* ox = g.nb.ox;
        const int* oz = g.nb.oz;
        float rest[NCOMP];
        collide_emit<PT, L, NCOMP, COLL>(
            p, st, g.qloc, pif, wall_lo, wall_hi,
            [&](int s, int a) { return pop_smem(sP, (s * (L::Q - 1) + a - 1) * T + t); },
            [&](int s, int a, PT va, PT vb, bool ba, bool bb) {
                PT* out = fout + (long long)s * (L::Q - 1) * N - N;
                const int ab = a + 1;
                const int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
                if (ba) out[ab * N + node] = va;
                else if (idx_ok(node + ox[cx + 1] + oy[cy + 1] + oz[cz + 1], N, b.status))
                    out[a * N + node + ox[cx + 1] + oy[cy + 1] + oz[cz + 1]] = va;
                if (bb) out[a * N + node] = vb;
                else if (idx_ok(node + ox[1 - cx] + oy[1 - cy] + oz[1 - cz], N, b.status))
                    out[ab * N + node + ox[1 - cx] + oy[1 - cy] + oz[1 - cz]] = vb;
                // this thread's own slots: its reads of them are done
                sP[(s * (L::Q - 1) + a - 1) * T + t] = va;
                sP[(s * (L::Q - 1) + ab - 1) * T + t] = vb;
            },
            rest);
        // the rest population stays at the node, in FP32, updated in place
#pragma unroll
        for (int s = 0; s < NCOMP; ++s) {
            b.frest[s * N + node] = rest[s];
            pc[s] += rest[s];
        }
        __syncthreads();
        // values arriving at this (x, y) from inside the column, in direction order
#pragma unroll
        for (int s = 0; s < NCOMP; ++s) {
#pragma unroll
            for (int a = 1; a < L::Q; ++a) {
                const int cx = L::cx(a), cy = L::cy(a), cz = L::cz(a);
                if (EDGE && ((cy > 0 && wall_lo) || (cy < 0 && wall_hi))) {
                    // the opposite population left through the wall and came back
                    pc[s] += pop_get(sP[(s * (L::Q - 1) + opposite(a) - 1) * T + t]);
                } else if (zm_inner(tx - cx, ty - cy, z + cz, z0, z1, topo)) {
                    const int src = ((ty - cy) & 7) * 32 + ((tx - cx) & 31);
                    const float fv = pop_get(sP[(s * (L::Q - 1) + a - 1) * T + src]);
                    if (cz == 0 || topo.nz1) pc[s] += fv;
                    else if (cz < 0) pm[s] += fv;
                    else pn[s] += fv;
                }
            }
        }
        // plane z - 1 is complete within the column and segment
        if (k > 0) dens_store<NCOMP>(b.drho_next, node - plane, pm);
#pragma unroll
        for (int s = 0; s < NCOMP; ++s) {
            pm[s] = pc[s];
            pc[s] = pn[s];
            pn[s] = 0.0f;
        }
        __syncthreads();  // the pulls are done before this buffer takes the copy after next
    }
    // the segment's last plane: what arrives from the next segment comes through memory
    if (nplanes > 0) dens_store<NCOMP>(b.drho_next, ((z1 - 1) * ny + y) * nx + x, pm);
}

template <class PT, int NCOMP, int COLL>
__global__ void __launch_bounds__(256, 3)
    k_lattice_zm(const __grid_constant__ CUtensorMap tm_fin, StepBufs b, StepParams p, int zs, int rev) {
    const int x0 = tile_index(blockIdx.x, gridDim.x, rev) * 32;
    const int y0 = p.ylo + tile_index(blockIdx.y, gridDim.y, rev) * 8;
    const int z0 = tile_index(blockIdx.z, gridDim.z, rev) * zs;
    const int z1 = min(z0 + zs, p.nz);
    // columns whose rows all have both y-neighbours inside the lattice take the
    // path without bounce-back and y-wrap logic (block-uniform branch)
    if (y0 > 0 && y0 + 8 < p.ny)
        lattice_column<PT, NCOMP, COLL, false>(&tm_fin, b, p, x0, y0, z0, z1);
    else
        lattice_column<PT, NCOMP, COLL, true>(&tm_fin, b, p, x0, y0, z0, z1);
}

inline int lattice_sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) n = 152;
    }
    return n;
}

template <class PT, class L, int NCOMP, int BX, int BY, int BZ>
cudaError_t launch_pers_tile(const CUtensorMap* tm, const StepParams& p, const StepBufs& b, int rev, cudaStream_t s) {
    constexpr int T = BX * BY * BZ;
    constexpr int smem = 2 * NCOMP * (L::Q - 1) * T * (int)sizeof(PT);
    static int per_sm = 0;  // resident blocks per SM of this instantiation
    if (!per_sm) {
        cudaError_t e = cudaFuncSetAttribute(k_lattice_pers<PT, L, NCOMP, BX, BY, BZ>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        int nb = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_lattice_pers<PT, L, NCOMP, BX, BY, BZ>, T, smem);
        if (e != cudaSuccess) return e;
        if (nb < 1) return cudaErrorInvalidConfiguration;
        per_sm = nb;
    }
    const int ntx = (p.nx + BX - 1) / BX, nty = (p.ny + BY - 1) / BY, ntz = (p.nz + BZ - 1) / BZ;
    const long long ntiles = (long long)ntx * nty * ntz;
    const long long grid = std::min<long long>(ntiles, (long long)per_sm * lattice_sm_count());
    k_lattice_pers<PT, L, NCOMP, BX, BY, BZ><<<(unsigned)grid, dim3(BX, BY, BZ), smem, s>>>(*tm, b, p, rev, ntx, nty,
                                                                                         (int)ntiles);
    return cudaGetLastError();
}

// Segment length of the column-marching kernel: one wave of
// (SMs x resident blocks) blocks over the columns and z-segments.
inline int zm_segment_length(const StepParams& p) {
    const int cols = (p.nx / 32) * (p.ny / 8);
    int nseg = 3 * lattice_sm_count() / (cols > 0 ? cols : 1);  // three resident blocks per SM
    if (nseg < 1) nseg = 1;
    if (nseg > p.nz) nseg = p.nz;
    return (p.nz + nseg - 1) / nseg;
}

template <class PT, int NCOMP, int COLL>
cudaError_t launch_zm(const CUtensorMap* tm, const StepParams& p, const StepBufs& b, int zs, int rev, cudaStream_t s) {
    constexpr int smem = 2 * NCOMP * 18 * 256 * (int)sizeof(PT);  // two staged planes
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_lattice_zm<PT, NCOMP, COLL>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    dim3 blk(32, 8, 1), grd(p.nx / 32, (p.yhi - p.ylo) / 8, (p.nz + zs - 1) / zs);
    k_lattice_zm<PT, NCOMP, COLL><<<grd, blk, smem, s>>>(*tm, b, p, zs, rev);
    return cudaGetLastError();
}

template <int COLL>
cudaError_t launch_zm_coll(int ncomp, const StepParams& p, const StepBufs& b, cudaStream_t s, const void* tensor_map,
                           int zs, int rev) {
    const CUtensorMap* tm = static_cast<const CUtensorMap*>(tensor_map);
    cudaError_t e = cudaSuccess;
    VEFD_WITH_PT(p.prec, {
        e = ncomp == 2 ? launch_zm<PT, 2, COLL>(tm, p, b, zs, rev, s) : launch_zm<PT, 1, COLL>(tm, p, b, zs, rev, s);
    });
    return e;
}

// Tiles 0..2 staged per block; 3..5 the persistent forms (single relaxation
// time only: the moment-space collision takes the staged form of the tile).
template <class PT, class L, int NCOMP, int COLL>
cudaError_t launch_tma(const CUtensorMap* tm, const StepParams& p, const StepBufs& b, int rev, cudaStream_t s,
                       int tile, Parts parts) {
    if (COLL != 0 && tile >= 3) tile -= 3;
    if constexpr (L::D == 3) {
        if (parts.part) {
            // partial densities: the 32 x 4 x 2 and 32 x 2 x 4 tiles (the host admits no other)
            if (tile == 1 && parts.by == 2 && parts.bz == 4)
                return launch_tma_tile_parts<PT, L, NCOMP, 32, 2, 4, COLL>(tm, p, b, rev, s, parts.part);
            if (tile == 0 && parts.by == 4 && parts.bz == 2)
                return launch_tma_tile_parts<PT, L, NCOMP, 32, 4, 2, COLL>(tm, p, b, rev, s, parts.part);
            return cudaErrorInvalidValue;
        }
        switch (tile) {
        case 1: return launch_tma_tile<PT, L, NCOMP, 32, 2, 4, COLL>(tm, p, b, rev, s);
        case 2: return launch_tma_tile<PT, L, NCOMP, 32, 8, 1, COLL>(tm, p, b, rev, s);
        case 3: if constexpr (COLL == 0) return launch_pers_tile<PT, L, NCOMP, 32, 4, 2>(tm, p, b, rev, s);
        case 4: if constexpr (COLL == 0) return launch_pers_tile<PT, L, NCOMP, 32, 2, 4>(tm, p, b, rev, s);
        case 5: if constexpr (COLL == 0) return launch_pers_tile<PT, L, NCOMP, 32, 8, 1>(tm, p, b, rev, s);
        default: return launch_tma_tile<PT, L, NCOMP, 32, 4, 2, COLL>(tm, p, b, rev, s);
        }
    } else {
        switch (tile) {
        case 1: return launch_tma_tile<PT, L, NCOMP, 32, 4, 1, COLL>(tm, p, b, rev, s);
        case 2: return launch_tma_tile<PT, L, NCOMP, 32, 16, 1, COLL>(tm, p, b, rev, s);
        case 3: if constexpr (COLL == 0) return launch_pers_tile<PT, L, NCOMP, 32, 8, 1>(tm, p, b, rev, s);
        case 4: if constexpr (COLL == 0) return launch_pers_tile<PT, L, NCOMP, 32, 4, 1>(tm, p, b, rev, s);
        case 5: if constexpr (COLL == 0) return launch_pers_tile<PT, L, NCOMP, 32, 16, 1>(tm, p, b, rev, s);
        default: return launch_tma_tile<PT, L, NCOMP, 32, 8, 1, COLL>(tm, p, b, rev, s);
        }
    }
}

// Collide-stream launch of one collision kind (TMA-staged when a tensor map
// is given, else the register kernel).
template <int COLL>
cudaError_t launch_lattice_coll(int lattice, int ncomp, const StepParams& p, const StepBufs& b, cudaStream_t s,
                                const void* tensor_map, int rev, int tile, Parts parts) {
    if (tensor_map) {
        const CUtensorMap* tm = static_cast<const CUtensorMap*>(tensor_map);
        cudaError_t e = cudaSuccess;
        VEFD_WITH_PT(p.prec, {
            if (lattice == 1)
                e = ncomp == 2 ? launch_tma<PT, D3Q19, 2, COLL>(tm, p, b, rev, s, tile, parts)
                               : launch_tma<PT, D3Q19, 1, COLL>(tm, p, b, rev, s, tile, parts);
            else
                e = ncomp == 2 ? launch_tma<PT, D2Q9, 2, COLL>(tm, p, b, rev, s, tile, parts)
                               : launch_tma<PT, D2Q9, 1, COLL>(tm, p, b, rev, s, tile, parts);
        });
        return e;
    }
    if (parts.part) return cudaErrorInvalidValue;  // partial densities need the staged kernel
    dim3 blk(32, 4, 1), grd = node_grid(p);
    VEFD_WITH_PT(p.prec, {
        if (lattice == 1) {
            if (ncomp == 2) k_lattice<PT, D3Q19, 2, true, COLL><<<grd, blk, 0, s>>>(b, p, rev);
            else k_lattice<PT, D3Q19, 1, true, COLL><<<grd, blk, 0, s>>>(b, p, rev);
        } else {
            if (ncomp == 2) k_lattice<PT, D2Q9, 2, true, COLL><<<grd, blk, 0, s>>>(b, p, rev);
            else k_lattice<PT, D2Q9, 1, true, COLL><<<grd, blk, 0, s>>>(b, p, rev);
        }
    });
    return cudaGetLastError();
}

using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

}  // namespace
}  // namespace vefd
