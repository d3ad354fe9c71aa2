/*
 * FP64 CPU oracle for the hybrid LBM / FD viscoelastic two-component step.
 *
 * TEST INFRASTRUCTURE ONLY: a plain, slow, serial restatement of the method
 * of Gupta, Sbragaglia & Scagliarini (Sec. 2), used to check the CUDA
 * library.  It shares no source with it.  Every loop runs over nodes in the
 * order x fastest, then y, then z; nothing is fused or reordered beyond what
 * the equations state.  Loops over independent nodes may run on several
 * OpenMP threads; every node's arithmetic is the same whatever the thread
 * count, and all sums across nodes (diagnostics) stay serial.
 *
 * One time step n -> n+1 (the paper leaves the ordering open; this is the
 * reading used throughout):
 *   1. moments       rho_sigma = sum_a f_a, rho u~ = sum_sigma sum_a c_a f_a     (Sec. 2, moments)
 *   2. Shan-Chen     g_sigma = -G rho_sigma sum_a w_a rho_sigma'(x+c_a) c_a       (Eq. SCforce)
 *   3. polymer force F_p = (eta_P/tau_P) div[(f(r_P) C - I) m(phi)]              (Eq. NS, Sec. 2 end)
 *   4. velocity      u = u~ + sum(forces)/(2 rho)                                (Eq. equilibrium:vel)
 *   5. viscosity     rho c_s^2 (tau - 1/2) = eta_A f_+ + eta_B f_-              (Eq. smoothingvisco)
 *   6. collision     BGK form of Eq. (LB) with the source S_a(u, F_sigma)
 *   7. streaming     periodic x, z; half-way bounce-back with moving walls in y
 *   8. FENE-P        R = -(u.grad)C + C.grad u + (grad u)^T.C - (f C - I)/tau_P
 *                        + kappa lap C                                           (Eq. FENE + diffusivity)
 *   9. AB2           C^{n+1} = C^n + 3/2 R^n - 1/2 R^{n-1}; Euler on the first step
 * Steps 8-9 use u^n and C^n of steps 1-4.
 *
 * Polymer feedback, two readings of Sec. 2: (a) the body force
 * (eta_P/tau_P) div[(f C - I) m(phi)] shared by rho_sigma/rho (coupling 0), or
 * (b) Eq. MODEtransformation: the stress T_sigma = -(rho_sigma/rho)(eta_P/tau_P)
 * (f C - I) m(phi) added to the second moment of each component's equilibrium
 * (coupling 1); in BGK form E_a += w_a (c_a c_a - c_s^2 I):T_sigma / (2 c_s^4),
 * which leaves mass and momentum unchanged and adds exactly T_sigma to the
 * second moment.
 *
 * Collision, two readings of Sec. 2: (a) a single relaxation time, the local
 * tau of the viscosity field (collision 0); (b) the paper's relaxation in
 * moment space (collision 1): every component's populations are mapped to
 * the orthogonal moments of Premnath & Abraham's transformation (the
 * polynomial rows of d'Humieres et al. for D3Q19, of Lallemand & Luo for
 * D2Q9), each moment relaxes towards the moment of E with its own time -
 * the shear and bulk modes with the local tau (tau_b = tau_s), the species
 * momentum with tau_M, all other modes with tau_g (the paper uses
 * tau_M = tau_g = 1) - and the source enters as (I - Lambda/2) S in the same
 * moment space.
 *
 * Conformation update, two readings of Sec. 2: (a) AB2 on C (chol 0); (b) the
 * Cholesky scheme (chol 1): sigma_P = f(r_P) C = L L^T with L lower
 * triangular; the same right-hand side dC/dt gives d sigma_P/dt = f dC/dt +
 * sigma_P f tr(dC/dt)/(L^2 - 3), then dL/dt = L Phi(L^-1 (d sigma_P/dt) L^-T)
 * with Phi the lower triangle with the diagonal halved; AB2 advances ln l_ii
 * and l_ij (i > j), and C = sigma_P / f with f = (L^2 - 3 + tr sigma_P)/L^2,
 * so C stays SPD with tr C < L^2 by construction.
 *
 * Boundary readings (the paper states the rules only in words):
 *   - densities seen by the Shan-Chen sum across a wall take the value of the
 *     adjacent fluid row (zero normal gradient, neutral wetting, Sec. 2);
 *   - C, u and the feedback stress take linearly extrapolated ghost values
 *     v(-1) = 2 v(0) - v(1), v(NY) = 2 v(NY-1) - v(NY-2) (Sec. 2, "linear
 *     extrapolation at the boundaries");
 *   - moving walls use Ladd's bounce-back term -2 w_a rho_sigma (c_a.U)/c_s^2
 *     with the local component density (Sec. 3.1, bounce-back rule).
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define CS2 (1.0 / 3.0)

/* D2Q9: rest, +-x, +-y, then diagonals as opposite pairs. Weights 4/9, 1/9, 1/36. */
static const int C9[9][3] = {
    {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0}};
static const double W9[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* D3Q19: rest, +-x, +-y, +-z, then the twelve face diagonals as opposite pairs.
 * Weights 1/3, 1/18 (a = 1..6), 1/36 (a = 7..18) (Sec. 2, D3Q19 weights). */
static const int C19[19][3] = {
    {0, 0, 0}, {1, 0, 0}, {-1, 0, 0}, {0, 1, 0}, {0, -1, 0}, {0, 0, 1}, {0, 0, -1},
    {1, 1, 0}, {-1, -1, 0}, {1, -1, 0}, {-1, 1, 0},
    {1, 0, 1}, {-1, 0, -1}, {1, 0, -1}, {-1, 0, 1},
    {0, 1, 1}, {0, -1, -1}, {0, 1, -1}, {0, -1, 1}};
static const double W19[19] = {
    1.0 / 3.0,
    1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0, 1.0 / 18.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0,
    1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

/* symmetric tensor component index (i, j) -> 0..5 in order xx xy xz yy yz zz */
static const int SYM[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};

struct orc_state {
    orc_params p;
    int Q;
    const int (*c)[3];
    const double *w;
    long N;
    double *f, *fn;        /* populations [ncomp][Q][N] */
    double *C, *Rp;        /* conformation tensor and AB2 history [6][N] */
    int have_prev;
    long step;
    unsigned status;
    /* derived fields of the current state */
    double *rho;           /* [2][N] */
    double *j;             /* [3][N] momentum sum_sigma sum_a c_a f_a */
    double *g;             /* [2][3][N] Shan-Chen forces */
    double *Qs;            /* [6][N] feedback stress (f C - I) m(phi) */
    double *Fp;            /* [3][N] polymer body force */
    double *u;             /* [3][N] equilibrium velocity */
    double *tau;           /* [N] local relaxation time */
    /* moment basis of the MRT collision */
    double Mb[19][19];
    double Mnorm[19];
    int Mkind[19];
};

static int opposite(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }

static long node(const orc_state *s, int x, int y, int z) {
    return ((long)z * s->p.ny + y) * s->p.nx + x;
}

/* periodic image of v in [0, n); offsets here never exceed one period */
static int wrap(int v, int n) {
    if (v < 0) return v + n;
    if (v >= n) return v - n;
    return v;
}

static double fplus(double phi, double delta) { return 0.5 * (1.0 + tanh(phi / delta)); }
static double fminus(double phi, double delta) { return 0.5 * (1.0 - tanh(phi / delta)); }

static double phi_of(const orc_state *s, long i) {
    if (s->p.ncomp == 1) return 1.0;
    double ra = s->rho[i], rb = s->rho[s->N + i];
    return (ra - rb) / (ra + rb);
}

/* FENE-P potential f(r_P) = (L^2 - 3) / (L^2 - tr C)  (Sec. 2) */
static double fene_f(double L2, double trC) { return (L2 - 3.0) / (L2 - trC); }

static double modulation(const orc_state *s, double phi) {
    if (s->p.phase > 0) return fplus(phi, s->p.delta);
    if (s->p.phase < 0) return fminus(phi, s->p.delta);
    return 1.0;
}

/* Value of component k of a node field at (x, y, z) where y may be -1 or NY
 * (ghost rows).  Periodic in x and z; in y either periodic or linearly
 * extrapolated from the two nearest fluid rows. */
static double field_at(const orc_state *s, const double *fld, int k, int x, int y, int z) {
    const int nx = s->p.nx, ny = s->p.ny, nz = s->p.nz;
    x = wrap(x, nx);
    z = wrap(z, nz);
    const double *F = fld + (long)k * s->N;
    if (!s->p.walls) return F[node(s, x, wrap(y, ny), z)];
    if (y < 0) return 2.0 * F[node(s, x, 0, z)] - F[node(s, x, 1, z)];
    if (y >= ny) return 2.0 * F[node(s, x, ny - 1, z)] - F[node(s, x, ny - 2, z)];
    return F[node(s, x, y, z)];
}

/* central first derivative along axis `ax` (0 x, 1 y, 2 z) */
static double d1(const orc_state *s, const double *fld, int k, int x, int y, int z, int ax) {
    int e[3] = {0, 0, 0};
    e[ax] = 1;
    return 0.5 * (field_at(s, fld, k, x + e[0], y + e[1], z + e[2]) -
                  field_at(s, fld, k, x - e[0], y - e[1], z - e[2]));
}

/* central second derivative along axis `ax` */
static double d2(const orc_state *s, const double *fld, int k, int x, int y, int z, int ax) {
    int e[3] = {0, 0, 0};
    e[ax] = 1;
    return field_at(s, fld, k, x + e[0], y + e[1], z + e[2]) - 2.0 * field_at(s, fld, k, x, y, z) +
           field_at(s, fld, k, x - e[0], y - e[1], z - e[2]);
}

static int ndim(const orc_state *s) { return s->p.lattice == ORC_D3Q19 ? 3 : 2; }

/* ---- single-node formulas ------------------------------------------------ */

/* E_a = w_a rho [1 + c.u/cs2 + uu:(cc - cs2 I)/(2 cs2^2)]  (Sec. 2, equilibrium) */
static double equilibrium(double w, const int c[3], double rho, const double u[3]) {
    double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    return w * rho * (1.0 + cu / CS2 + (cu * cu - CS2 * uu) / (2.0 * CS2 * CS2));
}

/* S_a = w_a [(c - u)/cs2 + (c.u) c / cs2^2] . F  (Sec. 2, source term) */
static double source(double w, const int c[3], const double u[3], const double F[3]) {
    double cu = c[0] * u[0] + c[1] * u[1] + c[2] * u[2];
    double s = 0.0;
    for (int k = 0; k < 3; ++k) s += ((c[k] - u[k]) / CS2 + cu * c[k] / (CS2 * CS2)) * F[k];
    return w * s;
}

/* ---- moment basis of the MRT collision (Sec. 2) -----------------------------
 * Rows are orthogonal polynomials in c evaluated on the lattice velocities:
 *   D3Q19: 1, 19c^2 - 30, (21c^4 - 53c^2 + 24)/2, c_x, (5c^2 - 9)c_x, c_y,
 *          (5c^2 - 9)c_y, c_z, (5c^2 - 9)c_z, 3c_x^2 - c^2,
 *          (3c^2 - 5)(3c_x^2 - c^2), c_y^2 - c_z^2, (3c^2 - 5)(c_y^2 - c_z^2),
 *          c_x c_y, c_y c_z, c_x c_z, (c_y^2 - c_z^2)c_x, (c_z^2 - c_x^2)c_y,
 *          (c_x^2 - c_y^2)c_z
 *   D2Q9:  1, 3c^2 - 4, (9c^4 - 21c^2 + 8)/2, c_x, (3c^2 - 5)c_x, c_y,
 *          (3c^2 - 5)c_y, c_x^2 - c_y^2, c_x c_y
 * and each row has a relaxation kind. */
enum { MK_RHO = 0, MK_BULK = 1, MK_MOM = 2, MK_SHEAR = 3, MK_GHOST = 4 };

static double mrt_row(int lattice, int k, const int c[3], int *kind) {
    const double x = c[0], y = c[1], z = c[2];
    const double c2 = x * x + y * y + z * z;
    if (lattice == ORC_D3Q19) {
        switch (k) {
        case 0: *kind = MK_RHO; return 1.0;
        case 1: *kind = MK_BULK; return 19.0 * c2 - 30.0;
        case 2: *kind = MK_GHOST; return (21.0 * c2 * c2 - 53.0 * c2 + 24.0) / 2.0;
        case 3: *kind = MK_MOM; return x;
        case 4: *kind = MK_GHOST; return (5.0 * c2 - 9.0) * x;
        case 5: *kind = MK_MOM; return y;
        case 6: *kind = MK_GHOST; return (5.0 * c2 - 9.0) * y;
        case 7: *kind = MK_MOM; return z;
        case 8: *kind = MK_GHOST; return (5.0 * c2 - 9.0) * z;
        case 9: *kind = MK_SHEAR; return 3.0 * x * x - c2;
        case 10: *kind = MK_GHOST; return (3.0 * c2 - 5.0) * (3.0 * x * x - c2);
        case 11: *kind = MK_SHEAR; return y * y - z * z;
        case 12: *kind = MK_GHOST; return (3.0 * c2 - 5.0) * (y * y - z * z);
        case 13: *kind = MK_SHEAR; return x * y;
        case 14: *kind = MK_SHEAR; return y * z;
        case 15: *kind = MK_SHEAR; return x * z;
        case 16: *kind = MK_GHOST; return (y * y - z * z) * x;
        case 17: *kind = MK_GHOST; return (z * z - x * x) * y;
        default: *kind = MK_GHOST; return (x * x - y * y) * z;
        }
    }
    switch (k) {
    case 0: *kind = MK_RHO; return 1.0;
    case 1: *kind = MK_BULK; return 3.0 * c2 - 4.0;
    case 2: *kind = MK_GHOST; return (9.0 * c2 * c2 - 21.0 * c2 + 8.0) / 2.0;
    case 3: *kind = MK_MOM; return x;
    case 4: *kind = MK_GHOST; return (3.0 * c2 - 5.0) * x;
    case 5: *kind = MK_MOM; return y;
    case 6: *kind = MK_GHOST; return (3.0 * c2 - 5.0) * y;
    case 7: *kind = MK_SHEAR; return x * x - y * y;
    default: *kind = MK_SHEAR; return x * y;
    }
}

static int mrt_basis_fill(int lattice, double M[19][19], double norm[19], int kind[19]) {
    const int Q = lattice == ORC_D3Q19 ? 19 : 9;
    const int (*c)[3] = lattice == ORC_D3Q19 ? C19 : C9;
    for (int k = 0; k < Q; ++k) {
        norm[k] = 0.0;
        for (int a = 0; a < Q; ++a) {
            M[k][a] = mrt_row(lattice, k, c[a], &kind[k]);
            norm[k] += M[k][a] * M[k][a];
        }
    }
    return Q;
}

/* ---- Cholesky scheme for sigma_P = f(r_P) C (Sec. 2) ----------------------- */

/* log-Cholesky variables of sigma_P and their rates for a given dC/dt */
static void chol_rates_node(const double C6[6], const double Cd6[6], double L2, double lam[6], double rl[6]) {
    const double fr = fene_f(L2, C6[0] + C6[3] + C6[5]);
    const double trCd = Cd6[0] + Cd6[3] + Cd6[5];
    double S[3][3], Sd[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            S[a][b] = fr * C6[SYM[a][b]];
            Sd[a][b] = fr * Cd6[SYM[a][b]] + S[a][b] * fr * trCd / (L2 - 3.0);
        }
    /* S = L L^T */
    double L[3][3] = {{0}};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j <= i; ++j) {
            double v = S[i][j];
            for (int k = 0; k < j; ++k) v -= L[i][k] * L[j][k];
            L[i][j] = (i == j) ? sqrt(v) : v / L[j][j];
        }
    /* inverse of the lower-triangular factor */
    double Li[3][3] = {{0}};
    for (int j = 0; j < 3; ++j) {
        Li[j][j] = 1.0 / L[j][j];
        for (int i = j + 1; i < 3; ++i) {
            double v = 0.0;
            for (int k = j; k < i; ++k) v -= L[i][k] * Li[k][j];
            Li[i][j] = v / L[i][i];
        }
    }
    /* A = L^-1 Sd L^-T; Phi(A) = lower triangle of A with the diagonal halved */
    double T[3][3], A[3][3], P[3][3] = {{0}};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double v = 0.0;
            for (int k = 0; k < 3; ++k) v += Li[i][k] * Sd[k][j];
            T[i][j] = v;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double v = 0.0;
            for (int k = 0; k < 3; ++k) v += T[i][k] * Li[j][k];
            A[i][j] = v;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j <= i; ++j) P[i][j] = (i == j) ? 0.5 * A[i][i] : A[i][j];
    /* dL/dt = L Phi(A) */
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j <= i; ++j) {
            double v = 0.0;
            for (int k = j; k <= i; ++k) v += L[i][k] * P[k][j];
            if (i == j) {
                lam[SYM[i][i]] = log(L[i][i]);
                rl[SYM[i][i]] = v / L[i][i];
            } else {
                lam[SYM[i][j]] = L[i][j];
                rl[SYM[i][j]] = v;
            }
        }
}

/* C from the log-Cholesky variables of sigma_P */
static void chol_to_C_node(const double lam[6], double L2, double C6[6]) {
    double L[3][3] = {{0}};
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j <= i; ++j) L[i][j] = (i == j) ? exp(lam[SYM[i][i]]) : lam[SYM[i][j]];
    double S[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            double v = 0.0;
            for (int k = 0; k < 3; ++k) v += L[a][k] * L[b][k];
            S[a][b] = v;
        }
    const double fr = (L2 - 3.0 + S[0][0] + S[1][1] + S[2][2]) / L2;
    for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b) C6[SYM[a][b]] = S[a][b] / fr;
}

/* ---- derived fields ------------------------------------------------------- */

static void compute_moments(orc_state *s) {
    const long N = s->N;
    const int Q = s->Q;
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < N; ++i) {
        double jx = 0, jy = 0, jz = 0;
        for (int sg = 0; sg < s->p.ncomp; ++sg) {
            double r = 0.0;
            for (int a = 0; a < Q; ++a) {
                double fa = s->f[((long)sg * Q + a) * N + i];
                r += fa;
                jx += s->c[a][0] * fa;
                jy += s->c[a][1] * fa;
                jz += s->c[a][2] * fa;
            }
            s->rho[sg * N + i] = r;
        }
        if (s->p.ncomp == 1) s->rho[N + i] = 0.0;
        s->j[i] = jx;
        s->j[N + i] = jy;
        s->j[2 * N + i] = jz;
    }
}

/* g_sigma(x) = -G rho_sigma(x) sum_a w_a rho_sigma'(x + c_a) c_a  (Eq. SCforce) */
static void compute_sc_force(orc_state *s) {
    const long N = s->N;
    memset(s->g, 0, sizeof(double) * 6 * N);
    if (s->p.ncomp < 2) return;
    #pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < s->p.nz; ++z)
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x) {
                long i = node(s, x, y, z);
                for (int sg = 0; sg < 2; ++sg) {
                    const double *rother = s->rho + (long)(1 - sg) * N;
                    double acc[3] = {0, 0, 0};
                    for (int a = 1; a < s->Q; ++a) {
                        int xx = wrap(x + s->c[a][0], s->p.nx);
                        int zz = wrap(z + s->c[a][2], s->p.nz);
                        int yy = y + s->c[a][1];
                        if (s->p.walls) {
                            if (yy < 0) yy = 0;             /* ghost row mirrors row 0 */
                            if (yy >= s->p.ny) yy = s->p.ny - 1;
                        } else {
                            yy = wrap(yy, s->p.ny);
                        }
                        double rn = rother[node(s, xx, yy, zz)];
                        for (int k = 0; k < 3; ++k) acc[k] += s->w[a] * rn * s->c[a][k];
                    }
                    double rs = s->rho[sg * N + i];
                    for (int k = 0; k < 3; ++k) s->g[((long)sg * 3 + k) * N + i] = -s->p.G * rs * acc[k];
                }
            }
}

/* F_p = (eta_P / tau_P) div[(f(r_P) C - I) m(phi)]  (Eq. NS with the phase
 * modulation of the last equation of Sec. 2; the identity is subtracted so
 * the feedback vanishes at rest) */
static void compute_polymer_force(orc_state *s) {
    const long N = s->N;
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < N; ++i) {
        double trC = s->C[0 * N + i] + s->C[3 * N + i] + s->C[5 * N + i];
        double fr = fene_f(s->p.L2, trC);
        double m = modulation(s, phi_of(s, i));
        for (int k = 0; k < 6; ++k) {
            double delta_ij = (k == 0 || k == 3 || k == 5) ? 1.0 : 0.0;
            s->Qs[k * N + i] = (fr * s->C[k * N + i] - delta_ij) * m;
        }
    }
    const double pref = s->p.eta_p / s->p.tau_p;
    const int nd = ndim(s);
    if (s->p.coupling == 1) {
        /* the stress enters the equilibrium instead of a force */
        memset(s->Fp, 0, sizeof(double) * 3 * N);
        return;
    }
    #pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < s->p.nz; ++z)
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x) {
                long i = node(s, x, y, z);
                for (int jj = 0; jj < 3; ++jj) {
                    double div = 0.0;
                    for (int ii = 0; ii < nd; ++ii) div += d1(s, s->Qs, SYM[ii][jj], x, y, z, ii);
                    s->Fp[(long)jj * N + i] = pref * div;
                }
            }
}

/* total force on component sigma: g_sigma + (rho_sigma/rho)(F_p + F_ext) */
static void component_force(const orc_state *s, long i, int sg, double F[3]) {
    const long N = s->N;
    double rho = s->rho[i] + s->rho[N + i];
    double share = s->rho[(long)sg * N + i] / rho;
    for (int k = 0; k < 3; ++k)
        F[k] = s->g[((long)sg * 3 + k) * N + i] + share * (s->Fp[(long)k * N + i] + s->p.fext[k]);
}

/* u = (rho u~ + 1/2 sum_sigma F_sigma) / rho  (Eq. equilibrium:vel) and the
 * local relaxation time from rho c_s^2 (tau - 1/2) = eta_A f_+ + eta_B f_- */
static void compute_velocity_tau(orc_state *s) {
    const long N = s->N;
    #pragma omp parallel for schedule(static)
    for (long i = 0; i < N; ++i) {
        double rho = s->rho[i] + s->rho[N + i];
        double Ftot[3] = {0, 0, 0};
        for (int sg = 0; sg < s->p.ncomp; ++sg) {
            double F[3];
            component_force(s, i, sg, F);
            for (int k = 0; k < 3; ++k) Ftot[k] += F[k];
        }
        for (int k = 0; k < 3; ++k) s->u[(long)k * N + i] = (s->j[(long)k * N + i] + 0.5 * Ftot[k]) / rho;
        double phi = phi_of(s, i);
        double eta = s->p.eta_A * fplus(phi, s->p.delta) + s->p.eta_B * fminus(phi, s->p.delta);
        s->tau[i] = 0.5 + eta / (rho * CS2);
    }
}

static void compute_derived(orc_state *s) {
    compute_moments(s);
    compute_sc_force(s);
    compute_polymer_force(s);
    compute_velocity_tau(s);
}

/* ---- one time step ------------------------------------------------------- */

static void collide_stream(orc_state *s) {
    const long N = s->N;
    const int Q = s->Q;
    #pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < s->p.nz; ++z)
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x) {
                long i = node(s, x, y, z);
                double u[3] = {s->u[i], s->u[N + i], s->u[2 * N + i]};
                double tau = s->tau[i];
                for (int sg = 0; sg < s->p.ncomp; ++sg) {
                    double F[3];
                    component_force(s, i, sg, F);
                    double rs = s->rho[(long)sg * N + i];
                    /* equilibrium stress of Eq. MODEtransformation (coupling 1) */
                    double T[3][3] = {{0}};
                    if (s->p.coupling == 1) {
                        double share = rs / (s->rho[i] + s->rho[N + i]);
                        for (int aa = 0; aa < 3; ++aa)
                            for (int bb = 0; bb < 3; ++bb)
                                T[aa][bb] = -share * s->p.eta_p / s->p.tau_p * s->Qs[(long)SYM[aa][bb] * N + i];
                    }
                    const int nd = ndim(s);
                    double fl[19], El[19], Sl[19], fp[19];
                    for (int a = 0; a < Q; ++a) {
                        fl[a] = s->f[((long)sg * Q + a) * N + i];
                        double E = equilibrium(s->w[a], s->c[a], rs, u);
                        if (s->p.coupling == 1) {
                            double cTc = 0.0, trT = 0.0;
                            for (int aa = 0; aa < nd; ++aa) {
                                trT += T[aa][aa];
                                for (int bb = 0; bb < nd; ++bb) cTc += s->c[a][aa] * s->c[a][bb] * T[aa][bb];
                            }
                            E += s->w[a] * (cTc - CS2 * trT) / (2.0 * CS2 * CS2);
                        }
                        El[a] = E;
                        Sl[a] = source(s->w[a], s->c[a], u, F);
                    }
                    if (s->p.collision == 1) {
                        /* Eq. (LB) in moment space: m = M f, relaxation of each moment
                         * towards M E with its rate, source (1 - rate/2) M S, back with
                         * M^-1 = M^T diag(1/|row|^2) */
                        double d[19];
                        for (int k = 0; k < Q; ++k) {
                            double m = 0.0, meq = 0.0, ms = 0.0;
                            for (int a = 0; a < Q; ++a) {
                                m += s->Mb[k][a] * fl[a];
                                meq += s->Mb[k][a] * El[a];
                                ms += s->Mb[k][a] * Sl[a];
                            }
                            double rate;
                            switch (s->Mkind[k]) {
                            case MK_MOM: rate = 1.0 / s->p.tau_M; break;
                            case MK_GHOST: rate = 1.0 / s->p.tau_g; break;
                            default: rate = 1.0 / tau; break; /* shear, bulk (conserved density: no change) */
                            }
                            d[k] = -rate * (m - meq) + (1.0 - 0.5 * rate) * ms;
                        }
                        for (int a = 0; a < Q; ++a) {
                            double v = fl[a];
                            for (int k = 0; k < Q; ++k) v += s->Mb[k][a] * d[k] / s->Mnorm[k];
                            fp[a] = v;
                        }
                    } else {
                        /* Eq. (LB) with Lambda = 1/tau: f* = f - (f - E)/tau + (1 - 1/(2 tau)) S */
                        for (int a = 0; a < Q; ++a) fp[a] = fl[a] - (fl[a] - El[a]) / tau + (1.0 - 0.5 / tau) * Sl[a];
                    }
                    for (int a = 0; a < Q; ++a) {
                        double fpost = fp[a];
                        int xt = wrap(x + s->c[a][0], s->p.nx);
                        int zt = wrap(z + s->c[a][2], s->p.nz);
                        int yt = y + s->c[a][1];
                        if (s->p.walls && (yt < 0 || yt >= s->p.ny)) {
                            /* half-way bounce-back; wall velocity +U at y=-1/2, -U at y=NY-1/2 */
                            double Uw = (yt < 0) ? s->p.u_wall : -s->p.u_wall;
                            double cU = s->c[a][0] * Uw;
                            s->fn[((long)sg * Q + opposite(a)) * N + i] = fpost - 2.0 * s->w[a] * rs * cU / CS2;
                        } else {
                            if (!s->p.walls) yt = wrap(yt, s->p.ny);
                            s->fn[((long)sg * Q + a) * N + node(s, xt, yt, zt)] = fpost;
                        }
                    }
                }
            }
    double *t = s->f;
    s->f = s->fn;
    s->fn = t;
}

/* Right-hand side of the conformation equation at one node,
 * R = -(u.grad)C + C.grad u + (grad u)^T.C - (f C - I)/tau_P + kappa lap C,
 * with (grad u)_ij = d_i u_j (Eq. FENE plus the artificial diffusivity).
 * adv[k] = (u.grad) C_k and lap[k] = lap C_k are given per component. */
static void fenep_rhs_node(const double Cm[3][3], const double Gu[3][3], const double adv[6],
                           const double lap[6], double tau_p, double L2, double kappa, double R[6]) {
    double fr = fene_f(L2, Cm[0][0] + Cm[1][1] + Cm[2][2]);
    for (int a = 0; a < 3; ++a)
        for (int b = a; b < 3; ++b) {
            int k = SYM[a][b];
            double up = 0.0;
            for (int e = 0; e < 3; ++e) up += Cm[a][e] * Gu[e][b] + Gu[e][a] * Cm[e][b];
            double delta_ab = (a == b) ? 1.0 : 0.0;
            R[k] = -adv[k] + up - (fr * Cm[a][b] - delta_ab) / tau_p + kappa * lap[k];
        }
}

/* one explicit FD step of the conformation tensor: central differences,
 * then Adams-Bashforth 2 (forward Euler when there is no history) */
static void fenep_update(orc_state *s, double *Cnew) {
    const long N = s->N;
    const int nd = ndim(s);
    #pragma omp parallel for collapse(2) schedule(static)
    for (int z = 0; z < s->p.nz; ++z)
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x) {
                long i = node(s, x, y, z);
                double Gu[3][3] = {{0}};
                for (int a = 0; a < nd; ++a)
                    for (int b = 0; b < 3; ++b) Gu[a][b] = d1(s, s->u, b, x, y, z, a);
                double Cm[3][3];
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) Cm[a][b] = s->C[(long)SYM[a][b] * N + i];
                double uu[3] = {s->u[i], s->u[N + i], s->u[2 * N + i]};
                double adv[6], lap[6], R[6];
                for (int k = 0; k < 6; ++k) {
                    adv[k] = 0.0;
                    lap[k] = 0.0;
                    for (int e = 0; e < nd; ++e) {
                        adv[k] += uu[e] * d1(s, s->C, k, x, y, z, e);
                        lap[k] += d2(s, s->C, k, x, y, z, e);
                    }
                }
                fenep_rhs_node(Cm, Gu, adv, lap, s->p.tau_p, s->p.L2, s->p.kappa, R);
                if (s->p.chol) {
                    /* AB2 on the log-Cholesky variables of sigma_P; the history holds their rates */
                    double C6[6], lam[6], rl[6], lamn[6], Cn[6];
                    for (int k = 0; k < 6; ++k) C6[k] = s->C[(long)k * N + i];
                    chol_rates_node(C6, R, s->p.L2, lam, rl);
                    for (int k = 0; k < 6; ++k) {
                        double inc = s->have_prev ? 1.5 * rl[k] - 0.5 * s->Rp[(long)k * N + i] : rl[k];
                        lamn[k] = lam[k] + inc;
                        s->Rp[(long)k * N + i] = rl[k];
                    }
                    chol_to_C_node(lamn, s->p.L2, Cn);
                    for (int k = 0; k < 6; ++k) Cnew[(long)k * N + i] = Cn[k];
                    continue;
                }
                for (int k = 0; k < 6; ++k) {
                    double inc = s->have_prev ? 1.5 * R[k] - 0.5 * s->Rp[(long)k * N + i] : R[k];
                    Cnew[(long)k * N + i] = s->C[(long)k * N + i] + inc;
                    /* the history is only read at this node, so it is replaced in place */
                    s->Rp[(long)k * N + i] = R[k];
                }
            }
}

static void guards(orc_state *s, const double *Cnext) {
    const long N = s->N;
    unsigned st = s->status;
    #pragma omp parallel for reduction(|:st) schedule(static)
    for (long i = 0; i < N; ++i) {
        double rho = s->rho[i] + s->rho[N + i];
        double u2 = 0;
        for (int k = 0; k < 3; ++k) u2 += s->u[(long)k * N + i] * s->u[(long)k * N + i];
        if (!(rho > 0.0)) st |= isnan(rho) ? ORC_ST_NAN : ORC_ST_RHO;
        if (isnan(u2)) st |= ORC_ST_NAN;
        if (u2 > 0.09) st |= ORC_ST_MACH;
        const double *Cs[2] = {s->C, Cnext};
        for (int q = 0; q < 2; ++q) {
            if (!Cs[q]) continue;
            double tr = Cs[q][i] + Cs[q][3 * N + i] + Cs[q][5 * N + i];
            if (isnan(tr)) st |= ORC_ST_NAN;
            else if (tr >= s->p.L2) st |= ORC_ST_TRACE;
        }
    }
    s->status = st;
}

int orc_step(orc_state *s, long nsteps) {
    if (!s || nsteps < 0) return -1;
    double *Cnew = (double *)malloc(sizeof(double) * 6 * s->N);
    if (!Cnew) return -2;
    for (long n = 0; n < nsteps; ++n) {
        compute_derived(s);
        collide_stream(s);
        if (s->p.fd_on) {
            fenep_update(s, Cnew);
            guards(s, Cnew);
            memcpy(s->C, Cnew, sizeof(double) * 6 * s->N);
            s->have_prev = 1;
        } else {
            guards(s, NULL);
        }
        s->step++;
    }
    free(Cnew);
    return 0;
}

/* ---- construction and field access --------------------------------------- */

static int params_ok(const orc_params *p) {
    if (p->lattice != ORC_D2Q9 && p->lattice != ORC_D3Q19) return 0;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return 0;
    if (p->lattice == ORC_D2Q9 && p->nz != 1) return 0;
    if (p->walls && p->ny < 2) return 0;
    if (p->ncomp != 1 && p->ncomp != 2) return 0;
    if (!(p->L2 > 3.0) || !(p->tau_p > 0.0) || !(p->delta > 0.0)) return 0;
    if (p->collision != 0 && p->collision != 1) return 0;
    if (p->collision == 1 && (!(p->tau_M > 0.5) || !(p->tau_g > 0.5))) return 0;
    if (p->chol != 0 && p->chol != 1) return 0;
    return 1;
}

orc_state *orc_create(const orc_params *p) {
    if (!p || !params_ok(p)) return NULL;
    orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
    if (!s) return NULL;
    s->p = *p;
    if (p->lattice == ORC_D3Q19) {
        s->Q = 19;
        s->c = C19;
        s->w = W19;
    } else {
        s->Q = 9;
        s->c = C9;
        s->w = W9;
    }
    mrt_basis_fill(p->lattice, s->Mb, s->Mnorm, s->Mkind);
    s->N = (long)p->nx * p->ny * p->nz;
    long N = s->N;
    s->f = (double *)calloc((size_t)2 * s->Q * N, sizeof(double));
    s->fn = (double *)calloc((size_t)2 * s->Q * N, sizeof(double));
    s->C = (double *)calloc((size_t)6 * N, sizeof(double));
    s->Rp = (double *)calloc((size_t)6 * N, sizeof(double));
    s->rho = (double *)calloc((size_t)2 * N, sizeof(double));
    s->j = (double *)calloc((size_t)3 * N, sizeof(double));
    s->g = (double *)calloc((size_t)6 * N, sizeof(double));
    s->Qs = (double *)calloc((size_t)6 * N, sizeof(double));
    s->Fp = (double *)calloc((size_t)3 * N, sizeof(double));
    s->u = (double *)calloc((size_t)3 * N, sizeof(double));
    s->tau = (double *)calloc((size_t)N, sizeof(double));
    if (!s->f || !s->fn || !s->C || !s->Rp || !s->rho || !s->j || !s->g || !s->Qs || !s->Fp || !s->u ||
        !s->tau) {
        orc_destroy(s);
        return NULL;
    }
    for (long i = 0; i < N; ++i) s->C[i] = s->C[3 * N + i] = s->C[5 * N + i] = 1.0;
    return s;
}

void orc_destroy(orc_state *s) {
    if (!s) return;
    free(s->f); free(s->fn); free(s->C); free(s->Rp); free(s->rho); free(s->j);
    free(s->g); free(s->Qs); free(s->Fp); free(s->u); free(s->tau);
    free(s);
}

int orc_set_params(orc_state *s, const orc_params *p) {
    if (!s || !p || !params_ok(p)) return -1;
    if (p->lattice != s->p.lattice || p->nx != s->p.nx || p->ny != s->p.ny || p->nz != s->p.nz ||
        p->ncomp != s->p.ncomp)
        return -1;
    s->p = *p;
    return 0;
}

int orc_num_c(const orc_state *s) { return s->p.lattice == ORC_D3Q19 ? 6 : 4; }
int orc_q(const orc_state *s) { return s->Q; }
unsigned orc_status(const orc_state *s) { return s->status; }
long orc_steps_done(const orc_state *s) { return s->step; }
int orc_set_have_prev(orc_state *s, int hp) { s->have_prev = hp ? 1 : 0; return 0; }

/* API component k of C (4 comps in 2D: xx xy yy zz) -> internal index 0..5 */
static int c_api_to_int(const orc_state *s, int k) {
    static const int map2d[4] = {0, 1, 3, 5};
    return s->p.lattice == ORC_D3Q19 ? k : map2d[k];
}

static void write_tensor(orc_state *s, double *dst_int, const double *src_api) {
    const long N = s->N;
    const int nc = orc_num_c(s);
    if (s->p.lattice == ORC_D2Q9) {
        memset(dst_int + 2 * N, 0, sizeof(double) * N); /* xz */
        memset(dst_int + 4 * N, 0, sizeof(double) * N); /* yz */
    }
    for (int k = 0; k < nc; ++k) memcpy(dst_int + (long)c_api_to_int(s, k) * N, src_api + (long)k * N, sizeof(double) * N);
}

static void read_tensor(const orc_state *s, const double *src_int, double *dst_api) {
    const long N = s->N;
    const int nc = orc_num_c(s);
    for (int k = 0; k < nc; ++k) memcpy(dst_api + (long)k * N, src_int + (long)c_api_to_int(s, k) * N, sizeof(double) * N);
}

int orc_init_fields(orc_state *s, const double *rhoA, const double *rhoB, const double *u, const double *C0) {
    if (!s || !rhoA || (s->p.ncomp == 2 && !rhoB)) return -1;
    const long N = s->N;
    for (long i = 0; i < N; ++i) {
        double uu[3] = {0, 0, 0};
        if (u) {
            uu[0] = u[i];
            uu[1] = u[N + i];
            if (s->p.lattice == ORC_D3Q19) uu[2] = u[2 * N + i];
        }
        for (int sg = 0; sg < s->p.ncomp; ++sg) {
            double r = sg == 0 ? rhoA[i] : rhoB[i];
            for (int a = 0; a < s->Q; ++a) s->f[((long)sg * s->Q + a) * N + i] = equilibrium(s->w[a], s->c[a], r, uu);
        }
    }
    if (C0) {
        write_tensor(s, s->C, C0);
    } else {
        memset(s->C, 0, sizeof(double) * 6 * N);
        for (long i = 0; i < N; ++i) s->C[i] = s->C[3 * N + i] = s->C[5 * N + i] = 1.0;
    }
    memset(s->Rp, 0, sizeof(double) * 6 * N);
    s->have_prev = 0;
    s->step = 0;
    s->status = 0;
    return 0;
}

int orc_write_field(orc_state *s, int field, const double *src) {
    if (!s || !src) return -1;
    const long N = s->N;
    switch (field) {
    case ORC_F_POPS:
        memcpy(s->f, src, sizeof(double) * s->p.ncomp * s->Q * N);
        return 0;
    case ORC_F_C:
        write_tensor(s, s->C, src);
        return 0;
    case ORC_F_RPREV:
        write_tensor(s, s->Rp, src);
        s->have_prev = 1;
        return 0;
    default:
        return -1;
    }
}

int orc_read_field(orc_state *s, int field, double *dst) {
    if (!s || !dst) return -1;
    const long N = s->N;
    const int nd = ndim(s);
    switch (field) {
    case ORC_F_POPS:
        memcpy(dst, s->f, sizeof(double) * s->p.ncomp * s->Q * N);
        return 0;
    case ORC_F_C:
        read_tensor(s, s->C, dst);
        return 0;
    case ORC_F_RPREV:
        read_tensor(s, s->Rp, dst);
        return 0;
    case ORC_F_SIGMA_P: {
        double *tmp = (double *)malloc(sizeof(double) * 6 * N);
        if (!tmp) return -2;
        for (long i = 0; i < N; ++i) {
            double fr = fene_f(s->p.L2, s->C[i] + s->C[3 * N + i] + s->C[5 * N + i]);
            for (int k = 0; k < 6; ++k) tmp[(long)k * N + i] = fr * s->C[(long)k * N + i];
        }
        read_tensor(s, tmp, dst);
        free(tmp);
        return 0;
    }
    default:
        break;
    }
    compute_derived(s);
    switch (field) {
    case ORC_F_RHO_A: memcpy(dst, s->rho, sizeof(double) * N); return 0;
    case ORC_F_RHO_B: memcpy(dst, s->rho + N, sizeof(double) * N); return 0;
    case ORC_F_PHI:
        for (long i = 0; i < N; ++i) dst[i] = phi_of(s, i);
        return 0;
    case ORC_F_U: memcpy(dst, s->u, sizeof(double) * nd * N); return 0;
    case ORC_F_G_A: memcpy(dst, s->g, sizeof(double) * nd * N); return 0;
    case ORC_F_G_B:
        for (int k = 0; k < nd; ++k) memcpy(dst + (long)k * N, s->g + (3L + k) * N, sizeof(double) * N);
        return 0;
    case ORC_F_F_P: memcpy(dst, s->Fp, sizeof(double) * nd * N); return 0;
    case ORC_F_TAU: memcpy(dst, s->tau, sizeof(double) * N); return 0;
    default: return -1;
    }
}

/* Diagnostics of the current state (all sums in FP64):
 *  0 mass_A  1 mass_B  2..4 momentum sum rho u  5 <sigma_P,xy>  6 <sigma_P,xx - sigma_P,yy>
 *  7 max tr C / L^2  8 max |u|  9 droplet area in the plane z = NZ/2 (phi > 0)
 *  10 deformation D = (a-b)/(a+b)  11 orientation theta (rad, major axis vs +x)
 *  12 centroid x  13 centroid y  14 droplet volume (phi > 0)  15 <tr sigma_P> - 3 */
int orc_diagnostics(orc_state *s, double out[16]) {
    if (!s || !out) return -1;
    compute_derived(s);
    const long N = s->N;
    memset(out, 0, sizeof(double) * 16);
    double sxy = 0, n1 = 0, trmax = 0, umax = 0, tr3 = 0, vol = 0;
    double m0 = 0, mx = 0, my = 0, mxx = 0, mxy = 0, myy = 0;
    const int zc = s->p.nz / 2;
    for (int z = 0; z < s->p.nz; ++z)
        for (int y = 0; y < s->p.ny; ++y)
            for (int x = 0; x < s->p.nx; ++x) {
                long i = node(s, x, y, z);
                double rho = s->rho[i] + s->rho[N + i];
                out[0] += s->rho[i];
                out[1] += s->rho[N + i];
                double u2 = 0;
                for (int k = 0; k < 3; ++k) {
                    out[2 + k] += rho * s->u[(long)k * N + i];
                    u2 += s->u[(long)k * N + i] * s->u[(long)k * N + i];
                }
                double trC = s->C[i] + s->C[3 * N + i] + s->C[5 * N + i];
                double fr = fene_f(s->p.L2, trC);
                sxy += fr * s->C[N + i];
                n1 += fr * (s->C[i] - s->C[3 * N + i]);
                tr3 += fr * trC - 3.0;
                if (trC / s->p.L2 > trmax) trmax = trC / s->p.L2;
                if (sqrt(u2) > umax) umax = sqrt(u2);
                double ind = phi_of(s, i) > 0.0 ? 1.0 : 0.0;
                vol += ind;
                if (z == zc && ind > 0) {
                    m0 += 1;
                    mx += x;
                    my += y;
                    mxx += (double)x * x;
                    mxy += (double)x * y;
                    myy += (double)y * y;
                }
            }
    out[5] = sxy / N;
    out[6] = n1 / N;
    out[7] = trmax;
    out[8] = umax;
    out[9] = m0;
    if (m0 > 0) {
        double cx = mx / m0, cy = my / m0;
        double ixx = mxx / m0 - cx * cx, ixy = mxy / m0 - cx * cy, iyy = myy / m0 - cy * cy;
        double tr = ixx + iyy, det = ixx * iyy - ixy * ixy;
        double disc = sqrt(fmax(0.25 * tr * tr - det, 0.0));
        double l1 = 0.5 * tr + disc, l2 = fmax(0.5 * tr - disc, 0.0);
        double a = sqrt(l1), b = sqrt(l2);
        out[10] = (a + b) > 0 ? (a - b) / (a + b) : 0.0;
        out[11] = 0.5 * atan2(2.0 * ixy, ixx - iyy);
        out[12] = cx;
        out[13] = cy;
    }
    out[14] = vol;
    out[15] = tr3 / N;
    return 0;
}

/* ---- single-node entry points -------------------------------------------- */

int orc_lattice(int lattice, int *c_out, double *w_out) {
    int Q = lattice == ORC_D3Q19 ? 19 : 9;
    const int (*c)[3] = lattice == ORC_D3Q19 ? C19 : C9;
    const double *w = lattice == ORC_D3Q19 ? W19 : W9;
    for (int a = 0; a < Q; ++a) {
        for (int k = 0; k < 3; ++k) c_out[a * 3 + k] = c[a][k];
        w_out[a] = w[a];
    }
    return Q;
}

int orc_equilibrium(int lattice, double rho, const double u[3], double *out) {
    int Q = lattice == ORC_D3Q19 ? 19 : 9;
    const int (*c)[3] = lattice == ORC_D3Q19 ? C19 : C9;
    const double *w = lattice == ORC_D3Q19 ? W19 : W9;
    for (int a = 0; a < Q; ++a) out[a] = equilibrium(w[a], c[a], rho, u);
    return Q;
}

int orc_source(int lattice, const double u[3], const double F[3], double *out) {
    int Q = lattice == ORC_D3Q19 ? 19 : 9;
    const int (*c)[3] = lattice == ORC_D3Q19 ? C19 : C9;
    const double *w = lattice == ORC_D3Q19 ? W19 : W9;
    for (int a = 0; a < Q; ++a) out[a] = source(w[a], c[a], u, F);
    return Q;
}

int orc_fenep_point(double *C, double *Rprev, int *have_prev, const double gradu[9], double tau_p, double L2,
                    long nsteps) {
    return orc_fenep_point_form(C, Rprev, have_prev, gradu, tau_p, L2, nsteps, 0);
}

int orc_fenep_point_form(double *C, double *Rprev, int *have_prev, const double gradu[9], double tau_p,
                         double L2, long nsteps, int chol) {
    /* uniform fields: the advection and diffusion terms vanish */
    const double zero[6] = {0, 0, 0, 0, 0, 0};
    double Gu[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) Gu[a][b] = gradu[a * 3 + b];
    for (long n = 0; n < nsteps; ++n) {
        double Cm[3][3], R[6];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) Cm[a][b] = C[SYM[a][b]];
        fenep_rhs_node(Cm, Gu, zero, zero, tau_p, L2, 0.0, R);
        if (chol) {
            double lam[6], rl[6];
            chol_rates_node(C, R, L2, lam, rl);
            for (int k = 0; k < 6; ++k) {
                lam[k] += *have_prev ? 1.5 * rl[k] - 0.5 * Rprev[k] : rl[k];
                Rprev[k] = rl[k];
            }
            chol_to_C_node(lam, L2, C);
        } else {
            for (int k = 0; k < 6; ++k) {
                C[k] += *have_prev ? 1.5 * R[k] - 0.5 * Rprev[k] : R[k];
                Rprev[k] = R[k];
            }
        }
        *have_prev = 1;
    }
    return 0;
}

int orc_chol_rates(const double C[6], const double Cdot[6], double L2, double lam[6], double lam_dot[6]) {
    chol_rates_node(C, Cdot, L2, lam, lam_dot);
    return 0;
}

int orc_chol_to_C(const double lam[6], double L2, double C[6]) {
    chol_to_C_node(lam, L2, C);
    return 0;
}

int orc_mrt_basis(int lattice, double *M, int *kind) {
    double Mb[19][19], norm[19];
    int kd[19];
    const int Q = mrt_basis_fill(lattice, Mb, norm, kd);
    for (int k = 0; k < Q; ++k) {
        if (kind) kind[k] = kd[k];
        for (int a = 0; a < Q; ++a) M[k * Q + a] = Mb[k][a];
    }
    return Q;
}

int orc_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}
