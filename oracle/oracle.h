/*
 * FP64 CPU oracle for the hybrid lattice-Boltzmann / finite-difference
 * viscoelastic two-component step (Gupta, Sbragaglia & Scagliarini,
 * "Hybrid Lattice Boltzmann/Finite Difference simulations of viscoelastic
 * multicomponent flows in confined geometries", Sec. 2).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is a plain, slow restatement of the
 * method used to check the CUDA library.  Only the test-suite, the smoke
 * check and the CPU-baseline leg of the benchmark may load it; the product
 * path never does.  It shares no source with the CUDA library.
 *
 * Layout of every field exchanged through this interface: double precision,
 * x fastest, index = ((comp*NZ + z)*NY + y)*NX + x.  Conformation-tensor
 * components are ordered xx, xy, xz, yy, yz, zz for D3Q19 and xx, xy, yy, zz
 * for D2Q9.
 */
#ifndef VEFD_ORACLE_H
#define VEFD_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_D2Q9 = 0, ORC_D3Q19 = 1 };

enum {
    ORC_F_RHO_A = 0, ORC_F_RHO_B = 1, ORC_F_PHI = 2, ORC_F_U = 3, ORC_F_C = 4,
    ORC_F_SIGMA_P = 5, ORC_F_POPS = 6, ORC_F_RPREV = 7,
    /* derived quantities of the current state, for stage-wise checks */
    ORC_F_G_A = 8, ORC_F_G_B = 9, ORC_F_F_P = 10, ORC_F_TAU = 11
};

/* status bits (sticky) */
enum { ORC_ST_NAN = 1, ORC_ST_TRACE = 2, ORC_ST_MACH = 4, ORC_ST_RHO = 8 };

typedef struct {
    int lattice;            /* ORC_D2Q9 or ORC_D3Q19 */
    int nx, ny, nz;         /* D2Q9 requires nz == 1 */
    int ncomp;              /* 1 or 2 */
    int walls;              /* 1: walls at y=-1/2 and y=NY-1/2; 0: periodic y */
    double G;               /* Shan-Chen coupling, Eq. (eq:SCforce) */
    double eta_A, eta_B;    /* phase shear viscosities, Eq. (smoothingvisco) */
    double delta;           /* smoothing width of f_+-(phi) */
    double u_wall;          /* +u_wall at y=-1/2, -u_wall at y=NY-1/2 */
    double fext[3];         /* external body force density */
    double tau_p, eta_p;    /* polymer relaxation time and viscosity */
    double L2;              /* FENE-P maximum extension squared */
    double kappa;           /* artificial stress diffusivity */
    int phase;              /* feedback modulation: 0 -> 1, +1 -> f_+, -1 -> f_- */
    int fd_on;              /* 1: evolve C; 0: C frozen (LBM only) */
    int coupling;           /* polymer feedback: 0 body force div Q (Eq. NS);
                               1 added to the equilibrium second moment (Eq. MODEtransformation) */
    int collision;          /* 0: single relaxation time tau (BGK form of Eq. LB);
                               1: relaxation in moment space (Sec. 2, MRT): shear and bulk
                                  modes with the local tau (tau_b = tau_s), the species
                                  momentum with tau_M, every other mode with tau_g */
    double tau_M, tau_g;    /* MRT relaxation times of the momentum and non-hydrodynamic modes */
    int chol;               /* conformation update: 0 AB2 on C; 1 AB2 on the Cholesky factor of
                               sigma_P = f(r_P) C with log diagonal (Sec. 2, Cholesky scheme) */
} orc_params;

typedef struct orc_state orc_state;

orc_state *orc_create(const orc_params *p);
void orc_destroy(orc_state *s);
int orc_num_c(const orc_state *s);     /* 4 (D2Q9) or 6 (D3Q19) */
int orc_q(const orc_state *s);

/* populations <- equilibrium(rho_sigma, u); C <- C0 (or identity when NULL);
 * AB2 history cleared (next step uses forward Euler). rhoB ignored for ncomp==1. */
int orc_init_fields(orc_state *s, const double *rhoA, const double *rhoB,
                    const double *u, const double *C0);
int orc_set_params(orc_state *s, const orc_params *p);
int orc_step(orc_state *s, long nsteps);
/* Writes a field into the state: POPS, C, RPREV (RPREV also sets have_prev). */
int orc_write_field(orc_state *s, int field, const double *src);
/* Reads a field of the current state (derived fields are recomputed). */
int orc_read_field(orc_state *s, int field, double *dst);
int orc_set_have_prev(orc_state *s, int have_prev);
unsigned orc_status(const orc_state *s);
long orc_steps_done(const orc_state *s);
int orc_diagnostics(orc_state *s, double out[16]);

/* lattice tables and single-node formulas, for the moment identities */
int orc_lattice(int lattice, int *c_out /* Q*3 */, double *w_out /* Q */);
int orc_equilibrium(int lattice, double rho, const double u[3], double *out);
int orc_source(int lattice, const double u[3], const double F[3], double *out);

/* Pointwise FENE-P conformation ODE under a prescribed uniform velocity
 * gradient gradu[i*3+j] = d_i u_j, advanced by the same right-hand side and
 * Adams-Bashforth-2 update as the lattice path.  C (6 comps, in/out), Rprev
 * (6, in/out), have_prev (in/out). */
int orc_fenep_point(double *C, double *Rprev, int *have_prev,
                    const double gradu[9], double tau_p, double L2, long nsteps);

/* Pointwise ODE as orc_fenep_point, with the conformation update chosen by
 * chol (0: AB2 on C; 1: AB2 on the log-Cholesky variables of sigma_P). */
int orc_fenep_point_form(double *C, double *Rprev, int *have_prev, const double gradu[9], double tau_p,
                         double L2, long nsteps, int chol);

/* Log-Cholesky variables of sigma_P = f(r_P) C (lam, 6 values in the tensor
 * slots: lam_ii = ln l_ii, lam_ij = l_ij for i > j) and their rates for a
 * given dC/dt (both C and dC/dt as 6 components xx xy xz yy yz zz). */
int orc_chol_rates(const double C[6], const double Cdot[6], double L2, double lam[6], double lam_dot[6]);
/* C of given log-Cholesky variables: sigma = L L^T, f = (L^2 - 3 + tr sigma)/L^2, C = sigma / f. */
int orc_chol_to_C(const double lam[6], double L2, double C[6]);

/* Moment basis of the MRT collision: M[k*Q + a] (row k, direction a) and the
 * relaxation kind of each row (0 conserved density, 1 bulk, 2 species
 * momentum, 3 shear, 4 non-hydrodynamic).  Returns Q. */
int orc_mrt_basis(int lattice, double *M, int *kind);

/* OpenMP threads used by node loops (n <= 0 leaves it unchanged); returns the count in use */
int orc_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
