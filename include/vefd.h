/*
 * vefd - GB300 (sm_103a) library for the hybrid lattice-Boltzmann / finite-
 * difference step of viscoelastic two-component flows (A. Gupta,
 * M. Sbragaglia, A. Scagliarini, "Hybrid Lattice Boltzmann/Finite Difference
 * simulations of viscoelastic multicomponent flows in confined geometries",
 * arXiv:1406.2686).
 *
 * One step advances, on one GPU:
 *   - a two-component Shan-Chen lattice-Boltzmann fluid (D2Q9 or D3Q19):
 *     moments, pseudo-potential force (Eq. SCforce), forced BGK collision
 *     (Eq. LB with Lambda = 1/tau, equilibrium and source of Sec. 2, velocity
 *     of Eq. equilibrium:vel), phase-dependent viscosity (Eq. smoothingvisco),
 *     streaming with periodic x, z and half-way bounce-back on moving walls at
 *     y = -1/2 and y = NY - 1/2 (Sec. 3.1);
 *   - the FENE-P conformation tensor C (Eq. FENE, f(r_P) of Sec. 2) by
 *     second-order central finite differences with an artificial diffusivity
 *     and Adams-Bashforth 2 in time, linear extrapolation at the walls (Sec. 2);
 *   - the polymer feedback (eta_P/tau_P) div[(f C - I) m(phi)] as a body force
 *     shared between components by rho_sigma/rho, m = 1, f_+ or f_- (Sec. 2).
 *
 * Conventions for every entry point:
 *   - every function returns a vefd_status and never aborts; on error the
 *     context (when there is one) keeps a message for vefd_last_error;
 *   - fields are FP32, x fastest: index = ((comp*NZ + z)*NY + y)*NX + x;
 *     tensor components are xx xy xz yy yz zz (D3Q19) or xx xy yy zz (D2Q9);
 *     velocities have 3 (D3Q19) or 2 (D2Q9) components;
 *   - pointers marked "host or device" are interpreted by the on_device flag;
 *     buffers passed in stay owned by the caller;
 *   - work is enqueued on the context's CUDA stream; calls that return data
 *     to the host synchronise that stream;
 *   - a context is not thread-safe.
 */
#ifndef VEFD_H
#define VEFD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vefd_ctx vefd_ctx;

typedef enum {
    VEFD_OK = 0,
    VEFD_ERR_ARG = -1,       /* bad argument or size; nothing was changed */
    VEFD_ERR_CUDA = -2,      /* a CUDA call failed; see vefd_last_error */
    VEFD_ERR_UNSTABLE = -3,  /* the device guard word is set (NaN, tr C >= L^2, |u| > 0.3, rho <= 0) */
    VEFD_ERR_TIMEOUT = -4,   /* a bounded device wait ran out (guard bit VEFD_ST_TIMEOUT) */
    VEFD_ERR_STATE = -5      /* call out of order (e.g. memory not bound, fields not initialised) */
} vefd_status;

typedef enum { VEFD_D2Q9 = 0, VEFD_D3Q19 = 1 } vefd_lattice;

typedef enum {
    VEFD_RHO_A = 0,    /* 1 comp: density of component A of the current state */
    VEFD_RHO_B = 1,    /* 1 comp: density of component B (zero for one component) */
    VEFD_PHI = 2,      /* 1 comp: order parameter (rho_A - rho_B)/(rho_A + rho_B) (Sec. 2) */
    VEFD_U = 3,        /* 2|3 comps: velocity of Eq. (equilibrium:vel) of the current state */
    VEFD_C = 4,        /* 4|6 comps: conformation tensor C */
    VEFD_SIGMA_P = 5,  /* 4|6 comps: polymer stress f(r_P) C (Eq. fluidstress) */
    VEFD_POPS = 6,     /* ncomp*Q comps: populations f_a^sigma, order [sigma][a] */
    VEFD_RPREV = 7,    /* 4|6 comps: right-hand side of the previous FD step (AB2 history) */
    VEFD_G_A = 8,      /* 2|3 comps: Shan-Chen force on A of the current state (Eq. SCforce) */
    VEFD_G_B = 9,      /* 2|3 comps: Shan-Chen force on B */
    VEFD_F_P = 10,     /* 2|3 comps: polymer feedback force (eta_P/tau_P) div[(f C - I) m(phi)] */
    VEFD_TAU = 11      /* 1 comp: local relaxation time (Eq. smoothingvisco) */
} vefd_field;

/* Guard bits of the device status word (sticky until vefd_clear_status). */
enum { VEFD_ST_NAN = 1, VEFD_ST_TRACE = 2, VEFD_ST_MACH = 4, VEFD_ST_RHO = 8, VEFD_ST_TIMEOUT = 16,
       VEFD_ST_BOUNDS = 32 /* debug library only (built with VEFD_BOUNDS_CHECK): a neighbour index of a
                              step kernel left the lattice; the access was skipped */ };

/* Lattice and two-component fluid (Sec. 2). */
typedef struct {
    int lattice;         /* vefd_lattice */
    int nx, ny, nz;      /* nodes; D2Q9 needs nz == 1; walls need ny >= 3 */
    int ncomp;           /* 1 or 2 components */
    int walls;           /* 1: walls at y = -1/2 and NY - 1/2; 0: periodic in y */
    double G;            /* Shan-Chen coupling (Eq. SCforce); ignored for one component */
    double eta_A;        /* shear viscosity of the A-rich phase (Eq. smoothingvisco) */
    double eta_B;        /* shear viscosity of the B-rich phase */
    double delta;        /* smoothing width of f_+-(phi), Eq. (smoothingvisco); paper: 0.1 */
    int external_memory; /* 1: the caller binds device memory with vefd_bind_device_memory */
    int precision;       /* storage of the population deviations f - w rho_ref: 0 FP32, 1 FP16,
                            2 BF16 (arithmetic is FP32 and C is FP32 in every case) */
} vefd_config;

/* Creates a context on the current CUDA device; `stream` is a cudaStream_t
 * (NULL = legacy default stream).  Validates cfg; allocates device buffers
 * unless cfg->external_memory.  The kernels index a population plane by
 * 32-bit offsets, so one lattice holds at most 2^31 / 40 = 53,687,091 nodes
 * (about 23 GB of state with FP32 storage); larger ones are refused with
 * VEFD_ERR_ARG.  Errors: VEFD_ERR_ARG, VEFD_ERR_CUDA. */
vefd_status vefd_create(const vefd_config *cfg, void *stream, vefd_ctx **out);
/* Bytes of device memory a context with this config needs. */
vefd_status vefd_required_bytes(const vefd_config *cfg, size_t *bytes);
/* Binds caller-owned device memory (>= vefd_required_bytes, 256-byte
 * aligned) to a context created with external_memory = 1.  The memory must
 * outlive the context.  Errors: VEFD_ERR_ARG, VEFD_ERR_STATE (already bound). */
vefd_status vefd_bind_device_memory(vefd_ctx *ctx, void *dev_ptr, size_t bytes);
/* Frees owned buffers (not bound ones) after synchronising the stream. */
void vefd_destroy(vefd_ctx *ctx);
vefd_status vefd_set_stream(vefd_ctx *ctx, void *stream);

/* Wall speed U: +U at y = -1/2, -U at y = NY - 1/2, moving-wall bounce-back
 * (Sec. 3.1: u_x(y=0) = -u_x(y=H) = U_w).  |U| < 0.1. */
vefd_status vefd_set_wall_shear(vefd_ctx *ctx, double u_wall);
/* External body-force density, shared between components by rho_sigma/rho. */
vefd_status vefd_set_body_force(vefd_ctx *ctx, double fx, double fy, double fz);
/* FENE-P parameters (Sec. 2): relaxation time tau_P > 0, viscosity eta_P >= 0,
 * maximum extension squared L2 > 3, artificial diffusivity kappa in
 * [0, 1/(2 dim)), feedback modulation phase: 0 -> 1, +1 -> f_+(phi),
 * -1 -> f_-(phi), and fd_on: 0 freezes C (pure lattice-Boltzmann runs). */
vefd_status vefd_set_fenep(vefd_ctx *ctx, double tau_p, double eta_p, double L2, double kappa, int phase,
                           int fd_on);

/* How the polymer stress reaches the fluid (Sec. 2): 0 (default) as the body
 * force (eta_P/tau_P) div[(f C - I) m(phi)] shared by rho_sigma/rho (Eq. NS);
 * 1 added to the second moment of each component's equilibrium with weight
 * rho_sigma/rho (Eq. MODEtransformation), in BGK form
 * E_a += w_a (c_a c_a - c_s^2 I):T_sigma / (2 c_s^4),
 * T_sigma = -(rho_sigma/rho)(eta_P/tau_P)(f C - I) m(phi).  Errors: VEFD_ERR_ARG. */
vefd_status vefd_set_polymer_coupling(vefd_ctx *ctx, int mode);

/* Collision operator of Eq. (LB) (Sec. 2): 0 (default) a single relaxation
 * time, the local tau of Eq. smoothingvisco; 1 relaxation in moment space
 * with the paper's times (Eq. TRANSPORTCOEFF and the text after it): shear
 * and bulk modes tau_s = tau_b = the local tau, species momentum tau_M = 1
 * (mobility 1/2), non-hydrodynamic modes 1, on the orthogonal moment basis
 * of the D3Q19 (D2Q9) lattice; the source enters as (I - Lambda/2) S.
 * Errors: VEFD_ERR_ARG. */
vefd_status vefd_set_collision(vefd_ctx *ctx, int model);

/* Conformation-tensor time stepping (Sec. 2): 0 (default) AB2 on C; 1 the
 * Cholesky scheme: AB2 on ln l_ii and l_ij (i > j) of sigma_P = f(r_P) C =
 * L L^T, driven by the same right-hand side, which keeps C symmetric positive
 * definite with tr C < L^2.  The stored field stays C; the AB2 history
 * (VEFD_RPREV) then holds the rates of the log-Cholesky variables in the C
 * component slots.  Changing the scheme clears the history (the next step is
 * forward Euler).  Errors: VEFD_ERR_ARG. */
vefd_status vefd_set_conformation_update(vefd_ctx *ctx, int scheme);

/* Initial state: populations at equilibrium E(rho_sigma, u), C = C0 (or I
 * when C0 is NULL), AB2 history cleared (the next step is forward Euler).
 * rho_A (N), rho_B (N, ignored for one component), u (dim*N or NULL for
 * rest), C0 (nc*N or NULL); host or device FP32 per on_device.
 * Also resets the step counter and the status word.  Each component's
 * domain-mean density (the reference of the stored deviations) is an FP64
 * sum on the device in a fixed order.  Densities that are not finite or are
 * negative give VEFD_ERR_ARG and leave the context uninitialised (VEFD_ERR_STATE
 * for stepping and reads until a valid call).  Synchronises the stream. */
vefd_status vefd_init_fields(vefd_ctx *ctx, const float *rho_A, const float *rho_B, const float *u,
                             const float *C0, int on_device);
/* Convenience droplet initialisation computed on the host: rho_A = rho_out +
 * (rho_in - rho_out)(1 + tanh(2 (R - r)/width))/2 about (cx, cy, cz), rho_B =
 * rho_in + rho_out - rho_A, order-parameter noise phi_amp * U[-1, 1) from
 * SplitMix64(seed) at node counter i, u = 0, C = I. */
vefd_status vefd_init_droplet(vefd_ctx *ctx, double cx, double cy, double cz, double R, double rho_in,
                              double rho_out, double width, uint64_t seed, double phi_amp);

/* Overwrites a stored field: VEFD_POPS (absolute populations), VEFD_C, or
 * VEFD_RPREV (also marks the history valid).  bytes must equal the field size. */
vefd_status vefd_write_field(vefd_ctx *ctx, vefd_field field, const void *src, size_t bytes, int src_on_device);
/* Enqueues nsteps >= 0 time steps on the context stream (asynchronous). */
vefd_status vefd_step(vefd_ctx *ctx, int64_t nsteps);
/* Copies a field of the current state to dst (host or device); derived
 * fields (rho, phi, u, sigma_P, forces, tau) are computed on the device
 * first.  Host destinations synchronise the stream. */
vefd_status vefd_read_field(vefd_ctx *ctx, vefd_field field, void *dst, size_t bytes, int dst_on_device);
/* Field size in bytes. */
vefd_status vefd_field_bytes(const vefd_ctx *ctx, vefd_field field, size_t *bytes);

/* FP64 reductions of the current state (synchronises), out[16]:
 *  0 mass_A  1 mass_B  2..4 total momentum sum rho u  5 <sigma_P,xy>
 *  6 <sigma_P,xx - sigma_P,yy>  7 max tr C / L^2  8 max |u|
 *  9 droplet area (phi > 0) in the plane z = NZ/2  10 deformation D = (a-b)/(a+b)
 *  11 orientation angle theta of the major axis from +x (Sec. 4.1)
 *  12, 13 droplet centroid x, y in that plane  14 droplet volume (phi > 0)
 *  15 <tr sigma_P> - 3 */
vefd_status vefd_diagnostics(vefd_ctx *ctx, double out[16]);
/* Reads the guard word (synchronises); returns VEFD_ERR_TIMEOUT when the
 * wait-timeout bit is set, else VEFD_ERR_UNSTABLE when any other bit is set. */
vefd_status vefd_get_status(vefd_ctx *ctx, uint32_t *bits);
/* Exercises the bounded-wait guard without a fault (the paper has no
 * counterpart).  Every device wait of the library (the mbarrier waits of the
 * bulk tensor copies and of the tensor-core GEMM) gives up after 2^31 SM
 * cycles of clock64 (about one second) or 2^22 polls, sets VEFD_ST_TIMEOUT
 * and leaves its kernel with no copy in flight.  This call runs one such wait
 * on the context's stream, with a budget of 2^24 cycles (about 8 ms), on an
 * mbarrier that one thread completes (arrive = 1: no bit is set) or that
 * nothing completes (arrive = 0: the wait runs out and VEFD_ST_TIMEOUT is set,
 * so vefd_get_status returns VEFD_ERR_TIMEOUT; vefd_clear_status resets it and
 * the context stays usable).  Asynchronous.  VEFD_ERR_ARG for a NULL context
 * or arrive not 0/1, VEFD_ERR_STATE without bound memory, VEFD_ERR_CUDA on a
 * launch error. */
vefd_status vefd_wait_selftest(vefd_ctx *ctx, int arrive);
vefd_status vefd_clear_status(vefd_ctx *ctx);
vefd_status vefd_steps_done(const vefd_ctx *ctx, int64_t *n);
/* Raw binary checkpoint of populations, C, AB2 history, counters and
 * parameters; restoring into a context of the same config continues
 * bit-identically. */
vefd_status vefd_checkpoint(vefd_ctx *ctx, const char *path);
vefd_status vefd_restore(vefd_ctx *ctx, const char *path);
/* Message of the last error of this context ("" when none). */
const char *vefd_last_error(const vefd_ctx *ctx);
/* Device kernels one time step enqueues. */
vefd_status vefd_kernels_per_step(const vefd_ctx *ctx, int *n);
/* Per-kernel timing of vefd_step: when on, every launch of a step is
 * bracketed by CUDA events on the context stream (turning it on clears the
 * record).  Tracing aid, not a hot-path requirement.  (Independently, the
 * library marks vefd_step, graph captures, diagnostics, checkpoints,
 * autotuning and ensemble steps as NVTX ranges, visible to a profiler such as
 * Nsight Systems and free otherwise.) */
vefd_status vefd_profile_kernels(vefd_ctx *ctx, int on);
/* Synchronises and returns, per kernel class (0 densities of the initial
 * populations, 1 lattice collide-stream, 2 densities of the new populations
 * fused with the FENE-P finite-difference update), the summed device time in
 * milliseconds and the number of timed launches since profiling was turned
 * on or last read; then clears the record. */
vefd_status vefd_kernel_times(vefd_ctx *ctx, double ms[3], int64_t launches[3]);

/* ---- kernel choice and autotuning (implementation detail; the paper has no
 * counterpart) ---------------------------------------------------------------
 * lattice_tile selects the node tile the collide-stream kernel (Sec. 2.1,
 * Eqs. 1-3) stages through shared memory: D3Q19 0 = 32x4x2 (default),
 * 1 = 32x2x4, 2 = 32x8x1 nodes (x by y by z); D2Q9 0 = 32x8 (default),
 * 1 = 32x4, 2 = 32x16.  3, 4 and 5 are the same tiles walked by a persistent
 * grid (one block per resident slot on every SM) that double-buffers the
 * staged populations.  post_mode selects how the densities of the new
 * populations and the FENE-P update are done: 0 = a column-marching lattice
 * kernel (32 x 8 columns walked along z) that also sums the new densities,
 * followed by a z-marching FENE-P pass that adds the populations which
 * crossed a column side or segment end (D3Q19 with NX % 32 == 0 and
 * NY % 8 == 0; lattice_tile is then unused; it moves fewer bytes but issues
 * about 2.7 times the lattice kernel's instructions); 1 = a 3-D tiled
 * densities/FENE-P pass; 2 (default) = the z-marching densities/FENE-P pass
 * after the tiled lattice kernel; 3 = the tiled lattice kernel (D3Q19 tiles 0
 * and 1, lattices of whole tiles) also sums, after its collision, the new
 * populations that stay inside its tile into partial densities and writes
 * what it pushes across each face and edge of the tile as per-node partial
 * sums, so that the z-marching pass completes the densities from those
 * (about 3 values per node) instead of reading the new populations back; the
 * partial sums use the staging planes, which are free inside a step.  Post
 * modes 1 and 2 with tiles 0-2 run the same arithmetic in the
 * same order and give bit-identical results; the persistent tiles (separately
 * compiled, multiply-adds contracted as the compiler sees fit) and post modes 0
 * and 3 (each node's new density summed in another order) agree to FP32
 * rounding.  A tile the lattice shape
 * does not admit falls back to tile 0, post_mode 0 or 2 falls back to 1 where
 * the column does not fit, post_mode 3 falls back to 2 where the tile or the
 * lattice does not admit it, and shapes that admit no staged tile use the
 * unstaged kernels.  Returns VEFD_ERR_ARG for values outside these ranges.
 * Not to be called while steps are in flight. */
vefd_status vefd_set_kernel_config(vefd_ctx *ctx, int lattice_tile, int post_mode);
/* Environment switches, read when memory is bound to a context (measurement
 * and testing; the defaults are the measured fastest, and results stay
 * within the agreements stated above):
 *   VEFD_NO_TMA=1        unstaged kernels only;
 *   VEFD_NO_ZMARCH=1     the 3-D tiled densities pass instead of the z-marching one;
 *   VEFD_NO_FUSED=1      post_mode 0 runs as post_mode 2;
 *   VEFD_NO_PDL=1        no programmatic dependent launch between a step's kernels;
 *   VEFD_SCHEDULE=b      bit 0 walks the lattice kernel's tiles, bit 1 the pass's
 *                        columns in reverse order (default 0);
 *   VEFD_ZM_SEGMENT=n    z-segment length of the column march (default: one wave);
 *   VEFD_SLAB_SEGMENT=n  z-segment of the step graph's slab passes (default 12);
 *   VEFD_SLAB_PDL=1      programmatic launch between a slab's consecutive kernels
 *                        inside the step graph (measured slower; off). */
/* The configuration in effect: lattice_tile -1 and post_mode -1 mean the
 * unstaged kernels; post_mode 1 also when the column does not fit. */
vefd_status vefd_get_kernel_config(const vefd_ctx *ctx, int *lattice_tile, int *post_mode);
/* Times every admitted (lattice_tile, post_mode) pair for `steps` steps on a
 * scratch lattice of the same configuration and parameters (droplet initial
 * state; the context's own state is untouched), then applies the fastest.
 * times_ms (host, 18 doubles or NULL) receives the times, index
 * post_mode * 6 + lattice_tile, -1 for pairs not admitted (post_mode 0 is
 * timed with lattice_tile 0 only; post_mode 3 is not timed: its lattice
 * kernel's extra work outweighs the bytes it saves).  Allocates and
 * frees the scratch lattice's device memory and synchronises the context
 * stream.  VEFD_ERR_UNSTABLE when the scratch run trips a guard. */
vefd_status vefd_autotune(vefd_ctx *ctx, int steps, double *times_ms);
/* Step graph (implementation detail; the paper steps the whole lattice).
 * vefd_step runs whole chunks of `chunk` steps (even, >= 2) as a replayed
 * CUDA graph, and the even remainder of the call (nsteps mod chunk, rounded
 * down to even) as one replay of a graph of that many steps, so calls of any
 * length replay graphs.  A context keeps up to four graph sizes (the chunk
 * and the remainders of recent calls, least recently used dropped first),
 * each captured on first use.  The graphs take one of two forms.
 * - Pipelined slabs (slabs >= 2): the lattice is split into `slabs` slabs of
 *   NY / slabs rows.  Each slab's lattice kernel and densities/FENE-P pass is
 *   a graph node that waits only for the nodes of the neighbouring slabs it
 *   exchanges data with: its lattice kernel of step n+1 waits for the passes
 *   of step n on slabs k-1, k, k+1, and its pass of step n waits for the
 *   lattice kernels of step n on those slabs.  Work on different slabs then
 *   overlaps, and a slab's new populations can be re-read while still in L2.
 *   Each slab's pass marches z-segments of 12 planes (shorter blocks than
 *   the whole-lattice pass, so the pass its neighbours wait for finishes
 *   sooner).  This form needs: D3Q19; a staged tile 0-2 with post mode 2;
 *   NY a multiple of 8 * slabs.  An explicit slab count the lattice does not
 *   admit means eager stepping.
 * - Whole-lattice (slabs = 1): the eager launch pairs of `chunk` steps,
 *   replayed as one graph; any lattice and kernel choice.  It saves the
 *   host-side launch cost, which bounds small lattices.
 * In both forms the kernels and their per-node arithmetic are those of the
 * eager step, so results are bit-identical.  slabs = 0 turns the graph off;
 * slabs = -1 (the default) chooses 8 slabs when NY is a multiple of 64, 4 when
 * of 32, where the split applies and each slab holds at least 100,000 nodes,
 * otherwise the whole-lattice form (on the 128 x 64 x 128 droplet, against
 * eager stepping: 8 slabs +7 to +8 %, 4 slabs +5 %; on smaller lattices the
 * slabs' kernels cannot fill the GPU and the whole-lattice form is faster,
 * e.g. 10042 against 6623 MLUPS on 64^3).  The graph is used when kernel timing is off and the
 * context stream is not being captured.  Some steps run eagerly: the Euler
 * start, steps with pending densities, the last step of an odd count, and
 * one step that brings the ping-pong buffers back to the parity the graphs
 * were captured at (rather than capturing the other parity; a call of fewer
 * than three steps at the other parity steps eagerly).  The graphs are
 * re-captured when the parameters or kernel choice change.
 * VEFD_ERR_ARG for slabs below -1 or above 64, or a bad chunk (default 256). */
vefd_status vefd_set_step_graph(vefd_ctx *ctx, int slabs, int chunk);
/* Captures and instantiates the step graph for the current state now, so the
 * next vefd_step call of at least one chunk replays it without capturing
 * first (capture records 2 x slabs x chunk launches).  Takes no step.  A no-op
 * when the graph does not apply or the state is not steady yet (the Euler
 * start or densities pending: take a step first).  VEFD_ERR_STATE before
 * initialisation, VEFD_ERR_CUDA on capture errors. */
vefd_status vefd_prepare_step_graph(vefd_ctx *ctx);
/* As vefd_prepare_step_graph, for a call of nsteps steps: captures now every
 * graph that vefd_step(ctx, nsteps) would replay from the current state (the
 * chunk when nsteps >= chunk, and the even remainder), so that call only
 * replays.  Graphs held for the other ping-pong parity are dropped first.
 * Takes no step; a no-op where the graph does not apply or the state is not
 * steady yet.  VEFD_ERR_ARG for nsteps < 0, VEFD_ERR_STATE before
 * initialisation, VEFD_ERR_CUDA on capture errors. */
vefd_status vefd_prepare_steps(vefd_ctx *ctx, int64_t nsteps);
/* The slab count in effect (0: no graph, 1: the whole-lattice form), the
 * chunk, and active = 1 when the next vefd_step would use the graph. */
vefd_status vefd_get_step_graph(vefd_ctx *ctx, int *slabs, int *chunk, int *active);

/* ---- ensembles of independent lattices (implementation detail: the paper
 * steps one lattice at a time) --------------------------------------------
 * An ensemble steps many independent lattices of any sizes and
 * configurations together: `chunk` steps of all members are captured once as
 * a CUDA graph and replayed, either as two batched launches per step over the
 * tiles of all members (vefd_ensemble_set_batched) or with every member's
 * step as one graph branch, so small lattices fill the GPU together and pay
 * no per-launch host cost.  Members stay
 * ordinary contexts (read, diagnose, checkpoint them as usual, between
 * ensemble calls); the ensemble does not own them and must be destroyed
 * before they are. */
typedef struct vefd_ensemble vefd_ensemble;
/* members: n distinct, initialised contexts on the current device.  stream:
 * the caller's stream (NULL = legacy default stream); ensemble work is
 * ordered after prior work on it and on every member's own stream, and work
 * later enqueued on those streams is ordered after it. */
vefd_status vefd_ensemble_create(vefd_ctx *const *members, int n, void *stream, vefd_ensemble **out);
/* Advances every member by nsteps >= 0 steps (asynchronous), each member's
 * results those of vefd_step on it alone (bit-identical with graph branches,
 * to FP32 rounding with batched launches).  chunk (even, >= 2) is the
 * number of steps per graph replay: members still in their first step (the
 * Euler start) or with densities pending take one eager step first,
 * then nsteps / chunk replays run and the remainder runs eagerly.  The graph
 * is re-captured whenever a member's parameters, kernel choice or buffer
 * parity differ from the capture (for example after vefd_set_wall_shear or an
 * odd eager remainder).  VEFD_ERR_ARG for a bad chunk, VEFD_ERR_STATE when a
 * member is not initialised, VEFD_ERR_CUDA on capture or launch errors
 * (see vefd_ensemble_last_error). */
vefd_status vefd_ensemble_step(vefd_ensemble *ens, int64_t nsteps, int64_t chunk);
/* Batched launches (default on): when every member is D3Q19 with the same
 * component count, storage type, collision operator, FENE-P switch and
 * programmatic-launch setting, and each takes the staged lattice kernel and
 * the separate z-marching densities/FENE-P pass (NX % 32 == 0, NY % 8 == 0,
 * kernel config post mode 2), the members are split into up to 4 groups of
 * about equal node count (contiguous in member order; the count is set by
 * vefd_ensemble_set_groups), and a replayed step
 * is, per group, ONE lattice-kernel launch over the 32 x 4 x 2 tiles of its
 * members and ONE densities/FENE-P launch over their 32 x 8 columns; each
 * group's launches are one graph branch, so the groups overlap.  Each block
 * finds its member by binary search
 * over a device table holding the member's parameters, the buffers and
 * tensor maps of both ping-pong parities, and its tile counts; the table is
 * rebuilt with every re-capture.  Per node the arithmetic is the member's own
 * kernels' (results agree with vefd_step to FP32 rounding: the batched
 * kernels are separate instantiations, so floating-point contraction may
 * differ in the last ulp).  on = 0 keeps one graph branch per member.
 * VEFD_ERR_ARG for a NULL ensemble or on not 0/1; takes effect at the next
 * replay (after waiting for earlier replays). */
vefd_status vefd_ensemble_set_batched(vefd_ensemble *ens, int on);
/* 1 when the currently captured graph uses the batched launches, else 0. */
int vefd_ensemble_is_batched(const vefd_ensemble *ens);
/* Kernel choices of the replayed steps: batched (0/1, as
 * vefd_ensemble_set_batched) and the z-segment length, in planes, of the
 * batched densities/FENE-P pass (0: automatic, the length that fills two
 * blocks per SM with the fewest planes per block; otherwise clamped to each
 * member's NZ).  Results do not depend on the segment length.  Takes effect
 * at the next replay.  VEFD_ERR_ARG for a NULL ensemble, batched not 0/1 or
 * a negative segment. */
vefd_status vefd_ensemble_set_config(vefd_ensemble *ens, int batched, int post_segment);
vefd_status vefd_ensemble_get_config(const vefd_ensemble *ens, int *batched, int *post_segment);
/* Group count of the batched launches (no counterpart in the paper; a
 * launch-layout choice): 0 (the default) means 4; otherwise 1..64, clamped to
 * the member count.  Members are split into that many contiguous groups of
 * about equal node count, each group one graph branch of two launches per
 * step.  Results do not depend on the group count (bit-identical).  Takes
 * effect at the next replay (after waiting for earlier replays).
 * VEFD_ERR_ARG for a NULL ensemble or groups outside 0..64. */
vefd_status vefd_ensemble_set_groups(vefd_ensemble *ens, int groups);
/* The group-count setting (0: automatic). */
vefd_status vefd_ensemble_get_groups(const vefd_ensemble *ens, int *groups);
/* Lattice tiles of the batched launches (no counterpart in the paper; a launch
 * shape): 0 (default) 32 x 4 x 2 nodes, 1 32 x 8 x 1.  Results agree with
 * vefd_step to FP32 rounding for both.  Takes effect at the next replay (after
 * waiting for earlier replays).  VEFD_ERR_ARG for a NULL ensemble or another
 * value. */
vefd_status vefd_ensemble_set_tile(vefd_ensemble *ens, int tile);
vefd_status vefd_ensemble_get_tile(const vefd_ensemble *ens, int *tile);
/* The ensemble's own autotuner.  It times seven configurations: graph
 * branches; and batched launches with each lattice tile (0, 1), each with the
 * automatic z-segment of the densities pass, twice it and half of it.
 * Each is timed as `steps` replayed steps (after one untimed replay that
 * captures it), and the fastest is kept.  The timed steps are real steps:
 * every member advances by 7 (steps + chunk) steps (plus one eager step if its
 * Euler start is pending), its results those of vefd_step to FP32 rounding.
 * times_ms (7 slots, or NULL) receives each configuration's milliseconds, -1
 * where the members do not allow batched launches.  Synchronises.
 * VEFD_ERR_ARG unless steps is a positive multiple of an even chunk;
 * otherwise as vefd_ensemble_step. */
vefd_status vefd_ensemble_autotune(vefd_ensemble *ens, int64_t steps, int64_t chunk, double *times_ms);
const char *vefd_ensemble_last_error(const vefd_ensemble *ens);
/* Waits for the ensemble's work and frees its streams, events and graph. */
void vefd_ensemble_destroy(vefd_ensemble *ens);

/* Allocation-free diagnostics (the paper has no counterpart; this is a
 * service for callers that cannot allocate device memory).  Some callers
 * cannot call cudaMalloc: their device memory is owned by another allocator
 * that reserves the GPU up front, or they run as a monitoring hook that must
 * not trigger the device-wide synchronisation cudaMalloc/cudaFree can cause.
 * This entry point reduces fields the caller already holds on the device and
 * allocates nothing; its only scratch is a fixed array inside the library's
 * device image (557,192 bytes, kept by every GPU that loads the library until
 * the process exits).
 * Inputs (device pointers, FP32, layout as vefd_read_field): rho_A and rho_B
 * (N each; rho_B may be NULL when ncomp == 1), u (2|3 planes), C (4|6 planes);
 * L2 is the FENE-P maximum extension squared.  out[16] (host) receives the
 * values listed for vefd_diagnostics.  Work runs on `stream` and the call
 * synchronises it.  Lattices above 8,388,608 nodes exceed the scratch array
 * and are rejected with VEFD_ERR_ARG, as are bad sizes and NULL inputs.
 * The first call in each CUDA context (on each device, and again after a
 * device reset replaced the context) looks up the scratch address with that
 * context current and caches it under the context's unique ID, so make that
 * first call before any stream capture.  Every
 * call shares the one scratch array and rewrites every row it reads, so
 * nothing needs clearing between calls; a lock held from the first launch to
 * the synchronisation makes host threads that call at the same time take
 * turns on it. */
vefd_status vefd_diagnostics_noalloc(int lattice, int nx, int ny, int nz, int ncomp, double L2,
                                     const float *rho_A, const float *rho_B, const float *u, const float *C,
                                     void *stream, double out[16]);

#ifdef __cplusplus
}
#endif
#endif
