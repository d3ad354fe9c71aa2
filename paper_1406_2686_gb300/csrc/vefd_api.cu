// C-ABI of libvefd (declared in include/vefd.h): context, memory, parameters,
// field I/O, time stepping, diagnostics and checkpoints of the hybrid
// lattice-Boltzmann / finite-difference viscoelastic step.
#include <algorithm>
#include <utility>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <cuda.h>
#include <nvtx3/nvToolsExt.h>

#include "vefd.h"
#include "vefd_internal.cuh"

using namespace vefd;

struct vefd_ctx {
    vefd_config cfg;
    int Q = 0, D = 0, NC = 0;
    long long N = 0;
    cudaStream_t stream = nullptr;
    // physical parameters
    double u_wall = 0.0, fext[3] = {0.0, 0.0, 0.0};
    double tau_p = 1.0, eta_p = 0.0, L2 = 100.0, kappa = 0.0;
    int phase = 0, fd_on = 1;
    int coupling = 0;  // polymer feedback: 0 body force, 1 equilibrium stress
    int collision = 0;  // 0 single relaxation time, 1 moment space (paper's rates)
    int chol = 0;       // conformation update: 0 AB2 on C, 1 log-Cholesky of f C
    double rho_ref[2] = {1.0, 1.0};
    // time-level state
    int have_prev = 0;
    int64_t steps = 0;
    int initialised = 0;
    int cur = 0, ccur = 0;
    // memory
    void* mem = nullptr;
    size_t mem_bytes = 0;
    bool owned = false;
    void* f[2] = {nullptr, nullptr};  // moving population deviations, storage type of cfg.precision
    float* frest = nullptr;           // rest population deviations (FP32, updated in place)
    size_t psize = 4;                 // bytes per stored population value
    float* drho = nullptr;      // densities of the current time level
    float* drho_alt = nullptr;  // the other density buffer (column-marching step writes the next level here)
    float* u = nullptr;
    float* C[2] = {nullptr, nullptr};
    float* R = nullptr;
    float* dbg = nullptr;
    float* qbuf = nullptr;  // feedback stress Q
    unsigned* status = nullptr;
    double* diag_part = nullptr;
    double* diag_out = nullptr;
    std::string err;
    // TMA descriptors of the two population buffers (when the shape allows)
    alignas(64) CUtensorMap tmap[2];       // lattice kernel: box = the selected staged tile
    alignas(64) CUtensorMap tmap_post[2];  // densities/FD pass (3-D tile variant): box 32x4x2 or 32x8x1
    bool tma_ok = false;
    int lat_tile = 0;                      // staged tile shape of the lattice kernel (lattice_tile_shape)
    int post_mode = 2;                     // 0 column march with fused densities, 1 3-D tiles, 2 separate z-march pass
    // tensor maps with a 32 x 8 x 1 box for the z-marching densities/FD pass
    alignas(64) CUtensorMap tmap_zm[2];
    bool zm_ok = false;
    // column-marching lattice kernel with the densities fused in (post_mode 0)
    bool fused_ok = false;
    // staged lattice kernel writing partial densities that the z-marching pass
    // completes (post_mode 3; D3Q19, 32 x 4 x 2 or 32 x 2 x 4 tiles)
    bool parts_ok = false;
    int zm_seg_fixed = 0;  // z-segment length of the column march (0: one wave of blocks)
    bool pdl = true;       // programmatic dependent launch between the step's kernels
    // densities and feedback stress of the current state are in drho and Q
    bool drho_valid = false;
    // tile traversal: bit0 lattice kernel backwards, bit1 densities/FD kernel
    // backwards; opposite orders make each kernel start on the tiles the other
    // touched last (still in L2)
    int sched = 1;
    // pipelined step graph: the lattice split into `slabs` y-slabs, each slab's
    // lattice kernel and densities/FENE-P pass a node that waits only for the
    // neighbouring slabs; `slab_chunk` steps per replayed graph
    int slabs = -1;  // -1 automatic (slab_count), 0 off
    int slab_chunk = 256;
    int slab_zs = 12;                      // z-segment of the slab passes (planes marched per block)
    bool slab_pdl = false;                 // programmatic launch between a slab's consecutive kernels
    cudaStream_t cap = nullptr;            // capture origin
    std::vector<cudaStream_t> slab_s;      // one capture stream per slab
    std::vector<cudaEvent_t> slab_evL, slab_evP;
    cudaEvent_t slab_fork = nullptr;
    // replayed step graphs, keyed by their (even) step count: the main chunk of
    // slab_chunk steps and up to kGraphSizes - 1 other sizes (the even
    // remainders of recent calls), most recently used first.  All of them are
    // captured from one state (slab_key) and ping-pong parity (slab_parity).
    std::vector<std::pair<int64_t, cudaGraphExec_t>> graphs;
    std::vector<double> slab_key;          // state the graphs were captured for
    int slab_parity = -1;                  // population buffer parity (cur) the graphs start from
    // optional per-kernel timing of vefd_step (events on the context stream)
    bool prof_on = false;
    std::vector<cudaEvent_t> prof_ev;
    std::vector<int> prof_kind;
    size_t prof_used = 0;
};

namespace {

// NVTX range for the duration of a scope (header-only NVTX3: a no-op unless a
// profiler such as Nsight Systems is attached).
struct Range {
    explicit Range(const char* name) { nvtxRangePushA(name); }
    ~Range() { nvtxRangePop(); }
};

vefd_status fail(vefd_ctx* c, vefd_status st, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return st;
}

#define VEFD_CUDA(ctx, call)                                                                      \
    do {                                                                                          \
        cudaError_t e_ = (call);                                                                  \
        if (e_ != cudaSuccess)                                                                    \
            return fail((ctx), VEFD_ERR_CUDA, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), \
                        __FILE__, __LINE__);                                                      \
    } while (0)

int lattice_Q(int lat) { return lat == VEFD_D3Q19 ? 19 : 9; }
int lattice_D(int lat) { return lat == VEFD_D3Q19 ? 3 : 2; }
int lattice_NC(int lat) { return lat == VEFD_D3Q19 ? 6 : 4; }

bool config_ok(const vefd_config* c, const char** why) {
    if (!c) return *why = "config is NULL", false;
    if (c->lattice != VEFD_D2Q9 && c->lattice != VEFD_D3Q19) return *why = "unknown lattice", false;
    if (c->nx < 1 || c->ny < 1 || c->nz < 1) return *why = "sizes must be >= 1", false;
    if (c->lattice == VEFD_D2Q9 && c->nz != 1) return *why = "D2Q9 needs nz == 1", false;
    if (c->walls && c->ny < 3) return *why = "walls need ny >= 3", false;
    if (c->ncomp != 1 && c->ncomp != 2) return *why = "ncomp must be 1 or 2", false;
    if (!(c->eta_A > 0.0) || !(c->eta_B > 0.0) || !std::isfinite(c->eta_A) || !std::isfinite(c->eta_B))
        return *why = "viscosities must be positive", false;
    if (!(c->delta > 0.0) || !std::isfinite(c->delta)) return *why = "delta must be positive", false;
    if (!(c->G >= 0.0) || !std::isfinite(c->G)) return *why = "G must be finite and >= 0", false;
    if (c->precision < 0 || c->precision > 2) return *why = "precision must be 0 (FP32), 1 (FP16) or 2 (BF16)", false;
    const long long N = (long long)c->nx * c->ny * c->nz;
    if (N > (1LL << 31) / 40) return *why = "lattice too large for 32-bit plane offsets", false;
    return true;
}

// staging planes (FP32): the initial fields (rho_A, rho_B, 3 velocity, 6 C) and
// the derived fields of reads and writes go through this buffer; inside a step
// of post_mode 3 it holds the 7 partial-density slots (7 x 2 planes)
constexpr int kStagePlanes = 14;

struct Layout {
    size_t f0, f1, frest, drho, u, c0, c1, r, dbg, q, status, dpart, dout, total;
};

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

Layout layout_of(const vefd_config* c) {
    const size_t N = (size_t)c->nx * c->ny * c->nz;
    const size_t Q = lattice_Q(c->lattice), NC = lattice_NC(c->lattice);
    Layout L;
    size_t o = 0;
    auto take = [&](size_t bytes) {
        size_t at = o;
        o = align256(o + bytes);
        return at;
    };
    const size_t ps = c->precision == 0 ? 4 : 2;
    L.f0 = take(ps * c->ncomp * (Q - 1) * N);
    L.f1 = take(ps * c->ncomp * (Q - 1) * N);
    L.frest = take(sizeof(float) * c->ncomp * N);
    L.drho = take(sizeof(float) * 4 * N);
    L.u = take(sizeof(float) * 3 * N);
    L.c0 = take(sizeof(float) * NC * N);
    L.c1 = take(sizeof(float) * NC * N);
    L.r = take(sizeof(float) * NC * N);
    L.dbg = take(sizeof(float) * kStagePlanes * N);
    L.q = take(sizeof(float) * 6 * N);
    L.status = take(256);
    L.dpart = take(sizeof(double) * kDiagBlocks * kDiagVals);
    L.dout = take(sizeof(double) * kDiagVals);
    L.total = o;
    return L;
}

void build_tensor_maps(vefd_ctx* c);

void carve(vefd_ctx* c) {
    const Layout L = layout_of(&c->cfg);
    char* b = (char*)c->mem;
    c->f[0] = b + L.f0;
    c->f[1] = b + L.f1;
    c->frest = (float*)(b + L.frest);
    c->drho = (float*)(b + L.drho);
    c->drho_alt = c->drho + 2 * (size_t)c->cfg.nx * c->cfg.ny * c->cfg.nz;
    c->u = (float*)(b + L.u);
    c->C[0] = (float*)(b + L.c0);
    c->C[1] = (float*)(b + L.c1);
    c->R = (float*)(b + L.r);
    c->dbg = (float*)(b + L.dbg);
    c->qbuf = (float*)(b + L.q);
    c->status = (unsigned*)(b + L.status);
    c->diag_part = (double*)(b + L.dpart);
    c->diag_out = (double*)(b + L.dout);
    c->tma_ok = false;
    build_tensor_maps(c);
    if (const char* e = getenv("VEFD_SCHEDULE")) c->sched = atoi(e) & 3;
    if (const char* e = getenv("VEFD_ZM_SEGMENT")) c->zm_seg_fixed = atoi(e) > 0 ? atoi(e) : 0;
    if (getenv("VEFD_NO_PDL")) c->pdl = false;
    if (const char* e = getenv("VEFD_SLAB_SEGMENT")) c->slab_zs = atoi(e) > 0 ? atoi(e) : 12;
    if (const char* e = getenv("VEFD_SLAB_PDL")) c->slab_pdl = atoi(e) != 0;
}

// (Re)builds the TMA descriptors of both population buffers for the selected
// kernel configuration; shapes the staged kernels cannot take use the
// register-only kernels.
void build_tensor_maps(vefd_ctx* c) {
    const int prec = c->cfg.precision;
    const int lat = c->cfg.lattice, nc = c->cfg.ncomp, nx = c->cfg.nx, ny = c->cfg.ny, nz = c->cfg.nz;
    c->tma_ok = false;
    c->zm_ok = false;
    c->fused_ok = false;
    c->parts_ok = false;
    if (getenv("VEFD_NO_TMA") || !pop_tile_eligible(lat, prec, nx, ny, nz, 0)) return;
    // the densities/FD pass keeps the default tile
    if (!(make_pop_tensor_map(lat, nc, prec, nx, ny, nz, c->f[0], &c->tmap_post[0]) &&
          make_pop_tensor_map(lat, nc, prec, nx, ny, nz, c->f[1], &c->tmap_post[1])))
        return;
    int tile = pop_tile_eligible(lat, prec, nx, ny, nz, c->lat_tile) ? c->lat_tile : 0;
    c->lat_tile = tile;
    int bx, by, bz;
    lattice_tile_shape(lat, tile, &bx, &by, &bz);
    if (!(make_pop_tensor_map_box(lat, nc, prec, nx, ny, nz, c->f[0], bx, by, bz, &c->tmap[0]) &&
          make_pop_tensor_map_box(lat, nc, prec, nx, ny, nz, c->f[1], bx, by, bz, &c->tmap[1])))
        return;
    c->tma_ok = true;
    if (c->post_mode != 1 && !getenv("VEFD_NO_ZMARCH") && post_zm_eligible(lat, nx, ny)) {
        c->zm_ok = make_pop_tensor_map_box(c->cfg.lattice, c->cfg.ncomp, prec, c->cfg.nx, c->cfg.ny, c->cfg.nz,
                                           c->f[0], 32, 8, 1, &c->tmap_zm[0]) &&
                   make_pop_tensor_map_box(c->cfg.lattice, c->cfg.ncomp, prec, c->cfg.nx, c->cfg.ny, c->cfg.nz,
                                           c->f[1], 32, 8, 1, &c->tmap_zm[1]);
        c->fused_ok = c->zm_ok && c->post_mode == 0 && !getenv("VEFD_NO_FUSED");
        // partial densities: every node of a whole tile (a node on at most one
        // face per axis), tiles 32 x 4 x 2 and 32 x 2 x 4
        c->parts_ok = c->zm_ok && c->post_mode == 3 && (tile == 0 || tile == 1) && ny % by == 0 && nz % bz == 0 &&
                      bz >= 2 && by >= 2;
    }
}

StepParams params_of(const vefd_ctx* c) {
    StepParams p;
    p.nx = c->cfg.nx;
    p.ny = c->cfg.ny;
    p.nz = c->cfg.nz;
    p.walls = c->cfg.walls;
    p.N = c->N;
    p.G = (float)c->cfg.G;
    p.eta_A = (float)c->cfg.eta_A;
    p.eta_B = (float)c->cfg.eta_B;
    p.inv_delta = (float)(1.0 / c->cfg.delta);
    p.u_wall = (float)c->u_wall;
    for (int k = 0; k < 3; ++k) p.fext[k] = (float)c->fext[k];
    if (c->D == 2) p.fext[2] = 0.0f;
    p.inv_tau_p = (float)(1.0 / c->tau_p);
    p.feedback = (float)(c->eta_p / c->tau_p);
    p.L2m3 = (float)(c->L2 - 3.0);
    p.kappa = (float)c->kappa;
    p.phase = c->phase;
    p.have_prev = c->have_prev;
    p.rho_ref[0] = (float)c->rho_ref[0];
    p.rho_ref[1] = (float)c->rho_ref[1];
    p.prec = c->cfg.precision;
    p.coupling = c->coupling;
    p.collision = c->collision;
    p.chol = c->chol;
    p.pdl = c->pdl ? 1 : 0;
    p.ylo = 0;
    p.yhi = c->cfg.ny;
    p.post_zs = 0;
    return p;
}

// The partial densities of post mode 3 (off otherwise); the staging planes are
// free inside a step.
Parts parts_of(const vefd_ctx* c) {
    Parts q{};
    if (!c->parts_ok) return q;
    int bx;
    lattice_tile_shape(c->cfg.lattice, c->lat_tile, &bx, &q.by, &q.bz);
    q.part = c->dbg;
    return q;
}

StepBufs bufs_of(vefd_ctx* c) {
    StepBufs b;
    b.fin = c->f[c->cur];
    b.fout = c->f[1 - c->cur];
    b.frest = c->frest;
    b.drho = c->drho;
    b.drho_next = c->drho_alt;
    b.u = c->u;
    b.Cin = c->C[c->ccur];
    b.Cout = c->C[1 - c->ccur];
    b.R = c->R;
    b.status = c->status;
    b.dbg = nullptr;
    b.Q = c->qbuf;
    return b;
}

vefd_status need_ready(vefd_ctx* c) {
    if (!c) return VEFD_ERR_ARG;
    if (!c->mem) return fail(c, VEFD_ERR_STATE, "device memory is not bound");
    if (!c->initialised) return fail(c, VEFD_ERR_STATE, "fields are not initialised");
    return VEFD_OK;
}

size_t field_planes(const vefd_ctx* c, int field) {
    switch (field) {
    case VEFD_RHO_A: case VEFD_RHO_B: case VEFD_PHI: case VEFD_TAU: return 1;
    case VEFD_U: case VEFD_G_A: case VEFD_G_B: case VEFD_F_P: return (size_t)c->D;
    case VEFD_C: case VEFD_SIGMA_P: case VEFD_RPREV: return (size_t)c->NC;
    case VEFD_POPS: return (size_t)c->cfg.ncomp * c->Q;
    default: return 0;
    }
}

// moments and the macroscopic pass (velocity, optionally forces and tau) of the current state
vefd_status macro_pass(vefd_ctx* c, bool with_dbg) {
    StepParams p = params_of(c);
    StepBufs b = bufs_of(c);
    b.dbg = with_dbg ? c->dbg : nullptr;
    // densities and feedback stress of the current state (kept by the step when current)
    if (!c->drho_valid) VEFD_CUDA(c, launch_pre(c->cfg.lattice, c->cfg.ncomp, p, b, c->stream));
    VEFD_CUDA(c, launch_lattice(c->cfg.lattice, c->cfg.ncomp, false, p, b, c->stream, nullptr, 0, 0));
    c->drho_valid = true;
    return VEFD_OK;
}

vefd_status copy_out(vefd_ctx* c, void* dst, const void* src, size_t bytes, int dst_on_device) {
    VEFD_CUDA(c, cudaMemcpyAsync(dst, src, bytes, dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                                 c->stream));
    if (!dst_on_device) VEFD_CUDA(c, cudaStreamSynchronize(c->stream));
    return VEFD_OK;
}

// SplitMix64 (Steele, Lea & Flood 2014): output for counter i of stream seed
uint64_t splitmix64(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

// The pipelined y-slab split applies for K slabs: staged lattice tiles (not
// the persistent forms) with the separate z-marching pass, D3Q19, and rows
// that split into K slabs of whole 32 x 8 columns.
bool slabs_fit(const vefd_ctx* c, int K) {
    return K >= 2 && c->cfg.lattice == VEFD_D3Q19 && c->tma_ok && c->zm_ok && !c->fused_ok && c->lat_tile <= 2 &&
           c->cfg.ny % (8 * K) == 0;
}

// Slabs of the step graph for this lattice and kernel choice (0: no graph,
// 1: whole-lattice launch pairs replayed as a graph): the setting, or
// automatically 8 slabs when NY is a multiple of 64 and 4 when of 32 where
// the split applies and every slab holds at least kSlabMinNodes nodes,
// otherwise 1.  Measured on D3Q19 droplets (MLUPS, slabs / whole-lattice
// graph): 128 x 64 x 128 10002 / 9281 and 128^3 10130 / 9629 with 8 slabs
// of 131k and 262k nodes, but 96 x 64 x 96 8574 / 9056, 64^3 6623 / 10042
// and 64 x 32 x 64 4654 / 8853 with slabs of 74k, 33k and 33k nodes: a
// slab's kernels must fill the GPU beside their neighbours.  An explicit
// slab count the lattice does not admit means no graph.
constexpr long long kSlabMinNodes = 100000;
int slab_count(const vefd_ctx* c) {
    if (c->slabs >= 2) return slabs_fit(c, c->slabs) ? c->slabs : 0;
    if (c->slabs >= 0) return c->slabs;
    const int K = c->cfg.ny % 64 == 0 ? 8 : (c->cfg.ny % 32 == 0 ? 4 : 0);
    return slabs_fit(c, K) && c->N / K >= kSlabMinNodes ? K : 1;
}

// Everything a captured step bakes into its launches: parameters, kernel
// choices, memory and the ping-pong parities.
std::vector<double> state_key(const vefd_ctx* m) {
    return {m->u_wall, m->fext[0], m->fext[1], m->fext[2], m->tau_p, m->eta_p, m->L2, m->kappa,
            (double)m->phase, (double)m->fd_on, (double)m->coupling, (double)m->collision, (double)m->chol,
            m->rho_ref[0], m->rho_ref[1], (double)m->lat_tile, (double)m->tma_ok, (double)m->zm_ok,
            (double)m->fused_ok, (double)m->parts_ok, (double)(m->drho < m->drho_alt), (double)m->sched,
            (double)m->cur,
            (double)m->ccur, (double)m->have_prev, (double)m->drho_valid, (double)m->pdl,
            (double)(uintptr_t)m->mem, (double)m->zm_seg_fixed, (double)slab_count(m), (double)m->slab_chunk};
}

// The next step is the plain AB2 step with current densities (not the Euler
// start or the densities-on-demand pass).
bool steady_state(const vefd_ctx* m) { return m->drho_valid && (m->have_prev || !m->fd_on); }

// The step graph applies: a slab count (or the whole-lattice graph), no
// kernel timing, and a stream that is not itself being captured.
bool slab_usable(vefd_ctx* c) {
    if (slab_count(c) < 1 || c->prof_on) return false;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(c->stream, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return false;
    return true;
}

// Records an event pair around one launch when kernel timing is on.
struct ProfScope {
    vefd_ctx* c;
    size_t slot;
    bool ok;
    ProfScope(vefd_ctx* ctx, int kind) : c(ctx), slot(0), ok(false) {
        if (!c->prof_on) return;
        if (c->prof_used * 2 + 2 > c->prof_ev.size()) {
            for (int k = 0; k < 256; ++k) {
                cudaEvent_t e;
                if (cudaEventCreate(&e) != cudaSuccess) return;
                c->prof_ev.push_back(e);
            }
        }
        slot = c->prof_used++;
        if (c->prof_kind.size() < c->prof_used) c->prof_kind.resize(c->prof_used);
        c->prof_kind[slot] = kind;
        ok = cudaEventRecord(c->prof_ev[2 * slot], c->stream) == cudaSuccess;
    }
    ~ProfScope() {
        if (ok) cudaEventRecord(c->prof_ev[2 * slot + 1], c->stream);
    }
};

}  // namespace

extern "C" {

vefd_status vefd_required_bytes(const vefd_config* cfg, size_t* bytes) {
    const char* why = nullptr;
    if (!bytes || !config_ok(cfg, &why)) return VEFD_ERR_ARG;
    *bytes = layout_of(cfg).total;
    return VEFD_OK;
}

vefd_status vefd_create(const vefd_config* cfg, void* stream, vefd_ctx** out) {
    const char* why = nullptr;
    if (!out) return VEFD_ERR_ARG;
    *out = nullptr;
    if (!config_ok(cfg, &why)) return VEFD_ERR_ARG;
    vefd_ctx* c = new (std::nothrow) vefd_ctx();
    if (!c) return VEFD_ERR_ARG;
    c->cfg = *cfg;
    c->Q = lattice_Q(cfg->lattice);
    c->D = lattice_D(cfg->lattice);
    c->NC = lattice_NC(cfg->lattice);
    c->N = (long long)cfg->nx * cfg->ny * cfg->nz;
    c->psize = cfg->precision == 0 ? 4 : 2;
    c->stream = (cudaStream_t)stream;
    if (!cfg->external_memory) {
        const size_t bytes = layout_of(cfg).total;
        cudaError_t e = cudaMalloc(&c->mem, bytes);
        if (e != cudaSuccess) {
            delete c;
            return VEFD_ERR_CUDA;
        }
        c->mem_bytes = bytes;
        c->owned = true;
        carve(c);
        if (cudaMemsetAsync(c->mem, 0, bytes, c->stream) != cudaSuccess) {
            cudaFree(c->mem);
            delete c;
            return VEFD_ERR_CUDA;
        }
    }
    *out = c;
    return VEFD_OK;
}

vefd_status vefd_bind_device_memory(vefd_ctx* c, void* dev_ptr, size_t bytes) {
    if (!c || !dev_ptr) return fail(c, VEFD_ERR_ARG, "NULL argument");
    if (c->mem) return fail(c, VEFD_ERR_STATE, "memory already bound");
    if (((uintptr_t)dev_ptr & 255u) != 0) return fail(c, VEFD_ERR_ARG, "device memory must be 256-byte aligned");
    const size_t need = layout_of(&c->cfg).total;
    if (bytes < need) return fail(c, VEFD_ERR_ARG, "need %zu bytes, got %zu", need, bytes);
    c->mem = dev_ptr;
    c->mem_bytes = bytes;
    c->owned = false;
    carve(c);
    VEFD_CUDA(c, cudaMemsetAsync(c->mem, 0, need, c->stream));
    return VEFD_OK;
}

void vefd_destroy(vefd_ctx* c) {
    if (!c) return;
    if (c->stream || c->mem) cudaStreamSynchronize(c->stream);
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.second);
    for (cudaStream_t s : c->slab_s) cudaStreamDestroy(s);
    for (cudaEvent_t e : c->slab_evL) cudaEventDestroy(e);
    for (cudaEvent_t e : c->slab_evP) cudaEventDestroy(e);
    if (c->slab_fork) cudaEventDestroy(c->slab_fork);
    if (c->cap) cudaStreamDestroy(c->cap);
    if (c->owned && c->mem) cudaFree(c->mem);
    for (cudaEvent_t e : c->prof_ev) cudaEventDestroy(e);
    delete c;
}

vefd_status vefd_set_stream(vefd_ctx* c, void* stream) {
    if (!c) return VEFD_ERR_ARG;
    c->stream = (cudaStream_t)stream;
    return VEFD_OK;
}

vefd_status vefd_set_wall_shear(vefd_ctx* c, double u_wall) {
    if (!c) return VEFD_ERR_ARG;
    if (!(std::fabs(u_wall) < 0.1)) return fail(c, VEFD_ERR_ARG, "|u_wall| must be < 0.1 (lattice Mach limit)");
    c->u_wall = u_wall;
    return VEFD_OK;
}

vefd_status vefd_set_body_force(vefd_ctx* c, double fx, double fy, double fz) {
    if (!c) return VEFD_ERR_ARG;
    if (!std::isfinite(fx) || !std::isfinite(fy) || !std::isfinite(fz))
        return fail(c, VEFD_ERR_ARG, "body force must be finite");
    c->fext[0] = fx;
    c->fext[1] = fy;
    c->fext[2] = fz;
    return VEFD_OK;
}

vefd_status vefd_set_fenep(vefd_ctx* c, double tau_p, double eta_p, double L2, double kappa, int phase, int fd_on) {
    if (!c) return VEFD_ERR_ARG;
    if (!(tau_p > 0.0) || !std::isfinite(tau_p)) return fail(c, VEFD_ERR_ARG, "tau_p must be > 0");
    if (!(eta_p >= 0.0) || !std::isfinite(eta_p)) return fail(c, VEFD_ERR_ARG, "eta_p must be >= 0");
    if (!(L2 > 3.0)) return fail(c, VEFD_ERR_ARG, "L2 must be > 3");
    if (!(kappa >= 0.0) || !(kappa < 0.5 / c->D)) return fail(c, VEFD_ERR_ARG, "kappa must be in [0, 1/(2 dim))");
    if (phase < -1 || phase > 1) return fail(c, VEFD_ERR_ARG, "phase must be -1, 0 or 1");
    c->tau_p = tau_p;
    c->eta_p = eta_p;
    c->L2 = L2;
    c->kappa = kappa;
    c->phase = phase;
    c->fd_on = fd_on ? 1 : 0;
    c->drho_valid = false;  // the feedback stress depends on these parameters
    return VEFD_OK;
}

vefd_status vefd_set_polymer_coupling(vefd_ctx* c, int mode) {
    if (!c) return VEFD_ERR_ARG;
    if (mode != 0 && mode != 1) return fail(c, VEFD_ERR_ARG, "coupling must be 0 (body force) or 1 (equilibrium)");
    c->coupling = mode;
    return VEFD_OK;
}

vefd_status vefd_set_collision(vefd_ctx* c, int model) {
    if (!c) return VEFD_ERR_ARG;
    if (model != 0 && model != 1) return fail(c, VEFD_ERR_ARG, "collision must be 0 (single time) or 1 (moment space)");
    c->collision = model;
    return VEFD_OK;
}

vefd_status vefd_set_conformation_update(vefd_ctx* c, int scheme) {
    if (!c) return VEFD_ERR_ARG;
    if (scheme != 0 && scheme != 1) return fail(c, VEFD_ERR_ARG, "scheme must be 0 (C) or 1 (log-Cholesky)");
    if (scheme != c->chol) c->have_prev = 0;  // the history holds rates of the other variables
    c->chol = scheme;
    return VEFD_OK;
}

vefd_status vefd_field_bytes(const vefd_ctx* c, vefd_field field, size_t* bytes) {
    if (!c || !bytes) return VEFD_ERR_ARG;
    const size_t planes = field_planes(c, field);
    if (!planes) return VEFD_ERR_ARG;
    *bytes = planes * (size_t)c->N * sizeof(float);
    return VEFD_OK;
}

vefd_status vefd_init_fields(vefd_ctx* c, const float* rho_A, const float* rho_B, const float* u, const float* C0,
                             int on_device) {
    if (!c || !rho_A || (c->cfg.ncomp == 2 && !rho_B)) return fail(c, VEFD_ERR_ARG, "density fields missing");
    if (!c->mem) return fail(c, VEFD_ERR_STATE, "device memory is not bound");
    const long long N = c->N;
    const size_t plane = sizeof(float) * (size_t)N;
    // stage the inputs in the staging planes
    c->cur = 0;
    c->ccur = 0;
    float* st = c->dbg;
    float* sA = st;
    float* sB = st + N;
    float* sU = st + 2 * N;
    float* sC = st + 5 * N;
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    VEFD_CUDA(c, cudaMemcpyAsync(sA, rho_A, plane, kind, c->stream));
    if (c->cfg.ncomp == 2) VEFD_CUDA(c, cudaMemcpyAsync(sB, rho_B, plane, kind, c->stream));
    if (u) VEFD_CUDA(c, cudaMemcpyAsync(sU, u, plane * c->D, kind, c->stream));
    if (C0) VEFD_CUDA(c, cudaMemcpyAsync(sC, C0, plane * c->NC, kind, c->stream));
    // reference densities: domain means (FP64 sums in a fixed order on the
    // device), so that the stored deviations are small; the densities must be
    // finite and non-negative
    double sums[3];
    VEFD_CUDA(c, launch_density_sums(sA, c->cfg.ncomp == 2 ? sB : nullptr, N, c->diag_part, c->diag_out, c->stream));
    VEFD_CUDA(c, cudaMemcpyAsync(sums, c->diag_out, sizeof sums, cudaMemcpyDeviceToHost, c->stream));
    VEFD_CUDA(c, cudaStreamSynchronize(c->stream));
    if (sums[2] != 0.0) {
        c->initialised = 0;
        return fail(c, VEFD_ERR_ARG, "densities must be finite and >= 0");
    }
    c->rho_ref[0] = (double)(float)(sums[0] / (double)N);
    c->rho_ref[1] = c->cfg.ncomp == 2 ? (double)(float)(sums[1] / (double)N) : 0.0;
    StepParams p = params_of(c);
    VEFD_CUDA(c, launch_init_equilibrium(c->cfg.lattice, c->cfg.ncomp, p, sA, sB, u ? sU : nullptr, c->f[0],
                                         c->frest, c->stream));
    if (C0) VEFD_CUDA(c, launch_tensor_shift(c->cfg.lattice, sC, c->C[0], N, -1.0f, c->stream));
    else VEFD_CUDA(c, cudaMemsetAsync(c->C[0], 0, plane * c->NC, c->stream));
    VEFD_CUDA(c, cudaMemsetAsync(c->R, 0, plane * c->NC, c->stream));
    VEFD_CUDA(c, cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream));
    VEFD_CUDA(c, cudaStreamSynchronize(c->stream));
    c->have_prev = 0;
    c->steps = 0;
    c->initialised = 1;
    c->drho_valid = false;
    return VEFD_OK;
}

vefd_status vefd_init_droplet(vefd_ctx* c, double cx, double cy, double cz, double R, double rho_in, double rho_out,
                              double width, uint64_t seed, double phi_amp) {
    if (!c) return VEFD_ERR_ARG;
    if (c->cfg.ncomp != 2) return fail(c, VEFD_ERR_ARG, "a droplet needs two components");
    if (!(R > 0.0) || !(width > 0.0) || !(rho_in >= 0.0) || !(rho_out >= 0.0))
        return fail(c, VEFD_ERR_ARG, "bad droplet parameters");
    const long long N = c->N;
    std::vector<float> rA((size_t)N), rB((size_t)N);
    const double tot = rho_in + rho_out;
    long long i = 0;
    for (int z = 0; z < c->cfg.nz; ++z)
        for (int y = 0; y < c->cfg.ny; ++y)
            for (int x = 0; x < c->cfg.nx; ++x, ++i) {
                const double dx = x - cx, dy = y - cy, dz = z - cz;
                const double r = std::sqrt(dx * dx + dy * dy + dz * dz);
                double a = rho_out + (rho_in - rho_out) * 0.5 * (1.0 + std::tanh(2.0 * (R - r) / width));
                double b = tot - a;
                if (phi_amp != 0.0) {
                    const double uni = (double)(splitmix64(seed, (uint64_t)i) >> 11) * (1.0 / 4503599627370496.0) - 1.0;
                    const double dphi = phi_amp * uni;
                    a += 0.5 * tot * dphi;
                    b -= 0.5 * tot * dphi;
                }
                rA[(size_t)i] = (float)a;
                rB[(size_t)i] = (float)b;
            }
    return vefd_init_fields(c, rA.data(), rB.data(), nullptr, nullptr, 0);
}

vefd_status vefd_write_field(vefd_ctx* c, vefd_field field, const void* src, size_t bytes, int src_on_device) {
    vefd_status st = need_ready(c);
    if (st != VEFD_OK) return st;
    if (!src) return fail(c, VEFD_ERR_ARG, "NULL source");
    size_t need = 0;
    if (vefd_field_bytes(c, field, &need) != VEFD_OK) return fail(c, VEFD_ERR_ARG, "unknown field");
    if (bytes != need) return fail(c, VEFD_ERR_ARG, "field needs %zu bytes, got %zu", need, bytes);
    const cudaMemcpyKind kind = src_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    float* stg = c->dbg;
    StepParams p = params_of(c);
    switch (field) {
    case VEFD_POPS: {
        // absolute FP32 populations -> stored deviations, a few planes at a time
        const int planes = c->cfg.ncomp * c->Q;
        const size_t plane = sizeof(float) * (size_t)c->N;
        for (int p0 = 0; p0 < planes; p0 += kStagePlanes) {
            const int k = planes - p0 < kStagePlanes ? planes - p0 : kStagePlanes;
            VEFD_CUDA(c, cudaMemcpyAsync(stg, (const char*)src + p0 * plane, k * plane, kind, c->stream));
            VEFD_CUDA(c, launch_pops_convert(c->cfg.lattice, c->cfg.ncomp, p, c->f[c->cur], c->frest, stg, p0, k, 0,
                                             c->stream));
        }
        c->drho_valid = false;
        break;
    }
    case VEFD_C:
        VEFD_CUDA(c, cudaMemcpyAsync(stg, src, bytes, kind, c->stream));
        VEFD_CUDA(c, launch_tensor_shift(c->cfg.lattice, stg, c->C[c->ccur], c->N, -1.0f, c->stream));
        c->drho_valid = false;
        break;
    case VEFD_RPREV:
        VEFD_CUDA(c, cudaMemcpyAsync(c->R, src, bytes, kind, c->stream));
        c->have_prev = 1;
        break;
    default:
        return fail(c, VEFD_ERR_ARG, "field %d cannot be written", (int)field);
    }
    if (!src_on_device) VEFD_CUDA(c, cudaStreamSynchronize(c->stream));
    return VEFD_OK;
}

// Captures `chunk` steps as the pipelined y-slab graph into *out.
// Slab k's lattice kernel of step t waits for the densities/FENE-P passes of
// step t - 1 on slabs k - 1, k, k + 1 (their densities, stress and velocity
// reads border its rows, and its pushes reach theirs); slab k's pass of step
// t waits for the lattice kernels of step t on slabs k - 1, k, k + 1 (their
// pushes and velocities reach its rows).  With walls the outer slabs have one
// neighbour, otherwise the slabs wrap.  Same-slab order is its stream's order.
static vefd_status step_eager(vefd_ctx* c, int64_t nsteps);

// Captures `chunk` eager steps (whole-lattice launch pairs) into *out:
// the graph form for lattices and kernel choices the slab split does not
// take; it saves the host-side launch cost of small lattices.  Capture only
// records the launches, so the host state they advanced is put back.
static vefd_status plain_capture(vefd_ctx* c, int64_t chunk, cudaGraphExec_t* out) {
    Range range("vefd capture step graph (whole lattice)");
    if (!c->cap && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess)
        return fail(c, VEFD_ERR_CUDA, "cannot create the capture stream");
    const int cur = c->cur, ccur = c->ccur, hp = c->have_prev;
    const int64_t steps = c->steps;
    float* const dr = c->drho;
    float* const dra = c->drho_alt;
    const bool dv = c->drho_valid;
    cudaStream_t own = c->stream;
    if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return fail(c, VEFD_ERR_CUDA, "cannot begin capture");
    c->stream = c->cap;
    const vefd_status st = step_eager(c, chunk);
    c->stream = own;
    cudaGraph_t graph = nullptr;
    const cudaError_t ce2 = cudaStreamEndCapture(c->cap, &graph);
    c->cur = cur;
    c->ccur = ccur;
    c->have_prev = hp;
    c->steps = steps;
    c->drho = dr;
    c->drho_alt = dra;
    c->drho_valid = dv;
    if (st != VEFD_OK || ce2 != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return st != VEFD_OK ? st : fail(c, VEFD_ERR_CUDA, "step graph capture failed: %s", cudaGetErrorString(ce2));
    }
    const cudaError_t ce = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
        *out = nullptr;
        return fail(c, VEFD_ERR_CUDA, "step graph instantiation failed");
    }
    return VEFD_OK;
}

static vefd_status slab_capture(vefd_ctx* c, int64_t chunk, cudaGraphExec_t* out) {
    Range range("vefd capture step graph (y-slabs)");
    const int K = slab_count(c);
    if (!c->cap && cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess)
        return fail(c, VEFD_ERR_CUDA, "cannot create the capture stream");
    if (!c->slab_fork && cudaEventCreateWithFlags(&c->slab_fork, cudaEventDisableTiming) != cudaSuccess)
        return fail(c, VEFD_ERR_CUDA, "cannot create events");
    while ((int)c->slab_s.size() < K) {
        cudaStream_t s = nullptr;
        cudaEvent_t a = nullptr, b = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
            return fail(c, VEFD_ERR_CUDA, "cannot create slab streams");
        c->slab_s.push_back(s);
        if (cudaEventCreateWithFlags(&a, cudaEventDisableTiming) != cudaSuccess)
            return fail(c, VEFD_ERR_CUDA, "cannot create events");
        c->slab_evL.push_back(a);
        if (cudaEventCreateWithFlags(&b, cudaEventDisableTiming) != cudaSuccess)
            return fail(c, VEFD_ERR_CUDA, "cannot create events");
        c->slab_evP.push_back(b);
    }
    const int rows = c->cfg.ny / K;
    const int lat_rev = c->sched & 1, post_rev = (c->sched >> 1) & 1;
    auto nbr = [&](int k, int d) -> int {
        const int j = k + d;
        if (j >= 0 && j < K) return j;
        return c->cfg.walls ? -1 : (j + K) % K;
    };
    if (cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return fail(c, VEFD_ERR_CUDA, "cannot begin capture");
    cudaError_t ce = cudaEventRecord(c->slab_fork, c->cap);
    for (int k = 0; k < K && ce == cudaSuccess; ++k) ce = cudaStreamWaitEvent(c->slab_s[k], c->slab_fork, 0);
    StepParams p0 = params_of(c);
    // a slab's kernels follow each other on its stream; with programmatic
    // launch the next one may start its prologue while the previous drains
    // (the cross-slab edges stay full dependencies)
    p0.pdl = c->pdl && c->slab_pdl ? 1 : 0;
    p0.post_zs = c->slab_zs;
    for (int64_t t = 0; t < chunk && ce == cudaSuccess; ++t) {
        const int par = (int)(t & 1);
        const int cur = c->cur ^ par, ccur = c->ccur ^ (c->fd_on ? par : 0);
        StepBufs b = bufs_of(c);
        b.fin = c->f[cur];
        b.fout = c->f[1 - cur];
        b.Cin = c->C[ccur];
        b.Cout = c->C[1 - ccur];
        auto lattice_node = [&](int k) {
            for (int d = -1; d <= 1 && t > 0 && ce == cudaSuccess; d += 2) {
                const int j = nbr(k, d);
                if (j >= 0 && j != k) ce = cudaStreamWaitEvent(c->slab_s[k], c->slab_evP[j], 0);
            }
            StepParams p = p0;
            p.ylo = k * rows;
            p.yhi = (k + 1) * rows;
            if (ce == cudaSuccess)
                ce = launch_lattice(c->cfg.lattice, c->cfg.ncomp, true, p, b, c->slab_s[k], &c->tmap[cur], lat_rev,
                                    c->lat_tile, parts_of(c));
            if (ce == cudaSuccess) ce = cudaEventRecord(c->slab_evL[k], c->slab_s[k]);
        };
        auto pass_node = [&](int k) {
            for (int d = -1; d <= 1 && ce == cudaSuccess; d += 2) {
                const int j = nbr(k, d);
                if (j >= 0 && j != k) ce = cudaStreamWaitEvent(c->slab_s[k], c->slab_evL[j], 0);
            }
            StepParams p = p0;
            p.ylo = k * rows;
            p.yhi = (k + 1) * rows;
            if (ce == cudaSuccess)
                ce = launch_post_zm(c->cfg.ncomp, c->fd_on != 0, p, b, &c->tmap_zm[1 - cur], c->slab_s[k], post_rev,
                                    parts_of(c));
            if (ce == cudaSuccess) ce = cudaEventRecord(c->slab_evP[k], c->slab_s[k]);
        };
        // (capturing each pass right after the lattice kernels it waits for
        // instead measured the same: the graph runs nodes as their inputs complete)
        for (int k = 0; k < K && ce == cudaSuccess; ++k) lattice_node(k);
        for (int k = 0; k < K && ce == cudaSuccess; ++k) pass_node(k);
    }
    for (int k = 0; k < K && ce == cudaSuccess; ++k) ce = cudaStreamWaitEvent(c->cap, c->slab_evP[k], 0);
    cudaGraph_t graph = nullptr;
    const cudaError_t ce2 = cudaStreamEndCapture(c->cap, &graph);
    if (ce != cudaSuccess || ce2 != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(c, VEFD_ERR_CUDA, "step graph capture failed: %s", cudaGetErrorString(ce != cudaSuccess ? ce : ce2));
    }
    ce = cudaGraphInstantiate(out, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
        *out = nullptr;
        return fail(c, VEFD_ERR_CUDA, "step graph instantiation failed");
    }
    return VEFD_OK;
}

// Graph sizes kept per context (the main chunk and recent remainders).
constexpr size_t kGraphSizes = 4;

// Destroys every captured step graph (after the replays in flight).
static void drop_graphs(vefd_ctx* c) {
    if (c->graphs.empty()) return;
    cudaStreamSynchronize(c->stream);
    for (auto& g : c->graphs) cudaGraphExecDestroy(g.second);
    c->graphs.clear();
}

// The step graph of `n` steps (n even) for the current setting and state: the
// slab pipeline or the whole-lattice form, captured on first use.  Graphs of a
// stale state are dropped first; beyond kGraphSizes sizes the least recently
// used one goes.
static vefd_status graph_get(vefd_ctx* c, int64_t n, cudaGraphExec_t* exec) {
    const std::vector<double> key = state_key(c);
    if (!c->graphs.empty() && (c->slab_key != key || c->slab_parity != c->cur)) drop_graphs(c);
    for (size_t k = 0; k < c->graphs.size(); ++k)
        if (c->graphs[k].first == n) {
            std::rotate(c->graphs.begin(), c->graphs.begin() + k, c->graphs.begin() + k + 1);
            *exec = c->graphs[0].second;
            return VEFD_OK;
        }
    cudaGraphExec_t e = nullptr;
    const vefd_status st = slab_count(c) >= 2 ? slab_capture(c, n, &e) : plain_capture(c, n, &e);
    if (st != VEFD_OK) return st;
    if (c->graphs.size() >= kGraphSizes) {
        cudaStreamSynchronize(c->stream);  // its replays may still be in flight
        cudaGraphExecDestroy(c->graphs.back().second);
        c->graphs.pop_back();
    }
    c->graphs.insert(c->graphs.begin(), std::make_pair(n, e));
    c->slab_key = key;
    c->slab_parity = c->cur;
    *exec = e;
    // upload now (in stream order), so that the first replay only launches
    VEFD_CUDA(c, cudaGraphUpload(e, c->stream));
    return VEFD_OK;
}

// How vefd_step replays `nsteps` steps from the current state: `pre` eager
// steps (the Euler start or densities pass, and one step that brings the
// ping-pong parity back to the captured graphs'), `full` replays of the main
// chunk, one replay of the even remainder `part`, then eager steps for the
// rest (none or one).  Graphs are used only where the step graph applies.
static void step_plan(const vefd_ctx* c, int64_t nsteps, int64_t* pre, int64_t* full, int64_t* part) {
    *pre = *full = *part = 0;
    if (nsteps <= 0) return;
    if (!steady_state(c)) {
        *pre = 1;
        --nsteps;
    }
    // graphs replay from one parity; realign with one eager step when that
    // still leaves a graph's worth of steps, otherwise step eagerly
    const int parity = c->cur ^ (int)(*pre & 1);
    if (!c->graphs.empty() && parity != c->slab_parity) {
        if (nsteps < 3) return;
        ++*pre;
        --nsteps;
    }
    *full = nsteps / c->slab_chunk;
    *part = (nsteps % c->slab_chunk) & ~(int64_t)1;
}

vefd_status vefd_step(vefd_ctx* c, int64_t nsteps) {
    Range range("vefd_step");
    vefd_status st = need_ready(c);
    if (st != VEFD_OK) return st;
    if (nsteps < 0) return fail(c, VEFD_ERR_ARG, "nsteps must be >= 0");
    if (nsteps > 0 && slab_usable(c)) {
        int64_t pre, full, part;
        step_plan(c, nsteps, &pre, &full, &part);
        if (pre > 0) {
            st = step_eager(c, pre);
            if (st != VEFD_OK) return st;
            nsteps -= pre;
        }
        cudaGraphExec_t exec = nullptr;
        if (full > 0) {
            st = graph_get(c, c->slab_chunk, &exec);
            if (st != VEFD_OK) return st;
            for (int64_t r = 0; r < full; ++r) VEFD_CUDA(c, cudaGraphLaunch(exec, c->stream));
        }
        if (part > 0) {
            st = graph_get(c, part, &exec);
            if (st != VEFD_OK) return st;
            VEFD_CUDA(c, cudaGraphLaunch(exec, c->stream));
        }
        // even step counts leave every ping-pong parity where it was
        c->steps += full * c->slab_chunk + part;
        nsteps -= full * c->slab_chunk + part;
    }
    return step_eager(c, nsteps);
}

// Steps one launch pair at a time on the context stream.
static vefd_status step_eager(vefd_ctx* c, int64_t nsteps) {
    const int lat_rev = c->sched & 1, post_rev = (c->sched >> 1) & 1;
    for (int64_t n = 0; n < nsteps; ++n) {
        StepParams p = params_of(c);
        StepBufs b = bufs_of(c);
        if (!c->drho_valid) {
            ProfScope ps(c, 0);
            VEFD_CUDA(c, launch_pre(c->cfg.lattice, c->cfg.ncomp, p, b, c->stream));
        }
        if (c->fused_ok) {
            // populations n -> n+1, velocity of time n and the partial densities of
            // n+1; then the densities completed, and the FENE-P update
            const int zs = c->zm_seg_fixed > 0 ? std::min(c->zm_seg_fixed, c->cfg.nz) : lattice_zm_segment(p);
            {
                ProfScope ps(c, 1);
                VEFD_CUDA(c, launch_lattice_zm(c->cfg.ncomp, p, b, c->stream, &c->tmap_zm[c->cur], zs, lat_rev));
            }
            {
                ProfScope ps(c, 2);
                VEFD_CUDA(c, launch_post_zm_fused(c->cfg.ncomp, c->fd_on != 0, p, b, c->stream, zs, post_rev));
            }
            std::swap(c->drho, c->drho_alt);
            if (c->fd_on) {
                c->ccur ^= 1;
                c->have_prev = 1;
            }
            c->drho_valid = true;
            c->cur ^= 1;
            c->steps++;
            continue;
        }
        {
            // populations n -> n+1, velocity of time n
            ProfScope ps(c, 1);
            VEFD_CUDA(c, launch_lattice(c->cfg.lattice, c->cfg.ncomp, true, p, b, c->stream,
                                        c->tma_ok ? (const void*)&c->tmap[c->cur] : nullptr, lat_rev, c->lat_tile,
                                        parts_of(c)));
        }
        {
            // densities of time n+1 (they only depend on the new populations)
            // and the conformation update n -> n+1 (it only needs u^n and C^n)
            ProfScope ps(c, 2);
            if (c->zm_ok)
                VEFD_CUDA(c, launch_post_zm(c->cfg.ncomp, c->fd_on != 0, p, b, &c->tmap_zm[1 - c->cur], c->stream,
                                            post_rev, parts_of(c)));
            else if (c->tma_ok)
                VEFD_CUDA(c, launch_post_tma(c->cfg.lattice, c->cfg.ncomp, c->fd_on != 0, p, b, &c->tmap_post[1 - c->cur],
                                             c->stream, post_rev));
            else
                VEFD_CUDA(c, launch_post(c->cfg.lattice, c->cfg.ncomp, c->fd_on != 0, p, b, c->f[1 - c->cur],
                                         c->stream, post_rev));
        }
        if (c->fd_on) {
            c->ccur ^= 1;
            c->have_prev = 1;
        }
        c->drho_valid = true;
        c->cur ^= 1;
        c->steps++;
    }
    return VEFD_OK;
}

vefd_status vefd_read_field(vefd_ctx* c, vefd_field field, void* dst, size_t bytes, int dst_on_device) {
    vefd_status st = need_ready(c);
    if (st != VEFD_OK) return st;
    if (!dst) return fail(c, VEFD_ERR_ARG, "NULL destination");
    size_t need = 0;
    if (vefd_field_bytes(c, field, &need) != VEFD_OK) return fail(c, VEFD_ERR_ARG, "unknown field");
    if (bytes != need) return fail(c, VEFD_ERR_ARG, "field needs %zu bytes, got %zu", need, bytes);
    float* stg = c->dbg;
    const long long N = c->N;
    StepParams p = params_of(c);
    switch (field) {
    case VEFD_POPS: {
        // stored deviations -> absolute FP32 populations, a few planes at a time
        const int planes = c->cfg.ncomp * c->Q;
        const size_t plane = sizeof(float) * (size_t)N;
        for (int p0 = 0; p0 < planes; p0 += kStagePlanes) {
            const int k = planes - p0 < kStagePlanes ? planes - p0 : kStagePlanes;
            VEFD_CUDA(c, launch_pops_convert(c->cfg.lattice, c->cfg.ncomp, p, c->f[c->cur], c->frest, stg, p0, k, 1,
                                             c->stream));
            VEFD_CUDA(c, cudaMemcpyAsync((char*)dst + p0 * plane, stg, k * plane,
                                         dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream));
        }
        if (!dst_on_device) VEFD_CUDA(c, cudaStreamSynchronize(c->stream));
        return VEFD_OK;
    }
    case VEFD_C:
        VEFD_CUDA(c, launch_tensor_shift(c->cfg.lattice, c->C[c->ccur], stg, N, 1.0f, c->stream));
        return copy_out(c, dst, stg, bytes, dst_on_device);
    case VEFD_RPREV:
        return copy_out(c, dst, c->R, bytes, dst_on_device);
    case VEFD_SIGMA_P:
        VEFD_CUDA(c, launch_derived(c->cfg.lattice, c->cfg.ncomp, 5, p, c->drho, c->C[c->ccur], stg, c->stream));
        return copy_out(c, dst, stg, bytes, dst_on_device);
    case VEFD_RHO_A:
    case VEFD_RHO_B:
    case VEFD_PHI: {
        // the densities of the current state: kept by the step, else computed from the populations
        if (!c->drho_valid) {
            StepBufs b = bufs_of(c);
            VEFD_CUDA(c, launch_pre(c->cfg.lattice, c->cfg.ncomp, p, b, c->stream));
            c->drho_valid = true;
        }
        VEFD_CUDA(c, launch_derived(c->cfg.lattice, c->cfg.ncomp, (int)field, p, c->drho, c->C[c->ccur], stg,
                                    c->stream));
        return copy_out(c, dst, stg, bytes, dst_on_device);
    }
    case VEFD_U:
        st = macro_pass(c, false);
        if (st != VEFD_OK) return st;
        return copy_out(c, dst, c->u, bytes, dst_on_device);
    case VEFD_G_A:
    case VEFD_G_B:
    case VEFD_F_P:
    case VEFD_TAU: {
        st = macro_pass(c, true);
        if (st != VEFD_OK) return st;
        const int plane0 = field == VEFD_G_A ? 0 : (field == VEFD_G_B ? 3 : (field == VEFD_F_P ? 6 : 9));
        return copy_out(c, dst, c->dbg + (size_t)plane0 * N, bytes, dst_on_device);
    }
    default:
        return fail(c, VEFD_ERR_ARG, "unknown field");
    }
}

vefd_status vefd_diagnostics(vefd_ctx* c, double out[16]) {
    Range range("vefd_diagnostics");
    vefd_status st = need_ready(c);
    if (st != VEFD_OK) return st;
    if (!out) return fail(c, VEFD_ERR_ARG, "NULL output");
    st = macro_pass(c, false);
    if (st != VEFD_OK) return st;
    StepParams p = params_of(c);
    VEFD_CUDA(c, launch_diagnostics(c->cfg.lattice, c->cfg.ncomp, p, c->drho, c->u, c->C[c->ccur], c->diag_part,
                                    c->diag_out, c->stream));
    double v[kDiagVals];
    VEFD_CUDA(c, cudaMemcpyAsync(v, c->diag_out, sizeof v, cudaMemcpyDeviceToHost, c->stream));
    VEFD_CUDA(c, cudaStreamSynchronize(c->stream));
    const double N = (double)c->N;
    for (int k = 0; k < 16; ++k) out[k] = 0.0;
    out[0] = N * (double)(float)c->rho_ref[0] + v[0];
    out[1] = c->cfg.ncomp == 2 ? N * (double)(float)c->rho_ref[1] + v[1] : 0.0;
    out[2] = v[2];
    out[3] = v[3];
    out[4] = c->D == 3 ? v[4] : 0.0;
    out[5] = v[5] / N;
    out[6] = v[6] / N;
    // the kernel keeps max tr(C - I) and max |u|^2 (empty: -inf and 0)
    out[7] = std::fmax(0.0, (v[15] + 3.0) / ((double)p.L2m3 + 3.0));
    out[8] = std::sqrt(v[16]);
    const double m0 = v[9];
    out[9] = m0;
    if (m0 > 0.0) {
        const double cx = v[10] / m0, cy = v[11] / m0;
        const double ixx = v[12] / m0 - cx * cx, ixy = v[13] / m0 - cx * cy, iyy = v[14] / m0 - cy * cy;
        const double tr = ixx + iyy, det = ixx * iyy - ixy * ixy;
        const double disc = std::sqrt(std::fmax(0.25 * tr * tr - det, 0.0));
        const double l1 = 0.5 * tr + disc, l2 = std::fmax(0.5 * tr - disc, 0.0);
        const double a = std::sqrt(l1), b = std::sqrt(l2);
        out[10] = (a + b) > 0.0 ? (a - b) / (a + b) : 0.0;
        out[11] = 0.5 * std::atan2(2.0 * ixy, ixx - iyy);
        out[12] = cx;
        out[13] = cy;
    }
    out[14] = v[8];
    out[15] = v[7] / N;
    return VEFD_OK;
}

vefd_status vefd_get_status(vefd_ctx* c, uint32_t* bits) {
    if (!c || !bits) return VEFD_ERR_ARG;
    if (!c->mem) return fail(c, VEFD_ERR_STATE, "device memory is not bound");
    unsigned v = 0;
    VEFD_CUDA(c, cudaMemcpyAsync(&v, c->status, sizeof v, cudaMemcpyDeviceToHost, c->stream));
    VEFD_CUDA(c, cudaStreamSynchronize(c->stream));
    *bits = v;
    if (!v) return VEFD_OK;
    return (v & kStTimeout) ? VEFD_ERR_TIMEOUT : VEFD_ERR_UNSTABLE;
}

vefd_status vefd_wait_selftest(vefd_ctx* c, int arrive) {
    if (!c || (arrive != 0 && arrive != 1)) return VEFD_ERR_ARG;
    if (!c->mem) return fail(c, VEFD_ERR_STATE, "device memory is not bound");
    // a budget of 2^24 cycles: about 8 ms at the maximum SM clock
    VEFD_CUDA(c, launch_wait_selftest(c->status, arrive, 1LL << 24, c->stream));
    return VEFD_OK;
}

vefd_status vefd_clear_status(vefd_ctx* c) {
    if (!c) return VEFD_ERR_ARG;
    if (!c->mem) return fail(c, VEFD_ERR_STATE, "device memory is not bound");
    VEFD_CUDA(c, cudaMemsetAsync(c->status, 0, sizeof(unsigned), c->stream));
    return VEFD_OK;
}

vefd_status vefd_set_step_graph(vefd_ctx* c, int slabs, int chunk) {
    if (!c || slabs < -1 || slabs > 64 || chunk < 2 || (chunk & 1)) return VEFD_ERR_ARG;
    if (c->slabs != slabs || c->slab_chunk != chunk) {
        drop_graphs(c);
        c->slabs = slabs;
        c->slab_chunk = chunk;
    }
    return VEFD_OK;
}

vefd_status vefd_prepare_step_graph(vefd_ctx* c) {
    vefd_status st = need_ready(c);
    if (st != VEFD_OK) return st;
    if (!slab_usable(c) || !steady_state(c)) return VEFD_OK;
    cudaGraphExec_t exec = nullptr;
    return graph_get(c, c->slab_chunk, &exec);
}

vefd_status vefd_prepare_steps(vefd_ctx* c, int64_t nsteps) {
    vefd_status st = need_ready(c);
    if (st != VEFD_OK) return st;
    if (nsteps < 0) return fail(c, VEFD_ERR_ARG, "nsteps must be >= 0");
    if (!slab_usable(c) || !steady_state(c)) return VEFD_OK;
    // graphs of the other ping-pong parity would cost the call an eager
    // realigning step: capture at this parity instead
    if (!c->graphs.empty() && c->slab_parity != c->cur) drop_graphs(c);
    int64_t pre, full, part;
    step_plan(c, nsteps, &pre, &full, &part);
    cudaGraphExec_t exec = nullptr;
    if (full > 0) st = graph_get(c, c->slab_chunk, &exec);
    if (st == VEFD_OK && part > 0) st = graph_get(c, part, &exec);
    return st;
}

vefd_status vefd_get_step_graph(vefd_ctx* c, int* slabs, int* chunk, int* active) {
    if (!c || !slabs || !chunk || !active) return VEFD_ERR_ARG;
    *slabs = slab_count(c);
    *chunk = c->slab_chunk;
    *active = slab_usable(c) ? 1 : 0;
    return VEFD_OK;
}

vefd_status vefd_steps_done(const vefd_ctx* c, int64_t* n) {
    if (!c || !n) return VEFD_ERR_ARG;
    *n = c->steps;
    return VEFD_OK;
}

vefd_status vefd_kernels_per_step(const vefd_ctx* c, int* n) {
    if (!c || !n) return VEFD_ERR_ARG;
    // lattice + (densities of the new populations with the FD update); the
    // first step after initialisation adds one densities pass
    *n = 2;
    return VEFD_OK;
}

const char* vefd_last_error(const vefd_ctx* c) { return c ? c->err.c_str() : "NULL context"; }

vefd_status vefd_profile_kernels(vefd_ctx* c, int on) {
    if (!c) return VEFD_ERR_ARG;
    c->prof_on = on != 0;
    c->prof_used = 0;
    return VEFD_OK;
}

vefd_status vefd_kernel_times(vefd_ctx* c, double ms[3], int64_t launches[3]) {
    if (!c || !ms || !launches) return fail(c, VEFD_ERR_ARG, "NULL output");
    VEFD_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < 3; ++k) {
        ms[k] = 0.0;
        launches[k] = 0;
    }
    for (size_t i = 0; i < c->prof_used; ++i) {
        float t = 0.0f;
        VEFD_CUDA(c, cudaEventElapsedTime(&t, c->prof_ev[2 * i], c->prof_ev[2 * i + 1]));
        const int k = c->prof_kind[i];
        ms[k] += t;
        launches[k] += 1;
    }
    c->prof_used = 0;
    return VEFD_OK;
}

// ---- checkpoints ------------------------------------------------------------

namespace {
const char kMagic[8] = {'V', 'E', 'F', 'D', 'C', 'K', 'P', '1'};

struct CkptHeader {
    char magic[8];
    int32_t version;
    int32_t lattice, nx, ny, nz, ncomp, walls;
    double G, eta_A, eta_B, delta;
    double u_wall, fext[3], tau_p, eta_p, L2, kappa;
    int32_t phase, fd_on, have_prev, precision;
    double rho_ref[2];
    int64_t steps;
    uint32_t status;
    int32_t coupling;
    int32_t collision, chol;
};
}  // namespace

vefd_status vefd_checkpoint(vefd_ctx* c, const char* path) {
    Range range("vefd_checkpoint");
    vefd_status st = need_ready(c);
    if (st != VEFD_OK) return st;
    if (!path) return fail(c, VEFD_ERR_ARG, "NULL path");
    CkptHeader h;
    memset(&h, 0, sizeof h);
    memcpy(h.magic, kMagic, 8);
    h.version = 4;
    h.lattice = c->cfg.lattice;
    h.nx = c->cfg.nx;
    h.ny = c->cfg.ny;
    h.nz = c->cfg.nz;
    h.ncomp = c->cfg.ncomp;
    h.walls = c->cfg.walls;
    h.G = c->cfg.G;
    h.eta_A = c->cfg.eta_A;
    h.eta_B = c->cfg.eta_B;
    h.delta = c->cfg.delta;
    h.u_wall = c->u_wall;
    for (int k = 0; k < 3; ++k) h.fext[k] = c->fext[k];
    h.tau_p = c->tau_p;
    h.eta_p = c->eta_p;
    h.L2 = c->L2;
    h.kappa = c->kappa;
    h.phase = c->phase;
    h.fd_on = c->fd_on;
    h.have_prev = c->have_prev;
    h.precision = c->cfg.precision;
    h.coupling = c->coupling;
    h.collision = c->collision;
    h.chol = c->chol;
    h.rho_ref[0] = c->rho_ref[0];
    h.rho_ref[1] = c->rho_ref[1];
    h.steps = c->steps;
    VEFD_CUDA(c, cudaMemcpyAsync(&h.status, c->status, sizeof(unsigned), cudaMemcpyDeviceToHost, c->stream));
    const size_t npb = (size_t)c->cfg.ncomp * (c->Q - 1) * c->N * c->psize, nc = (size_t)c->NC * c->N;
    const size_t nrb = (size_t)c->cfg.ncomp * c->N * 4;
    std::vector<char> buf(npb + nrb + 2 * nc * 4);
    VEFD_CUDA(c, cudaMemcpyAsync(buf.data(), c->f[c->cur], npb, cudaMemcpyDeviceToHost, c->stream));
    VEFD_CUDA(c, cudaMemcpyAsync(buf.data() + npb, c->frest, nrb, cudaMemcpyDeviceToHost, c->stream));
    VEFD_CUDA(c, cudaMemcpyAsync(buf.data() + npb + nrb, c->C[c->ccur], nc * 4, cudaMemcpyDeviceToHost, c->stream));
    VEFD_CUDA(c, cudaMemcpyAsync(buf.data() + npb + nrb + nc * 4, c->R, nc * 4, cudaMemcpyDeviceToHost, c->stream));
    VEFD_CUDA(c, cudaStreamSynchronize(c->stream));
    FILE* fh = fopen(path, "wb");
    if (!fh) return fail(c, VEFD_ERR_ARG, "cannot open %s for writing", path);
    bool ok = fwrite(&h, sizeof h, 1, fh) == 1 && fwrite(buf.data(), 1, buf.size(), fh) == buf.size();
    ok = (fclose(fh) == 0) && ok;
    return ok ? VEFD_OK : fail(c, VEFD_ERR_ARG, "short write to %s", path);
}

vefd_status vefd_restore(vefd_ctx* c, const char* path) {
    Range range("vefd_restore");
    if (!c || !path) return fail(c, VEFD_ERR_ARG, "NULL argument");
    if (!c->mem) return fail(c, VEFD_ERR_STATE, "device memory is not bound");
    FILE* fh = fopen(path, "rb");
    if (!fh) return fail(c, VEFD_ERR_ARG, "cannot open %s", path);
    CkptHeader h;
    const size_t npb = (size_t)c->cfg.ncomp * (c->Q - 1) * c->N * c->psize, nc = (size_t)c->NC * c->N;
    const size_t nrb = (size_t)c->cfg.ncomp * c->N * 4;
    std::vector<char> buf(npb + nrb + 2 * nc * 4);
    bool ok = fread(&h, sizeof h, 1, fh) == 1;
    ok = ok && memcmp(h.magic, kMagic, 8) == 0 && h.version == 4 && h.precision == c->cfg.precision;
    ok = ok && h.lattice == c->cfg.lattice && h.nx == c->cfg.nx && h.ny == c->cfg.ny && h.nz == c->cfg.nz &&
         h.ncomp == c->cfg.ncomp && h.walls == c->cfg.walls;
    ok = ok && fread(buf.data(), 1, buf.size(), fh) == buf.size();
    fclose(fh);
    if (!ok) return fail(c, VEFD_ERR_ARG, "%s is not a checkpoint of this lattice", path);
    c->cfg.G = h.G;
    c->cfg.eta_A = h.eta_A;
    c->cfg.eta_B = h.eta_B;
    c->cfg.delta = h.delta;
    c->u_wall = h.u_wall;
    for (int k = 0; k < 3; ++k) c->fext[k] = h.fext[k];
    c->tau_p = h.tau_p;
    c->eta_p = h.eta_p;
    c->L2 = h.L2;
    c->kappa = h.kappa;
    c->phase = h.phase;
    c->fd_on = h.fd_on;
    c->coupling = h.coupling;
    c->collision = h.collision;
    c->chol = h.chol;
    c->have_prev = h.have_prev;
    c->rho_ref[0] = h.rho_ref[0];
    c->rho_ref[1] = h.rho_ref[1];
    c->steps = h.steps;
    c->cur = 0;
    c->ccur = 0;
    VEFD_CUDA(c, cudaMemcpyAsync(c->f[0], buf.data(), npb, cudaMemcpyHostToDevice, c->stream));
    VEFD_CUDA(c, cudaMemcpyAsync(c->frest, buf.data() + npb, nrb, cudaMemcpyHostToDevice, c->stream));
    VEFD_CUDA(c, cudaMemcpyAsync(c->C[0], buf.data() + npb + nrb, nc * 4, cudaMemcpyHostToDevice, c->stream));
    VEFD_CUDA(c, cudaMemcpyAsync(c->R, buf.data() + npb + nrb + nc * 4, nc * 4, cudaMemcpyHostToDevice, c->stream));
    VEFD_CUDA(c, cudaMemcpyAsync(c->status, &h.status, sizeof(unsigned), cudaMemcpyHostToDevice, c->stream));
    VEFD_CUDA(c, cudaStreamSynchronize(c->stream));
    c->initialised = 1;
    c->drho_valid = false;
    return VEFD_OK;
}


// ---- kernel configuration and autotuning ------------------------------------

vefd_status vefd_set_kernel_config(vefd_ctx* c, int lattice_tile, int post_mode) {
    if (!c) return VEFD_ERR_ARG;
    if (lattice_tile < 0 || lattice_tile > 5) return fail(c, VEFD_ERR_ARG, "lattice_tile must be in 0..5");
    if (post_mode < 0 || post_mode > 3) return fail(c, VEFD_ERR_ARG, "post_mode must be 0, 1, 2 or 3");
    c->lat_tile = lattice_tile;
    c->post_mode = post_mode;
    if (c->mem) build_tensor_maps(c);
    return VEFD_OK;
}

vefd_status vefd_get_kernel_config(const vefd_ctx* c, int* lattice_tile, int* post_mode) {
    if (!c || !lattice_tile || !post_mode) return VEFD_ERR_ARG;
    *lattice_tile = c->tma_ok ? c->lat_tile : -1;
    *post_mode = c->fused_ok ? 0 : (c->parts_ok ? 3 : (c->zm_ok ? 2 : (c->tma_ok ? 1 : -1)));
    return VEFD_OK;
}

vefd_status vefd_autotune(vefd_ctx* c, int steps, double* times_ms) {
    Range range("vefd_autotune");
    if (!c || steps < 1) return fail(c, VEFD_ERR_ARG, "steps must be >= 1");
    if (!c->mem) return fail(c, VEFD_ERR_STATE, "device memory is not bound");
    if (times_ms)
        for (int k = 0; k < 18; ++k) times_ms[k] = -1.0;
    // scratch lattice of the same shape and parameters, so the context's own
    // state is not advanced
    vefd_config cfg = c->cfg;
    cfg.external_memory = 0;
    vefd_ctx* t = nullptr;
    vefd_status st = vefd_create(&cfg, c->stream, &t);
    if (st != VEFD_OK) return fail(c, st, "autotune: cannot create the scratch lattice");
    t->slabs = 0;  // the kernels are timed one launch pair at a time
    t->u_wall = c->u_wall;
    for (int k = 0; k < 3; ++k) t->fext[k] = c->fext[k];
    t->tau_p = c->tau_p;
    t->eta_p = c->eta_p;
    t->L2 = c->L2;
    t->kappa = c->kappa;
    t->phase = c->phase;
    t->fd_on = c->fd_on;
    t->coupling = c->coupling;
    t->collision = c->collision;
    t->chol = c->chol;
    if (cfg.ncomp == 2)
        st = vefd_init_droplet(t, 0.5 * (cfg.nx - 1), 0.5 * (cfg.ny - 1), 0.5 * (cfg.nz - 1),
                               0.25 * std::min(cfg.nx, std::min(cfg.ny, cfg.lattice == VEFD_D3Q19 ? cfg.nz : cfg.ny)),
                               2.0, 0.1, 5.0, 1, 1e-3);
    else {
        std::vector<float> one((size_t)t->N, 1.0f);
        st = vefd_init_fields(t, one.data(), nullptr, nullptr, nullptr, 0);
    }
    if (st == VEFD_OK) st = vefd_step(t, 2);
    double best = 1e300;
    int best_tile = c->lat_tile, best_post = c->post_mode;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (st == VEFD_OK && (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) st = VEFD_ERR_CUDA;
    for (int pm = 0; pm < 3 && st == VEFD_OK; ++pm)
        for (int tile = 0; tile < 6 && st == VEFD_OK; ++tile) {
            if (!pop_tile_eligible(cfg.lattice, cfg.precision, cfg.nx, cfg.ny, cfg.nz, tile)) continue;
            if (pm != 1 && !post_zm_eligible(cfg.lattice, cfg.nx, cfg.ny)) continue;
            vefd_set_kernel_config(t, tile, pm);
            if (!t->tma_ok) continue;
            if (pm == 0 && (!t->fused_ok || tile != 0)) continue;  // the column march has its own tile
            st = vefd_step(t, 2);  // warm the configuration
            if (st != VEFD_OK) break;
            cudaEventRecord(e0, t->stream);
            st = vefd_step(t, steps);
            cudaEventRecord(e1, t->stream);
            if (st != VEFD_OK || cudaEventSynchronize(e1) != cudaSuccess) {
                st = st != VEFD_OK ? st : VEFD_ERR_CUDA;
                break;
            }
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (times_ms) times_ms[pm * 6 + tile] = ms;
            if (ms < best) {
                best = ms;
                best_tile = tile;
                best_post = pm;
            }
        }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    uint32_t bits = 0;
    if (st == VEFD_OK && vefd_get_status(t, &bits) != VEFD_OK) st = VEFD_ERR_UNSTABLE;
    if (st != VEFD_OK) {
        const std::string why = vefd_last_error(t);
        vefd_destroy(t);
        return fail(c, st, "autotune failed: %s", why.c_str());
    }
    vefd_destroy(t);
    return vefd_set_kernel_config(c, best_tile, best_post);
}

// ---- ensembles --------------------------------------------------------------

}  // extern "C"

struct vefd_ensemble {
    std::vector<vefd_ctx*> members;
    std::vector<cudaStream_t> branch;  // one capture/eager branch per member
    std::vector<cudaEvent_t> join;
    cudaStream_t user = nullptr;       // caller's stream
    cudaStream_t main = nullptr;       // capture origin and graph launch stream
    cudaEvent_t fork = nullptr, done = nullptr;
    int64_t chunk = 0;                 // steps per graph launch
    cudaGraphExec_t exec = nullptr;
    std::vector<std::vector<double>> key;  // member state the graph was captured for
    std::string err;
    // batched launches: one lattice kernel and one densities/FENE-P pass per
    // step over the tiles of all members, from a device table of members
    int batched_pref = 1;       // use them when the members allow
    int post_seg = 0;           // z-segment of the batched densities pass: 0 automatic, else planes
    int tile = 0;               // batched lattice tiles: 0 32 x 4 x 2, 1 32 x 8 x 1
    bool batched = false;       // the captured graph uses them
    std::vector<EnsMember> table;
    std::vector<int> start;     // lattice tiles then z-march columns: first item of each member
    EnsMember* d_table = nullptr;
    int* d_start = nullptr;
    size_t d_cap = 0;           // members the device table holds
    // members split into contiguous groups of about equal node count; each
    // group's launches form one graph branch, so groups overlap like the
    // per-member branches do (start[] is relative to the group's first member)
    int groups = 0;             // 0: automatic
    std::vector<int> gbeg;      // first member of each group, then the member count
    std::vector<int> glat, gpost;  // lattice tiles and z-march columns of each group
};

namespace {

vefd_status ens_fail(vefd_ensemble* e, vefd_status st, const std::string& msg) {
    if (e) e->err = msg;
    return st;
}

std::vector<double> ens_key(const vefd_ctx* m) { return state_key(m); }

// Members can share batched launches when they agree on everything the
// kernels are specialised for and each takes the 32 x 4 x 2 staged lattice
// tile and the separate z-marching densities/FENE-P pass.
bool ens_batchable(const vefd_ensemble* e) {
    const vefd_ctx* a = e->members[0];
    for (const vefd_ctx* m : e->members) {
        if (m->cfg.lattice != VEFD_D3Q19 || m->cfg.ncomp != a->cfg.ncomp || m->cfg.precision != a->cfg.precision ||
            m->collision != a->collision || m->fd_on != a->fd_on || m->pdl != a->pdl)
            return false;
        if (!m->tma_ok || !m->zm_ok || m->fused_ok) return false;
    }
    return true;
}

constexpr int kEnsTuneSlots = 7;  // configurations vefd_ensemble_autotune times

// z-segment length of the batched z-march pass: fewest (waves x planes per
// block), counting two planes of ring prologue per block.
int ens_post_segment(const vefd_ensemble* e, int sms) {
    int maxnz = 1;
    for (const vefd_ctx* m : e->members) maxnz = std::max(maxnz, m->cfg.nz);
    const long long slots = 2LL * sms;  // two blocks per SM
    int best = maxnz;
    long long best_cost = -1;
    for (int zs = 1; zs <= maxnz; ++zs) {
        long long items = 0;
        for (const vefd_ctx* m : e->members) {
            const int z = std::min(zs, m->cfg.nz);
            items += (long long)(m->cfg.nx / 32) * (m->cfg.ny / 8) * ((m->cfg.nz + z - 1) / z);
        }
        const long long cost = ((items + slots - 1) / slots) * (zs + 2);
        if (best_cost < 0 || cost < best_cost) {
            best_cost = cost;
            best = zs;
        }
    }
    return best;
}

// Builds and uploads the member table (both ping-pong parities of every
// member) for the batched launches; the upload is ordered on e->main after
// every earlier replay that reads the old table.
vefd_status ens_build_table(vefd_ensemble* e) {
    const size_t n = e->members.size();
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 152;
    const int zs = e->post_seg > 0 ? e->post_seg : ens_post_segment(e, sms);
    e->table.assign(n, EnsMember{});
    e->start.assign(2 * n, 0);
    // groups: contiguous members, split at equal shares of the total nodes
    int G = e->groups > 0 ? e->groups : 4;
    G = std::max(1, std::min(G, (int)n));
    long long total = 0;
    for (const vefd_ctx* m : e->members) total += m->N;
    e->gbeg.assign(1, 0);
    {
        long long acc = 0;
        for (size_t k = 0; k < n; ++k) {
            acc += e->members[k]->N;
            const int g = (int)e->gbeg.size();  // groups opened so far
            if (k + 1 < n && g < G && acc * G >= total * g) e->gbeg.push_back((int)k + 1);
        }
        e->gbeg.push_back((int)n);
    }
    const int ng = (int)e->gbeg.size() - 1;
    e->glat.assign(ng, 0);
    e->gpost.assign(ng, 0);
    long long lat = 0, post = 0, lat_max = 0, post_max = 0;
    int grp = 0;
    for (size_t k = 0; k < n; ++k) {
        if ((int)k == e->gbeg[grp + 1]) {
            ++grp;
            lat = 0;
            post = 0;
        }
        vefd_ctx* m = e->members[k];
        EnsMember& M = e->table[k];
        M.p = params_of(m);
        M.cur0 = m->cur;
        for (int j = 0; j < 2; ++j) {
            M.tm_lat[j] = e->tile == 1 ? m->tmap_zm[j] : m->tmap_post[j];  // box of the lattice tile
            M.tm_post[j] = m->tmap_zm[j];                                    // box 32 x 8 x 1
        }
        for (int par = 0; par < 2; ++par) {
            const int cur = m->cur ^ par, ccur = m->ccur ^ (m->fd_on ? par : 0);
            StepBufs b = bufs_of(m);
            b.fin = m->f[cur];
            b.fout = m->f[1 - cur];
            b.Cin = m->C[ccur];
            b.Cout = m->C[1 - ccur];
            M.b[par] = b;
        }
        const int tby = e->tile == 1 ? 8 : 4, tbz = e->tile == 1 ? 1 : 2;
        M.ntx = (m->cfg.nx + 31) / 32;
        M.nty = (m->cfg.ny + tby - 1) / tby;
        M.ntz = (m->cfg.nz + tbz - 1) / tbz;
        M.ncx = m->cfg.nx / 32;
        M.ncy = m->cfg.ny / 8;
        M.zs = std::min(zs, m->cfg.nz);
        M.nseg = (m->cfg.nz + M.zs - 1) / M.zs;
        e->start[k] = (int)lat;
        e->start[n + k] = (int)post;
        lat += (long long)M.ntx * M.nty * M.ntz;
        post += (long long)M.ncx * M.ncy * M.nseg;
        lat_max = std::max(lat_max, lat);
        post_max = std::max(post_max, post);
        e->glat[grp] = (int)std::min(lat, 0x7fffffffLL);
        e->gpost[grp] = (int)std::min(post, 0x7fffffffLL);
    }
    if (lat_max > 0x7fffffffLL || post_max > 0x7fffffffLL)
        return ens_fail(e, VEFD_ERR_ARG, "ensemble too large for one launch");
    if (e->d_cap < n) {
        if (e->main) cudaStreamSynchronize(e->main);
        if (e->d_table) cudaFree(e->d_table);
        if (e->d_start) cudaFree(e->d_start);
        e->d_table = nullptr;
        e->d_start = nullptr;
        e->d_cap = 0;
        if (cudaMalloc((void**)&e->d_table, n * sizeof(EnsMember)) != cudaSuccess ||
            cudaMalloc((void**)&e->d_start, 2 * n * sizeof(int)) != cudaSuccess)
            return ens_fail(e, VEFD_ERR_CUDA, "cannot allocate the member table");
        e->d_cap = n;
    }
    if (cudaMemcpyAsync(e->d_table, e->table.data(), n * sizeof(EnsMember), cudaMemcpyHostToDevice, e->main) !=
            cudaSuccess ||
        cudaMemcpyAsync(e->d_start, e->start.data(), 2 * n * sizeof(int), cudaMemcpyHostToDevice, e->main) !=
            cudaSuccess ||
        cudaStreamSynchronize(e->main) != cudaSuccess)
        return ens_fail(e, VEFD_ERR_CUDA, "cannot upload the member table");
    return VEFD_OK;
}

// Captures `chunk` steps of all members as two batched launches per step.
vefd_status ens_capture_batched(vefd_ensemble* e, int64_t chunk) {
    vefd_status st = ens_build_table(e);
    if (st != VEFD_OK) return st;
    const vefd_ctx* a = e->members[0];
    const int nm = (int)e->members.size();
    const int nc = a->cfg.ncomp, prec = a->cfg.precision;
    const bool fd = a->fd_on != 0, pdl = a->pdl;
    if (cudaStreamBeginCapture(e->main, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return ens_fail(e, VEFD_ERR_CUDA, "cannot begin capture");
    cudaError_t ce = cudaEventRecord(e->fork, e->main);
    const int ng = (int)e->gbeg.size() - 1;
    for (int g = 0; g < ng && ce == cudaSuccess; ++g) {
        const int m0 = e->gbeg[g], gm = e->gbeg[g + 1] - m0;
        cudaStream_t s = e->branch[g];
        ce = cudaStreamWaitEvent(s, e->fork, 0);
        for (int64_t k = 0; k < chunk && ce == cudaSuccess; ++k) {
            const int par = (int)(k & 1);
            ce = launch_lattice_batch(nc, prec, a->collision, e->tile, e->d_table + m0, e->d_start + m0, gm,
                                      e->glat[g], par, pdl, s);
            if (ce == cudaSuccess)
                ce = launch_post_batch(nc, prec, fd, e->d_table + m0, e->d_start + nm + m0, gm, e->gpost[g], par, pdl,
                                       s);
        }
        if (ce == cudaSuccess) ce = cudaEventRecord(e->join[g], s);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(e->main, e->join[g], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ce2 = cudaStreamEndCapture(e->main, &graph);
    if (ce != cudaSuccess || ce2 != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return ens_fail(e, VEFD_ERR_CUDA, std::string("batched graph capture failed: ") +
                                              cudaGetErrorString(ce != cudaSuccess ? ce : ce2));
    }
    ce = cudaGraphInstantiate(&e->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
        e->exec = nullptr;
        return ens_fail(e, VEFD_ERR_CUDA, "graph instantiation failed");
    }
    e->batched = true;
    // upload now (in stream order), so that the first replay only launches
    if (cudaGraphUpload(e->exec, e->main) != cudaSuccess) return ens_fail(e, VEFD_ERR_CUDA, "graph upload failed");
    return VEFD_OK;
}

// A member is steady when its next step is the plain AB2 step with current
// densities (not the Euler start or the densities-on-demand pass).
bool ens_steady(const vefd_ctx* m) { return steady_state(m); }

// `target` waits for the caller's stream and every member's own stream.
cudaError_t ens_wait_inputs(vefd_ensemble* e, cudaStream_t target) {
    cudaError_t ce = cudaEventRecord(e->fork, e->user);
    if (ce == cudaSuccess) ce = cudaStreamWaitEvent(target, e->fork, 0);
    for (size_t k = 0; k < e->members.size() && ce == cudaSuccess; ++k) {
        cudaStream_t ms = e->members[k]->stream;
        if (ms == e->user) continue;
        ce = cudaEventRecord(e->join[k], ms);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(target, e->join[k], 0);
    }
    return ce;
}

// The caller's stream and every member's own stream wait for `ev`.
cudaError_t ens_release(vefd_ensemble* e, cudaEvent_t ev) {
    cudaError_t ce = cudaStreamWaitEvent(e->user, ev, 0);
    for (size_t k = 0; k < e->members.size() && ce == cudaSuccess; ++k)
        if (e->members[k]->stream != e->user) ce = cudaStreamWaitEvent(e->members[k]->stream, ev, 0);
    return ce;
}

// n eager steps of every member, each on its own branch.
vefd_status ens_eager(vefd_ensemble* e, int64_t n) {
    if (n <= 0) return VEFD_OK;
    if (ens_wait_inputs(e, e->main) != cudaSuccess || cudaEventRecord(e->fork, e->main) != cudaSuccess)
        return ens_fail(e, VEFD_ERR_CUDA, "ordering after the inputs failed");
    for (size_t k = 0; k < e->members.size(); ++k) {
        vefd_ctx* m = e->members[k];
        const cudaStream_t own = m->stream;
        if (cudaStreamWaitEvent(e->branch[k], e->fork, 0) != cudaSuccess)
            return ens_fail(e, VEFD_ERR_CUDA, "branch ordering failed");
        m->stream = e->branch[k];
        const vefd_status st = vefd_step(m, n);
        m->stream = own;
        if (st != VEFD_OK) return ens_fail(e, st, std::string("member step failed: ") + m->err);
        if (cudaEventRecord(e->join[k], e->branch[k]) != cudaSuccess ||
            cudaStreamWaitEvent(e->main, e->join[k], 0) != cudaSuccess)
            return ens_fail(e, VEFD_ERR_CUDA, "branch join failed");
    }
    if (cudaEventRecord(e->done, e->main) != cudaSuccess || ens_release(e, e->done) != cudaSuccess)
        return ens_fail(e, VEFD_ERR_CUDA, "ordering before the caller failed");
    return VEFD_OK;
}

// Captures `chunk` steps of every member, one branch each, into e->exec.
vefd_status ens_capture(vefd_ensemble* e, int64_t chunk) {
    const size_t n = e->members.size();
    std::vector<int> cur(n), ccur(n), hp(n);
    std::vector<int64_t> steps(n);
    std::vector<cudaStream_t> own(n);
    std::vector<bool> prof(n);
    std::vector<float*> dr(n), dra(n);
    for (size_t k = 0; k < n; ++k) {
        vefd_ctx* m = e->members[k];
        dr[k] = m->drho;
        dra[k] = m->drho_alt;
        cur[k] = m->cur;
        ccur[k] = m->ccur;
        hp[k] = m->have_prev;
        steps[k] = m->steps;
        own[k] = m->stream;
        prof[k] = m->prof_on;
    }
    if (cudaStreamBeginCapture(e->main, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
        return ens_fail(e, VEFD_ERR_CUDA, "cannot begin capture");
    vefd_status st = VEFD_OK;
    std::string why;
    cudaError_t ce = cudaEventRecord(e->fork, e->main);
    for (size_t k = 0; k < n && ce == cudaSuccess && st == VEFD_OK; ++k) {
        vefd_ctx* m = e->members[k];
        ce = cudaStreamWaitEvent(e->branch[k], e->fork, 0);
        if (ce != cudaSuccess) break;
        m->stream = e->branch[k];
        m->prof_on = false;
        // record the member's launch pairs in its branch, not a nested launch
        // of its own step graph
        const int slabs = m->slabs;
        m->slabs = 0;
        st = vefd_step(m, chunk);
        m->slabs = slabs;
        if (st != VEFD_OK) why = m->err;
        if (st == VEFD_OK) ce = cudaEventRecord(e->join[k], e->branch[k]);
        if (st == VEFD_OK && ce == cudaSuccess) ce = cudaStreamWaitEvent(e->main, e->join[k], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t ce2 = cudaStreamEndCapture(e->main, &graph);
    // capture only recorded the launches: restore the members' host state
    for (size_t k = 0; k < n; ++k) {
        vefd_ctx* m = e->members[k];
        m->cur = cur[k];
        m->ccur = ccur[k];
        m->have_prev = hp[k];
        m->steps = steps[k];
        m->stream = own[k];
        m->prof_on = prof[k];
        m->drho = dr[k];
        m->drho_alt = dra[k];
    }
    if (st != VEFD_OK || ce != cudaSuccess || ce2 != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return ens_fail(e, st != VEFD_OK ? st : VEFD_ERR_CUDA, "graph capture failed: " + why);
    }
    ce = cudaGraphInstantiate(&e->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ce != cudaSuccess) {
        e->exec = nullptr;
        return ens_fail(e, VEFD_ERR_CUDA, "graph instantiation failed");
    }
    e->batched = false;
    // upload now (in stream order), so that the first replay only launches
    if (cudaGraphUpload(e->exec, e->main) != cudaSuccess) return ens_fail(e, VEFD_ERR_CUDA, "graph upload failed");
    return VEFD_OK;
}

}  // namespace

extern "C" {

vefd_status vefd_ensemble_create(vefd_ctx* const* members, int n, void* stream, vefd_ensemble** out) {
    if (!members || n < 1 || !out) return VEFD_ERR_ARG;
    *out = nullptr;
    for (int k = 0; k < n; ++k) {
        if (!members[k]) return VEFD_ERR_ARG;
        for (int j = 0; j < k; ++j)
            if (members[j] == members[k]) return fail(members[k], VEFD_ERR_ARG, "a lattice appears twice in the ensemble");
        if (need_ready(members[k]) != VEFD_OK) return VEFD_ERR_STATE;
    }
    vefd_ensemble* e = new (std::nothrow) vefd_ensemble();
    if (!e) return VEFD_ERR_ARG;
    e->members.assign(members, members + n);
    e->user = (cudaStream_t)stream;
    e->branch.assign(n, nullptr);
    e->join.assign(n, nullptr);
    bool ok = cudaStreamCreateWithFlags(&e->main, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&e->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&e->done, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < n && ok; ++k)
        ok = cudaStreamCreateWithFlags(&e->branch[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&e->join[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        vefd_ensemble_destroy(e);
        return VEFD_ERR_CUDA;
    }
    *out = e;
    return VEFD_OK;
}

void vefd_ensemble_destroy(vefd_ensemble* e) {
    if (!e) return;
    if (e->main) cudaStreamSynchronize(e->main);
    for (cudaStream_t s : e->branch)
        if (s) cudaStreamSynchronize(s);
    if (e->exec) cudaGraphExecDestroy(e->exec);
    if (e->d_table) cudaFree(e->d_table);
    if (e->d_start) cudaFree(e->d_start);
    for (cudaStream_t s : e->branch)
        if (s) cudaStreamDestroy(s);
    for (cudaEvent_t v : e->join)
        if (v) cudaEventDestroy(v);
    if (e->fork) cudaEventDestroy(e->fork);
    if (e->done) cudaEventDestroy(e->done);
    if (e->main) cudaStreamDestroy(e->main);
    delete e;
}

vefd_status vefd_ensemble_step(vefd_ensemble* e, int64_t nsteps, int64_t chunk) {
    Range range("vefd_ensemble_step");
    if (!e) return VEFD_ERR_ARG;
    if (nsteps < 0) return ens_fail(e, VEFD_ERR_ARG, "nsteps must be >= 0");
    if (chunk < 2 || (chunk & 1)) return ens_fail(e, VEFD_ERR_ARG, "chunk must be even and >= 2");
    for (vefd_ctx* m : e->members)
        if (need_ready(m) != VEFD_OK) return ens_fail(e, VEFD_ERR_STATE, "a member is not initialised");
    if (nsteps == 0) return VEFD_OK;
    // every captured step must be the steady AB2 step with current densities
    bool steady = true;
    for (vefd_ctx* m : e->members) steady = steady && ens_steady(m);
    if (!steady) {
        const vefd_status st = ens_eager(e, 1);
        if (st != VEFD_OK) return st;
        nsteps -= 1;
    }
    const int64_t full = nsteps / chunk;
    if (full > 0) {
        bool stale = !e->exec || e->chunk != chunk;
        for (size_t k = 0; k < e->members.size() && !stale; ++k) stale = ens_key(e->members[k]) != e->key[k];
        if (stale) {
            if (e->exec) cudaGraphExecDestroy(e->exec);
            e->exec = nullptr;
            const vefd_status st =
                e->batched_pref && ens_batchable(e) ? ens_capture_batched(e, chunk) : ens_capture(e, chunk);
            if (st != VEFD_OK) return st;
            e->chunk = chunk;
            e->key.resize(e->members.size());
            for (size_t k = 0; k < e->members.size(); ++k) e->key[k] = ens_key(e->members[k]);
        }
        if (ens_wait_inputs(e, e->main) != cudaSuccess) return ens_fail(e, VEFD_ERR_CUDA, "ordering after the inputs failed");
        for (int64_t r = 0; r < full; ++r)
            if (cudaGraphLaunch(e->exec, e->main) != cudaSuccess) return ens_fail(e, VEFD_ERR_CUDA, "graph launch failed");
        // an even chunk leaves every ping-pong parity where it was
        for (vefd_ctx* m : e->members) m->steps += full * chunk;
        if (cudaEventRecord(e->done, e->main) != cudaSuccess || ens_release(e, e->done) != cudaSuccess)
            return ens_fail(e, VEFD_ERR_CUDA, "ordering before the caller failed");
    }
    return ens_eager(e, nsteps - full * chunk);
}

vefd_status vefd_ensemble_set_config(vefd_ensemble* e, int batched, int post_segment) {
    if (!e || (batched != 0 && batched != 1) || post_segment < 0) return VEFD_ERR_ARG;
    if (e->batched_pref != batched || e->post_seg != post_segment) {
        // the next replay re-captures; earlier replays may still be in flight
        if (e->exec) {
            cudaStreamSynchronize(e->main);
            cudaGraphExecDestroy(e->exec);
        }
        e->exec = nullptr;
        e->batched_pref = batched;
        e->post_seg = post_segment;
    }
    return VEFD_OK;
}

vefd_status vefd_ensemble_get_config(const vefd_ensemble* e, int* batched, int* post_segment) {
    if (!e || !batched || !post_segment) return VEFD_ERR_ARG;
    *batched = e->batched_pref;
    *post_segment = e->post_seg;
    return VEFD_OK;
}

vefd_status vefd_ensemble_set_tile(vefd_ensemble* e, int tile) {
    if (!e || (tile != 0 && tile != 1)) return VEFD_ERR_ARG;
    if (e->tile != tile) {
        // the next replay re-captures; earlier replays may still be in flight
        if (e->exec) {
            cudaStreamSynchronize(e->main);
            cudaGraphExecDestroy(e->exec);
        }
        e->exec = nullptr;
        e->tile = tile;
    }
    return VEFD_OK;
}

vefd_status vefd_ensemble_get_tile(const vefd_ensemble* e, int* tile) {
    if (!e || !tile) return VEFD_ERR_ARG;
    *tile = e->tile;
    return VEFD_OK;
}

vefd_status vefd_ensemble_set_groups(vefd_ensemble* e, int groups) {
    if (!e || groups < 0 || groups > 64) return VEFD_ERR_ARG;
    if (e->groups != groups) {
        // the next replay re-captures; earlier replays may still be in flight
        if (e->exec) {
            cudaStreamSynchronize(e->main);
            cudaGraphExecDestroy(e->exec);
        }
        e->exec = nullptr;
        e->groups = groups;
    }
    return VEFD_OK;
}

vefd_status vefd_ensemble_get_groups(const vefd_ensemble* e, int* groups) {
    if (!e || !groups) return VEFD_ERR_ARG;
    *groups = e->groups;
    return VEFD_OK;
}

vefd_status vefd_ensemble_set_batched(vefd_ensemble* e, int on) {
    if (!e) return VEFD_ERR_ARG;
    return vefd_ensemble_set_config(e, on, e->post_seg);
}

vefd_status vefd_ensemble_autotune(vefd_ensemble* e, int64_t steps, int64_t chunk, double* times_ms) {
    if (!e) return VEFD_ERR_ARG;
    if (chunk < 2 || (chunk & 1) || steps < chunk || steps % chunk)
        return ens_fail(e, VEFD_ERR_ARG, "steps must be a positive multiple of an even chunk");
    for (vefd_ctx* m : e->members)
        if (need_ready(m) != VEFD_OK) return ens_fail(e, VEFD_ERR_STATE, "a member is not initialised");
    // the Euler start or pending densities first, so that every timed step is a replay
    bool steady = true;
    for (vefd_ctx* m : e->members) steady = steady && ens_steady(m);
    if (!steady) {
        const vefd_status st = ens_eager(e, 1);
        if (st != VEFD_OK) return st;
    }
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 152;
    const int auto_zs = ens_post_segment(e, sms);
    // graph branches; batched with lattice tiles 32 x 4 x 2 and 32 x 8 x 1, each
    // with the automatic z-segment of the pass, twice and half as long
    const int half = std::max(1, auto_zs / 2);
    const int cand[kEnsTuneSlots][3] = {{0, 0, 0},        {1, 0, 0}, {1, 2 * auto_zs, 0}, {1, half, 0},
                                        {1, 0, 1},        {1, 2 * auto_zs, 1}, {1, half, 1}};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return ens_fail(e, VEFD_ERR_CUDA, "cannot create timing events");
    }
    const int keep_b = e->batched_pref, keep_s = e->post_seg, keep_t = e->tile;
    vefd_status st = VEFD_OK;
    double best = 1e300;
    int best_k = -1;
    for (int k = 0; k < kEnsTuneSlots && st == VEFD_OK; ++k) {
        if (times_ms) times_ms[k] = -1.0;
        st = vefd_ensemble_set_config(e, cand[k][0], cand[k][1]);
        if (st == VEFD_OK) st = vefd_ensemble_set_tile(e, cand[k][2]);
        // one untimed replay, which captures the graph
        if (st == VEFD_OK) st = vefd_ensemble_step(e, chunk, chunk);
        if (st != VEFD_OK) break;
        if (cand[k][0] == 1 && !e->batched) continue;  // the members do not allow batched launches
        if (cudaEventRecord(e0, e->main) != cudaSuccess) st = VEFD_ERR_CUDA;
        if (st == VEFD_OK) st = vefd_ensemble_step(e, steps, chunk);
        if (st == VEFD_OK && (cudaEventRecord(e1, e->main) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess))
            st = VEFD_ERR_CUDA;
        if (st != VEFD_OK) break;
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (times_ms) times_ms[k] = ms;
        if (ms < best) {
            best = ms;
            best_k = k;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != VEFD_OK || best_k < 0) {
        vefd_ensemble_set_config(e, keep_b, keep_s);
        vefd_ensemble_set_tile(e, keep_t);
        return st != VEFD_OK ? st : ens_fail(e, VEFD_ERR_CUDA, "no configuration was timed");
    }
    st = vefd_ensemble_set_config(e, cand[best_k][0], cand[best_k][1]);
    return st != VEFD_OK ? st : vefd_ensemble_set_tile(e, cand[best_k][2]);
}

int vefd_ensemble_is_batched(const vefd_ensemble* e) { return e && e->exec && e->batched ? 1 : 0; }

const char* vefd_ensemble_last_error(const vefd_ensemble* e) { return e ? e->err.c_str() : "NULL ensemble"; }

}  // extern "C"
