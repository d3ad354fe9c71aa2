// Internal declarations shared by the CUDA translation units of libvefd.
//
// Storage (all FP32, x fastest, node i = (z*NY + y)*NX + x):
//   populations  moving a >= 1: fd[(s*(Q-1) + a-1)*N + i] = f_a^s - w_a rho_ref_s  (deviation form,
//                storage type PT, ping-pong); rest a = 0: frest[s*N + i], always FP32,
//                updated in place (it does not stream) and carrying each node's mass exactly
//   densities    drho[i*ncomp + s] = rho_s - rho_ref_s        (sum of deviations; interleaved so a
//                node's densities are one 8-byte access)
//   velocity     u[k*N + i], k < D                             (Eq. equilibrium:vel)
//   conformation Ct[k*N + i] = C_k - delta_k                   (k < NC)
//   AB2 history  R[k*N + i]                                    (right-hand side of the last FD step)
//   feedback     Q[k*N + i] = (f(r_P) C - I) m(phi), k < NQ    (the stress whose divergence is the
//                polymer force; derived from C and the densities of the same time level)
// Storing deviations keeps FP32 rounding relative to the small departures
// from a uniform rest state instead of to the full populations.  The
// population deviations may also be stored in 16 bits (FP16 or BF16, type PT
// below); all arithmetic stays FP32 and C stays FP32.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <utility>
#include <stdint.h>

namespace vefd {

constexpr float kCs2 = 1.0f / 3.0f;

// D2Q9: rest, +-x, +-y, diagonals as opposite pairs; weights 4/9, 1/9, 1/36.
struct D2Q9 {
    static constexpr int Q = 9, D = 2, NC = 4, NQ = 3;  // NQ: xx xy yy of the feedback stress
    __host__ __device__ static constexpr int cx(int a) {
        return a == 1 || a == 5 || a == 7 ? 1 : (a == 2 || a == 6 || a == 8 ? -1 : 0);
    }
    __host__ __device__ static constexpr int cy(int a) {
        return a == 3 || a == 5 || a == 8 ? 1 : (a == 4 || a == 6 || a == 7 ? -1 : 0);
    }
    __host__ __device__ static constexpr int cz(int) { return 0; }
    __host__ __device__ static constexpr float w(int a) {
        return a == 0 ? 4.0f / 9.0f : (a <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f);
    }
};

// D3Q19: rest, +-x, +-y, +-z, then the twelve face diagonals as opposite
// pairs; weights 1/3, 1/18, 1/36 (Sec. 2).
struct D3Q19 {
    static constexpr int Q = 19, D = 3, NC = 6, NQ = 6;
    __host__ __device__ static constexpr int cx(int a) {
        return (a == 1 || a == 7 || a == 9 || a == 11 || a == 13) ? 1
             : (a == 2 || a == 8 || a == 10 || a == 12 || a == 14) ? -1 : 0;
    }
    __host__ __device__ static constexpr int cy(int a) {
        return (a == 3 || a == 7 || a == 10 || a == 15 || a == 17) ? 1
             : (a == 4 || a == 8 || a == 9 || a == 16 || a == 18) ? -1 : 0;
    }
    __host__ __device__ static constexpr int cz(int a) {
        return (a == 5 || a == 11 || a == 14 || a == 15 || a == 18) ? 1
             : (a == 6 || a == 12 || a == 13 || a == 16 || a == 17) ? -1 : 0;
    }
    __host__ __device__ static constexpr float w(int a) {
        return a == 0 ? 1.0f / 3.0f : (a <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
    }
};

__host__ __device__ constexpr int opposite(int a) { return a == 0 ? 0 : ((a & 1) ? a + 1 : a - 1); }

// --- population storage types: FP32, FP16 or BF16 deviations ------------------

enum { kPrecFp32 = 0, kPrecFp16 = 1, kPrecBf16 = 2 };

// Densities of node i (interleaved by node, see above).
template <int NCOMP>
__device__ __forceinline__ void dens_store(float* drho, long long i, const float d[NCOMP]) {
    if constexpr (NCOMP == 2) reinterpret_cast<float2*>(drho)[i] = make_float2(d[0], d[1]);
    else drho[i] = d[0];
}
template <int NCOMP>
__device__ __forceinline__ void dens_ldg(const float* __restrict__ drho, long long i, float d[NCOMP]) {
    if constexpr (NCOMP == 2) {
        const float2 v = __ldg(reinterpret_cast<const float2*>(drho) + i);
        d[0] = v.x;
        d[1] = v.y;
    } else {
        d[0] = __ldg(drho + i);
    }
}
// plain (coherent) read, for values this kernel also writes
template <int NCOMP>
__device__ __forceinline__ void dens_get(const float* drho, long long i, float d[NCOMP]) {
    if constexpr (NCOMP == 2) {
        const float2 v = reinterpret_cast<const float2*>(drho)[i];
        d[0] = v.x;
        d[1] = v.y;
    } else {
        d[0] = drho[i];
    }
}

// A tensor map the host copied into global memory (rather than passed as a
// kernel parameter) is made visible to the tensor-map proxy before use; the
// bulk tensor copies would otherwise be allowed to use a descriptor cached from
// earlier contents at the same address.
__device__ __forceinline__ void tensormap_acquire(const void* tm) {
    asm volatile("fence.proxy.tensormap::generic.acquire.sys [%0], 128;" ::"l"(tm) : "memory");
}

// Member of a batched ensemble that work item `item` belongs to: the last m
// with start[m] <= item (start is increasing, start[0] = 0).
__device__ __forceinline__ int batch_member(const int* __restrict__ start, int nm, int item) {
    int lo = 0, hi = nm - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (start[mid] <= item) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ float pop_load(const float* p) { return __ldg(p); }
__device__ __forceinline__ float pop_load(const __half* p) { return __half2float(__ldg(p)); }
__device__ __forceinline__ float pop_load(const __nv_bfloat16* p) { return __bfloat162float(__ldg(p)); }

// plain (non read-only-path) loads, for buffers the same kernel also writes
__device__ __forceinline__ float pop_get(float v) { return v; }
__device__ __forceinline__ float pop_get(__half v) { return __half2float(v); }
__device__ __forceinline__ float pop_get(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class PT>
__device__ __forceinline__ PT pop_put(float v);
template <>
__device__ __forceinline__ float pop_put<float>(float v) { return v; }
template <>
__device__ __forceinline__ __half pop_put<__half>(float v) { return __float2half_rn(v); }
template <>
__device__ __forceinline__ __nv_bfloat16 pop_put<__nv_bfloat16>(float v) { return __float2bfloat16_rn(v); }

// volatile shared-memory read of a staged population (keeps it out of registers)
__device__ __forceinline__ float pop_smem(const float* base, int idx) {
    return static_cast<const volatile float*>(base)[idx];
}
__device__ __forceinline__ float pop_smem(const __half* base, int idx) {
    return __half2float(__ushort_as_half(reinterpret_cast<const volatile unsigned short*>(base)[idx]));
}
__device__ __forceinline__ float pop_smem(const __nv_bfloat16* base, int idx) {
    return __bfloat162float(__ushort_as_bfloat16(reinterpret_cast<const volatile unsigned short*>(base)[idx]));
}

// Runs the statements that follow `prec` with PT bound to the population
// storage type of `prec`.
#define VEFD_WITH_PT(prec, ...)             \
    do {                                    \
        if ((prec) == kPrecFp16) {          \
            using PT = __half;              \
            __VA_ARGS__;                    \
        } else if ((prec) == kPrecBf16) {   \
            using PT = __nv_bfloat16;       \
            __VA_ARGS__;                    \
        } else {                            \
            using PT = float;               \
            __VA_ARGS__;                    \
        }                                   \
    } while (0)

// Scalars every kernel needs, passed by value.
struct StepParams {
    int nx, ny, nz;
    int walls;             // 1: walls in y; 0: periodic
    long long N;
    float G;               // Shan-Chen coupling
    float eta_A, eta_B;    // phase viscosities
    float inv_delta;       // 1 / smoothing width
    float u_wall;          // +u_wall at the lower wall
    float fext[3];         // body force density
    float inv_tau_p;       // 1 / tau_P
    float feedback;        // eta_P / tau_P
    float L2m3;            // L^2 - 3
    float kappa;           // artificial diffusivity
    int phase;             // 0: m = 1, +1: f_+, -1: f_-
    int have_prev;         // AB2 history valid
    float rho_ref[2];      // deviation reference densities
    int prec;              // population storage: kPrecFp32, kPrecFp16, kPrecBf16
    int coupling;          // polymer feedback: 0 body force div Q; 1 stress in the equilibrium
    int collision;         // 0: single relaxation time; 1: moment space with the paper's rates
    int chol;              // conformation update: 0 AB2 on C; 1 AB2 on the log-Cholesky factor of f C
    int pdl;               // launch the step's kernels with programmatic dependencies
    int ylo, yhi;          // rows [ylo, yhi) the staged lattice and z-marching launches cover
                           // (0, ny: the whole lattice; a y-slab of the pipelined step graph)
    int post_zs;           // z-segment of the z-marching pass (0: fill two blocks per SM)
};

// --- TMA staging helpers (inline PTX, sm_90 and later) -----------------------

__device__ __forceinline__ unsigned smem_u32(const void* ptr) {
    return static_cast<unsigned>(__cvta_generic_to_shared(ptr));
}

// One-shot transaction barrier: init for one arrival, made visible to the
// asynchronous proxy before any copy is issued against it.
__device__ __forceinline__ void mbar_init(unsigned bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Arrive once, announcing `bytes` of incoming copies, and issue a 4-D tiled
// bulk tensor copy of the box at (c0, c1, c2, c3) into shared memory.
__device__ __forceinline__ void tma_load_4d(unsigned dst, const void* tmap, int c0, int c1, int c2, int c3,
                                            unsigned bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(reinterpret_cast<unsigned long long>(tmap)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

// Waits for the given phase parity of the barrier for a bounded number of
// polls; returns false when the copy has not landed (the caller reports a
// timeout).
// Budget of every bounded wait: 2^31 SM cycles (about one second at the
// 2.07 GHz maximum clock), and at most 2^22 polls whatever the clock reads.
constexpr long long kWaitCycles = 1LL << 31;

__device__ __forceinline__ unsigned mbar_try_wait(unsigned bar, unsigned parity) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    return done;
}

// Waits for the phase with the given parity to complete; false when the
// budget (`cycles` of clock64, or 2^22 polls) runs out first.
__device__ __forceinline__ bool mbar_wait_budget(unsigned bar, unsigned parity, long long cycles) {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    for (int it = 0; it < (1 << 22); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if (clock64() - t0 > cycles) break;
    }
    return false;
}

__device__ __forceinline__ bool mbar_wait_bounded_parity(unsigned bar, unsigned parity) {
    return mbar_wait_budget(bar, parity, kWaitCycles);
}

__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar) { return mbar_wait_bounded_parity(bar, 0u); }

// --- programmatic dependent launch ------------------------------------------
// The two kernels of a step are launched so that the next one may start while
// the previous one drains.  pdl_wait() blocks until the preceding kernel in
// the stream has completed and its memory is visible (a no-op when the launch
// carried no programmatic dependency); pdl_trigger() lets the next kernel
// launch once every block of this one has triggered or exited.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Launches kernel<<<grid, block, smem, stream>>>(args...) with programmatic
// stream serialisation unless disabled (pdl == false).
template <class... KArgs, class... Args>
cudaError_t launch_pdl(bool pdl, void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                       Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// --- column-marching step with fused densities (D3Q19) ----------------------
// The lattice kernel k_lattice_zm walks 32 x 8 columns along z in segments of
// planes [z0, z1).  A population that moves from a source node to a
// destination node inside the same column and segment is stored by the
// destination's thread and counted in that node's partial density; every other
// population (crossing a column side or a segment end) is stored by the
// source's thread, and the densities pass adds it.  Half-way bounce-back
// returns to the node itself and always counts as inside.  `lane` and `row`
// are column-relative, before wrapping.
struct ColumnTopo {
    bool nx32;  // NX == 32: the column spans x (periodic wrap inside the warp)
    bool ny8p;  // NY == 8 and periodic in y: the column spans y
    bool nz1;   // NZ == 1: z neighbours are the plane itself
};

__device__ __forceinline__ bool zm_inner(int lane, int row, int zp, int z0, int z1, ColumnTopo t) {
    return (t.nx32 || (unsigned)lane < 32u) && (t.ny8p || (unsigned)row < 8u) && (t.nz1 || (zp >= z0 && zp < z1));
}

// Device guard bits (mirror VEFD_ST_*).
constexpr unsigned kStNan = 1u, kStTrace = 2u, kStMach = 4u, kStRho = 8u, kStTimeout = 16u, kStBounds = 32u;

// Debug builds (-DVEFD_BOUNDS_CHECK, a separate library): every neighbour
// index the step kernels compute (pushes, density and stress gathers, the
// FENE-P stencil) is checked against the lattice; an index outside [0, N)
// sets kStBounds and the access is skipped (a skipped load reads 0).  In the
// regular build the check is compiled out.
#ifdef VEFD_BOUNDS_CHECK
__device__ __forceinline__ bool idx_ok(long long j, long long N, unsigned* status) {
    if (j >= 0 && j < N) return true;
    atomicOr(status, kStBounds);
    return false;
}
#else
__device__ __forceinline__ constexpr bool idx_ok(long long, long long, unsigned*) { return true; }
#endif

// Pointers of one step.
struct StepBufs {
    const void* fin;       // populations at time n (deviation form, storage type of p.prec)
    void* fout;            // populations at time n+1
    float* frest;          // rest populations (FP32, in place: time n before the lattice kernel, n+1 after)
    float* drho;           // densities of time n
    float* drho_next;      // densities of time n+1 (column-marching step: partial, completed by the densities pass)
    float* u;              // velocity of time n (written by the lattice kernel)
    const float* Cin;      // C - I at time n
    float* Cout;           // C - I at time n+1
    float* R;              // AB2 history (in: n-1, out: n)
    unsigned* status;
    float* dbg;            // optional: g_A(3), g_B(3), F_p(3), tau(1) planes of N
    float* Q;              // feedback stress of time n (read by the lattice kernel; the
                           // densities/FD pass overwrites it with time n+1)
};

// Partial densities of time n+1 (post mode 3), passed beside StepBufs to the
// staged lattice kernel that writes them and the z-marching pass that
// completes them: 7 slots of N x NCOMP floats, interleaved by node like the
// densities; slot 0 holds what reached a node from inside its lattice tile
// (with its rest population and wall bounce-back), slots 1-6 what the
// neighbouring tile across x, y, z, xy, xz, yz pushed into it.  by, bz: the
// lattice tile's rows and planes (its width is 32).  part == nullptr: off.
struct Parts {
    float* part;
    int by, bz;
};

// One lattice of a batched ensemble step, as the batched kernels read it from
// device memory: parameters, the buffers of both ping-pong parities, the tensor
// maps of the two population buffers f[0], f[1] (lattice kernel: 32 x 4 x 2
// tiles; densities/FENE-P pass: 32 x 8 x 1 planes), the buffer parity 0 reads
// (cur0; parity q reads f[cur0 ^ q] and writes the other), and the work split
// (lattice tiles; z-marching columns and segments of zs planes).  The tensor
// maps depend on the buffers only, so rebuilding the table for the other
// parity rewrites them with the same bytes.
struct EnsMember {  // aligned as CUtensorMap
    CUtensorMap tm_lat[2];
    CUtensorMap tm_post[2];
    StepParams p;
    StepBufs b[2];
    int cur0;
    int ntx, nty, ntz;
    int ncx, ncy, nseg, zs;
};

// Launchers (return cudaGetLastError of the launch).  `rev` walks the tiles in
// reverse order, so that a kernel starts on the data its predecessor touched
// last (still in L2).
cudaError_t launch_moments(int lattice, int ncomp, const StepParams& p, const StepBufs& b, cudaStream_t s, int rev);
// tensor_map: a CUtensorMap of b.fin for the TMA-staged kernel (streaming
// steps only), or nullptr for the register-only kernel; `tile` selects the
// staged tile shape (lattice_tile_shape), and the map's box must match it.
// parts.part != nullptr (D3Q19 staged tiles 0 and 1 only): the kernel also
// writes the partial densities of time n+1 (post mode 3).
cudaError_t launch_lattice(int lattice, int ncomp, bool stream_pops, const StepParams& p, const StepBufs& b,
                           cudaStream_t s, const void* tensor_map, int rev, int tile, Parts parts = Parts{});
// The streaming launch with the moment-space collision (instantiated in its
// own translation unit); same arguments as launch_lattice.
cudaError_t launch_lattice_mrt(int lattice, int ncomp, const StepParams& p, const StepBufs& b, cudaStream_t s,
                               const void* tensor_map, int rev, int tile, Parts parts = Parts{});
// Column-marching lattice kernel with fused partial densities (D3Q19,
// NX % 32 == 0, NY % 8 == 0): reads b.fin through `tensor_map` (box 32 x 8 x 1
// x P), writes b.fout, b.frest, b.u and the partial densities into
// b.drho_next; zs is the z-segment length (the densities pass needs the same).
cudaError_t launch_lattice_zm(int ncomp, const StepParams& p, const StepBufs& b, cudaStream_t s,
                              const void* tensor_map, int zs, int rev);
int lattice_zm_segment(const StepParams& p);
cudaError_t launch_lattice_zm_mrt(int ncomp, const StepParams& p, const StepBufs& b, cudaStream_t s,
                                  const void* tensor_map, int zs, int rev);
// Batched ensemble step: one launch of the lattice kernel over the tiles of
// every member (item i belongs to the last member m with start[m] <= i), then
// one launch of the z-marching densities/FENE-P pass over their columns; all
// members share lattice D3Q19, ncomp, storage type, collision and fd_on.
// One bounded wait on an mbarrier that one thread completes (arrive != 0) or
// that nothing completes; on running out of `cycles` it sets kStTimeout.
cudaError_t launch_wait_selftest(unsigned* status, int arrive, long long cycles, cudaStream_t s);
// `tile` 0: 32 x 4 x 2 tiles, 1: 32 x 8 x 1 (the member table's tile counts and
// lattice tensor maps must be built for the same tile).
cudaError_t launch_lattice_batch(int ncomp, int prec, int coll, int tile, const EnsMember* members, const int* start,
                                 int nm, int items, int parity, bool pdl, cudaStream_t s);
cudaError_t launch_lattice_batch_mrt(int ncomp, int prec, int tile, const EnsMember* members, const int* start,
                                     int nm, int items, int parity, bool pdl, cudaStream_t s);
cudaError_t launch_post_batch(int ncomp, int prec, bool fd, const EnsMember* members, const int* start, int nm,
                              int items, int parity, bool pdl, cudaStream_t s);
// Staged tile shapes of the lattice kernel: tile 0..2 ->
// D3Q19 32x4x2, 32x2x4, 32x8x1; D2Q9 32x8x1, 32x4x1, 32x16x1.
void lattice_tile_shape(int lattice, int tile, int* bx, int* by, int* bz);
// Densities of the populations `fnew` into b.drho, when fd the FENE-P update
// b.Cin -> b.Cout with the AB2 history b.R and velocity b.u, and the feedback
// stress of the new time level into b.Q.
cudaError_t launch_post(int lattice, int ncomp, bool fd, const StepParams& p, const StepBufs& b,
                        const void* fnew, cudaStream_t s, int rev);
// With a tensor map of `fnew` (TMA-eligible shapes), the same pass stages the
// tile's populations with one bulk copy while the stencil loads are in flight.
cudaError_t launch_post_tma(int lattice, int ncomp, bool fd, const StepParams& p, const StepBufs& b,
                            const void* tensor_map_fnew, cudaStream_t s, int rev);
// D3Q19 z-marching variant of the pass (needs NX % 32 == 0 and NY % 8 == 0 and a
// tensor map of `fnew` with box 32 x 8 x 1 x P).
bool post_zm_eligible(int lattice, int nx, int ny);
// parts.part != nullptr: the densities are completed from the partial
// densities of post mode 3 (no population is read).
cudaError_t launch_post_zm(int ncomp, bool fd, const StepParams& p, const StepBufs& b, const void* tensor_map_fnew,
                           cudaStream_t s, int rev, Parts parts = Parts{});
// The same pass after k_lattice_zm: completes the partial densities in
// b.drho_next with the populations that crossed a column side or a segment
// end (segment length zs of the lattice kernel), then the FENE-P update and
// the feedback stress.
cudaError_t launch_post_zm_fused(int ncomp, bool fd, const StepParams& p, const StepBufs& b, cudaStream_t s,
                                 int zs, int rev);
// Densities of b.fin and the feedback stress of (b.fin, b.Cin): the derived
// state the lattice kernel needs, for the initial state and after writes.
cudaError_t launch_pre(int lattice, int ncomp, const StepParams& p, const StepBufs& b, cudaStream_t s);

// TMA staging of populations: lattice shapes it applies to, and the tensor
// map over one population buffer ([ncomp*Q][NZ][NY][NX] FP32) written to `out`
// (a 64-byte aligned CUtensorMap).  Returns false when the driver entry point
// is unavailable or the encoding is refused.
bool pop_tile_eligible(int lattice, int prec, int nx, int ny, int nz, int tile);
bool make_pop_tensor_map(int lattice, int ncomp, int prec, int nx, int ny, int nz, const void* base, void* out);
// Tensor map over one population buffer with an explicit box (bx, by, bz, all planes).
bool make_pop_tensor_map_box(int lattice, int ncomp, int prec, int nx, int ny, int nz, const void* base, int bx,
                             int by, int bz, void* out);

// Field conversions.
cudaError_t launch_init_equilibrium(int lattice, int ncomp, const StepParams& p, const float* rhoA,
                                    const float* rhoB, const float* u, void* fd, float* frest, cudaStream_t s);
// Planes [plane0, plane0 + nplanes) of the population buffer: stored deviations
// `pops` -> absolute FP32 `absf` (to_absolute) or back.
cudaError_t launch_pops_convert(int lattice, int ncomp, const StepParams& p, void* pops, float* frest, float* absf,
                                int plane0, int nplanes, int to_absolute, cudaStream_t s);
cudaError_t launch_tensor_shift(int lattice, const float* src, float* dst, long long N, float sign,
                                cudaStream_t s);
// which: 0 rho_A, 1 rho_B, 2 phi, 4 C, 5 sigma_P = f(r_P) C
cudaError_t launch_derived(int lattice, int ncomp, int which, const StepParams& p, const float* drho,
                           const float* Ct, float* dst, cudaStream_t s);

// Diagnostics: per-block FP64 partials then a fixed-order final reduction.
constexpr int kDiagSums = 15, kDiagMax = 2, kDiagVals = kDiagSums + kDiagMax;
// out[0..2] = FP64 sums of rho_A and rho_B (rho_B may be NULL) and the count of
// values that are not finite or negative; partial holds kDiagBlocks x 3 doubles.
cudaError_t launch_density_sums(const float* rho_A, const float* rho_B, long long N, double* partial, double* out,
                                cudaStream_t s);
constexpr int kDiagBlocks = 608;  // 4 x 152 SMs
cudaError_t launch_diagnostics(int lattice, int ncomp, const StepParams& p, const float* drho, const float* u,
                               const float* Ct, double* partial, double* out, cudaStream_t s);

}  // namespace vefd
