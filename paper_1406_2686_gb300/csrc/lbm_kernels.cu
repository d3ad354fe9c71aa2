// Instantiations of the lattice kernels for the single-relaxation-time
// collision, the initial equilibrium, the population conversions and the
// tensor maps of the staged kernels (templates in lbm_impl.cuh).
#include "lbm_impl.cuh"

namespace vefd {

namespace {

template <class PT, class L, int NCOMP>
__global__ void k_init_eq(const float* __restrict__ rhoA, const float* __restrict__ rhoB,
                          const float* __restrict__ u, PT* __restrict__ fd, float* __restrict__ frest, StepParams p) {
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
                const PT e = pop_put<PT>(L::w(a) * (d + r * (3.0f * cu + 4.5f * cu * cu - 1.5f * usq)));
                fd[(s * (L::Q - 1) + a - 1) * N + i] = e;
                moved += pop_get(e);
            }
            frest[s * N + i] = d - moved;
        }
    }
}

// Planes [plane0, plane0 + nplanes) of the population buffer (plane = s*Q + a):
// stored deviations <-> absolute FP32 populations f = deviation + w_a rho_ref_s.
template <class PT, class L>
__global__ void k_pops_convert(PT* __restrict__ pops, float* __restrict__ frest, float* __restrict__ absf, int plane0,
                               int nplanes, int to_abs, StepParams p) {
    const long long N = p.N;
    const long long total = N * nplanes;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
         e += (long long)gridDim.x * blockDim.x) {
        const int pl = plane0 + (int)(e / N);
        const long long i = e % N;
        const int s = pl / L::Q, a = pl % L::Q;
        const float sh = L::w(a) * p.rho_ref[s];
        if (a == 0) {
            if (to_abs) absf[e] = frest[s * N + i] + sh;
            else frest[s * N + i] = absf[e] - sh;
        } else {
            const long long k = (long long)(s * (L::Q - 1) + a - 1) * N + i;
            if (to_abs) absf[e] = pop_get(pops[k]) + sh;
            else pops[k] = pop_put<PT>(absf[e] - sh);
        }
    }
}

int grid_1d(long long n) {
    long long b = (n + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (int)(b < 1 ? 1 : b);
}

}  // namespace

void lattice_tile_shape(int lattice, int tile, int* bx, int* by, int* bz) {
    static const int t3[3][3] = {{32, 4, 2}, {32, 2, 4}, {32, 8, 1}};
    static const int t2[3][3] = {{32, 8, 1}, {32, 4, 1}, {32, 16, 1}};
    const int(*t)[3] = lattice == 1 ? t3 : t2;
    // tiles 3..5 are the persistent forms of tiles 0..2
    const int k = tile < 0 || tile > 5 ? 0 : tile % 3;
    *bx = t[k][0];
    *by = t[k][1];
    *bz = t[k][2];
}

bool pop_tile_eligible(int lattice, int prec, int nx, int ny, int nz, int tile) {
    int bx, by, bz;
    lattice_tile_shape(lattice, tile, &bx, &by, &bz);
    const int align = prec == kPrecFp32 ? 4 : 8;  // rows must be 16-byte multiples
    return nx % align == 0 && nx >= bx && ny >= by && nz >= bz;
}

bool make_pop_tensor_map_box(int lattice, int ncomp, int prec, int nx, int ny, int nz, const void* base, int bx,
                             int by, int bz, void* out) {
    static EncodeTiled encode = nullptr;
    if (!encode) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) !=
                cudaSuccess ||
            q != cudaDriverEntryPointSuccess || !fn)
            return false;
        encode = reinterpret_cast<EncodeTiled>(fn);
    }
    const int Q = lattice == 1 ? 19 : 9;
    const cuuint64_t dims[4] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz, (cuuint64_t)(ncomp * (Q - 1))};
    const cuuint64_t es = prec == kPrecFp32 ? 4 : 2;
    const cuuint64_t strides[3] = {(cuuint64_t)nx * es, (cuuint64_t)nx * ny * es, (cuuint64_t)nx * ny * nz * es};
    const cuuint32_t box[4] = {(cuuint32_t)bx, (cuuint32_t)by, (cuuint32_t)bz, (cuuint32_t)(ncomp * (Q - 1))};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUtensorMapDataType dt = prec == kPrecFp16   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                   : prec == kPrecBf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                       : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUresult r = encode(static_cast<CUtensorMap*>(out), dt, 4, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

bool make_pop_tensor_map(int lattice, int ncomp, int prec, int nx, int ny, int nz, const void* base, void* out) {
    return make_pop_tensor_map_box(lattice, ncomp, prec, nx, ny, nz, base, 32, lattice == 1 ? 4 : 8,
                                   lattice == 1 ? 2 : 1, out);
}

cudaError_t launch_moments(int lattice, int ncomp, const StepParams& p, const StepBufs& b, cudaStream_t s, int rev) {
    dim3 blk(32, 4, 1), grd = node_grid(p);
    VEFD_WITH_PT(p.prec, {
        const PT* fin = static_cast<const PT*>(b.fin);
        if (lattice == 1) {
            if (ncomp == 2) k_moments<PT, D3Q19, 2><<<grd, blk, 0, s>>>(fin, b.frest, b.drho, p, rev);
            else k_moments<PT, D3Q19, 1><<<grd, blk, 0, s>>>(fin, b.frest, b.drho, p, rev);
        } else {
            if (ncomp == 2) k_moments<PT, D2Q9, 2><<<grd, blk, 0, s>>>(fin, b.frest, b.drho, p, rev);
            else k_moments<PT, D2Q9, 1><<<grd, blk, 0, s>>>(fin, b.frest, b.drho, p, rev);
        }
    });
    return cudaGetLastError();
}

cudaError_t launch_lattice(int lattice, int ncomp, bool stream_pops, const StepParams& p, const StepBufs& b,
                           cudaStream_t s, const void* tensor_map, int rev, int tile, Parts parts) {
    if (stream_pops) {
        if (p.collision == 1) return launch_lattice_mrt(lattice, ncomp, p, b, s, tensor_map, rev, tile, parts);
        return launch_lattice_coll<0>(lattice, ncomp, p, b, s, tensor_map, rev, tile, parts);
    }
    if (parts.part) return cudaErrorInvalidValue;
    // macroscopic pass (moments, forces, velocity; no streaming)
    dim3 blk(32, 4, 1), grd = node_grid(p);
    VEFD_WITH_PT(p.prec, {
        if (lattice == 1) {
            if (ncomp == 2) k_lattice<PT, D3Q19, 2, false, 0><<<grd, blk, 0, s>>>(b, p, rev);
            else k_lattice<PT, D3Q19, 1, false, 0><<<grd, blk, 0, s>>>(b, p, rev);
        } else {
            if (ncomp == 2) k_lattice<PT, D2Q9, 2, false, 0><<<grd, blk, 0, s>>>(b, p, rev);
            else k_lattice<PT, D2Q9, 1, false, 0><<<grd, blk, 0, s>>>(b, p, rev);
        }
    });
    return cudaGetLastError();
}

cudaError_t launch_lattice_zm(int ncomp, const StepParams& p, const StepBufs& b, cudaStream_t s,
                              const void* tensor_map, int zs, int rev) {
    if (p.collision == 1) return launch_lattice_zm_mrt(ncomp, p, b, s, tensor_map, zs, rev);
    return launch_zm_coll<0>(ncomp, p, b, s, tensor_map, zs, rev);
}

int lattice_zm_segment(const StepParams& p) { return zm_segment_length(p); }

namespace {
__global__ void k_wait_selftest(unsigned* status, int arrive, long long cycles) {
    __shared__ __align__(8) unsigned long long bar;
    const unsigned a = smem_u32(&bar);
    if (threadIdx.x == 0) mbar_init(a);  // one arrival completes the phase
    __syncthreads();
    if (arrive && threadIdx.x == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(a) : "memory");
    const bool ok = mbar_wait_budget(a, 0u, cycles);
    if (!ok && threadIdx.x == 0) atomicOr(status, kStTimeout);
}
}  // namespace

cudaError_t launch_wait_selftest(unsigned* status, int arrive, long long cycles, cudaStream_t s) {
    k_wait_selftest<<<1, 32, 0, s>>>(status, arrive, cycles);
    return cudaGetLastError();
}

cudaError_t launch_lattice_batch(int ncomp, int prec, int coll, int tile, const EnsMember* members, const int* start,
                                 int nm, int items, int parity, bool pdl, cudaStream_t s) {
    if (coll == 1) return launch_lattice_batch_mrt(ncomp, prec, tile, members, start, nm, items, parity, pdl, s);
    return launch_lattice_batch_coll<0>(ncomp, prec, tile, members, start, nm, items, parity, pdl, s);
}

cudaError_t launch_init_equilibrium(int lattice, int ncomp, const StepParams& p, const float* rhoA,
                                    const float* rhoB, const float* u, void* fd, float* frest, cudaStream_t s) {
    const int g = grid_1d(p.N);
    VEFD_WITH_PT(p.prec, {
        PT* out = static_cast<PT*>(fd);
        if (lattice == 1) {
            if (ncomp == 2) k_init_eq<PT, D3Q19, 2><<<g, 256, 0, s>>>(rhoA, rhoB, u, out, frest, p);
            else k_init_eq<PT, D3Q19, 1><<<g, 256, 0, s>>>(rhoA, rhoB, u, out, frest, p);
        } else {
            if (ncomp == 2) k_init_eq<PT, D2Q9, 2><<<g, 256, 0, s>>>(rhoA, rhoB, u, out, frest, p);
            else k_init_eq<PT, D2Q9, 1><<<g, 256, 0, s>>>(rhoA, rhoB, u, out, frest, p);
        }
    });
    return cudaGetLastError();
}

cudaError_t launch_pops_convert(int lattice, int ncomp, const StepParams& p, void* pops, float* frest, float* absf,
                                int plane0, int nplanes, int to_absolute, cudaStream_t s) {
    (void)ncomp;
    const int g = grid_1d(p.N * nplanes);
    VEFD_WITH_PT(p.prec, {
        PT* pp = static_cast<PT*>(pops);
        if (lattice == 1)
            k_pops_convert<PT, D3Q19><<<g, 256, 0, s>>>(pp, frest, absf, plane0, nplanes, to_absolute, p);
        else k_pops_convert<PT, D2Q9><<<g, 256, 0, s>>>(pp, frest, absf, plane0, nplanes, to_absolute, p);
    });
    return cudaGetLastError();
}

}  // namespace vefd
