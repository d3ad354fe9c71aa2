// Allocation-free variant of the FP64 diagnostics reduction.
//
// Some callers cannot call cudaMalloc: their device memory is owned by
// another allocator that reserves the GPU up front (a framework's caching
// pool, a co-scheduled job), or they run as a monitoring hook that must not
// trigger the device-wide synchronisation that cudaMalloc and cudaFree can
// cause.  For them, vefd_diagnostics_noalloc reduces fields the caller
// already holds on the device, using only a fixed scratch array that is part
// of this library's device image.
//
// Scratch: kNoallocRows rows of kDiagVals doubles (one row per block of the
// reduction, plus one result row), 4097 x 17 x 8 = 557,192 bytes, held by
// every GPU that loads the library until the process exits.  One block
// reduces kNodesPerBlock = 2048 nodes, so lattices of at most
// kNoallocRows * 2048 = 8,388,608 nodes are accepted; larger ones are
// rejected with VEFD_ERR_ARG.  Every row that is read was written by the same
// call, so nothing needs clearing between calls; but all calls share the one
// array, so calls that overlap on the GPU (different streams, different host
// threads) race on it.
#include <cmath>
#include <mutex>
#include <vector>

#include <cuda.h>

#include "vefd.h"
#include "vefd_internal.cuh"

namespace vefd {
namespace {

constexpr int kNoallocRows = 4096;
constexpr int kNodesPerBlock = 2048;
constexpr int kThreads = 256;

static __device__ __align__(256) double g_noalloc_scratch[(kNoallocRows + 1) * kDiagVals];

__device__ __forceinline__ double wsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__device__ __forceinline__ double wmax(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    return v;
}

// Exactly (n / d > 0) without the division, for differences and sums of FP32
// values (the quotient never underflows): a finite nonzero d keeps or flips
// the sign of n; d = +-0 gives +-inf of the sign n and d share (NaN for n = 0
// or NaN); an infinite or NaN d gives a zero or NaN quotient.
__device__ __forceinline__ bool ratio_positive(double n, double d) {
    if (d != 0.0 && isfinite(d)) return d > 0.0 ? n > 0.0 : n < 0.0;
    if (d == 0.0) return n != 0.0 && !isnan(n) && signbit(n) == signbit(d);
    return false;
}

// Same sums and maxima as the context's diagnostics kernel, from absolute
// densities: one row of partials per block of kNodesPerBlock nodes.  The
// maxima are kept of tr C and |u|^2; the host maps them to max tr C / L^2 and
// max |u| (monotone maps, so the same as mapping every node).
template <int D, int NC>
__global__ void __launch_bounds__(kThreads) k_diag_rows_abs(const float* __restrict__ rA, const float* __restrict__ rB,
                                                            const float* __restrict__ u, const float* __restrict__ Ct,
                                                            int nx, int ny, int nz, double L2, double* __restrict__ rows) {
    const long long N = (long long)nx * ny * nz;
    const int zc = nz / 2;
    double acc[kDiagVals];
#pragma unroll
    for (int k = 0; k < kDiagVals; ++k) acc[k] = 0.0;
    acc[15] = -INFINITY;
    const long long first = (long long)blockIdx.x * kNodesPerBlock;
    for (int t = threadIdx.x; t < kNodesPerBlock; t += kThreads) {
        const long long i = first + t;
        if (i >= N) break;
        // N is at most the scratch capacity (8,388,608 nodes)
        const int ii = (int)i;
        const int x = ii % nx;
        const int r = ii / nx;
        const int y = r % ny;
        const int z = r / ny;
        const double a = rA[i];
        const double b = rB ? (double)rB[i] : 0.0;
        const double rho = a + b;
        acc[0] += a;
        acc[1] += b;
        double u2 = 0.0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const double uk = u[k * N + i];
            acc[2 + k] += rho * uk;
            u2 += uk * uk;
        }
        double c[NC];
#pragma unroll
        for (int k = 0; k < NC; ++k) c[k] = Ct[k * N + i];
        const double tr = NC == 6 ? c[0] + c[3] + c[5] : c[0] + c[2] + c[3];
        const double f = (L2 - 3.0) / (L2 - tr);
        const double cyy = NC == 6 ? c[3] : c[2];
        acc[5] += f * c[1];
        acc[6] += f * (c[0] - cyy);
        acc[7] += f * tr - 3.0;
        const bool ind = rB ? ratio_positive(a - b, rho) : true;
        if (ind) {
            acc[8] += 1.0;
            if (z == zc) {
                acc[9] += 1.0;
                acc[10] += x;
                acc[11] += y;
                acc[12] += (double)x * x;
                acc[13] += (double)x * y;
                acc[14] += (double)y * y;
            }
        }
        acc[15] = fmax(acc[15], tr);
        acc[16] = fmax(acc[16], u2);
    }
    __shared__ double sh[kDiagVals][kThreads / 32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < kDiagVals; ++k) {
        const double v = k < kDiagSums ? wsum(acc[k]) : wmax(acc[k]);
        if (lane == 0) sh[k][wid] = v;
    }
    __syncthreads();
    if (threadIdx.x < kDiagVals) {
        const int k = threadIdx.x;
        double v = sh[k][0];
        for (int w = 1; w < kThreads / 32; ++w) v = k < kDiagSums ? v + sh[k][w] : fmax(v, sh[k][w]);
        rows[(long long)blockIdx.x * kDiagVals + k] = v;
    }
}

// Combines the rows into the result row kNoallocRows: one warp per value,
// lane l taking rows l, l + 32, ... in index order, then a fixed shuffle tree.
__global__ void k_diag_rows_final(double* __restrict__ rows, int nrows) {
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k >= kDiagVals) return;
    const bool sum = k < kDiagSums;
    double v = sum ? 0.0 : -INFINITY;
    for (int r = lane; r < nrows; r += 32) {
        const double t = rows[(long long)r * kDiagVals + k];
        v = sum ? v + t : fmax(v, t);
    }
    v = sum ? wsum(v) : wmax(v);
    if (lane == 0) rows[(long long)kNoallocRows * kDiagVals + k] = v;
}

std::mutex g_setup_mutex;
// Held from the first launch to the synchronisation, so that host threads
// calling at the same time take turns on the one scratch array.
std::mutex g_run_mutex;

// Scratch addresses by CUDA context.  A context's ID is unique for the life
// of the process, so a device reset (which destroys the context and, with it,
// the module holding the array) leads to a fresh lookup in the new context
// instead of a stale address.
struct ScratchEntry {
    unsigned long long ctx_id;
    double* addr;
};
std::vector<ScratchEntry> g_scratch;

using PfnCtxGetCurrent = CUresult (*)(CUcontext*);
using PfnCtxGetId = CUresult (*)(CUcontext, unsigned long long*);
PfnCtxGetCurrent g_ctx_get_current = nullptr;
PfnCtxGetId g_ctx_get_id = nullptr;

cudaError_t driver_entry_points() {
    if (g_ctx_get_current && g_ctx_get_id) return cudaSuccess;
    void* a = nullptr;
    void* b = nullptr;
    cudaDriverEntryPointQueryResult qa, qb;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) != cudaSuccess ||
        qa != cudaDriverEntryPointSuccess || !a)
        return cudaErrorNotSupported;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) != cudaSuccess ||
        qb != cudaDriverEntryPointSuccess || !b)
        return cudaErrorNotSupported;
    g_ctx_get_current = reinterpret_cast<PfnCtxGetCurrent>(a);
    g_ctx_get_id = reinterpret_cast<PfnCtxGetId>(b);
    return cudaSuccess;
}

// ID of the calling thread's current context (0 when there is none).
unsigned long long current_ctx_id() {
    CUcontext ctx = nullptr;
    unsigned long long id = 0;
    if (g_ctx_get_current(&ctx) != CUDA_SUCCESS || !ctx) return 0;
    if (g_ctx_get_id(ctx, &id) != CUDA_SUCCESS) return 0;
    return id;
}

// Device address of the scratch array in the current context.  In host code
// the array's name is only a handle, so the address is looked up with
// cudaGetSymbolAddress, once per context (which also makes the device's
// primary context current if no context is yet), and cached under the
// context's ID.
cudaError_t scratch_on_current_device(double** out) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    e = driver_entry_points();
    if (e != cudaSuccess) return e;
    unsigned long long id = current_ctx_id();
    if (id != 0)
        for (const ScratchEntry& s : g_scratch)
            if (s.ctx_id == id) {
                *out = s.addr;
                return cudaSuccess;
            }
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    id = current_ctx_id();
    if (id == 0) return cudaErrorInvalidValue;
    g_scratch.push_back(ScratchEntry{id, static_cast<double*>(p)});
    *out = static_cast<double*>(p);
    return cudaSuccess;
}

}  // namespace
}  // namespace vefd

using namespace vefd;

extern "C" vefd_status vefd_diagnostics_noalloc(int lattice, int nx, int ny, int nz, int ncomp, double L2,
                                                const float* rho_A, const float* rho_B, const float* u,
                                                const float* C, void* stream, double out[16]) {
    if (!out || !rho_A || !u || !C) return VEFD_ERR_ARG;
    if (lattice != VEFD_D2Q9 && lattice != VEFD_D3Q19) return VEFD_ERR_ARG;
    if (nx < 1 || ny < 1 || nz < 1 || (lattice == VEFD_D2Q9 && nz != 1)) return VEFD_ERR_ARG;
    if (ncomp != 1 && ncomp != 2) return VEFD_ERR_ARG;
    if (ncomp == 2 && !rho_B) return VEFD_ERR_ARG;
    if (!(L2 > 3.0)) return VEFD_ERR_ARG;
    const long long N = (long long)nx * ny * nz;
    // lattices beyond the scratch array's capacity are refused
    if (N > (long long)kNoallocRows * kNodesPerBlock) return VEFD_ERR_ARG;
    double* rows = nullptr;
    if (scratch_on_current_device(&rows) != cudaSuccess) return VEFD_ERR_CUDA;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int nblocks = (int)((N + kNodesPerBlock - 1) / kNodesPerBlock);
    const float* rB = ncomp == 2 ? rho_B : nullptr;
    double v[kDiagVals];
    std::unique_lock<std::mutex> run(g_run_mutex);
    if (lattice == VEFD_D3Q19)
        k_diag_rows_abs<3, 6><<<nblocks, kThreads, 0, s>>>(rho_A, rB, u, C, nx, ny, nz, L2, rows);
    else
        k_diag_rows_abs<2, 4><<<nblocks, kThreads, 0, s>>>(rho_A, rB, u, C, nx, ny, nz, L2, rows);
    k_diag_rows_final<<<1, kDiagVals * 32, 0, s>>>(rows, nblocks);
    if (cudaGetLastError() != cudaSuccess) return VEFD_ERR_CUDA;
    if (cudaMemcpyAsync(v, rows + (size_t)kNoallocRows * kDiagVals, sizeof v, cudaMemcpyDeviceToHost, s) !=
        cudaSuccess)
        return VEFD_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return VEFD_ERR_CUDA;
    run.unlock();
    const double n = (double)N;
    for (int k = 0; k < 16; ++k) out[k] = 0.0;
    out[0] = v[0];
    out[1] = v[1];
    out[2] = v[2];
    out[3] = v[3];
    out[4] = lattice == VEFD_D3Q19 ? v[4] : 0.0;
    out[5] = v[5] / n;
    out[6] = v[6] / n;
    // the kernel keeps max tr C and max |u|^2 (empty: -inf and 0)
    out[7] = std::fmax(0.0, v[15] / L2);
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
    out[15] = v[7] / n;
    return VEFD_OK;
}
