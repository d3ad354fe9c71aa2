// Tensor-core GEMM for the convolution layers of the warm-start network:
//   C[M x N] (FP32) = A[M x K] (BF16) * B[N x K]^T (BF16)  (+ C when accumulate)
// A and B are K-major (row-major with K contiguous).  Every CTA owns one
// 128 x BN tile of C; K advances in chunks of 64.  Per chunk the 128 threads
// copy the two operand tiles into shared memory in the canonical
// no-swizzle K-major layout (8-row x 16-byte core matrices), one elected
// thread issues four tcgen05.mma (M = 128, N = BN, K = 16, BF16 inputs, FP32
// accumulator in tensor memory) and commits them to an mbarrier, which every
// thread waits on (bounded) before the tiles are overwritten.  At the end the
// four warps read their 32 accumulator lanes with tcgen05.ld and store C.
// Tensor memory is allocated by warp 0 and freed on every exit path.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "vefd_nn.h"

namespace vefd_nn {
namespace {

constexpr int kBM = 128, kBK = 64, kThreads = 128;
constexpr unsigned kStatusTimeout = 1u;

__device__ __forceinline__ unsigned smem_addr(const void* p) {
    return static_cast<unsigned>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor (no swizzle): start address, leading
// (between core matrices along K) and stride (between 8-row groups) byte
// offsets, all in 16-byte units, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(unsigned addr, unsigned lbo, unsigned sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 and M >> 4 in their fields.
__host__ __device__ constexpr uint32_t instr_desc(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mbar_init1(unsigned bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Bounded wait for the phase with the given parity: at most 2^31 SM cycles
// of clock64 (about one second at 2.07 GHz) and 2^22 polls.
__device__ __forceinline__ bool mbar_wait(unsigned bar, unsigned parity) {
    const long long t0 = clock64();
    for (int it = 0; it < (1 << 22); ++it) {
        unsigned done;
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
        if (clock64() - t0 > (1LL << 31)) break;
    }
    return false;
}

// Byte offset of element (r, k) of a rows x 64 K-major tile in the core-matrix
// layout: core matrix (r / 8, k / 8) at (r / 8) * sbo + (k / 8) * lbo, its row
// r % 8 at 16 * (r % 8).
__device__ __forceinline__ unsigned tile_off(int r, int kc, unsigned lbo, unsigned sbo) {
    return (unsigned)(r >> 3) * sbo + (unsigned)kc * lbo + (unsigned)(r & 7) * 16u;
}

// Copies rows [r0, r0 + rows) x K-chunk [k0, k0 + 64) of a K-major BF16 matrix
// into a tile, zero beyond the matrix (K must be a multiple of 8).
__device__ __forceinline__ void load_tile(unsigned char* tile, const __nv_bfloat16* __restrict__ g, int ld,
                                          int nrows_total, int K, int r0, int k0, int rows, unsigned lbo,
                                          unsigned sbo) {
    const int chunks = rows * (kBK / 8);
    for (int c = threadIdx.x; c < chunks; c += kThreads) {
        const int r = c >> 3, kc = c & 7;
        const int gr = r0 + r, gk = k0 + kc * 8;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (gr < nrows_total && gk < K) v = *reinterpret_cast<const uint4*>(g + (size_t)gr * ld + gk);
        *reinterpret_cast<uint4*>(tile + tile_off(r, kc, lbo, sbo)) = v;
    }
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    k_gemm_bf16(const __nv_bfloat16* __restrict__ A, int lda, const __nv_bfloat16* __restrict__ B, int ldb,
                float* __restrict__ C, int ldc, int M, int N, int K, int accumulate, unsigned lbo, unsigned sbo,
                int desc_swap, int k_split, long long c_split_stride, unsigned* __restrict__ status) {
    static_assert(BN % 16 == 0 && BN >= 32 && BN <= 256, "tcgen05 M = 128 needs N in [16, 256], a multiple of 16");
    constexpr unsigned kTmemCols = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
    __shared__ __align__(128) unsigned char sA[kBM * kBK * 2];
    __shared__ __align__(128) unsigned char sB[BN * kBK * 2];
    __shared__ __align__(8) unsigned long long bar;
    __shared__ unsigned tmem_base;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * kBM, n0 = blockIdx.y * BN;
    // split K: block z reduces K range [kb, ke) into its own slice of C
    const int kb = blockIdx.z * k_split, ke = min(K, kb + k_split);
    C += blockIdx.z * c_split_stride;
    const unsigned bar_a = smem_addr(&bar);
    if (threadIdx.x == 0) mbar_init1(bar_a);
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const unsigned tmem = tmem_base;
    constexpr uint32_t idesc = instr_desc(kBM, BN);
    const int nk = (ke - kb + kBK - 1) / kBK;
    bool ok = true;
    int last = -1;  // last chunk whose matrix operations were committed
    for (int kt = 0; kt < nk && ok; ++kt) {
        load_tile(sA, A, lda, M, ke, m0, kb + kt * kBK, kBM, lbo, sbo);
        load_tile(sB, B, ldb, N, ke, n0, kb + kt * kBK, BN, lbo, sbo);
        // generic-proxy writes of the tiles become visible to the tensor cores
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
            for (int kk = 0; kk < kBK / 16; ++kk) {
                // K = 16 is two core matrices along K
                const unsigned dl = desc_swap ? sbo : lbo, ds = desc_swap ? lbo : sbo;
                const uint64_t ad = smem_desc(smem_addr(sA) + kk * 2 * lbo, dl, ds);
                const uint64_t bd = smem_desc(smem_addr(sB) + kk * 2 * lbo, dl, ds);
                const unsigned acc = (kt > 0 || kk > 0) ? 1u : 0u;
                asm volatile(
                    "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
                    "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
                    : "memory");
            }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar_a)
                         : "memory");
        }
        last = kt;
        const bool done = mbar_wait(bar_a, (unsigned)(kt & 1));
        ok = !__syncthreads_or(!done);
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    }
    if (ok && nk > 0) {
        // accumulator row 32 * warp + lane, 16 columns per load
        const int row = m0 + warp * 32 + lane;
        for (int c0 = 0; c0 < BN; c0 += 16) {
            uint32_t v[16];
            const unsigned taddr = tmem + ((unsigned)(warp * 32) << 16) + (unsigned)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                "%13, %14, %15}, [%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(taddr)
                : "memory");
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < M) {
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int col = n0 + c0 + j;
                    if (col < N) {
                        float* c = C + (size_t)row * ldc + col;
                        *c = accumulate ? *c + __uint_as_float(v[j]) : __uint_as_float(v[j]);
                    }
                }
            }
        }
    } else if (threadIdx.x == 0) {
        atomicOr(status, kStatusTimeout);
        // bounded: let the outstanding matrix operations finish before tensor memory is freed
        if (last >= 0) mbar_wait(bar_a, (unsigned)(last & 1));
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace
}  // namespace vefd_nn

using namespace vefd_nn;

namespace {
int launch_gemm(const void* A, int lda, const void* B, int ldb, float* C, int ldc, int M, int N, int K, int accumulate,
                unsigned lbo, unsigned sbo, int desc_swap, int k_split, long long c_split_stride, unsigned* status,
                void* stream) {
    if (!A || !B || !C || !status || M < 1 || N < 1 || K < 8) return VEFD_NN_ERR_ARG;
    if (K % 8 != 0 || lda % 8 != 0 || ldb % 8 != 0 || lda < K || ldb < K || ldc < N) return VEFD_NN_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15u) return VEFD_NN_ERR_ARG;
    if (k_split < kBK || k_split % kBK != 0) return VEFD_NN_ERR_ARG;
    const int bn = N <= 32 ? 32 : (N <= 64 ? 64 : 128);
    // the layout must keep every 16-byte core-matrix row of both tiles inside
    // its staging buffer: last row group at (rows/8 - 1) * sbo, last K block
    // at 7 * lbo (64 / 8 - 1), plus one core matrix
    if (lbo % 16 || sbo % 16 || lbo == 0 || sbo == 0) return VEFD_NN_ERR_ARG;
    if (15u * sbo + 7u * lbo + 128u > (unsigned)(kBM * kBK * 2)) return VEFD_NN_ERR_ARG;
    if ((unsigned)(bn / 8 - 1) * sbo + 7u * lbo + 128u > (unsigned)(bn * kBK * 2)) return VEFD_NN_ERR_ARG;
    const int splits = (K + k_split - 1) / k_split;
    if (splits > 65535) return VEFD_NN_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    dim3 grd((M + kBM - 1) / kBM, (N + bn - 1) / bn, splits);
    const __nv_bfloat16* a = (const __nv_bfloat16*)A;
    const __nv_bfloat16* b = (const __nv_bfloat16*)B;
    if (bn == 32)
        k_gemm_bf16<32><<<grd, kThreads, 0, s>>>(a, lda, b, ldb, C, ldc, M, N, K, accumulate, lbo, sbo, desc_swap,
                                                 k_split, c_split_stride, status);
    else if (bn == 64)
        k_gemm_bf16<64><<<grd, kThreads, 0, s>>>(a, lda, b, ldb, C, ldc, M, N, K, accumulate, lbo, sbo, desc_swap,
                                                 k_split, c_split_stride, status);
    else
        k_gemm_bf16<128><<<grd, kThreads, 0, s>>>(a, lda, b, ldb, C, ldc, M, N, K, accumulate, lbo, sbo, desc_swap,
                                                  k_split, c_split_stride, status);
    return cudaGetLastError() == cudaSuccess ? VEFD_NN_OK : VEFD_NN_ERR_CUDA;
}
}  // namespace

extern "C" int vefd_nn_gemm_bf16(const void* A, int lda, const void* B, int ldb, float* C, int ldc, int M, int N,
                                 int K, int accumulate, unsigned* status, void* stream) {
    const int ks = ((K + kBK - 1) / kBK) * kBK;
    return launch_gemm(A, lda, B, ldb, C, ldc, M, N, K, accumulate, 128u, 1024u, 0, ks < kBK ? kBK : ks, 0, status,
                       stream);
}

extern "C" int vefd_nn_gemm_bf16_splitk(const void* A, int lda, const void* B, int ldb, float* C, int ldc, int M,
                                        int N, int K, int k_split, long long c_split_stride, unsigned* status,
                                        void* stream) {
    if (c_split_stride < (long long)M * ldc) return VEFD_NN_ERR_ARG;
    return launch_gemm(A, lda, B, ldb, C, ldc, M, N, K, 0, 128u, 1024u, 0, k_split, c_split_stride, status, stream);
}

extern "C" int vefd_nn_gemm_bf16_layout(const void* A, int lda, const void* B, int ldb, float* C, int ldc, int M,
                                        int N, int K, int accumulate, unsigned lbo, unsigned sbo, int desc_swap,
                                        unsigned* status, void* stream) {
    const int ks = ((K + kBK - 1) / kBK) * kBK;
    return launch_gemm(A, lda, B, ldb, C, ldc, M, N, K, accumulate, lbo, sbo, desc_swap, ks < kBK ? kBK : ks, 0,
                       status, stream);
}
