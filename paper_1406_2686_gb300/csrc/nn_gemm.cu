// Tensor-core GEMM for the convolution layers of the warm-start network:
//   C[M x N] (FP32) = A[M x K] (BF16) * B[N x K]^T (BF16)  (+ C when accumulate)
// A and B are K-major (row-major with K contiguous).
//
// k_gemm_tma (vefd_nn_gemm_bf16 and its split-K form): a persistent grid of at
// most one CTA per SM walks the 128 x BN tiles of C (BN = 32, 64, 128 or 256;
// split-K slices are further tiles), K in chunks of 64 through a ring of
// kStages shared-memory stages.  One thread issues the bulk tensor copies of
// both operand chunks (TMA, 128-byte swizzle, zero fill beyond the matrices)
// into a free stage; another issues the four tcgen05.mma (M = 128, N = BN,
// K = 16 each, BF16 inputs, FP32 accumulator in tensor memory) of each loaded
// stage and commits them to the stage's "empty" barrier, which frees the
// stage for the copy kStages chunks later.  Two accumulators alternate
// between tiles, so four epilogue warps read one tile's accumulator with
// tcgen05.ld and store C while the next tile's matrix operations run.
//
// k_gemm_bf16 (vefd_nn_gemm_bf16_layout only): the threads copy both tiles into
// the no-swizzle K-major core-matrix layout with plain loads, one chunk at a
// time; it exists to test the descriptor's byte offsets of that layout.
//
// Tensor memory is allocated by warp 0 and freed on every exit path; every
// wait is bounded.
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

constexpr int kStages = 4;

// Shared-memory matrix descriptor of a K-major operand tile in the 128-byte
// swizzled layout (rows of 64 BF16 = 128 bytes, 8-row atoms of 1024 bytes,
// atom-aligned): start address, leading byte offset unused (16), stride byte
// offset 1024 between 8-row groups, descriptor version 1, layout 2 (128-byte
// swizzle).  Along K the start address advances 32 bytes per 16 elements.
__device__ __forceinline__ uint64_t smem_desc_sw128(unsigned addr) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)1u << 16) | ((uint64_t)(1024u >> 4) << 32) | (1ull << 46) |
           (2ull << 61);
}

__device__ __forceinline__ void tma_load_2d(unsigned dst, const CUtensorMap* tm, int c0, int c1, unsigned bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<unsigned long long>(tm)), "r"(c0), "r"(c1), "r"(bar)
        : "memory");
}

// Persistent form: a grid of at most one CTA per SM walks the output tiles
// (tile = blockIdx.x + j * gridDim.x; split-K slices are further tiles) with
// two tensor-memory accumulators, so that the epilogue of tile j overlaps the
// main loop of tile j + 1.  Warp roles (192 threads):
//   warp 0, one thread: bulk tensor copies of both operand chunks into the
//     ring of kStages stages, each stage reused once the matrix operations of
//     the chunk kStages earlier have released it (barrier "empty");
//   warp 1, one thread: waits for each loaded stage ("full"), issues its four
//     tcgen05.mma into accumulator j % 2, commits them to the stage's "empty"
//     barrier, and after the tile's last chunk commits to "acc_full[j % 2]";
//     before the first chunk of tile j (j >= 2) it waits for "acc_empty",
//     which the epilogue arrives on once it has read that accumulator;
//   warps 2-5: the epilogue; warp w reads tensor-memory lanes 32 (w % 4) ...
//     (its lane quarter), i.e. rows 32 (w % 4) + lane of the tile.
// Every wait is bounded; a timeout sets the status bit and an abort flag that
// the other roles see at their next wait; the block then waits (bounded) for
// its copies and matrix operations in flight before freeing tensor memory.
constexpr int kPersistThreads = 192;

template <int BN>
__global__ void __launch_bounds__(kPersistThreads, 1)
    k_gemm_tma(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               float* __restrict__ C, int ldc, int M, int N, int K, int accumulate, int k_split,
               long long c_split_stride, unsigned* __restrict__ status) {
    static_assert(BN % 16 == 0 && BN >= 32 && BN <= 256, "tcgen05 M = 128 needs N in [16, 256], a multiple of 16");
    constexpr unsigned kAccCols = BN <= 32 ? 32 : (BN <= 64 ? 64 : (BN <= 128 ? 128 : 256));
    constexpr unsigned kTmemCols = 2 * kAccCols;  // two accumulators
    constexpr unsigned kABytes = kBM * kBK * 2, kBBytes = BN * kBK * 2, kStageBytes = kABytes + kBBytes;
    extern __shared__ unsigned char dsm[];
    __shared__ __align__(8) unsigned long long full[kStages], empty[kStages], acc_full[2], acc_empty[2];
    __shared__ unsigned tmem_base;
    __shared__ int abort_flag;
    const unsigned base = (smem_addr(dsm) + 1023u) & ~1023u;  // stages at the 1024-byte swizzle atom
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tiles_m = (M + kBM - 1) / kBM, tiles_n = (N + BN - 1) / BN;
    const int splits = (K + k_split - 1) / k_split;
    const int ntiles = tiles_m * tiles_n * splits;
    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init1(smem_addr(&full[s]));
            mbar_init1(smem_addr(&empty[s]));
        }
        for (int a = 0; a < 2; ++a) {
            mbar_init1(smem_addr(&acc_full[a]));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" ::"r"(smem_addr(&acc_empty[a])) : "memory");
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
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
    volatile int* abortp = &abort_flag;
    auto tile_coords = [&](int t, int& m0, int& n0, int& kb, int& ke) {
        const int mt = t % tiles_m, r = t / tiles_m;
        m0 = mt * kBM;
        n0 = (r % tiles_n) * BN;
        kb = (r / tiles_n) * k_split;
        ke = min(K, kb + k_split);
    };
    bool failed = false;
    if (threadIdx.x == 0) {
        // producer
        int it = 0;
        for (int t = blockIdx.x; t < ntiles && !failed; t += gridDim.x) {
            int m0, n0, kb, ke;
            tile_coords(t, m0, n0, kb, ke);
            const int nk = (ke - kb + kBK - 1) / kBK;
            for (int kt = 0; kt < nk; ++kt, ++it) {
                const int s = it % kStages;
                if (it >= kStages && !mbar_wait(smem_addr(&empty[s]), (unsigned)((it / kStages - 1) & 1))) {
                    failed = true;
                    break;
                }
                if (*abortp) {
                    failed = true;
                    break;
                }
                const unsigned fb = smem_addr(&full[s]);
                asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(fb), "r"(kStageBytes)
                             : "memory");
                const unsigned sa = base + (unsigned)s * kStageBytes;
                tma_load_2d(sa, &tmA, kb + kt * kBK, m0, fb);
                tma_load_2d(sa + kABytes, &tmB, kb + kt * kBK, n0, fb);
            }
        }
        if (failed) *abortp = 1;
        // bounded: the copies in flight (the last kStages issued) land before the block leaves
        for (int q = it > kStages ? it - kStages : 0; q < it; ++q)
            mbar_wait(smem_addr(&full[q % kStages]), (unsigned)((q / kStages) & 1));
    } else if (threadIdx.x == 32) {
        // matrix operations
        constexpr uint32_t idesc = instr_desc(kBM, BN);
        int it = 0, j = 0;
        for (int t = blockIdx.x; t < ntiles && !failed; t += gridDim.x, ++j) {
            int m0, n0, kb, ke;
            tile_coords(t, m0, n0, kb, ke);
            const int nk = (ke - kb + kBK - 1) / kBK;
            const int acc = j & 1;
            // the epilogue has read this accumulator's previous tile
            if (j >= 2 && !mbar_wait(smem_addr(&acc_empty[acc]), (unsigned)((j / 2 - 1) & 1))) {
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const unsigned dcol = tmem + (unsigned)acc * kAccCols;
            for (int kt = 0; kt < nk; ++kt, ++it) {
                const int s = it % kStages;
                if (!mbar_wait(smem_addr(&full[s]), (unsigned)((it / kStages) & 1)) || *abortp) {
                    failed = true;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const unsigned sa = base + (unsigned)s * kStageBytes;
#pragma unroll
                for (int kk = 0; kk < kBK / 16; ++kk) {
                    const uint64_t ad = smem_desc_sw128(sa + kk * 32);
                    const uint64_t bd = smem_desc_sw128(sa + kABytes + kk * 32);
                    const unsigned accum = (kt > 0 || kk > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dcol),
                        "l"(ad), "l"(bd), "r"(idesc), "r"(accum)
                        : "memory");
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                                 smem_addr(&empty[s]))
                             : "memory");
            }
            if (failed) break;
            // arrives once the tile's matrix operations have completed
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(&acc_full[acc]))
                         : "memory");
        }
        if (failed) {
            *abortp = 1;
            // bounded: every matrix operation issued has completed before tensor memory is freed
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                             smem_addr(&acc_full[j & 1]))
                         : "memory");
            mbar_wait(smem_addr(&acc_full[j & 1]), (unsigned)((j / 2) & 1));
        }
    } else if (warp >= 2) {
        // epilogue: lane quarter of this warp
        const int q = warp & 3;
        int j = 0;
        for (int t = blockIdx.x; t < ntiles; t += gridDim.x, ++j) {
            const int acc = j & 1;
            // warp-uniform decision: the tensor-memory loads below need all 32 lanes
            const bool ready = mbar_wait(smem_addr(&acc_full[acc]), (unsigned)((j / 2) & 1)) && !*abortp;
            if (!__all_sync(0xffffffffu, ready)) {
                failed = true;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            int m0, n0, kb, ke;
            tile_coords(t, m0, n0, kb, ke);
            float* Ct = C + (long long)(kb / k_split) * c_split_stride;
            const int row = m0 + q * 32 + lane;
            const unsigned tbase = tmem + ((unsigned)(q * 32) << 16) + (unsigned)acc * kAccCols;
            for (int c0 = 0; c0 < BN; c0 += 16) {
                uint32_t v[16];
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
                    "%13, %14, %15}, [%16];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                      "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                      "=r"(v[15])
                    : "r"(tbase + (unsigned)c0)
                    : "memory");
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
                if (row < M) {
                    float* c = Ct + (size_t)row * ldc + n0 + c0;
                    if (n0 + c0 + 16 <= N && !accumulate && ((reinterpret_cast<uintptr_t>(c) & 15u) == 0)) {
#pragma unroll
                        for (int jj = 0; jj < 16; jj += 4)
                            *reinterpret_cast<float4*>(c + jj) =
                                make_float4(__uint_as_float(v[jj]), __uint_as_float(v[jj + 1]),
                                            __uint_as_float(v[jj + 2]), __uint_as_float(v[jj + 3]));
                    } else {
#pragma unroll
                        for (int jj = 0; jj < 16; ++jj)
                            if (n0 + c0 + jj < N)
                                c[jj] = accumulate ? c[jj] + __uint_as_float(v[jj]) : __uint_as_float(v[jj]);
                    }
                }
            }
            // this warp has read its lanes of the accumulator
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(&acc_empty[acc])) : "memory");
        }
        if (failed) *abortp = 1;
    }
    __syncwarp();
    if (failed && lane == 0) atomicOr(status, kStatusTimeout);
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

namespace {
using EncodeTiled = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                 const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Tensor map of a K-major BF16 matrix [rows][K] (leading dimension ld
// elements): boxes of 64 K x box_rows rows, 128-byte swizzle, zero fill.
bool kmajor_map(CUtensorMap* out, const void* base, int rows, int K, int ld, int box_rows) {
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
    const cuuint64_t dims[2] = {(cuuint64_t)K, (cuuint64_t)rows};
    const cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
    const cuuint32_t estr[2] = {1, 1};
    return encode(out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN>
cudaError_t launch_tma_bn(const CUtensorMap& ta, const CUtensorMap& tb, float* C, int ldc, int M, int N, int K,
                          int accumulate, int k_split, long long c_split_stride, unsigned* status, cudaStream_t s) {
    constexpr int smem = kStages * (kBM * kBK * 2 + BN * kBK * 2) + 1024;  // + alignment slack
    static bool attr_set = false;
    if (!attr_set) {
        const cudaError_t e =
            cudaFuncSetAttribute(k_gemm_tma<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) sms = 152;
    }
    const long long tiles = (long long)((M + kBM - 1) / kBM) * ((N + BN - 1) / BN) * ((K + k_split - 1) / k_split);
    if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
    const int grid = (int)(tiles < sms ? tiles : sms);
    k_gemm_tma<BN><<<grid, kPersistThreads, smem, s>>>(ta, tb, C, ldc, M, N, K, accumulate, k_split, c_split_stride,
                                                        status);
    return cudaGetLastError();
}

int launch_gemm_tma(const void* A, int lda, const void* B, int ldb, float* C, int ldc, int M, int N, int K,
                    int accumulate, int k_split, long long c_split_stride, unsigned* status, void* stream) {
    if (!A || !B || !C || !status || M < 1 || N < 1 || K < 8) return VEFD_NN_ERR_ARG;
    if (K % 8 != 0 || lda % 8 != 0 || ldb % 8 != 0 || lda < K || ldb < K || ldc < N) return VEFD_NN_ERR_ARG;
    if ((reinterpret_cast<uintptr_t>(A) | reinterpret_cast<uintptr_t>(B)) & 15u) return VEFD_NN_ERR_ARG;
    if (k_split < kBK || k_split % kBK != 0) return VEFD_NN_ERR_ARG;
    if ((K + k_split - 1) / k_split > 65535) return VEFD_NN_ERR_ARG;
    const int bn = N <= 32 ? 32 : (N <= 64 ? 64 : (N <= 128 ? 128 : 256));
    CUtensorMap ta, tb;
    if (!kmajor_map(&ta, A, M, K, lda, kBM) || !kmajor_map(&tb, B, N, K, ldb, bn)) return VEFD_NN_ERR_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaError_t e;
    switch (bn) {
    case 32: e = launch_tma_bn<32>(ta, tb, C, ldc, M, N, K, accumulate, k_split, c_split_stride, status, s); break;
    case 64: e = launch_tma_bn<64>(ta, tb, C, ldc, M, N, K, accumulate, k_split, c_split_stride, status, s); break;
    case 128: e = launch_tma_bn<128>(ta, tb, C, ldc, M, N, K, accumulate, k_split, c_split_stride, status, s); break;
    default: e = launch_tma_bn<256>(ta, tb, C, ldc, M, N, K, accumulate, k_split, c_split_stride, status, s); break;
    }
    return e == cudaSuccess ? VEFD_NN_OK : VEFD_NN_ERR_CUDA;
}
}  // namespace

extern "C" int vefd_nn_gemm_bf16(const void* A, int lda, const void* B, int ldb, float* C, int ldc, int M, int N,
                                 int K, int accumulate, unsigned* status, void* stream) {
    const int ks = ((K + kBK - 1) / kBK) * kBK;
    return launch_gemm_tma(A, lda, B, ldb, C, ldc, M, N, K, accumulate, ks < kBK ? kBK : ks, 0, status, stream);
}

extern "C" int vefd_nn_gemm_bf16_splitk(const void* A, int lda, const void* B, int ldb, float* C, int ldc, int M,
                                        int N, int K, int k_split, long long c_split_stride, unsigned* status,
                                        void* stream) {
    if (c_split_stride < (long long)M * ldc) return VEFD_NN_ERR_ARG;
    return launch_gemm_tma(A, lda, B, ldb, C, ldc, M, N, K, 0, k_split, c_split_stride, status, stream);
}

extern "C" int vefd_nn_gemm_bf16_layout(const void* A, int lda, const void* B, int ldb, float* C, int ldc, int M,
                                        int N, int K, int accumulate, unsigned lbo, unsigned sbo, int desc_swap,
                                        unsigned* status, void* stream) {
    const int ks = ((K + kBK - 1) / kBK) * kBK;
    return launch_gemm(A, lda, B, ldb, C, ldc, M, N, K, accumulate, lbo, sbo, desc_swap, ks < kBK ? kBK : ks, 0,
                       status, stream);
}
