// Learned proposal scores on the 5th-generation tensor cores (tcgen05).
//
// For a tile of 128 queries (rows of A) and 128 series (rows of B) with
// 64-dimensional BF16 embeddings, D = A B^T is accumulated in FP32 in tensor
// memory by four tcgen05.mma instructions of K = 16 (issued by one thread);
// each thread then reads its query's row of D with tcgen05.ld and forms the
// predicted distance ||e_q - e_c||^2 = |e_q|^2 + |e_c|^2 - 2 e_q.e_c,
// keeping per query the lowest score of each 64-series tile and its series.
//
// Operands are staged in shared memory in the no-swizzle K-major layout of
// 8-row x 16-byte core matrices: element (r, k) of a [R][64] BF16 tile lies
// at byte (r / 8) * 1024 + (k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2, so the
// core matrices adjacent along K are 128 bytes apart (the descriptor's
// leading-dimension offset) and the 8-row groups 1024 bytes apart (its
// stride-dimension offset).  The accumulator takes 128 of the SM's 512 TMEM
// columns; the MMAs' completion is signalled through an mbarrier whose wait
// is bounded (KNN_DEV_TIMEOUT, the TMEM freed, no hang).
#include <cuda_bf16.h>

#include "common.cuh"
#include "encoder.cuh"
#include "internal.h"

namespace knn {

namespace {

constexpr int TC_M = 128;         // queries per CTA (MMA M)
constexpr int TC_N = 128;         // series per CTA (MMA N)
constexpr int TC_K = 64;          // embedding width
constexpr int TC_THREADS = 128;   // four warps: TMEM lanes 0..127, one query each
constexpr int TC_COLS = 128;      // TMEM columns allocated (power of two >= 32)
constexpr uint32_t TC_LBO = 128;  // bytes between K-adjacent core matrices
constexpr uint32_t TC_SBO = 1024; // bytes between 8-row groups

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address, leading / stride byte
// offsets (all >> 4), the fixed version bit 46, no swizzle.
__device__ __forceinline__ uint64_t tc_desc(uint32_t addr)
{
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(TC_LBO >> 4) << 16) |
           ((uint64_t)(TC_SBO >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator (bits 4-5 = 1), BF16
// A and B (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 in
// bits 17-22, M >> 4 in bits 24-28.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) |
                              ((uint32_t)(TC_N >> 3) << 17) | ((uint32_t)(TC_M >> 4) << 24);

// Byte offset of element row r, 16-byte chunk kc (8 BF16) in a staged tile.
__device__ __forceinline__ uint32_t tc_offset(int r, int kc)
{
    return (uint32_t)(r >> 3) * TC_SBO + (uint32_t)kc * TC_LBO + (uint32_t)(r & 7) * 16u;
}

__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase 0 of the barrier.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar)
{
    for (uint32_t it = 0; it < KNN_SPIN_LIMIT; ++it) {
        if (mbar_try(bar, 0))
            return true;
        if (it > 64)
            __nanosleep(256);
    }
    return false;
}

// 32 consecutive FP32 columns of the warp's 32 TMEM lanes (one per thread).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
        "[%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]),
          "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]),
          "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i)
        v[i] = __uint_as_float(r[i]);
}

// Unused dynamic shared memory that caps residency at 4 CTAs per SM, so that
// 4 x TC_COLS TMEM columns always fit and tcgen05.alloc never waits.
constexpr size_t TC_PAD_SMEM = 20 * 1024;

__global__ void __launch_bounds__(TC_THREADS) score_tc_kernel(
    const __nv_bfloat16 *__restrict__ eq, const float *__restrict__ nq2, int nq,
    const __nv_bfloat16 *__restrict__ ec, const float *__restrict__ nc2, int n,
    float *__restrict__ score, int *__restrict__ tile_idx, int64_t stride, int *status)
{
    __shared__ __align__(1024) unsigned char As[TC_M * TC_K * 2];
    __shared__ __align__(1024) unsigned char Bs[TC_N * TC_K * 2];
    __shared__ __align__(8) uint64_t bar;
    __shared__ uint32_t tmem_base;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q0 = blockIdx.y * TC_M, c0 = blockIdx.x * TC_N;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "r"(TC_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&bar)), "r"(1u)
                     : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // stage both tiles in 16-byte chunks (8 BF16 of one row), zero beyond the data
    for (int i = tid; i < TC_M * 8; i += TC_THREADS) {
        const int r = i >> 3, kc = i & 7;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (q0 + r < nq)
            v = __ldg(reinterpret_cast<const uint4 *>(eq + (size_t)(q0 + r) * TC_K) + kc);
        *reinterpret_cast<uint4 *>(As + tc_offset(r, kc)) = v;
    }
    for (int i = tid; i < TC_N * 8; i += TC_THREADS) {
        const int r = i >> 3, kc = i & 7;
        uint4 v = make_uint4(0u, 0u, 0u, 0u);
        if (c0 + r < n)
            v = __ldg(reinterpret_cast<const uint4 *>(ec + (size_t)(c0 + r) * TC_K) + kc);
        *reinterpret_cast<uint4 *>(Bs + tc_offset(r, kc)) = v;
    }
    // the tensor cores read shared memory through the async proxy
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tbase = tmem_base;
    if (tid == 0) {
        const uint32_t a0 = smem_u32(As), b0 = smem_u32(Bs);
#pragma unroll
        for (int ks = 0; ks < TC_K / 16; ++ks) {
            // K = 16 BF16 = two core matrices along K
            const uint64_t ad = tc_desc(a0 + ks * 2 * TC_LBO);
            const uint64_t bd = tc_desc(b0 + ks * 2 * TC_LBO);
            asm volatile(
                "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tbase),
                "l"(ad), "l"(bd), "r"(TC_IDESC), "r"(ks)
                : "memory");
        }
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                smem_u32(&bar))
            : "memory");
    }
    const bool done = __syncthreads_and(mbar_wait_bounded(smem_u32(&bar)));
    if (!done) {
        // the MMAs may still run: wait once more (bounded) before freeing TMEM
        mbar_wait_bounded(smem_u32(&bar));
        if (tid == 0)
            atomicOr(status, KNN_DEV_TIMEOUT);
    } else {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const int q = q0 + warp * 32 + lane;  // this thread's TMEM lane = query row
        const float qn = q < nq ? nq2[q] : 0.f;
        const uint32_t row = tbase + ((uint32_t)(warp * 32) << 16);
#pragma unroll
        for (int h = 0; h < TC_N / 64; ++h) {
            float best = KNN_INF;
            int bidx = -1;
#pragma unroll
            for (int part = 0; part < 2; ++part) {
                float dv[32];
                tmem_ld32(row + (uint32_t)(64 * h + 32 * part), dv);
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    const int c = c0 + 64 * h + 32 * part + j;
                    if (c < n) {
                        const float v = fmaxf(qn + nc2[c] - 2.f * dv[j], 0.f);
                        if (v < best) {
                            best = v;
                            bidx = c;
                        }
                    }
                }
            }
            const int tile = (c0 >> 6) + h;
            if (q < nq && c0 + 64 * h < n) {
                score[(int64_t)q * stride + tile] = best;
                tile_idx[(int64_t)q * stride + tile] = bidx;
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (warp == 0) {
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase),
                     "r"(TC_COLS)
                     : "memory");
    }
}

}  // namespace

// Lowest predicted distance of each 64-series tile per query and its series
// ([nq][stride], stride >= ceil(n / 64)).
void launch_score_tc(const __nv_bfloat16 *eq, const float *nq2, int nq, const __nv_bfloat16 *ec,
                     const float *nc2, int n, float *score, int *tile_idx, int64_t stride,
                     int *status, cudaStream_t st)
{
    static bool attr = false;
    if (!attr) {  // static 32 KB + padding: above the 48 KB default
        cudaFuncSetAttribute(score_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)TC_PAD_SMEM);
        attr = true;
    }
    const dim3 grid((n + TC_N - 1) / TC_N, (nq + TC_M - 1) / TC_M);
    score_tc_kernel<<<grid, TC_THREADS, TC_PAD_SMEM, st>>>(eq, nq2, nq, ec, nc2, n, score,
                                                          tile_idx, stride, status);
}

}  // namespace knn
