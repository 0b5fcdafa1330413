// LB_Box stream (Section 3, Eq. 1) and the query envelope (Sections 2.3, 3).
//
// LB_Box(X, env(Q)) = sum_i sum_j (x_ij - clamp(x_ij, l_ij, u_ij))^2 over the
// points i of a database series X, with the per-dimension band envelope
// [l, u] of the query Q.  Banded DTW is symmetric, so putting the envelope on
// the query (computed once per query) bounds DTW(Q, X) just as the paper's
// envelope on the candidate does.  The max form max_i sum_j (...)^2 bounds
// DK^2: every point of X is coupled to some query point inside its box.
//
// Layout: a series is stored as whole "chunks" of lcm(d, 4) floats (whole
// points and whole float4 vectors); lane L of a warp takes chunks L, L+32,
// ... of one series, so consecutive lanes read consecutive 16-byte vectors
// (coalesced, vectorised), and the envelope of the query, staged once per
// CTA into shared memory by a TMA bulk copy, is read with the same indices.
#include "common.cuh"
#include "internal.h"

namespace knn {

constexpr int LB_THREADS = 256;
constexpr int LB_WARPS = LB_THREADS / 32;

// ---------------------------------------------------------------------------
// envelope: direct window scan, one thread per (position, coordinate)

__global__ void envelope_kernel(const EnvArgs a)
{
    const int qb = blockIdx.y;
    const int m = a.q_len[qb];
    const float *q = a.q + a.q_off[qb];
    const int r = a.radius >= 0 ? a.radius : band_radius(m, a.n_hi, a.band);
    const int d = a.d;
    float *lo = a.lo + (int64_t)qb * a.env_stride;
    float *hi = a.hi + (int64_t)qb * a.env_stride;
    const int total = (int)a.env_stride;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
        const int i = e / d, j = e - (e / d) * d;
        float l = KNN_INF, u = -KNN_INF;
        if (i < a.n_hi) {
            const int p0 = max(0, i - r), p1 = min(m - 1, i + r);
            for (int p = p0; p <= p1; ++p) {
                const float v = q[(int64_t)p * d + j];
                l = fminf(l, v);
                u = fmaxf(u, v);
            }
        } else {
            l = 0.f;  // chunk padding, never read for a real point
            u = 0.f;
        }
        lo[e] = l;
        hi[e] = u;
    }
}

void launch_envelope(const EnvArgs &a, cudaStream_t st)
{
    const int threads = 256;
    int bx = (int)((a.env_stride + threads - 1) / threads);
    bx = bx < 64 ? bx : 64;
    dim3 grid(bx > 0 ? bx : 1, a.nq);
    envelope_kernel<<<grid, threads, 0, st>>>(a);
}

// ---------------------------------------------------------------------------
// TMA bulk copy global -> shared, completion tracked by an mbarrier

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void tma_bulk_g2s(void *dst, const void *src, uint32_t bytes,
                                             uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// Bounded wait for phase 0 of the barrier; false if it gave up.
__device__ __forceinline__ bool mbar_wait0(uint64_t *bar, uint32_t limit = KNN_SPIN_LIMIT)
{
    for (uint32_t it = 0; it < limit; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_addr(bar)), "r"(0u)
            : "memory");
        if (ok)
            return true;
        if (it > 64)
            __nanosleep(256);
    }
    return false;
}

// Fault injection for tests (a.fault_wait_spins > 0): one thread waits, with
// that short limit, on a barrier that no arrival and no copy will ever
// complete (nothing is in flight on it), gives up, and reports
// KNN_DEV_TIMEOUT the way every bounded wait of the library does; the
// kernel then carries on normally.
__device__ __noinline__ void lb_fault_wait(const LbArgs &a)
{
    __shared__ __align__(8) uint64_t never;
    mbar_init(&never, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    if (!mbar_wait0(&never, a.fault_wait_spins))
        atomicOr(a.status, KNN_DEV_TIMEOUT);
}

// Record which LB_Box kernel ran (bit of knn_stats.lb_kernels), once per
// launch; the same thread runs the injected wait when one is requested.
__device__ __forceinline__ void lb_mark(const LbArgs &a, unsigned long long bit)
{
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) {
        if (a.stats)
            atomicOr(a.stats + STAT_LB_KERNELS, bit);
        if (a.fault_wait_spins)
            lb_fault_wait(a);
    }
}

// One chunk of PPC whole points: accumulate the squared box distance of
// each point (sum form) or its max (max form) into acc.
template <int D, int PPC, int F4, int FORM>
__device__ __forceinline__ void lb_chunk(const float4 (&xv)[F4], const float4 *lo_s,
                                         const float4 *hi_s, int ch, int n, float &acc)
{
    float v[4 * F4], l[4 * F4], u[4 * F4];
#pragma unroll
    for (int f = 0; f < F4; ++f) {
        const float4 lv = lo_s[ch * F4 + f];
        const float4 uv = hi_s[ch * F4 + f];
        v[4 * f] = xv[f].x; v[4 * f + 1] = xv[f].y; v[4 * f + 2] = xv[f].z; v[4 * f + 3] = xv[f].w;
        l[4 * f] = lv.x; l[4 * f + 1] = lv.y; l[4 * f + 2] = lv.z; l[4 * f + 3] = lv.w;
        u[4 * f] = uv.x; u[4 * f + 1] = uv.y; u[4 * f + 2] = uv.z; u[4 * f + 3] = uv.w;
    }
#pragma unroll
    for (int p = 0; p < PPC; ++p) {
        float box = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const float e = box_gap(v[p * D + k], l[p * D + k], u[p * D + k]);
            box = __fmaf_rn(e, e, box);
        }
        if (ch * PPC + p < n)
            acc = FORM == 0 ? acc + box : fmaxf(acc, box);
    }
}

// ---------------------------------------------------------------------------
// LB_Box stream kernel: grid (x: series tiles, y: queries of the batch)

template <int D, int FORM>
__global__ void __launch_bounds__(LB_THREADS) lb_kernel(const LbArgs a)
{
    lb_mark(a, 1ull);
    constexpr int CH = chunk_floats(D);
    constexpr int PPC = chunk_points(D);
    constexpr int F4 = CH / 4;
    extern __shared__ __align__(128) float4 env_s[];  // lo chunks then hi chunks
    __shared__ __align__(8) uint64_t bar;

    const int qb = blockIdx.y;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const float4 *lo_s = env_s;
    const float4 *hi_s = env_s + a.env_floats / 4;

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t bytes = (uint32_t)a.env_floats * 4u;
        mbar_expect_tx(&bar, 2u * bytes);
        tma_bulk_g2s(env_s, a.env_lo + (int64_t)qb * a.env_stride, bytes, &bar);
        tma_bulk_g2s(env_s + a.env_floats / 4, a.env_hi + (int64_t)qb * a.env_stride, bytes, &bar);
    }
    if (!mbar_wait0(&bar)) {
        mbar_wait0(&bar);  // once more (bounded) for the copies still in flight
        if (lane == 0)
            atomicOr(a.status, KNN_DEV_TIMEOUT);
        return;
    }

    const int m = a.q_len[qb];
    const int nser = a.c_end - a.c_begin;
    const int ntiles = (nser + 31) / 32;
    unsigned long long st_pairs = 0, st_inf = 0, st_pruned = 0, st_points = 0;

    for (int t = blockIdx.x + gridDim.x * warp; t < ntiles; t += gridDim.x * LB_WARPS) {
        const int c0 = a.c_begin + t * 32;
        const int cnt = min(32, a.c_end - c0);
        float my_lb = KNN_INF;
        bool my_feasible = false;
        for (int jj = 0; jj < cnt; ++jj) {
            const int c = c0 + jj;
            const int n = a.db_len[c];
            const int r = band_radius(m, n, a.band);
            const bool feasible = abs(m - n) <= r;
            float acc = 0.f;
            if (feasible && D % 4 == 0) {
                // points of whole float4 vectors (one point per chunk): the
                // lanes take consecutive float4 of the series and of the
                // envelope, so each warp load covers 512 contiguous bytes and
                // each shared-memory read is free of bank conflicts; 16
                // independent 16-byte loads in flight per lane.  The max form
                // joins the FPP lanes of a point (xor shuffles) first.
                constexpr int FPP = D / 4, NV = 16;
                const float4 *x4 = reinterpret_cast<const float4 *>(a.db + a.db_off[c]);
                const int nf4 = n * FPP;
                float acc4[4] = {0.f, 0.f, 0.f, 0.f};  // sum form: four FMA chains
                for (int j0 = 0; j0 < nf4; j0 += 32 * NV) {
                    float4 xv[NV];
#pragma unroll
                    for (int u = 0; u < NV; ++u) {
                        const int j = j0 + 32 * u + lane;
                        xv[u] = __ldg(x4 + min(j, nf4 - 1));  // clamped; masked below
                    }
#pragma unroll
                    for (int u = 0; u < NV; ++u) {
                        const int j = j0 + 32 * u + lane;
                        // beyond the series: a zero element in a zero box
                        const bool in = j < nf4;
                        const float4 l4 = lo_s[min(j, nf4 - 1)], h4 = hi_s[min(j, nf4 - 1)];
                        const float ex = in ? box_gap(xv[u].x, l4.x, h4.x) : 0.f;
                        const float ey = in ? box_gap(xv[u].y, l4.y, h4.y) : 0.f;
                        const float ez = in ? box_gap(xv[u].z, l4.z, h4.z) : 0.f;
                        const float ew = in ? box_gap(xv[u].w, l4.w, h4.w) : 0.f;
                        if constexpr (FORM == 0) {
                            float &t = acc4[u & 3];
                            t = __fmaf_rn(ex, ex, t);
                            t = __fmaf_rn(ey, ey, t);
                            t = __fmaf_rn(ez, ez, t);
                            t = __fmaf_rn(ew, ew, t);
                        } else {
                            float t = __fmaf_rn(ex, ex, 0.f);
                            t = __fmaf_rn(ey, ey, t);
                            t = __fmaf_rn(ez, ez, t);
                            t = __fmaf_rn(ew, ew, t);
#pragma unroll
                            for (int o = 1; o < FPP; o <<= 1)
                                t += __shfl_xor_sync(KNN_FULL_MASK, t, o);
                            acc = fmaxf(acc, t);
                        }
                    }
                }
                if constexpr (FORM == 0)
                    acc = (acc4[0] + acc4[1]) + (acc4[2] + acc4[3]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float other = __shfl_xor_sync(KNN_FULL_MASK, acc, o);
                    acc = FORM == 0 ? acc + other : fmaxf(acc, other);
                }
            } else if (feasible) {
                const float4 *x4 = reinterpret_cast<const float4 *>(a.db + a.db_off[c]);
                const int nch = (n + PPC - 1) / PPC;
                // UNR chunks per lane per iteration: 16 independent 16-byte
                // loads in flight per lane before any arithmetic
                constexpr int UNR = F4 <= 2 ? 8 : 4;
                for (int ch0 = lane; ch0 < nch; ch0 += 32 * UNR) {
                    float4 xv[UNR][F4];
#pragma unroll
                    for (int u = 0; u < UNR; ++u) {
                        const int ch = ch0 + 32 * u;
                        if (ch < nch) {
#pragma unroll
                            for (int f = 0; f < F4; ++f)
                                xv[u][f] = __ldg(x4 + ch * F4 + f);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < UNR; ++u) {
                        const int ch = ch0 + 32 * u;
                        if (ch < nch)
                            lb_chunk<D, PPC, F4, FORM>(xv[u], lo_s, hi_s, ch, n, acc);
                    }
                }
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float other = __shfl_xor_sync(KNN_FULL_MASK, acc, o);
                    acc = FORM == 0 ? acc + other : fmaxf(acc, other);
                }
            } else {
                acc = KNN_INF;
            }
            if (lane == jj) {
                my_lb = acc;
                my_feasible = feasible;
                st_points += feasible ? (unsigned long long)n : 0ull;
            }
        }
        const int c = c0 + lane;
        const bool valid = lane < cnt;
        bool keep = valid && my_feasible;
        if (keep && a.skip) {
            const int id = c;  // skip bitmap is indexed by bucket-ordered series
            keep = !((a.skip[(int64_t)qb * a.skip_words + (id >> 5)] >> (id & 31)) & 1u);
        }
        const float thr = ld_volatile_f32(a.thr + qb);
        const bool pruned = keep && !(my_lb <= thr * a.mu_prune);
        keep = keep && !pruned;
        if (valid && a.out_lb)
            a.out_lb[(int64_t)qb * a.out_lb_stride + c] = my_lb;
        st_pairs += valid;
        st_inf += valid && !my_feasible;
        st_pruned += pruned;
        const unsigned kb = __ballot_sync(KNN_FULL_MASK, keep);
        if (kb && a.items) {
            int base = 0;
            if (lane == 0)
                base = atomicAdd(a.n_items, __popc(kb));
            base = __shfl_sync(KNN_FULL_MASK, base, 0);
            if (keep) {
                const int64_t pos = (int64_t)base + __popc(kb & ((1u << lane) - 1u));
                if (pos < a.capacity) {
                    a.items[pos] = make_int2(c, qb);
                    a.item_lb[pos] = my_lb;
                } else {
                    atomicOr(a.status, KNN_DEV_CAPACITY);
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        st_pairs += __shfl_xor_sync(KNN_FULL_MASK, st_pairs, o);
        st_inf += __shfl_xor_sync(KNN_FULL_MASK, st_inf, o);
        st_pruned += __shfl_xor_sync(KNN_FULL_MASK, st_pruned, o);
        st_points += __shfl_xor_sync(KNN_FULL_MASK, st_points, o);
    }
    if (lane == 0 && a.stats) {
        atomicAdd(a.stats + STAT_PAIRS, st_pairs);
        atomicAdd(a.stats + STAT_INFEASIBLE, st_inf);
        atomicAdd(a.stats + STAT_LB_PRUNED, st_pruned);
        atomicAdd(a.stats + STAT_LB_POINTS, st_points);
    }
}

// ---------------------------------------------------------------------------
// Multi-query LB_Box kernels: grid (x: blocks of 256 series, y: query tiles).
//
// One thread owns one series and QT queries: it loads a chunk of its series
// once and bounds it against the QT query envelopes held in shared memory;
// when the series of a warp have the same length every lane reads the same
// envelope address (a broadcast).  So the database is read once per QT
// queries and each element costs 4 FP32 operations per query (two
// subtractions, a three-input max, an FMA).

// Bound one chunk of a thread's series against QT envelopes: lo/hi point at
// the chunk's envelope of the tile's first query, the next query's lies
// qstride4 float4 further.  p_first = index of the chunk's first point.
// The subtractions and squares run on packed FP32 pairs; a chunk's squares
// are summed on their own before joining the series' total, so a bound of n
// points carries at most CH/2 + 2 + n roundings in the sum form (d in the
// max form).
template <int D, int FORM, int QT>
__device__ __forceinline__ void lb_multi_chunk(const float4 (&xv)[chunk_floats(D) / 4],
                                               const float4 *lo, const float4 *hi, int qstride4,
                                               bool full, int p_first, int n, float (&acc)[QT])
{
    constexpr int CH = chunk_floats(D);
    constexpr int PPC = chunk_points(D);
    constexpr int F4 = CH / 4;
#pragma unroll
    for (int j = 0; j < QT; ++j) {
        // e = distance of every element to its box, max(l - x, x - u, 0)
        float e[CH];
#pragma unroll
        for (int f = 0; f < F4; ++f) {
            const float4 lv = lo[j * qstride4 + f];
            const float4 uv = hi[j * qstride4 + f];
            const float2 x01 = make_float2(xv[f].x, xv[f].y), x23 = make_float2(xv[f].z, xv[f].w);
            const float2 a01 = sub2(make_float2(lv.x, lv.y), x01);
            const float2 a23 = sub2(make_float2(lv.z, lv.w), x23);
            const float2 b01 = sub2(x01, make_float2(uv.x, uv.y));
            const float2 b23 = sub2(x23, make_float2(uv.z, uv.w));
            e[4 * f] = fmax3(a01.x, b01.x, 0.f);
            e[4 * f + 1] = fmax3(a01.y, b01.y, 0.f);
            e[4 * f + 2] = fmax3(a23.x, b23.x, 0.f);
            e[4 * f + 3] = fmax3(a23.y, b23.y, 0.f);
        }
        if (full && FORM == 0) {
            // whole chunk inside the series: no per-point test
            float2 s = make_float2(0.f, 0.f);
#pragma unroll
            for (int i = 0; i < CH; i += 2) {
                const float2 t = make_float2(e[i], e[i + 1]);
                s = __ffma2_rn(t, t, s);
            }
            acc[j] += s.x + s.y;
        } else if constexpr (D % 2 == 0) {
            // points hold whole pairs
#pragma unroll
            for (int p = 0; p < PPC; ++p) {
                float2 s = make_float2(0.f, 0.f);
#pragma unroll
                for (int k = 0; k < D; k += 2) {
                    const float2 t = make_float2(e[p * D + k], e[p * D + k + 1]);
                    s = __ffma2_rn(t, t, s);
                }
                const float box = s.x + s.y;
                if (full || p_first + p < n)
                    acc[j] = FORM == 0 ? acc[j] + box : fmaxf(acc[j], box);
            }
        } else {
            float sq[CH];
#pragma unroll
            for (int i = 0; i < CH; i += 2) {
                const float2 t = make_float2(e[i], e[i + 1]);
                const float2 q2 = __fmul2_rn(t, t);
                sq[i] = q2.x;
                sq[i + 1] = q2.y;
            }
#pragma unroll
            for (int p = 0; p < PPC; ++p) {
                float box = sq[p * D];
#pragma unroll
                for (int k = 1; k < D; ++k)
                    box += sq[p * D + k];
                if (full || p_first + p < n)
                    acc[j] = FORM == 0 ? acc[j] + box : fmaxf(acc[j], box);
            }
        }
    }
}

template <int QT>
__device__ __forceinline__ bool lb_all_over(const float (&acc)[QT], const float *lim)
{
    bool all_over = true;
#pragma unroll
    for (int j = 0; j < QT; ++j)
        all_over &= acc[j] > lim[j];
    return all_over;
}

// Chunks [ka, ke) of one series against the tile's envelopes (chunk ch of
// the envelopes at lo/hi + (ch - cbase) * F4), the next chunk's load in
// flight while the current one is bounded; with `abandon`, stops once every
// bound exceeds its limit (checked every 4 chunks).
template <int D, int FORM, int QT>
__device__ __forceinline__ void lb_run_chunks(const float4 *__restrict__ x4, const float4 *lo,
                                              const float4 *hi, int cbase, int st4, int ka, int ke,
                                              int n, int nqt, bool abandon, const float *lim,
                                              float (&acc)[QT], unsigned long long &st_points)
{
    constexpr int CH = chunk_floats(D);
    constexpr int PPC = chunk_points(D);
    constexpr int F4 = CH / 4;
    if (ka >= ke)
        return;
    float4 nx[F4];
#pragma unroll
    for (int f = 0; f < F4; ++f)
        nx[f] = __ldg(x4 + ka * F4 + f);
    for (int ch = ka; ch < ke; ++ch) {
        if (abandon && ((ch - ka) & 3) == 0 && lb_all_over<QT>(acc, lim))
            break;
        float4 xv[F4];
#pragma unroll
        for (int f = 0; f < F4; ++f)
            xv[f] = nx[f];
        if (ch + 1 < ke) {
#pragma unroll
            for (int f = 0; f < F4; ++f)
                nx[f] = __ldg(x4 + (ch + 1) * F4 + f);
        }
        st_points += (unsigned long long)PPC * nqt;
        lb_multi_chunk<D, FORM, QT>(xv, lo + (ch - cbase) * F4, hi + (ch - cbase) * F4, st4,
                                    (ch + 1) * PPC <= n, ch * PPC, n, acc);
    }
}

// Query of slot j of the tile starting at q0 (tiles follow the length order).
__device__ __forceinline__ int lb_qslot(const LbArgs &a, int q0, int j)
{
    return a.q_order ? a.q_order[q0 + j] : q0 + j;
}

// Set-up shared by the multi-query kernels, into shared memory: query
// lengths and the pruning limits of the tile (filter mode; -1 for missing
// queries so that they never hold a series back).  Ends with a barrier.
template <int QT>
__device__ __forceinline__ void lb_multi_setup(const LbArgs &a, int q0, int nqt, int *mq, float *lim)
{
    const int j = threadIdx.x;
    if (j < QT) {
        const int qb = j < nqt ? lb_qslot(a, q0, j) : 0;
        mq[j] = j < nqt ? a.q_len[qb] : 1;
        lim[j] = j >= nqt ? -1.f : a.items ? ld_volatile_f32(a.thr + qb) * a.mu_prune : KNN_INF;
    }
    __syncthreads();
}

// Bounds of a new series start at 0, or at +inf for a query whose band
// cannot reach the end cell (|m - n| > r): such a pair is never a candidate,
// and an infinite bound lets the series be abandoned as soon as the feasible
// queries are done with it.
template <int QT>
__device__ __forceinline__ void lb_multi_init(const LbArgs &a, const int *mq, int n,
                                              float (&acc)[QT])
{
#pragma unroll
    for (int j = 0; j < QT; ++j)
        acc[j] = abs(mq[j] - n) <= band_radius(mq[j], n, a.band) ? 0.f : KNN_INF;
}

// True if some query of the tile can reach the end cell of some series
// length of the bucket; a CTA whose tile has none skips the bucket.
template <int QT>
__device__ __forceinline__ bool lb_tile_feasible(const LbArgs &a, const int *mq, int nqt)
{
    bool any = false;
    for (int n = a.n_lo + (int)threadIdx.x; n <= a.n_hi && !any; n += blockDim.x)
#pragma unroll
        for (int j = 0; j < QT; ++j)
            any |= j < nqt && abs(mq[j] - n) <= band_radius(mq[j], n, a.band);
    return __syncthreads_or(any) != 0;
}

// The CTA's series against a tile with no feasible pair: bounds +inf
// (store mode), counted as band-infeasible.
template <int QT>
__device__ __forceinline__ void lb_tile_skip(const LbArgs &a, int q0, int nqt, int i0, int stride,
                                             unsigned long long &st_pairs,
                                             unsigned long long &st_inf)
{
    const int nser = a.c_end - a.c_begin;
    for (int i = i0; i < nser; i += stride) {
        const int c = a.c_begin + i;
        if (a.out_lb)
            for (int j = 0; j < nqt; ++j)
                a.out_lb[(int64_t)lb_qslot(a, q0, j) * a.out_lb_stride + c] = KNN_INF;
        st_pairs += nqt;
        st_inf += nqt;
    }
}

// Results of one series against the tile: bound output (store mode) or the
// survivor queue (filter mode), and the counters.  Warp-converged.
template <int QT>
__device__ __forceinline__ void lb_multi_finish(const LbArgs &a, int q0, int nqt,
                                                const int *mq, const float *lim,
                                                const float (&acc)[QT], bool valid, int c, int n,
                                                int lane, unsigned long long &st_pairs,
                                                unsigned long long &st_inf,
                                                unsigned long long &st_pruned)
{
#pragma unroll
    for (int j = 0; j < QT; ++j) {
        if (j >= nqt)
            break;
        const int qb = lb_qslot(a, q0, j);
        const int r = band_radius(mq[j], n, a.band);
        const bool feasible = valid && abs(mq[j] - n) <= r;
        const float lb = feasible ? acc[j] : KNN_INF;
        if (valid && a.out_lb)
            a.out_lb[(int64_t)qb * a.out_lb_stride + c] = lb;
        st_pairs += valid;
        st_inf += valid && !feasible;
        if (a.items) {
            bool seeded = false;
            if (a.skip && valid)
                seeded = (a.skip[(int64_t)qb * a.skip_words + (c >> 5)] >> (c & 31)) & 1u;
            const bool keep = feasible && !seeded && lb <= lim[j];
            // proposals already scored count as pruned: they are not queued again
            st_pruned += feasible && !keep;
            const unsigned kb = __ballot_sync(KNN_FULL_MASK, keep);
            if (kb) {
                int base = 0;
                if (lane == 0)
                    base = atomicAdd(a.n_items, __popc(kb));
                base = __shfl_sync(KNN_FULL_MASK, base, 0);
                if (keep) {
                    const int64_t pos = (int64_t)base + __popc(kb & ((1u << lane) - 1u));
                    if (pos < a.capacity) {
                        a.items[pos] = make_int2(c, qb);
                        a.item_lb[pos] = lb;
                    } else {
                        atomicOr(a.status, KNN_DEV_CAPACITY);
                    }
                }
            }
        }
    }
}

__device__ __forceinline__ void lb_flush_stats(const LbArgs &a, int lane, unsigned long long st_pairs,
                                               unsigned long long st_inf,
                                               unsigned long long st_pruned,
                                               unsigned long long st_points)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        st_pairs += __shfl_xor_sync(KNN_FULL_MASK, st_pairs, o);
        st_inf += __shfl_xor_sync(KNN_FULL_MASK, st_inf, o);
        st_pruned += __shfl_xor_sync(KNN_FULL_MASK, st_pruned, o);
        st_points += __shfl_xor_sync(KNN_FULL_MASK, st_points, o);
    }
    if (lane == 0 && a.stats) {
        atomicAdd(a.stats + STAT_PAIRS, st_pairs);
        atomicAdd(a.stats + STAT_INFEASIBLE, st_inf);
        atomicAdd(a.stats + STAT_LB_PRUNED, st_pruned);
        atomicAdd(a.stats + STAT_LB_POINTS, st_points);
    }
}

// Whole envelopes: the CTA stages its QT envelopes of this bucket once
// (one TMA bulk copy per array and query) and walks several 256-series
// batches.
template <int D, int FORM, int QT>
__global__ void __launch_bounds__(LB_THREADS, 2) lb_multi_kernel(const LbArgs a)
{
    lb_mark(a, 2ull);
    constexpr int CH = chunk_floats(D);
    constexpr int PPC = chunk_points(D);
    // [QT][env_floats] lo, then [QT][env_floats] hi: this bucket's envelopes
    extern __shared__ __align__(128) float4 env_s[];
    __shared__ __align__(8) uint64_t bar;

    const int q0 = blockIdx.y * QT;
    const int nqt = min(QT, a.nq - q0);
    const int lane = threadIdx.x & 31;
    const int st4 = a.env_floats / 4;
    const float4 *lo_s = env_s;
    const float4 *hi_s = env_s + QT * st4;
    unsigned long long st_pairs = 0, st_inf = 0, st_pruned = 0, st_points = 0;

    // filter mode: a series is done once every bound exceeds its limit
    __shared__ int mq[QT];
    __shared__ float lim[QT];
    lb_multi_setup<QT>(a, q0, nqt, mq, lim);
    if (!lb_tile_feasible<QT>(a, mq, nqt)) {
        lb_tile_skip<QT>(a, q0, nqt, blockIdx.x * LB_THREADS + threadIdx.x, gridDim.x * LB_THREADS,
                         st_pairs, st_inf);
        lb_flush_stats(a, lane, st_pairs, st_inf, st_pruned, st_points);
        return;
    }

    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t bytes = (uint32_t)a.env_floats * 4u;
        mbar_expect_tx(&bar, 2u * bytes * (uint32_t)nqt);
        for (int j = 0; j < nqt; ++j) {
            const int64_t src = (int64_t)lb_qslot(a, q0, j) * a.env_stride;
            tma_bulk_g2s(env_s + j * st4, a.env_lo + src, bytes, &bar);
            tma_bulk_g2s(env_s + (QT + j) * st4, a.env_hi + src, bytes, &bar);
        }
    }
    if (!mbar_wait0(&bar)) {
        mbar_wait0(&bar);  // once more (bounded) for the copies still in flight
        if (lane == 0)
            atomicOr(a.status, KNN_DEV_TIMEOUT);
        return;
    }

    const int nser = a.c_end - a.c_begin;
    const int span = (nser + LB_THREADS - 1) / LB_THREADS * LB_THREADS;
    for (int i = blockIdx.x * LB_THREADS + threadIdx.x; i < span; i += gridDim.x * LB_THREADS) {
        const bool valid = i < nser;
        const int c = a.c_begin + (valid ? i : 0);
        const int n = valid ? a.db_len[c] : 0;
        float acc[QT];
        lb_multi_init<QT>(a, mq, n, acc);
        const float4 *x4 = reinterpret_cast<const float4 *>(a.db + a.db_off[c]);
        const int nch = (n + PPC - 1) / PPC;
        // early abandoning of the bound (Section 4): partial sums and maxima
        // only grow, so once all exceed their limits the series is pruned for
        // every query of the tile
        lb_run_chunks<D, FORM, QT>(x4, lo_s, hi_s, 0, st4, 0, nch, n, nqt, a.items != nullptr, lim,
                                   acc, st_points);
        lb_multi_finish<QT>(a, q0, nqt, mq, lim, acc, valid, c, n, lane, st_pairs, st_inf,
                            st_pruned);
    }
    lb_flush_stats(a, lane, st_pairs, st_inf, st_pruned, st_points);
}

// Whole envelopes with compaction of the early abandoning (filter mode).  In
// a 256-series batch every thread walks its series in lockstep with the
// others, so the batch runs as long as its slowest series even when most are
// already past every limit.  Here a batch runs to a first checkpoint K1; the
// series still alive for some query (index and QT partial bounds) go to a
// per-CTA queue in global scratch, and whenever 256 of them are waiting they
// run together to K2, the survivors of that to a second queue and on to the
// end.  Every group of 256 starts at the same chunk, so envelope reads stay
// broadcasts.  Bounds and decisions are those of lb_multi_kernel.
constexpr int LBQ_CAP = 512;  // entries per queue: < 256 waiting + 256 arriving

template <int D, int FORM, int QT>
__global__ void __launch_bounds__(LB_THREADS, 2) lb_compact_kernel(const LbArgs a)
{
    lb_mark(a, 8ull);
    constexpr int CH = chunk_floats(D);
    constexpr int PPC = chunk_points(D);
    extern __shared__ __align__(128) float4 env_s[];
    __shared__ __align__(8) uint64_t bar;
    __shared__ int qcnt[2], qhead[2], qpush[2];

    const int q0 = blockIdx.y * QT;
    const int nqt = min(QT, a.nq - q0);
    const int lane = threadIdx.x & 31;
    const int st4 = a.env_floats / 4;
    const float4 *lo_s = env_s;
    const float4 *hi_s = env_s + QT * st4;
    unsigned long long st_pairs = 0, st_inf = 0, st_pruned = 0, st_points = 0;

    __shared__ int mq[QT];
    __shared__ float lim[QT];
    lb_multi_setup<QT>(a, q0, nqt, mq, lim);
    if (!lb_tile_feasible<QT>(a, mq, nqt)) {
        lb_tile_skip<QT>(a, q0, nqt, blockIdx.x * LB_THREADS + threadIdx.x, gridDim.x * LB_THREADS,
                         st_pairs, st_inf);
        lb_flush_stats(a, lane, st_pairs, st_inf, st_pruned, st_points);
        return;
    }
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (threadIdx.x < 2) {
        qcnt[threadIdx.x] = 0;
        qhead[threadIdx.x] = 0;
        qpush[threadIdx.x] = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t bytes = (uint32_t)a.env_floats * 4u;
        mbar_expect_tx(&bar, 2u * bytes * (uint32_t)nqt);
        for (int j = 0; j < nqt; ++j) {
            const int64_t src = (int64_t)lb_qslot(a, q0, j) * a.env_stride;
            tma_bulk_g2s(env_s + j * st4, a.env_lo + src, bytes, &bar);
            tma_bulk_g2s(env_s + (QT + j) * st4, a.env_hi + src, bytes, &bar);
        }
    }
    if (!mbar_wait0(&bar)) {
        mbar_wait0(&bar);  // once more (bounded) for the copies still in flight
        if (lane == 0)
            atomicOr(a.status, KNN_DEV_TIMEOUT);
        return;
    }

    // queue q of this CTA: [CAP] series indices (as float bits), then QT rows
    // of [CAP] partial bounds
    float *qmem = a.lbq + (size_t)(blockIdx.y * gridDim.x + blockIdx.x) * 2 * LBQ_CAP * (QT + 1);
    const int nser = a.c_end - a.c_begin;
    int next = blockIdx.x * LB_THREADS;  // first series of the next new batch
    for (;;) {
        // job 0: a new batch to K1; 1: 256 (or the last) from queue 0 to K2;
        // 2: from queue 1 to the end.  A queue with 256 waiting goes first,
        // so neither holds more than 511 entries.
        int job;
        if (qcnt[1] >= LB_THREADS)
            job = 2;
        else if (qcnt[0] >= LB_THREADS)
            job = 1;
        else if (next < nser)
            job = 0;
        else if (qcnt[0] > 0)
            job = 1;
        else if (qcnt[1] > 0)
            job = 2;
        else
            break;
        int cnt = 0, ka = 0, kb = a.k1, c = a.c_begin, n = 0;
        bool valid;
        float acc[QT];
        if (job == 0) {
            const int i = next + threadIdx.x;
            valid = i < nser;
            c = a.c_begin + (valid ? i : 0);
            n = valid ? a.db_len[c] : 0;
            lb_multi_init<QT>(a, mq, n, acc);
            next += gridDim.x * LB_THREADS;
        } else {
            const int q = job - 1;
            cnt = min(LB_THREADS, qcnt[q]);
            valid = (int)threadIdx.x < cnt;
            const float *qs = qmem + (size_t)q * LBQ_CAP * (QT + 1);
            const int pos = (qhead[q] + (int)threadIdx.x) % LBQ_CAP;
#pragma unroll
            for (int j = 0; j < QT; ++j)
                acc[j] = valid ? qs[(1 + j) * LBQ_CAP + pos] : KNN_INF;
            if (valid) {
                c = __float_as_int(qs[pos]);
                n = a.db_len[c];
            }
            ka = q == 0 ? a.k1 : a.k2;
            kb = q == 0 ? a.k2 : (1 << 30);
        }
        const int nch = (n + PPC - 1) / PPC;
        const float4 *x4 = reinterpret_cast<const float4 *>(a.db + a.db_off[c]);
        const int ke = min(kb, nch);
        lb_run_chunks<D, FORM, QT>(x4, lo_s, hi_s, 0, st4, ka, ke, n, nqt, true, lim, acc,
                                   st_points);
        const bool done = !valid || nch <= kb || lb_all_over<QT>(acc, lim);
        lb_multi_finish<QT>(a, q0, nqt, mq, lim, acc, valid && done, c, n, lane, st_pairs, st_inf,
                            st_pruned);
        if (job < 2) {
            const bool push = valid && !done;
            const unsigned pb = __ballot_sync(KNN_FULL_MASK, push);
            int base = 0;
            if (lane == 0 && pb)
                base = atomicAdd(&qpush[job], __popc(pb));
            base = __shfl_sync(KNN_FULL_MASK, base, 0);
            if (push) {
                const int pos = (qhead[job] + qcnt[job] + base + __popc(pb & ((1u << lane) - 1u))) %
                                LBQ_CAP;
                float *qd = qmem + (size_t)job * LBQ_CAP * (QT + 1);
                qd[pos] = __int_as_float(c);
#pragma unroll
                for (int j = 0; j < QT; ++j)
                    qd[(1 + j) * LBQ_CAP + pos] = acc[j];
            }
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (job >= 1) {
                qhead[job - 1] = (qhead[job - 1] + cnt) % LBQ_CAP;
                qcnt[job - 1] -= cnt;
            }
            if (job < 2) {
                qcnt[job] += qpush[job];
                qpush[job] = 0;
            }
        }
        __syncthreads();
    }
    lb_flush_stats(a, lane, st_pairs, st_inf, st_pruned, st_points);
}

size_t lb_queue_floats(int n_sm, int nq)
{
    // a launch has at most n_sm * 8 + query tiles CTAs (tile of 4 or more)
    const size_t ctas = (size_t)n_sm * 8 + (size_t)(nq + 3) / 4;
    return ctas * 2 * LBQ_CAP * 17;
}

// Bounded wait for the given phase parity of an mbarrier.
__device__ __forceinline__ bool mbar_wait_parity(uint64_t *bar, uint32_t parity)
{
    for (uint32_t it = 0; it < KNN_SPIN_LIMIT; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(smem_addr(bar)), "r"(parity)
            : "memory");
        if (ok)
            return true;
        if (it > 64)
            __nanosleep(256);
    }
    return false;
}

// Windowed envelopes, for envelopes too large to stage whole (long series,
// high d): the CTA owns one batch of 256 series and walks the bucket's
// chunks in windows of a.win_chunks; the QT envelopes of each window are
// brought in by TMA bulk copies into one of two buffers while the other is
// being read.  Between windows the CTA votes: once every series of the batch
// exceeds its limits for every query (filter mode), the rest is skipped.
template <int D, int FORM, int QT>
__global__ void __launch_bounds__(LB_THREADS, 2) lb_win_kernel(const LbArgs a)
{
    lb_mark(a, 4ull);
    constexpr int CH = chunk_floats(D);
    constexpr int PPC = chunk_points(D);
    constexpr int F4 = CH / 4;
    // two buffers, each [QT][win] lo then [QT][win] hi (float4 units)
    extern __shared__ __align__(128) float4 env_s[];
    __shared__ __align__(8) uint64_t bar[2];

    const int WCH = a.win_chunks;
    const int wst4 = WCH * F4;
    const int buf4 = 2 * QT * wst4;
    const int q0 = blockIdx.y * QT;
    const int nqt = min(QT, a.nq - q0);
    const int lane = threadIdx.x & 31;
    const int nch_env = a.env_floats / CH;
    const int W = (nch_env + WCH - 1) / WCH;
    unsigned long long st_pairs = 0, st_inf = 0, st_pruned = 0, st_points = 0;

    __shared__ int mq[QT];
    __shared__ float lim[QT];
    lb_multi_setup<QT>(a, q0, nqt, mq, lim);
    if (!lb_tile_feasible<QT>(a, mq, nqt)) {
        lb_tile_skip<QT>(a, q0, nqt, blockIdx.x * LB_THREADS + threadIdx.x, 1 << 30, st_pairs,
                         st_inf);
        lb_flush_stats(a, lane, st_pairs, st_inf, st_pruned, st_points);
        return;
    }

    if (threadIdx.x == 0) {
        mbar_init(&bar[0], 1);
        mbar_init(&bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    // window w goes to buffer w & 1; it is that barrier's (w >> 1)-th phase
    auto issue = [&](int w) {
        const int c0 = w * WCH;
        const int cnt = min(WCH, nch_env - c0);
        const uint32_t bytes = (uint32_t)cnt * CH * 4u;
        float4 *dst = env_s + (w & 1) * buf4;
        mbar_expect_tx(&bar[w & 1], 2u * bytes * (uint32_t)nqt);
        for (int j = 0; j < nqt; ++j) {
            const int64_t src = (int64_t)lb_qslot(a, q0, j) * a.env_stride + (int64_t)c0 * CH;
            tma_bulk_g2s(dst + j * wst4, a.env_lo + src, bytes, &bar[w & 1]);
            tma_bulk_g2s(dst + (QT + j) * wst4, a.env_hi + src, bytes, &bar[w & 1]);
        }
    };
    if (threadIdx.x == 0) {
        issue(0);
        if (W > 1)
            issue(1);
    }

    const int nser = a.c_end - a.c_begin;
    const int i = blockIdx.x * LB_THREADS + threadIdx.x;
    const bool valid = i < nser;
    const int c = a.c_begin + (valid ? i : 0);
    const int n = valid ? a.db_len[c] : 0;
    const int nch = (n + PPC - 1) / PPC;
    const float4 *x4 = reinterpret_cast<const float4 *>(a.db + a.db_off[c]);
    float acc[QT];
    lb_multi_init<QT>(a, mq, n, acc);

    int w = 0;
    bool failed = false;
    for (; w < W; ++w) {
        const bool ok = mbar_wait_parity(&bar[w & 1], (uint32_t)(w >> 1) & 1u);
        if (__syncthreads_or(!ok)) {
            failed = true;
            break;
        }
        const float4 *lo_w = env_s + (w & 1) * buf4;
        const float4 *hi_w = lo_w + QT * wst4;
        const int cb = w * WCH;
        const int ce = min(cb + WCH, nch);
        lb_run_chunks<D, FORM, QT>(x4, lo_w, hi_w, cb, wst4, cb, ce, n, nqt, a.items != nullptr, lim,
                                   acc, st_points);
        const bool finished = nch <= cb + WCH || (a.items && lb_all_over<QT>(acc, lim));
        // every thread is done with buffer w & 1 after this barrier
        const bool all_finished = __syncthreads_and(finished);
        if (all_finished)
            break;
        if (threadIdx.x == 0 && w + 2 < W)
            issue(w + 2);
    }
    // copies still in flight into this CTA's shared memory end before it exits
    if (threadIdx.x == 0) {
        // issued: windows [0, min(W, w + 2)); waited for: [0, w) or [0, w]
        const int first = failed ? w : w + 1;
        for (int v = first; v < min(W, w + 2); ++v)
            mbar_wait_parity(&bar[v & 1], (uint32_t)(v >> 1) & 1u);
    }
    if (failed) {
        if (lane == 0)
            atomicOr(a.status, KNN_DEV_TIMEOUT);
        return;
    }
    lb_multi_finish<QT>(a, q0, nqt, mq, lim, acc, valid, c, n, lane, st_pairs, st_inf, st_pruned);
    lb_flush_stats(a, lane, st_pairs, st_inf, st_pruned, st_points);
}

template <int D, int QT>
static void lb_attr_q()
{
    cudaFuncSetAttribute(lb_multi_kernel<D, 0, QT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(lb_multi_kernel<D, 1, QT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(lb_win_kernel<D, 0, QT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(lb_compact_kernel<D, 0, QT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(lb_compact_kernel<D, 1, QT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(lb_win_kernel<D, 1, QT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
}

template <int D>
static void lb_attr_d()
{
    cudaFuncSetAttribute(lb_kernel<D, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(lb_kernel<D, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    lb_attr_q<D, 4>();
    lb_attr_q<D, 8>();
    lb_attr_q<D, 16>();
}

void lb_init_attributes()
{
    lb_attr_d<1>(); lb_attr_d<2>(); lb_attr_d<3>(); lb_attr_d<4>(); lb_attr_d<5>();
    lb_attr_d<6>(); lb_attr_d<7>(); lb_attr_d<8>(); lb_attr_d<16>();
}

template <int D, int QT>
static void lb_multi_launch(const LbArgs &a, int form, int n_sm, cudaStream_t st)
{
    constexpr int CH = chunk_floats(D);
    const size_t smem = (size_t)QT * a.env_floats * 4 * 2;
    const int nser = a.c_end - a.c_begin;
    const int qtiles = (a.nq + QT - 1) / QT;
    const int batches = (nser + LB_THREADS - 1) / LB_THREADS;
    int bx = batches;
    const int want = (n_sm * 8 + qtiles - 1) / qtiles;
    bx = bx < want ? bx : want;
    if (bx < 1)
        bx = 1;
    // compaction pays when a CTA walks several batches of long enough series
    const int nch_env = a.env_floats / CH;
    const bool compact = a.items && a.lbq && a.compact != 1 && nch_env >= 8 &&
                         (a.compact == 2 || (nch_env >= 16 && batches >= 4 * bx));
    if (compact) {
        LbArgs c = a;
        c.k1 = (nch_env / 4 + 3) / 4 * 4;
        c.k2 = (nch_env / 2 + 3) / 4 * 4;
        if (c.k1 < 4)
            c.k1 = 4;
        if (c.k2 <= c.k1)
            c.k2 = c.k1 + 4;
        if (a.compact == 2 && batches < 4 * bx)
            bx = (batches + 3) / 4;  // several batches per CTA, so that queues fill
        dim3 grid(bx, qtiles);
        if (form == 0)
            lb_compact_kernel<D, 0, QT><<<grid, LB_THREADS, smem, st>>>(c);
        else
            lb_compact_kernel<D, 1, QT><<<grid, LB_THREADS, smem, st>>>(c);
        return;
    }
    dim3 grid(bx, qtiles);
    if (form == 0)
        lb_multi_kernel<D, 0, QT><<<grid, LB_THREADS, smem, st>>>(a);
    else
        lb_multi_kernel<D, 1, QT><<<grid, LB_THREADS, smem, st>>>(a);
}

// Shared memory of the windowed kernel: two buffers of lo and hi windows.
constexpr size_t lb_win_bytes(int qt, int ch, int win) { return (size_t)16 * qt * ch * win; }

template <int D, int QT>
static void lb_win_launch(const LbArgs &a, int form, cudaStream_t st)
{
    constexpr int CH = chunk_floats(D);
    const int nch_env = a.env_floats / CH;
    LbArgs w = a;
    if (w.win_chunks <= 0) {
        // about 96 KB of windows: two CTAs per SM
        int win = (int)((96 * 1024) / lb_win_bytes(QT, CH, 1));
        w.win_chunks = win < nch_env ? win : nch_env;
    }
    if (lb_win_bytes(QT, CH, w.win_chunks) > 192 * 1024)
        w.win_chunks = (int)((192 * 1024) / lb_win_bytes(QT, CH, 1));
    if (w.win_chunks < 1)
        w.win_chunks = 1;
    const size_t smem = lb_win_bytes(QT, CH, w.win_chunks);
    const int nser = a.c_end - a.c_begin;
    dim3 grid((nser + LB_THREADS - 1) / LB_THREADS, (a.nq + QT - 1) / QT);
    if (form == 0)
        lb_win_kernel<D, 0, QT><<<grid, LB_THREADS, smem, st>>>(w);
    else
        lb_win_kernel<D, 1, QT><<<grid, LB_THREADS, smem, st>>>(w);
}

template <int D>
static void lb_launch_d(const LbArgs &a, int form, int n_sm, cudaStream_t st)
{
    // several queries: the multi-query kernel with the requested tile (16
    // unless set), whole envelopes when they fit in shared memory, else
    // windows of them
    const size_t per_q = (size_t)a.env_floats * 4 * 2;
    if (a.nq >= 4 && !a.single_query_kernel) {
        const int want = a.qtile > 0 ? a.qtile : 16;
        const int qt = (want >= 16 && a.nq >= 16) ? 16 : (want >= 8 && a.nq >= 8) ? 8 : 4;
        const bool whole = a.win_chunks <= 0 && qt * per_q <= 192 * 1024;
        if (qt == 16)
            return whole ? lb_multi_launch<D, 16>(a, form, n_sm, st) : lb_win_launch<D, 16>(a, form, st);
        if (qt == 8)
            return whole ? lb_multi_launch<D, 8>(a, form, n_sm, st) : lb_win_launch<D, 8>(a, form, st);
        return whole ? lb_multi_launch<D, 4>(a, form, n_sm, st) : lb_win_launch<D, 4>(a, form, st);
    }
    const size_t smem = (size_t)a.env_floats * 4 * 2;
    auto kern = form == 0 ? lb_kernel<D, 0> : lb_kernel<D, 1>;
    const int nser = a.c_end - a.c_begin;
    const int ntiles = (nser + 31) / 32;
    // one full wave of the CTAs that fit with this envelope size (the kernel
    // loops over the tiles)
    int resident = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&resident, kern, LB_THREADS, smem);
    if (resident < 1)
        resident = 1;
    int want = (n_sm * resident + a.nq - 1) / a.nq;
    int maxx = (ntiles + LB_WARPS - 1) / LB_WARPS;
    int bx = want < maxx ? want : maxx;
    if (bx < 1)
        bx = 1;
    dim3 grid(bx, a.nq);
    kern<<<grid, LB_THREADS, smem, st>>>(a);
}

void launch_lb(const LbArgs &a, int d, int form, int n_sm, cudaStream_t st)
{
    switch (d) {
    case 1: lb_launch_d<1>(a, form, n_sm, st); break;
    case 2: lb_launch_d<2>(a, form, n_sm, st); break;
    case 3: lb_launch_d<3>(a, form, n_sm, st); break;
    case 4: lb_launch_d<4>(a, form, n_sm, st); break;
    case 5: lb_launch_d<5>(a, form, n_sm, st); break;
    case 6: lb_launch_d<6>(a, form, n_sm, st); break;
    case 7: lb_launch_d<7>(a, form, n_sm, st); break;
    case 8: lb_launch_d<8>(a, form, n_sm, st); break;
    case 16: lb_launch_d<16>(a, form, n_sm, st); break;
    default: break;
    }
}

}  // namespace knn
