// Coarse first stage of the LB_Box cascade, and the exact LB_Box of the
// pairs that pass it.
//
// Eq. 1 (Section 3) bounds DTW by the squared distances of the points x_j of
// a series to the boxes B_j of the query's envelope.  Group the points into
// segments of W consecutive points and let B_s be the smallest box holding
// every B_j of segment s.  Then dist(x_j, B_s) <= dist(x_j, B_j) (B_j lies in
// B_s), and the squared distance to a box is convex, so
//     sum_{j in s} dist(x_j, B_s)^2 >= W dist(mean_s(x), B_s)^2.
// Summed over the segments:
//     LB_seg = sum_s W dist(mean_s(x), B_s)^2 <= LB_Box <= DTW,
// and for the max form (the DK^2 bound)
//     max_s dist(mean_s(x), B_s)^2 <= max_j dist(x_j, B_j)^2 <= DK^2.
// A partial last segment is left out (fewer terms: still a bound).
//
// The segment means of every series are computed once when the database is
// built; a bound then costs 1/W of LB_Box.  Pairs it cannot prune get the
// exact LB_Box (one lane group per pair), and only those that survive that
// reach the dynamic program: the paper's LB_Box stage stays, with a cheaper
// stage in front of it.
//
// Scaling: means and box bounds are stored multiplied by sqrt(W), W a power
// of 4 (so the scaling is exact), and the kernels sum plain squared gaps.
//
// Rounding: each mean is rounded once (FP64 sum, one rounding to FP32), so a
// coordinate of it is off by at most u * M (M = the largest magnitude in the
// database, u = 2^-24); box bounds are query coordinates and exact.  For K
// (segment, coordinate) terms the computed norm of the gap vector differs
// from the exact one by at most sqrt(K W) u M plus relative (K/2 + 3) u, so
// a bound is compared with lim_c = ((sqrt(lim) + c2) / (1 - c1))^2 instead of
// lim (coarse_limit below): no pair is pruned whose exact coarse bound is
// within the limit.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace knn {

namespace {

constexpr int LBC_THREADS = 256;
constexpr int LBP_THREADS = 256;
constexpr int LBP_GROUP = 8;       // lanes per pair in the exact stage

// ---------------------------------------------------------------------------
// Database side: scaled segment means, one warp per series.

__global__ void seg_means_kernel(const float *__restrict__ data, const int64_t *__restrict__ off,
                                 const int *__restrict__ len, int N, int deff, int W, float scale,
                                 const int64_t *__restrict__ sg_off, const int64_t *sg_end,
                                 float *__restrict__ sg)
{
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= N)
        return;
    const int n = len[warp];
    const int nseg = n / W;
    const float *x = data + off[warp];
    float *dst = sg + sg_off[warp];
    const int64_t span = sg_end[warp] - sg_off[warp];
    for (int64_t f = lane; f < span; f += 32) {
        float v = 0.f;
        if (f < (int64_t)nseg * deff) {
            const int s = (int)(f / deff), k = (int)(f - (int64_t)s * deff);
            double acc = 0.0;
            for (int t = 0; t < W; ++t)
                acc += (double)x[(int64_t)(s * W + t) * deff + k];
            v = (float)(acc / (double)W) * scale;  // scale is a power of two: exact
        }
        dst[f] = v;
    }
}

// Largest magnitude of a float array (non-negative floats order like their
// bit patterns).
__global__ void absmax_kernel(const float *__restrict__ x, int64_t n, unsigned int *out)
{
    float m = 0.f;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        m = fmaxf(m, fabsf(x[i]));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        m = fmaxf(m, __shfl_xor_sync(KNN_FULL_MASK, m, o));
    if ((threadIdx.x & 31) == 0)
        atomicMax(out, __float_as_uint(m));
}

// ---------------------------------------------------------------------------
// Query side: scaled segment boxes of one bucket's envelopes, one CTA per
// query.  Box s covers envelope points [s W, (s + 1) W).

__global__ void seg_boxes_kernel(const SegBoxArgs a)
{
    const int q = blockIdx.x;
    const float *lo = a.env_lo + (int64_t)q * a.env_stride;
    const float *hi = a.env_hi + (int64_t)q * a.env_stride;
    float *blo = a.box_lo + (int64_t)q * a.box_stride;
    float *bhi = a.box_hi + (int64_t)q * a.box_stride;
    const int total = a.nseg * a.d;
    for (int f = threadIdx.x; f < a.box_floats; f += blockDim.x) {
        float l = KNN_INF, h = -KNN_INF;
        if (f < total) {
            const int s = f / a.d, k = f - s * a.d;
            for (int t = 0; t < a.W; ++t) {
                const int64_t e = (int64_t)(s * a.W + t) * a.d + k;
                l = fminf(l, lo[e]);
                h = fmaxf(h, hi[e]);
            }
        }
        blo[f] = l * a.scale;
        bhi[f] = h * a.scale;
    }
}

// Limit a coarse bound is compared with so that rounding never prunes a pair
// whose exact coarse bound is within `lim` (see the rounding note above): K
// (segment, coordinate) terms, segment width W, database magnitude M.  A
// negative limit marks a missing query of a tile and is passed through.
__device__ __forceinline__ float coarse_limit(float lim, int K, int W, float M)
{
    if (!(lim < KNN_INF))
        return KNN_INF;
    if (lim < 0.f)
        return lim;
    const double u = 1.0 / 16777216.0;
    const double c1 = (0.5 * K + 3.0) * u;
    const double c2 = sqrt((double)K * W) * u * (double)M;
    const double r = (sqrt((double)lim) + c2) / (1.0 - c1);
    return __double2float_ru(r * r);
}

// Fault injection for tests (spins > 0): one thread waits, with that short
// limit, on an mbarrier that no arrival and no copy will complete (nothing is
// in flight on it), gives up, and reports KNN_DEV_TIMEOUT as every bounded
// wait of the library does; the kernel then carries on normally.
__device__ __noinline__ void coarse_fault_wait(uint32_t spins, int *status)
{
    __shared__ __align__(8) uint64_t never;
    const uint32_t bar = (uint32_t)__cvta_generic_to_shared(&never);
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(1u) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    for (uint32_t it = 0; it < spins; ++it) {
        uint32_t ok;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(ok)
            : "r"(bar), "r"(0u)
            : "memory");
        if (ok)
            return;
        if (it > 64)
            __nanosleep(256);
    }
    atomicOr(status, KNN_DEV_TIMEOUT);
}

template <int QT>
__device__ __forceinline__ bool all_over(const float (&acc)[QT], const float *lim)
{
    bool over = true;
#pragma unroll
    for (int j = 0; j < QT; ++j)
        over &= acc[j] > lim[j];
    return over;
}

__device__ __forceinline__ void flush_stat(unsigned long long *stats, int slot, unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(KNN_FULL_MASK, v, o);
    if ((threadIdx.x & 31) == 0 && stats && v)
        atomicAdd(stats + slot, v);
}

// Coarse stage: QT queries per CTA (their segment boxes in shared memory),
// one series per thread, batches of LBC_THREADS series in a grid-stride loop;
// a series stops once every query's bound exceeds its limit (checked every 4
// chunks).  Pairs within their limit go to the coarse queue.
template <int D, int FORM, int QT>
__global__ void __launch_bounds__(LBC_THREADS, 2) lb_coarse_kernel(const CoarseArgs a)
{
    constexpr int CH = chunk_floats(D), PPC = chunk_points(D), F4 = CH / 4;
    extern __shared__ __align__(16) float4 cbox[];  // [QT][bf4] lo, then [QT][bf4] hi
    const int bf4 = a.box_floats / 4;
    const int q0 = blockIdx.y * QT;
    const int nqt = min(QT, a.nq - q0);
    const int tid = threadIdx.x, lane = tid & 31;
    __shared__ int mq[QT], qbs[QT];
    __shared__ float lim[QT];
    __shared__ unsigned feas_one;  // bucket of one length: bit j = query j reaches it
    if (tid == 0 && blockIdx.x == 0 && blockIdx.y == 0) {
        if (a.stats)
            atomicOr(a.stats + STAT_LB_KERNELS, 16ull);
        if (a.fault_wait_spins)
            coarse_fault_wait(a.fault_wait_spins, a.status);
    }
    if (tid < QT) {
        const int qb = tid < nqt ? (a.q_order ? a.q_order[q0 + tid] : q0 + tid) : 0;
        qbs[tid] = qb;
        mq[tid] = tid < nqt ? a.q_len[qb] : 1;
        const float l = tid < nqt ? ld_volatile_f32(a.thr + qb) * a.mu_prune : -1.f;
        // max form: one segment's D terms, unscaled (W = 1 in the bound)
        lim[tid] = FORM == 0 ? coarse_limit(l, a.nseg_hi * D, a.W, a.M)
                             : coarse_limit(l, D, 1, a.M);
    }
    for (int i = tid; i < nqt * bf4; i += blockDim.x) {
        const int j = i / bf4, t = i - j * bf4;
        const int qb = a.q_order ? a.q_order[q0 + j] : q0 + j;
        cbox[j * bf4 + t] =
            reinterpret_cast<const float4 *>(a.box_lo + (int64_t)qb * a.box_stride)[t];
        cbox[(QT + j) * bf4 + t] =
            reinterpret_cast<const float4 *>(a.box_hi + (int64_t)qb * a.box_stride)[t];
    }
    __syncthreads();
    // the band test |m - n| <= r(m, n) once per query when the bucket has a
    // single length (published by the __syncthreads_or below)
    static_assert(QT <= 32, "one warp holds the tile's queries");
    if (tid < 32) {
        const bool f = tid < nqt && abs(mq[tid] - a.n_lo) <= band_radius(mq[tid], a.n_lo, a.band);
        const unsigned b = __ballot_sync(KNN_FULL_MASK, f);
        if (tid == 0)
            feas_one = b;
    }
    const int nser = a.c_end - a.c_begin;
    unsigned long long st_pairs = 0, st_inf = 0, st_pruned = 0, st_cpr = 0, st_segs = 0;
    // a tile none of whose queries reaches a length of the bucket skips it
    bool any = false;
    for (int n = a.n_lo + tid; n <= a.n_hi && !any; n += blockDim.x)
        for (int j = 0; j < nqt; ++j)
            any |= abs(mq[j] - n) <= band_radius(mq[j], n, a.band);
    const bool tile_ok = __syncthreads_or(any) != 0;
    const float4 *lo_s = cbox, *hi_s = cbox + QT * bf4;
    for (int base = blockIdx.x * LBC_THREADS; base < nser; base += gridDim.x * LBC_THREADS) {
        const int i = base + tid;
        const bool valid = i < nser;
        if (!tile_ok) {
            st_pairs += valid ? nqt : 0;
            st_inf += valid ? nqt : 0;
            continue;
        }
        const int c = a.c_begin + (valid ? i : 0);
        const int n = valid ? a.db_len[c] : 0;
        const int nseg = n / a.W;
        const int nch = (nseg + PPC - 1) / PPC;
        const float4 *x4 = reinterpret_cast<const float4 *>(a.sg + a.sg_off[c]);
        // bit j: query j's band reaches this series' end cell
        unsigned fm = 0;
        if (a.n_lo == a.n_hi) {
            fm = valid ? feas_one : 0u;
        } else {
#pragma unroll
            for (int j = 0; j < QT; ++j)
                if (valid && j < nqt && abs(mq[j] - n) <= band_radius(mq[j], n, a.band))
                    fm |= 1u << j;
        }
        float acc[QT];
#pragma unroll
        for (int j = 0; j < QT; ++j)
            acc[j] = (fm >> j) & 1u ? 0.f : KNN_INF;
        float4 nx[F4];
        if (nch > 0) {
#pragma unroll
            for (int f = 0; f < F4; ++f)
                nx[f] = __ldg(x4 + f);
        }
        for (int ch = 0; ch < nch; ++ch) {
            if ((ch & 3) == 0 && all_over<QT>(acc, lim))
                break;
            float xv[CH];
#pragma unroll
            for (int f = 0; f < F4; ++f) {
                xv[4 * f] = nx[f].x; xv[4 * f + 1] = nx[f].y;
                xv[4 * f + 2] = nx[f].z; xv[4 * f + 3] = nx[f].w;
            }
            if (ch + 1 < nch) {
#pragma unroll
                for (int f = 0; f < F4; ++f)
                    nx[f] = __ldg(x4 + (ch + 1) * F4 + f);
            }
            const int live = min(PPC, nseg - ch * PPC);
            st_segs += (unsigned long long)live * nqt;
#pragma unroll
            for (int j = 0; j < QT; ++j) {
                if (j >= nqt)
                    break;
                float lv[CH], hv[CH];
#pragma unroll
                for (int f = 0; f < F4; ++f) {
                    const float4 l4 = lo_s[j * bf4 + ch * F4 + f];
                    const float4 h4 = hi_s[j * bf4 + ch * F4 + f];
                    lv[4 * f] = l4.x; lv[4 * f + 1] = l4.y; lv[4 * f + 2] = l4.z; lv[4 * f + 3] = l4.w;
                    hv[4 * f] = h4.x; hv[4 * f + 1] = h4.y; hv[4 * f + 2] = h4.z; hv[4 * f + 3] = h4.w;
                }
#pragma unroll
                for (int p = 0; p < PPC; ++p) {
                    float box = 0.f;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const float e = box_gap(xv[p * D + k], lv[p * D + k], hv[p * D + k]);
                        box = __fmaf_rn(e, e, box);
                    }
                    // box = W dist^2 (scaled values); the max form keeps dist^2
                    if (p < live)
                        acc[j] = FORM == 0 ? acc[j] + box : fmaxf(acc[j], box * a.inv_w);
                }
            }
        }
        // results of this series against the tile
#pragma unroll
        for (int j = 0; j < QT; ++j) {
            if (j >= nqt)
                break;
            const int qb = qbs[j];
            const bool feasible = (fm >> j) & 1u;
            bool seeded = false;
            if (a.skip && feasible)
                seeded = (a.skip[(int64_t)qb * a.skip_words + (c >> 5)] >> (c & 31)) & 1u;
            const bool keep = a.cq && feasible && !seeded && acc[j] <= lim[j];
            if (a.out_lb && valid)
                a.out_lb[(int64_t)qb * a.out_lb_stride + c] = feasible ? acc[j] : KNN_INF;
            st_pairs += valid;
            st_inf += valid && !feasible;
            st_pruned += feasible && !keep;
            st_cpr += feasible && !seeded && !keep;
            const unsigned kb = __ballot_sync(KNN_FULL_MASK, keep);
            if (kb) {
                // one query per ballot: the warp's survivors go to its list
                int *count = a.cq_qcount ? a.cq_qcount + qb : a.cq_count;
                int2 *list = a.cq_qcount ? a.cq + (int64_t)qb * a.cq_stride : a.cq;
                const int64_t cap = a.cq_qcount ? a.cq_stride : a.cq_cap;
                int pos0 = 0;
                if (lane == 0)
                    pos0 = atomicAdd(count, __popc(kb));
                pos0 = __shfl_sync(KNN_FULL_MASK, pos0, 0);
                if (keep) {
                    const int64_t pos = (int64_t)pos0 + __popc(kb & ((1u << lane) - 1u));
                    if (pos < cap)
                        list[pos] = make_int2(c, qb);
                    else
                        atomicOr(a.status, KNN_DEV_CAPACITY);
                }
            }
        }
    }
    flush_stat(a.stats, STAT_PAIRS, st_pairs);
    flush_stat(a.stats, STAT_INFEASIBLE, st_inf);
    flush_stat(a.stats, STAT_LB_PRUNED, st_pruned);
    flush_stat(a.stats, STAT_LB_COARSE_PRUNED, st_cpr);
    flush_stat(a.stats, STAT_LB_SEGMENTS, st_segs);
}

// Exact LB_Box (Eq. 1, envelope on the query) of the pairs of the coarse
// queue: a group of LBP_GROUP lanes per pair takes the pair's chunks in turn
// (coalesced along the series), the group's partial bounds are combined every
// 4 rounds and the pair is dropped once they exceed its limit.  Pairs within
// the limit go to the DP queue with their bound.
template <int D, int FORM>
__global__ void __launch_bounds__(LBP_THREADS) lb_pair_kernel(const PairLbArgs a)
{
    constexpr int CH = chunk_floats(D), PPC = chunk_points(D), F4 = CH / 4;
    constexpr int GPW = 32 / LBP_GROUP;
    const int lane = threadIdx.x & 31, grp = lane / LBP_GROUP, gl = lane % LBP_GROUP;
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    const int total = (int)min((int64_t)*a.cq_count, a.cq_cap);
    unsigned long long st_pruned = 0, st_points = 0;
    for (int base = warp * GPW; base < total; base += nwarps * GPW) {
        const int idx = base + grp;
        const bool valid = idx < total;
        const int2 it = valid ? a.cq[idx] : make_int2(0, 0);
        const int c = it.x, qb = it.y;
        const int n = valid ? a.db_len[c] : 0;
        const float lim = valid ? ld_volatile_f32(a.thr + qb) * a.mu_prune : -1.f;
        const float4 *x4 = reinterpret_cast<const float4 *>(a.db + a.db_off[c]);
        const float4 *lo4 = reinterpret_cast<const float4 *>(a.env_lo + (int64_t)qb * a.env_stride);
        const float4 *hi4 = reinterpret_cast<const float4 *>(a.env_hi + (int64_t)qb * a.env_stride);
        const int nch = (n + PPC - 1) / PPC;
        const int nch_max = __reduce_max_sync(KNN_FULL_MASK, nch);
        float acc = 0.f, tot = 0.f;
        bool alive = valid;
        for (int ch0 = 0, round = 0; ch0 < nch_max; ch0 += LBP_GROUP, ++round) {
            const int ch = ch0 + gl;
            if (alive && ch < nch) {
                float xv[CH], lv[CH], hv[CH];
#pragma unroll
                for (int f = 0; f < F4; ++f) {
                    const float4 x = __ldg(x4 + ch * F4 + f);
                    const float4 l = __ldg(lo4 + ch * F4 + f);
                    const float4 h = __ldg(hi4 + ch * F4 + f);
                    xv[4 * f] = x.x; xv[4 * f + 1] = x.y; xv[4 * f + 2] = x.z; xv[4 * f + 3] = x.w;
                    lv[4 * f] = l.x; lv[4 * f + 1] = l.y; lv[4 * f + 2] = l.z; lv[4 * f + 3] = l.w;
                    hv[4 * f] = h.x; hv[4 * f + 1] = h.y; hv[4 * f + 2] = h.z; hv[4 * f + 3] = h.w;
                }
                const int live = min(PPC, n - ch * PPC);
#pragma unroll
                for (int p = 0; p < PPC; ++p) {
                    float box = 0.f;
#pragma unroll
                    for (int k = 0; k < D; ++k) {
                        const float e = box_gap(xv[p * D + k], lv[p * D + k], hv[p * D + k]);
                        box = __fmaf_rn(e, e, box);
                    }
                    if (p < live)
                        acc = FORM == 0 ? acc + box : fmaxf(acc, box);
                }
                st_points += live;
            }
            if ((round & 3) == 3 || ch0 + LBP_GROUP >= nch_max) {
                tot = acc;
#pragma unroll
                for (int o = 1; o < LBP_GROUP; o <<= 1) {
                    const float other = __shfl_xor_sync(KNN_FULL_MASK, tot, o);
                    tot = FORM == 0 ? tot + other : fmaxf(tot, other);
                }
                alive = alive && tot <= lim;
                if (!__any_sync(KNN_FULL_MASK, alive))
                    break;
            }
        }
        // alive: the bound over every chunk is within the limit
        const bool keep = alive && gl == 0;
        st_pruned += valid && gl == 0 && !alive;
        const unsigned kb = __ballot_sync(KNN_FULL_MASK, keep);
        if (kb) {
            int pos0 = 0;
            if (lane == 0)
                pos0 = atomicAdd(a.n_items, __popc(kb));
            pos0 = __shfl_sync(KNN_FULL_MASK, pos0, 0);
            if (keep) {
                const int64_t pos = (int64_t)pos0 + __popc(kb & ((1u << lane) - 1u));
                if (pos < a.capacity) {
                    a.items[pos] = make_int2(c, qb);
                    a.item_lb[pos] = tot;
                } else {
                    atomicOr(a.status, KNN_DEV_CAPACITY);
                }
            }
        }
    }
    flush_stat(a.stats, STAT_LB_PRUNED, st_pruned);
    flush_stat(a.stats, STAT_LB_POINTS, st_points);
}

// The same exact stage for point widths that are whole float4 vectors
// (D = 4, 8, 16: one point per chunk, FPP float4 per point).  The group's 8
// lanes read consecutive float4 of the series and of the envelope, so every
// load instruction of a group covers 128 contiguous bytes (the chunk-per-lane
// order above puts the lanes 16 D bytes apart and needs D/4 times the L1
// wavefronts).  The sum form adds every element's squared gap; the max form
// first joins the FPP lanes that hold one point (xor shuffles), then takes
// the maximum over points.
template <int D, int FORM>
__global__ void __launch_bounds__(LBP_THREADS) lb_pair4_kernel(const PairLbArgs a)
{
    static_assert(D % 4 == 0 && D <= 32, "whole float4 points");
    constexpr int FPP = D / 4;                 // float4 per point
    constexpr int UNR = 4;                     // float4 per lane per round
    constexpr int RF4 = LBP_GROUP * UNR;       // float4 per group per round
    constexpr int GPW = 32 / LBP_GROUP;
    const int lane = threadIdx.x & 31, grp = lane / LBP_GROUP, gl = lane % LBP_GROUP;
    const int warp = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    const int nwarps = (int)(((int64_t)gridDim.x * blockDim.x) >> 5);
    const int total = (int)min((int64_t)*a.cq_count, a.cq_cap);
    unsigned long long st_pruned = 0, st_points = 0;
    for (int base = warp * GPW; base < total; base += nwarps * GPW) {
        const int idx = base + grp;
        const bool valid = idx < total;
        const int2 it = valid ? a.cq[idx] : make_int2(0, 0);
        const int c = it.x, qb = it.y;
        const int n = valid ? a.db_len[c] : 0;
        const float lim = valid ? ld_volatile_f32(a.thr + qb) * a.mu_prune : -1.f;
        const float4 *x4 = reinterpret_cast<const float4 *>(a.db + a.db_off[c]);
        const float4 *lo4 = reinterpret_cast<const float4 *>(a.env_lo + (int64_t)qb * a.env_stride);
        const float4 *hi4 = reinterpret_cast<const float4 *>(a.env_hi + (int64_t)qb * a.env_stride);
        const int nf4 = n * FPP;
        const int nf4_max = __reduce_max_sync(KNN_FULL_MASK, nf4);
        float acc[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u)
            acc[u] = 0.f;
        float tot = 0.f;
        bool alive = valid;
        for (int r0 = 0, round = 0; r0 < nf4_max; r0 += RF4, ++round) {
            float4 xv[UNR], lv[UNR], hv[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const int j = r0 + u * LBP_GROUP + gl;
                if (alive && j < nf4) {
                    xv[u] = __ldg(x4 + j);
                    lv[u] = __ldg(lo4 + j);
                    hv[u] = __ldg(hi4 + j);
                    st_points += (j % FPP) == 0;
                } else {
                    // a zero element with a zero box: gap 0, adds nothing
                    xv[u] = lv[u] = hv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const float ex = box_gap(xv[u].x, lv[u].x, hv[u].x);
                const float ey = box_gap(xv[u].y, lv[u].y, hv[u].y);
                const float ez = box_gap(xv[u].z, lv[u].z, hv[u].z);
                const float ew = box_gap(xv[u].w, lv[u].w, hv[u].w);
                if constexpr (FORM == 0) {
                    float t = acc[u];
                    t = __fmaf_rn(ex, ex, t);
                    t = __fmaf_rn(ey, ey, t);
                    t = __fmaf_rn(ez, ez, t);
                    acc[u] = __fmaf_rn(ew, ew, t);
                } else {
                    float t = __fmaf_rn(ex, ex, 0.f);
                    t = __fmaf_rn(ey, ey, t);
                    t = __fmaf_rn(ez, ez, t);
                    t = __fmaf_rn(ew, ew, t);
#pragma unroll
                    for (int o = 1; o < FPP; o <<= 1)
                        t += __shfl_xor_sync(KNN_FULL_MASK, t, o);
                    acc[u] = fmaxf(acc[u], t);
                }
            }
            if ((round & 3) == 3 || r0 + RF4 >= nf4_max) {
                tot = acc[0];
#pragma unroll
                for (int u = 1; u < UNR; ++u)
                    tot = FORM == 0 ? tot + acc[u] : fmaxf(tot, acc[u]);
#pragma unroll
                for (int o = 1; o < LBP_GROUP; o <<= 1) {
                    const float other = __shfl_xor_sync(KNN_FULL_MASK, tot, o);
                    tot = FORM == 0 ? tot + other : fmaxf(tot, other);
                }
                alive = alive && tot <= lim;
                if (!__any_sync(KNN_FULL_MASK, alive))
                    break;
            }
        }
        const bool keep = alive && gl == 0;
        st_pruned += valid && gl == 0 && !alive;
        const unsigned kb = __ballot_sync(KNN_FULL_MASK, keep);
        if (kb) {
            int pos0 = 0;
            if (lane == 0)
                pos0 = atomicAdd(a.n_items, __popc(kb));
            pos0 = __shfl_sync(KNN_FULL_MASK, pos0, 0);
            if (keep) {
                const int64_t pos = (int64_t)pos0 + __popc(kb & ((1u << lane) - 1u));
                if (pos < a.capacity) {
                    a.items[pos] = make_int2(c, qb);
                    a.item_lb[pos] = tot;
                } else {
                    atomicOr(a.status, KNN_DEV_CAPACITY);
                }
            }
        }
    }
    flush_stat(a.stats, STAT_LB_PRUNED, st_pruned);
    flush_stat(a.stats, STAT_LB_POINTS, st_points);
}

// The exact stage with its pairs grouped by query: CTA (slice, qb) copies
// query qb's envelope (lower and upper, env_floats each) into shared memory
// once and bounds its share of qb's survivors; lanes read the series as in
// lb_pair4_kernel (consecutive float4, 128 B per group per load) and the
// envelope from shared memory, where the four groups of a warp, in step on
// the same query, read the same float4 (broadcast); eight float4 of the
// series in flight per lane, the bound tested every two rounds (as often per
// point as lb_pair4_kernel).  The series then come from DRAM alone instead of
// series plus two envelope rows per point.
template <int D, int FORM>
__global__ void __launch_bounds__(LBP_THREADS, 3) lb_pairq4_kernel(const PairLbArgs a)
{
    static_assert(D % 4 == 0 && D <= 32, "whole float4 points");
    constexpr int FPP = D / 4, UNR = 8, RF4 = LBP_GROUP * UNR, GPW = 32 / LBP_GROUP;
    constexpr int GPB = (LBP_THREADS / 32) * GPW;  // pair groups per CTA
    extern __shared__ __align__(16) float4 envq[];  // lo then hi, env_floats / 4 each
    const int qb = blockIdx.y;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / LBP_GROUP, gl = lane % LBP_GROUP;
    const int ef4 = a.env_floats / 4;
    const float4 *lo_g = reinterpret_cast<const float4 *>(a.env_lo + (int64_t)qb * a.env_stride);
    const float4 *hi_g = reinterpret_cast<const float4 *>(a.env_hi + (int64_t)qb * a.env_stride);
    for (int i = threadIdx.x; i < ef4; i += blockDim.x) {
        envq[i] = __ldg(lo_g + i);
        envq[ef4 + i] = __ldg(hi_g + i);
    }
    __syncthreads();
    const float4 *lo4 = envq, *hi4 = envq + ef4;
    const int total = (int)min((int64_t)a.cq_qcount[qb], a.cq_stride);
    const int2 *list = a.cq + (int64_t)qb * a.cq_stride;
    const float lim = ld_volatile_f32(a.thr + qb) * a.mu_prune;
    unsigned long long st_pruned = 0, st_points = 0;
    const int stride = gridDim.x * GPB;
    for (int base = blockIdx.x * GPB + warp * GPW; base < total; base += stride) {
        const int idx = base + grp;
        const bool valid = idx < total;
        const int c = valid ? list[idx].x : 0;
        const int n = valid ? a.db_len[c] : 0;
        const float4 *x4 = reinterpret_cast<const float4 *>(a.db + a.db_off[c]);
        const int nf4 = n * FPP;
        const int nf4_max = __reduce_max_sync(KNN_FULL_MASK, nf4);
        float acc[UNR];
#pragma unroll
        for (int u = 0; u < UNR; ++u)
            acc[u] = 0.f;
        float tot = 0.f;
        bool alive = valid;
        for (int r0 = 0, round = 0; r0 < nf4_max; r0 += RF4, ++round) {
            float4 xv[UNR];
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const int j = r0 + u * LBP_GROUP + gl;
                if (alive && j < nf4) {
                    xv[u] = __ldg(x4 + j);
                    st_points += (j % FPP) == 0;
                } else {
                    xv[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < UNR; ++u) {
                const int j = r0 + u * LBP_GROUP + gl;
                // beyond the series (or the pair decided): a zero gap
                const bool in = alive && j < nf4;
                const int js = in ? j : 0;
                const float4 l = lo4[js], h = hi4[js];
                const float ex = in ? box_gap(xv[u].x, l.x, h.x) : 0.f;
                const float ey = in ? box_gap(xv[u].y, l.y, h.y) : 0.f;
                const float ez = in ? box_gap(xv[u].z, l.z, h.z) : 0.f;
                const float ew = in ? box_gap(xv[u].w, l.w, h.w) : 0.f;
                if constexpr (FORM == 0) {
                    float t = acc[u];
                    t = __fmaf_rn(ex, ex, t);
                    t = __fmaf_rn(ey, ey, t);
                    t = __fmaf_rn(ez, ez, t);
                    acc[u] = __fmaf_rn(ew, ew, t);
                } else {
                    float t = __fmaf_rn(ex, ex, 0.f);
                    t = __fmaf_rn(ey, ey, t);
                    t = __fmaf_rn(ez, ez, t);
                    t = __fmaf_rn(ew, ew, t);
#pragma unroll
                    for (int o = 1; o < FPP; o <<= 1)
                        t += __shfl_xor_sync(KNN_FULL_MASK, t, o);
                    acc[u] = fmaxf(acc[u], t);
                }
            }
            if ((round & 1) == 1 || r0 + RF4 >= nf4_max) {
                tot = acc[0];
#pragma unroll
                for (int u = 1; u < UNR; ++u)
                    tot = FORM == 0 ? tot + acc[u] : fmaxf(tot, acc[u]);
#pragma unroll
                for (int o = 1; o < LBP_GROUP; o <<= 1) {
                    const float other = __shfl_xor_sync(KNN_FULL_MASK, tot, o);
                    tot = FORM == 0 ? tot + other : fmaxf(tot, other);
                }
                alive = alive && tot <= lim;
                if (!__any_sync(KNN_FULL_MASK, alive))
                    break;
            }
        }
        const bool keep = alive && gl == 0;
        st_pruned += valid && gl == 0 && !alive;
        const unsigned kb = __ballot_sync(KNN_FULL_MASK, keep);
        if (kb) {
            int pos0 = 0;
            if (lane == 0)
                pos0 = atomicAdd(a.n_items, __popc(kb));
            pos0 = __shfl_sync(KNN_FULL_MASK, pos0, 0);
            if (keep) {
                const int64_t pos = (int64_t)pos0 + __popc(kb & ((1u << lane) - 1u));
                if (pos < a.capacity) {
                    a.items[pos] = make_int2(c, qb);
                    a.item_lb[pos] = tot;
                } else {
                    atomicOr(a.status, KNN_DEV_CAPACITY);
                }
            }
        }
    }
    flush_stat(a.stats, STAT_LB_PRUNED, st_pruned);
    flush_stat(a.stats, STAT_LB_POINTS, st_points);
}

}  // namespace

void launch_seg_means(const float *data, const int64_t *off, const int *len, int N, int deff,
                      int W, const int64_t *sg_off, const int64_t *sg_end, float *sg,
                      cudaStream_t st)
{
    const float scale = coarse_scale(W);
    const int blocks = (int)(((int64_t)N * 32 + 255) / 256);
    seg_means_kernel<<<blocks, 256, 0, st>>>(data, off, len, N, deff, W, scale, sg_off, sg_end,
                                             sg);
}

void launch_absmax(const float *x, int64_t n, unsigned int *out, cudaStream_t st)
{
    cudaMemsetAsync(out, 0, sizeof(unsigned int), st);
    const int blocks = (int)std::min<int64_t>((n + 255) / 256, 4096);
    absmax_kernel<<<blocks > 0 ? blocks : 1, 256, 0, st>>>(x, n, out);
}

void launch_seg_boxes(const SegBoxArgs &a, cudaStream_t st)
{
    seg_boxes_kernel<<<a.nq, 256, 0, st>>>(a);
}

namespace {

constexpr size_t LBC_SMEM_MAX = 100 * 1024;  // two CTAs per SM

template <int D, int FORM, int QT>
void coarse_launch(const CoarseArgs &a, int n_sm, cudaStream_t st)
{
    const int ntiles = (a.nq + QT - 1) / QT;
    const int nbatch = (a.c_end - a.c_begin + LBC_THREADS - 1) / LBC_THREADS;
    const int gx = std::max(1, std::min(nbatch, n_sm * 8 / ntiles));
    const size_t smem = (size_t)2 * QT * a.box_floats * sizeof(float);
    lb_coarse_kernel<D, FORM, QT><<<dim3(gx, ntiles), LBC_THREADS, smem, st>>>(a);
}

template <int D, int FORM>
bool coarse_launch_q(const CoarseArgs &a, int qt, int n_sm, cudaStream_t st)
{
    switch (qt) {
    case 16: coarse_launch<D, FORM, 16>(a, n_sm, st); return true;
    case 8: coarse_launch<D, FORM, 8>(a, n_sm, st); return true;
    case 4: coarse_launch<D, FORM, 4>(a, n_sm, st); return true;
    default: return false;
    }
}

template <int D>
bool coarse_launch_d(const CoarseArgs &a, int form, int qt, int n_sm, cudaStream_t st)
{
    return form == 0 ? coarse_launch_q<D, 0>(a, qt, n_sm, st)
                     : coarse_launch_q<D, 1>(a, qt, n_sm, st);
}

constexpr size_t LBPQ_SMEM_MAX = 200 * 1024;

template <int D>
void pair_launch_d(const PairLbArgs &a, int form, int n_sm, cudaStream_t st)
{
    if constexpr (D % 4 == 0) {
        if (a.cq_qcount) {
            static bool attr = false;
            if (!attr) {
                cudaFuncSetAttribute(lb_pairq4_kernel<D, 0>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)LBPQ_SMEM_MAX);
                cudaFuncSetAttribute(lb_pairq4_kernel<D, 1>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)LBPQ_SMEM_MAX);
                attr = true;
            }
            // slices per query: about six CTAs' worth per SM over the batch
            const int slices = std::max(1, (6 * n_sm + a.nq - 1) / a.nq);
            const size_t smem = (size_t)2 * a.env_floats * sizeof(float);
            const dim3 grid(slices, a.nq);
            if (form == 0)
                lb_pairq4_kernel<D, 0><<<grid, LBP_THREADS, smem, st>>>(a);
            else
                lb_pairq4_kernel<D, 1><<<grid, LBP_THREADS, smem, st>>>(a);
            return;
        }
        if (form == 0)
            lb_pair4_kernel<D, 0><<<n_sm * 8, LBP_THREADS, 0, st>>>(a);
        else
            lb_pair4_kernel<D, 1><<<n_sm * 8, LBP_THREADS, 0, st>>>(a);
    } else {
        if (form == 0)
            lb_pair_kernel<D, 0><<<n_sm * 8, LBP_THREADS, 0, st>>>(a);
        else
            lb_pair_kernel<D, 1><<<n_sm * 8, LBP_THREADS, 0, st>>>(a);
    }
}

template <int D, int QT>
void coarse_attr_q()
{
    cudaFuncSetAttribute(lb_coarse_kernel<D, 0, QT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)LBC_SMEM_MAX);
    cudaFuncSetAttribute(lb_coarse_kernel<D, 1, QT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)LBC_SMEM_MAX);
}

template <int D>
void coarse_attr_d()
{
    coarse_attr_q<D, 16>();
    coarse_attr_q<D, 8>();
    coarse_attr_q<D, 4>();
}

}  // namespace

int coarse_qtile(int box_floats)
{
    for (int qt = 16; qt >= 4; qt /= 2)
        if ((size_t)2 * qt * box_floats * sizeof(float) <= LBC_SMEM_MAX)
            return qt;
    return 0;
}

bool launch_lb_coarse(const CoarseArgs &a, int deff, int form, int n_sm, cudaStream_t st)
{
    int qt = coarse_qtile(a.box_floats);
    if (a.qtile_req > 0 && a.qtile_req < qt)
        qt = a.qtile_req;
    switch (deff) {
    case 1: return coarse_launch_d<1>(a, form, qt, n_sm, st);
    case 2: return coarse_launch_d<2>(a, form, qt, n_sm, st);
    case 3: return coarse_launch_d<3>(a, form, qt, n_sm, st);
    case 4: return coarse_launch_d<4>(a, form, qt, n_sm, st);
    case 5: return coarse_launch_d<5>(a, form, qt, n_sm, st);
    case 6: return coarse_launch_d<6>(a, form, qt, n_sm, st);
    case 7: return coarse_launch_d<7>(a, form, qt, n_sm, st);
    case 8: return coarse_launch_d<8>(a, form, qt, n_sm, st);
    case 16: return coarse_launch_d<16>(a, form, qt, n_sm, st);
    default: return false;
    }
}

bool lb_pairs_by_query(int deff, int env_floats)
{
    return deff % 4 == 0 && (size_t)2 * env_floats * sizeof(float) <= LBPQ_SMEM_MAX;
}

bool launch_lb_pairs(const PairLbArgs &a, int deff, int form, int n_sm, cudaStream_t st)
{
    switch (deff) {
    case 1: pair_launch_d<1>(a, form, n_sm, st); return true;
    case 2: pair_launch_d<2>(a, form, n_sm, st); return true;
    case 3: pair_launch_d<3>(a, form, n_sm, st); return true;
    case 4: pair_launch_d<4>(a, form, n_sm, st); return true;
    case 5: pair_launch_d<5>(a, form, n_sm, st); return true;
    case 6: pair_launch_d<6>(a, form, n_sm, st); return true;
    case 7: pair_launch_d<7>(a, form, n_sm, st); return true;
    case 8: pair_launch_d<8>(a, form, n_sm, st); return true;
    case 16: pair_launch_d<16>(a, form, n_sm, st); return true;
    default: return false;
    }
}

void lbc_init_attributes()
{
    coarse_attr_d<1>();
    coarse_attr_d<2>();
    coarse_attr_d<3>();
    coarse_attr_d<4>();
    coarse_attr_d<5>();
    coarse_attr_d<6>();
    coarse_attr_d<7>();
    coarse_attr_d<8>();
    coarse_attr_d<16>();
}

}  // namespace knn
