// Seed selection and survivor filtering for the seeded scan.
//
// A seeded scan computes LB_Box for every (query, series) pair first, picks
// per query the S series with the lowest score (the bound itself, or a
// learned predicted distance), scores those exactly, and only then filters
// the remaining pairs against the now tight threshold (the k-th best exact
// distance among the seeds, which bounds the final k-th distance from above
// because the seeds are k distinct series).  Any subset of series is a valid
// seed set, so the selection only has to be cheap, not exact.
#include "common.cuh"
#include "internal.h"

namespace knn {

constexpr int SEL_THREADS = 512;
constexpr int SEL_BINS = 4096;  // histogram over the top 12 bits of a non-negative float

// One block per query.  Picks at most S series with finite score and
// finite bound, appends them to the seed queue and marks their bound
// negative so that the filter skips them.
__global__ void __launch_bounds__(SEL_THREADS) select_kernel(const SelArgs a)
{
    __shared__ unsigned int hist[SEL_BINS];
    __shared__ int s_bin, s_before, s_taken, s_count;
    const int q = blockIdx.x;
    const float *score = a.score + (int64_t)q * a.score_stride;
    const int *cand = a.cand ? a.cand + (int64_t)q * a.score_stride : nullptr;
    float *lb = a.lb_all ? a.lb_all + (int64_t)q * a.lb_stride : nullptr;
    const int m = a.lb_all ? 0 : a.q_len[q];
    // a series can be a seed if its end cell is inside the band
    auto series = [&](int c) -> int { return cand ? cand[c] : a.c_base + c; };
    auto feasible = [&](int c) -> bool {
        if (lb)
            return lb[c] < KNN_INF;
        const int sidx = series(c);
        if (sidx < 0)
            return false;
        const int n = a.db_len[sidx];
        return abs(m - n) <= band_radius(m, n, a.band);
    };
    for (int i = threadIdx.x; i < SEL_BINS; i += blockDim.x)
        hist[i] = 0;
    if (threadIdx.x == 0) {
        s_taken = 0;
        s_count = 0;
    }
    __syncthreads();
    for (int c = threadIdx.x; c < a.n; c += blockDim.x) {
        const float s = score[c];
        if (s < KNN_INF && feasible(c))
            atomicAdd(&hist[__float_as_uint(fmaxf(s, 0.f)) >> 20], 1u);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned int cum = 0;
        int b = 0;
        for (; b < SEL_BINS; ++b) {
            if (cum + hist[b] >= (unsigned)a.S)
                break;
            cum += hist[b];
        }
        s_bin = b;  // SEL_BINS if fewer than S candidates exist: take all
        s_before = (int)cum;
    }
    __syncthreads();
    const int bin = s_bin, quota = a.S - s_before;
    for (int c = threadIdx.x; c < a.n; c += blockDim.x) {
        const float s = score[c];
        if (!(s < KNN_INF) || !feasible(c))
            continue;
        const int sb = (int)(__float_as_uint(fmaxf(s, 0.f)) >> 20);
        bool take = sb < bin;
        if (sb == bin)
            take = atomicAdd(&s_taken, 1) < quota;
        if (take) {
            const int pos = atomicAdd(a.n_seed, 1);
            if (pos < a.seed_cap) {
                const int sidx = series(c);
                a.seed_items[pos] = make_int2(sidx, q);
                a.seed_lb[pos] = lb ? lb[c] : 0.f;
                if (lb)
                    lb[c] = -1.f;  // scored as a seed; the filter skips it
                if (a.seed_bits)   // scored as a seed; the LB_Box stream skips it
                    atomicOr(a.seed_bits + (int64_t)q * a.bits_words + (sidx >> 5),
                             1u << (sidx & 31));
                atomicAdd(&s_count, 1);
            } else {
                atomicOr(a.status, KNN_DEV_CAPACITY);
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && a.stats)
        atomicAdd(a.stats + STAT_SEEDS, (unsigned long long)s_count);
}

void launch_select(const SelArgs &a, cudaStream_t st)
{
    select_kernel<<<a.nq, SEL_THREADS, 0, st>>>(a);
}

// Filter: grid (x: series of the bucket, y: queries).  Keeps pairs whose bound
// is not above the (seeded) threshold; bounds of seeds are negative.
__global__ void __launch_bounds__(256) filter_kernel(const FilterArgs a)
{
    const int q = blockIdx.y;
    const int lane = threadIdx.x & 31;
    const float lim = ld_volatile_f32(a.thr + q) * a.mu_prune;
    const float *lb = a.lb_all + (int64_t)q * a.lb_stride;
    unsigned long long pruned = 0;
    const int nser = a.c_end - a.c_begin;
    const int span = (nser + 31) / 32 * 32;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < span; i += gridDim.x * blockDim.x) {
        const int c = a.c_begin + i;
        bool keep = false;
        float v = 0.f;
        if (i < nser) {
            v = lb[c];
            const bool feasible = v >= 0.f && v < KNN_INF;
            keep = feasible && v <= lim;
            pruned += feasible && !keep;
        }
        const unsigned kb = __ballot_sync(KNN_FULL_MASK, keep);
        if (kb) {
            int base = 0;
            if (lane == 0)
                base = atomicAdd(a.n_items, __popc(kb));
            base = __shfl_sync(KNN_FULL_MASK, base, 0);
            if (keep) {
                const int64_t pos = (int64_t)base + __popc(kb & ((1u << lane) - 1u));
                if (pos < a.capacity) {
                    a.items[pos] = make_int2(c, q);
                    a.item_lb[pos] = v;
                } else {
                    atomicOr(a.status, KNN_DEV_CAPACITY);
                }
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1)
        pruned += __shfl_xor_sync(KNN_FULL_MASK, pruned, o);
    if (lane == 0 && a.stats && pruned)
        atomicAdd(a.stats + STAT_LB_PRUNED, pruned);
}

void launch_filter(const FilterArgs &a, int n_sm, cudaStream_t st)
{
    const int nser = a.c_end - a.c_begin;
    int bx = (nser + 255) / 256;
    const int cap = (n_sm * 8 + a.nq - 1) / a.nq;
    if (bx > cap)
        bx = cap;
    if (bx < 1)
        bx = 1;
    filter_kernel<<<dim3(bx, a.nq), 256, 0, st>>>(a);
}

}  // namespace knn
