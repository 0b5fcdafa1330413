// Greedy upper bound (Section 4.1, Algorithm 1) and the threshold pre-pass of
// Section 4.3.
//
// One thread walks one (query, series) pair from cell (0,0): at (i,j) it
// steps to the cheapest of (i+1,j), (i+1,j+1), (i,j+1) (first minimum in
// that order; cells outside the matrix or the band cost +inf) until it
// reaches (m-1, n-1).  form 0 keeps the max of the squared costs (GDK^2, an
// upper bound of DK^2); form 1 keeps their sum (the cost of one admissible
// path, an upper bound of DTW).  The walk stops as soon as the running value
// exceeds the current k-th smallest bound of its query (the threshold eps of
// Algorithm 1), and a finished bound enters the query's k smallest; the k-th
// of those is a valid initial threshold for the exact scan, because each
// bound is at least the exact distance of its own series.
#include "common.cuh"
#include "internal.h"

namespace knn {

constexpr int GR_THREADS = 128;

template <int D, int FORM>
__global__ void __launch_bounds__(GR_THREADS) greedy_kernel(const GreedyArgs a)
{
    const int qb = blockIdx.y;
    const int m = a.q_len[qb];
    const float *qp = a.q + a.q_off[qb];
    unsigned long long *slots = a.ub_slots ? a.ub_slots + (size_t)qb * a.k : nullptr;
    unsigned long long st_walks = 0;

    for (int c = a.c_begin + blockIdx.x * blockDim.x + threadIdx.x; c < a.c_end;
         c += gridDim.x * blockDim.x) {
        const int n = a.db_len[c];
        const int r = band_radius(m, n, a.band);
        if (abs(m - n) > r) {
            if (a.out_ub)
                a.out_ub[(int64_t)qb * a.out_stride + c] = KNN_INF;
            continue;
        }
        ++st_walks;
        const float *xp = a.db + a.db_off[c];
        float eps = KNN_INF;
        if (slots) {
            const unsigned long long kth = ld_volatile_u64(slots + a.k - 1);
            if (kth != KNN_EMPTY_KEY)
                eps = key_dist(kth);
        }
        float qi[D], qn[D], xj[D], xn[D];
        load_point<D>(qp, qi);
        load_point<D>(qp + min(1, m - 1) * D, qn);
        load_point<D>(xp, xj);
        load_point<D>(xp + min(1, n - 1) * D, xn);
        int i = 0, j = 0;
        float g = sqdist_acc<D>(qi, xj, 0.f);
        int steps = 0;
        const int max_steps = m + n;  // a walk reaches (m-1, n-1) in at most m+n-2 steps
        while (g <= eps && !(i == m - 1 && j == n - 1) && steps < max_steps) {
            const bool can_i = i + 1 < m, can_j = j + 1 < n;
            const float c_dn = (can_i && abs(i + 1 - j) <= r) ? sqdist_acc<D>(qn, xj, 0.f) : KNN_INF;
            const float c_dg = (can_i && can_j) ? sqdist_acc<D>(qn, xn, 0.f) : KNN_INF;
            const float c_rt = (can_j && abs(i - j - 1) <= r) ? sqdist_acc<D>(qi, xn, 0.f) : KNN_INF;
            // first minimum in the order (i+1,j), (i+1,j+1), (i,j+1)
            float best = c_dn;
            int mv = 0;
            if (c_dg < best) { best = c_dg; mv = 1; }
            if (c_rt < best) { best = c_rt; mv = 2; }
            if (!(best < KNN_INF)) {  // no finite successor (cost overflow): no bound
                g = KNN_INF;
                break;
            }
            const bool mi = mv != 2, mj = mv != 0;
            i += mi;
            j += mj;
#pragma unroll
            for (int k = 0; k < D; ++k) {
                qi[k] = mi ? qn[k] : qi[k];
                xj[k] = mj ? xn[k] : xj[k];
            }
            if (mi)
                load_point<D>(qp + min(i + 1, m - 1) * D, qn);
            if (mj)
                load_point<D>(xp + min(j + 1, n - 1) * D, xn);
            g = FORM == 0 ? fmaxf(g, best) : g + best;
            ++steps;
            if (slots && ((steps & 31) == 0)) {
                const unsigned long long kth = ld_volatile_u64(slots + a.k - 1);
                if (kth != KNN_EMPTY_KEY)
                    eps = key_dist(kth);
            }
        }
        if (!(i == m - 1 && j == n - 1) && g <= eps)
            g = KNN_INF;  // stopped early without exceeding eps: no valid bound
        if (a.out_ub)
            a.out_ub[(int64_t)qb * a.out_stride + c] = g;
        if (slots && g <= eps && g < KNN_INF) {
            topk_insert(slots, a.k, make_key(g, (uint32_t)a.db_id[c]));
            const unsigned long long kth = ld_volatile_u64(slots + a.k - 1);
            if (kth != KNN_EMPTY_KEY && a.thr)
                atomic_min_pos_float(a.thr + qb, key_dist(kth));
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        st_walks += __shfl_xor_sync(KNN_FULL_MASK, st_walks, o);
    if ((threadIdx.x & 31) == 0 && a.stats)
        atomicAdd(a.stats + STAT_UB_WALKS, st_walks);
}

template <int D>
static void greedy_launch_d(const GreedyArgs &a, int form, cudaStream_t st)
{
    const int nser = a.c_end - a.c_begin;
    int bx = (nser + GR_THREADS - 1) / GR_THREADS;
    dim3 grid(bx > 0 ? bx : 1, a.nq);
    if (form == 0)
        greedy_kernel<D, 0><<<grid, GR_THREADS, 0, st>>>(a);
    else
        greedy_kernel<D, 1><<<grid, GR_THREADS, 0, st>>>(a);
}

void launch_greedy(const GreedyArgs &a, int d, int form, cudaStream_t st)
{
    switch (d) {
    case 1: greedy_launch_d<1>(a, form, st); break;
    case 2: greedy_launch_d<2>(a, form, st); break;
    case 3: greedy_launch_d<3>(a, form, st); break;
    case 4: greedy_launch_d<4>(a, form, st); break;
    case 5: greedy_launch_d<5>(a, form, st); break;
    case 6: greedy_launch_d<6>(a, form, st); break;
    case 7: greedy_launch_d<7>(a, form, st); break;
    case 8: greedy_launch_d<8>(a, form, st); break;
    case 16: greedy_launch_d<16>(a, form, st); break;
    default: break;
    }
}

}  // namespace knn
