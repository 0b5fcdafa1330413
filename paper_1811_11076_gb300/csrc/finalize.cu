// Result assembly: FP64 re-scoring of the boundary band, (distance, id) order,
// output; plus the FP64 pair program.
//
// The scan computes in FP32.  A candidate whose FP32 distance lies within
// the FP32 error band of the k-th distance (or of eps), or within that band of
// a neighbour inside the top k, could be ordered differently by exact
// arithmetic, so such candidates are re-scored by an FP64 dynamic program
// (Section 2.1 recurrences, no pruning) before the cut is taken.  Candidates
// outside the band are ordered correctly by their FP32 values already.
//
// Three launches: mark (sort, pick entries to re-score), rescore (one CTA per
// picked entry, band rows in shared memory), output (final order, cut).
#include "common.cuh"
#include "internal.h"

namespace knn {

constexpr int FIN_THREADS = 128;
// Threads that share one cell of the FP64 program (a power of two <= 32): four
// give the SM seven warps per CTA at d = 16 (eight measured 35 % slower: three
// shuffles per cell and half-empty FMA chains).
constexpr int FP64_TPC = 4;

// Banded DP in FP64 for one pair, computed by the threads of one CTA along
// anti-diagonals t = i + j: every cell of an anti-diagonal is independent,
// groups of FP64_TPC threads take the band diagonals delta = j - i of the
// right parity in strides of 2 * blockDim.x / FP64_TPC, and the two previous
// anti-diagonals live in shared memory (indexed by delta + r + 1, with an
// infinite sentinel on both sides).  Every in-band slot is rewritten on each
// anti-diagonal of its parity (with +inf outside the matrix) and slots of the
// other parity are never read, so the three rows rotate without clearing.
// kind 0: DTW (sum of squared costs); kind 1: DK^2 (max of squared costs).
// Each cell applies the operations of the recurrence in a fixed order (the
// difference of two FP32 coordinates is exact in double precision; thread q
// of the cell's group adds the squares of the coordinates k = q mod FP64_TPC
// with fused multiply-adds, and the group joins its partial sums pairwise by
// xor shuffles, neighbours first), so the value does not depend on the sweep
// order and agrees with a sequential double-precision evaluation to rounding
// (about 1e-15 relative per cell).  Shared memory: 3 * (2r + 3) doubles.
// Called by all threads of the CTA (a multiple of FP64_TPC); returns the
// value in every thread.
//
// stage != nullptr: the two series are first converted to double in shared
// memory (rows of d + 1 doubles, so the rows that the threads of an
// anti-diagonal read, one apart, fall in different banks), and every cell
// then costs one subtraction and one fused multiply-add per coordinate
// instead of two conversions more.  Same value either way.
__device__ double dp_fp64_cta(const float *s, int m, const float *t, int n, int d, int r,
                              int kind, double *buf, double *stage = nullptr)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    if (abs(m - n) > r)
        return (double)KNN_INF;
    const int W = 2 * r + 3;
    double *A = buf, *B = buf + W, *Cc = buf + 2 * W;  // t-2, t-1, t
    for (int b = tid; b < 3 * W; b += nt)
        buf[b] = (double)KNN_INF;
    const int ds = d + 1;
    double *ss = stage, *st = stage ? stage + (int64_t)m * ds : nullptr;
    if (stage) {
        for (int i = tid; i < m; i += nt)
            for (int k = 0; k < d; ++k)
                ss[i * ds + k] = (double)s[(int64_t)i * d + k];
        for (int j = tid; j < n; j += nt)
            for (int k = 0; k < d; ++k)
                st[j * ds + k] = (double)t[(int64_t)j * d + k];
    }
    __syncthreads();
    const int tmax = m + n - 2;
    // FP64_TPC threads per cell: thread q of a group sums the squares of the
    // coordinates k = q (mod FP64_TPC) (one FMA chain each), and the group
    // joins the partial sums pairwise, ((c0 + c1) + (c2 + c3)) + ..., by shuffles
    const int g = tid / FP64_TPC, ng = nt / FP64_TPC, q = tid % FP64_TPC;
    const unsigned gmask = (FP64_TPC == 32 ? 0xFFFFFFFFu : ((1u << FP64_TPC) - 1u))
                           << ((tid & 31) & ~(FP64_TPC - 1));
    for (int tt = 0; tt <= tmax; ++tt) {
        // diagonals delta in [-r, r] with delta = tt (mod 2)
        const int d0 = -r + (((tt + r) & 1) ? 1 : 0);
        for (int dl = d0 + 2 * g; dl <= r; dl += 2 * ng) {
            const int i2 = tt - dl, j2 = tt + dl;  // 2i, 2j
            const int i = i2 >> 1, j = j2 >> 1;
            const bool in = i >= 0 && i < m && j >= 0 && j < n;
            double c = 0.0;
            if (in) {
                if (stage) {
                    const double *si = ss + i * ds, *tj = st + j * ds;
                    for (int k = q; k < d; k += FP64_TPC) {
                        const double df = __dsub_rn(si[k], tj[k]);
                        c = __fma_rn(df, df, c);
                    }
                } else {
                    const float *sf = s + (int64_t)i * d, *tf = t + (int64_t)j * d;
                    for (int k = q; k < d; k += FP64_TPC) {
                        const double df = __dsub_rn((double)sf[k], (double)tf[k]);
                        c = __fma_rn(df, df, c);
                    }
                }
            }
#pragma unroll
            for (int o = 1; o < FP64_TPC; o <<= 1)
                c = __dadd_rn(c, __shfl_xor_sync(gmask, c, o));
            if (q != 0)
                continue;
            double v = (double)KNN_INF;
            if (in) {
                if (tt == 0) {
                    v = c;
                } else {
                    const int x = dl + r + 1;
                    const double best = fmin(fmin(B[x - 1], B[x + 1]), A[x]);
                    v = kind == 0 ? __dadd_rn(c, best) : fmax(c, best);
                }
            }
            Cc[dl + r + 1] = v;
        }
        __syncthreads();
        // rotate: the new t-2 is the old t-1
        double *old = A;
        A = B;
        B = Cc;
        Cc = old;
    }
    // the end cell (m-1, n-1) lies on anti-diagonal tmax, now in B
    return B[(n - m) + r + 1];
}

// Threads of the re-scoring CTA for band rows of `row` slots: about one
// diagonal of each parity per group of FP64_TPC threads.
static int fp64_threads(int row)
{
    const int half = (row + 1) / 2;
    int t = (FP64_TPC * half + 31) / 32 * 32;
    return t < 32 ? 32 : (t > 512 ? 512 : t);
}

// ---------------------------------------------------------------------------
// 1. mark: per query, sort (eps lists), pick entries to re-score

__global__ void __launch_bounds__(FIN_THREADS) fin_mark_kernel(const FinArgs a)
{
    extern __shared__ unsigned long long keys[];
    const int qb = blockIdx.x;
    const int tid = threadIdx.x;
    const bool knn_mode = a.k > 0;
    unsigned long long *src = knn_mode ? a.slots + (size_t)qb * a.kslots
                                       : a.eps_list + (size_t)qb * a.eps_cap;
    int cnt = knn_mode ? a.kslots : min(a.eps_count[qb], a.eps_cap);
    int p2 = 1;
    while (p2 < cnt)
        p2 <<= 1;
    if (p2 > a.sort_cap) {  // host sizes sort_cap >= every list; defensive
        if (tid == 0)
            atomicOr(a.status, KNN_DEV_BAD_SHAPE);
        return;
    }
    for (int i = tid; i < p2; i += blockDim.x)
        keys[i] = i < cnt ? src[i] : KNN_EMPTY_KEY;
    __syncthreads();
    if (!knn_mode) {
        for (int kk = 2; kk <= p2; kk <<= 1)
            for (int j = kk >> 1; j > 0; j >>= 1) {
                for (int i = tid; i < p2; i += blockDim.x) {
                    const int l = i ^ j;
                    if (l > i) {
                        const bool up = (i & kk) == 0;
                        const unsigned long long x = keys[i], y = keys[l];
                        if ((x > y) == up) {
                            keys[i] = y;
                            keys[l] = x;
                        }
                    }
                }
                __syncthreads();
            }
        for (int i = tid; i < cnt; i += blockDim.x)
            src[i] = keys[i];
    }
    __syncthreads();
    // number of real entries
    int valid = 0;
    for (int i = tid; i < cnt; i += blockDim.x)
        valid += keys[i] != KNN_EMPTY_KEY;
    for (int o = 16; o > 0; o >>= 1)
        valid += __shfl_xor_sync(KNN_FULL_MASK, valid, o);
    __shared__ int part[FIN_THREADS / 32];
    if ((tid & 31) == 0)
        part[tid >> 5] = valid;
    __syncthreads();
    if (tid == 0) {
        int t = 0;
        for (int w = 0; w < FIN_THREADS / 32; ++w)
            t += part[w];
        a.fin_valid[qb] = t;
    }
    __syncthreads();
    cnt = a.fin_valid[qb];

    const float w = a.rerank_rel;
    const float pivot = knn_mode ? (cnt >= a.k ? key_dist(keys[a.k - 1]) : KNN_INF) : a.eps_int;
    double *vals = a.fin_vals + (size_t)qb * a.fin_width;
    // k-NN: the cut can only move if a second entry shares the boundary band
    __shared__ int s_band;
    if (tid == 0)
        s_band = 0;
    __syncthreads();
    if (knn_mode && pivot < KNN_INF)
        for (int i = tid; i < cnt; i += blockDim.x) {
            const float di = key_dist(keys[i]);
            if (di >= pivot * (1.f - w) && di <= pivot * (1.f + w) && di != pivot)
                atomicAdd(&s_band, 1);
        }
    __syncthreads();
    const bool band_matters = !knn_mode || s_band > 0;
    for (int i = tid; i < cnt; i += blockDim.x) {
        const float di = key_dist(keys[i]);
        bool nd = band_matters && pivot < KNN_INF && di >= pivot * (1.f - w) &&
                  di <= pivot * (1.f + w);
        if (knn_mode && i <= a.k) {
            if (i > 0) {
                const float dp = key_dist(keys[i - 1]);
                nd |= di != dp && di <= dp * (1.f + w);
            }
            if (i + 1 < cnt) {
                const float dn = key_dist(keys[i + 1]);
                nd |= di != dn && dn <= di * (1.f + w);
            }
        }
        vals[i] = (double)di;
        if (nd) {
            const int pos = atomicAdd(a.rer_count, 1);
            if (pos < a.rer_cap)
                a.rer_list[pos] = make_int2(qb, i);
            else
                atomicOr(a.status, KNN_DEV_CAPACITY);
        }
    }
}

// ---------------------------------------------------------------------------
// 2. rescore: one CTA per picked entry

__global__ void __launch_bounds__(512) fin_rescore_kernel(const FinArgs a)
{
    extern __shared__ double rbuf[];
    const int n_rer = min(*a.rer_count, a.rer_cap);
    for (int e = blockIdx.x; e < n_rer; e += gridDim.x) {
        const int2 it = a.rer_list[e];
        const int qb = it.x, i = it.y;
        const unsigned long long key = a.k > 0 ? a.slots[(size_t)qb * a.kslots + i]
                                               : a.eps_list[(size_t)qb * a.eps_cap + i];
        const uint32_t id = key_id(key);
        const int m = a.q_len[qb];
        const int n = a.db_len_by_id[id];
        const int r = band_radius(m, n, a.band);
        if (2 * r + 1 > a.rer_row) {
            if (threadIdx.x == 0)
                atomicOr(a.status, KNN_DEV_BAD_SHAPE);
            continue;
        }
        // both series staged as doubles when they fit the launch's allotment
        double *stage = (int64_t)(m + n) <= (int64_t)a.stage_pts ? rbuf + 3 * (a.rer_row + 2)
                                                                 : nullptr;
        const double v = dp_fp64_cta(a.q + a.q_off[qb], m, a.db + a.db_off_by_id[id], n, a.d, r,
                                     a.kind, rbuf, stage);
        if (threadIdx.x == 0)
            a.fin_vals[(size_t)qb * a.fin_width + i] = v;
        __syncthreads();
    }
    if (blockIdx.x == 0 && threadIdx.x == 0 && a.stats)
        atomicAdd(a.stats + STAT_RERANKED, (unsigned long long)n_rer);
}

// ---------------------------------------------------------------------------
// 3. output: order by (value, id), exact eps test, cut, write

__global__ void __launch_bounds__(FIN_THREADS) fin_out_kernel(const FinArgs a)
{
    extern __shared__ unsigned long long keys[];
    double *val = reinterpret_cast<double *>(keys + a.sort_cap);
    const int qb = blockIdx.x;
    const int tid = threadIdx.x;
    const bool knn_mode = a.k > 0;
    const int cnt = a.fin_valid[qb];
    const unsigned long long *src = knn_mode ? a.slots + (size_t)qb * a.kslots
                                             : a.eps_list + (size_t)qb * a.eps_cap;
    const double *vals = a.fin_vals + (size_t)qb * a.fin_width;
    for (int i = tid; i < cnt; i += blockDim.x) {
        keys[i] = src[i];
        val[i] = vals[i];
    }
    __syncthreads();
    __shared__ int s_kept;
    if (tid == 0) {
        // entries arrive ordered by FP32 value; only re-scored ones move, so
        // an insertion sort does little work
        for (int i = 1; i < cnt; ++i) {
            const double v = val[i];
            const unsigned long long k = keys[i];
            int j = i - 1;
            while (j >= 0 && (val[j] > v || (val[j] == v && key_id(keys[j]) > key_id(k)))) {
                val[j + 1] = val[j];
                keys[j + 1] = keys[j];
                --j;
            }
            val[j + 1] = v;
            keys[j + 1] = k;
        }
        int kept = cnt;
        if (!knn_mode) {
            int o = 0;
            for (int i = 0; i < cnt; ++i)
                if (val[i] <= (double)a.eps_int) {
                    val[o] = val[i];
                    keys[o] = keys[i];
                    ++o;
                }
            kept = o;
        }
        s_kept = kept;
    }
    __syncthreads();
    const int kept = s_kept;
    const int width = a.out_width;
    const int lim = knn_mode ? min(kept, a.k) : kept;
    for (int i = tid; i < width; i += blockDim.x) {
        int64_t id = -1;
        float dist = KNN_INF;
        if (i < lim) {
            id = (int64_t)key_id(keys[i]);
            dist = a.kind == 0 ? (float)val[i] : (float)sqrt(val[i]);
        }
        a.out_ids[(size_t)qb * width + i] = id;
        a.out_dist[(size_t)qb * width + i] = dist;
    }
    if (tid == 0 && a.out_counts) {
        if (knn_mode) {
            a.out_counts[qb] = lim;
        } else {
            const int raw = a.eps_count[qb];
            // entries beyond capacity were never stored, so they could not be
            // re-checked in FP64; they are counted as found
            a.out_counts[qb] = raw > a.eps_cap ? raw - (cnt - kept) : kept;
            if (raw > a.eps_cap)
                atomicOr(a.status, KNN_DEV_CAPACITY);
        }
    }
}

// ---------------------------------------------------------------------------
// eps-NN lists longer than the shared-memory sort holds (eps_cap above
// FIN_SMALL_CAP): a merge sort in global memory (runs of FIN_RUN keys sorted
// in shared memory, then merge passes), a mark pass over the sorted list, the
// same FP64 re-scoring, and an output pass that re-orders only the tail of
// the list near eps.  Keys are (FP32 value bits, id), unique per query.

constexpr int FIN_RUN = 4096;           // keys per run sorted in shared memory
constexpr int FIN_RUN_THREADS = 512;
constexpr int FIN_MERGE_PER_THREAD = 8; // consecutive outputs per merge thread
constexpr int FIN_MERGE_THREADS = 256;
constexpr int FIN_MERGE_TILE = FIN_MERGE_PER_THREAD * FIN_MERGE_THREADS;
constexpr int FIN_TAIL_CAP = 8192;      // keys near eps re-ordered in shared memory

__device__ __forceinline__ int fin_list_len(const int *eps_count, int cap, int qb)
{
    return min(eps_count[qb], cap);
}

// Lower edge of the tail that may be re-ordered: FP32 values below it are
// more than the FP32 error band below every re-scored value.
__device__ __forceinline__ float fin_tail_lo(const FinArgs &a)
{
    return a.eps_int * (1.f - 2.f * a.rerank_rel);
}

__global__ void __launch_bounds__(FIN_RUN_THREADS) fin_run_sort_kernel(const FinArgs a)
{
    __shared__ unsigned long long keys[FIN_RUN];
    const int qb = blockIdx.x;
    const int cnt = fin_list_len(a.eps_count, a.eps_cap, qb);
    const int r0 = blockIdx.y * FIN_RUN;
    if (r0 >= cnt)
        return;
    const int len = min(FIN_RUN, cnt - r0);
    unsigned long long *src = a.eps_list + (size_t)qb * a.eps_cap + r0;
    for (int i = threadIdx.x; i < FIN_RUN; i += blockDim.x)
        keys[i] = i < len ? src[i] : KNN_EMPTY_KEY;
    __syncthreads();
    for (int kk = 2; kk <= FIN_RUN; kk <<= 1)
        for (int j = kk >> 1; j > 0; j >>= 1) {
            for (int i = threadIdx.x; i < FIN_RUN; i += blockDim.x) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & kk) == 0;
                    const unsigned long long x = keys[i], y = keys[l];
                    if ((x > y) == up) {
                        keys[i] = y;
                        keys[l] = x;
                    }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < len; i += blockDim.x)
        src[i] = keys[i];
}

// Number of keys taken from A among the first o keys of merge(A, B) (keys
// unique): the smallest i with A[i] > B[o - i - 1].
__device__ __forceinline__ int merge_corank(const unsigned long long *A, int la,
                                            const unsigned long long *B, int lb, int o)
{
    int lo = max(0, o - lb), hi = min(o, la);
    while (lo < hi) {
        const int i = (lo + hi) >> 1;
        if (A[i] < B[o - i - 1])
            lo = i + 1;
        else
            hi = i;
    }
    return lo;
}

// One merge pass: sorted runs of width w (the last one shorter) are merged
// pairwise from src into dst.  A thread writes FIN_MERGE_PER_THREAD
// consecutive outputs, which lie in one pair of runs because 2w is a
// multiple of that count.
__global__ void __launch_bounds__(FIN_MERGE_THREADS)
    fin_merge_kernel(const unsigned long long *__restrict__ src, unsigned long long *__restrict__ dst,
                     const int *__restrict__ eps_count, int cap, int w)
{
    const int qb = blockIdx.x;
    const int cnt = fin_list_len(eps_count, cap, qb);
    const int o0 = blockIdx.y * FIN_MERGE_TILE + threadIdx.x * FIN_MERGE_PER_THREAD;
    if (o0 >= cnt)
        return;
    const unsigned long long *s = src + (size_t)qb * cap;
    unsigned long long *d = dst + (size_t)qb * cap;
    const int base = o0 / (2 * w) * (2 * w);
    const int la = min(w, cnt - base);
    const int lb = max(0, min(w, cnt - base - w));
    const unsigned long long *A = s + base, *B = s + base + la;
    int i = merge_corank(A, la, B, lb, o0 - base);
    int j = o0 - base - i;
    const int end = min(o0 + FIN_MERGE_PER_THREAD, cnt);
    for (int o = o0; o < end; ++o) {
        const unsigned long long x = i < la ? A[i] : KNN_EMPTY_KEY;
        const unsigned long long y = j < lb ? B[j] : KNN_EMPTY_KEY;
        if (x < y) {
            d[o] = x;
            ++i;
        } else {
            d[o] = y;
            ++j;
        }
    }
}

// Mark the entries near eps for FP64 re-scoring; record the list length and
// the values of the tail.
__global__ void __launch_bounds__(FIN_THREADS) fin_big_mark_kernel(const FinArgs a)
{
    const int qb = blockIdx.x;
    const int cnt = fin_list_len(a.eps_count, a.eps_cap, qb);
    if (threadIdx.x == 0)
        a.fin_valid[qb] = cnt;
    const unsigned long long *keys = a.eps_list + (size_t)qb * a.eps_cap;
    double *vals = a.fin_vals + (size_t)qb * a.fin_width;
    const float w = a.rerank_rel, pivot = a.eps_int, lo = fin_tail_lo(a);
    for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
        const float di = key_dist(keys[i]);
        if (di < lo)
            continue;
        vals[i] = (double)di;
        if (di >= pivot * (1.f - w) && di <= pivot * (1.f + w)) {
            const int pos = atomicAdd(a.rer_count, 1);
            if (pos < a.rer_cap)
                a.rer_list[pos] = make_int2(qb, i);
            else
                atomicOr(a.status, KNN_DEV_CAPACITY);
        }
    }
}

// Output: the prefix below the tail is already in (value, id) order and is
// written as it stands; the tail is re-ordered by (FP64 value where
// re-scored, id) and cut at eps.
__global__ void __launch_bounds__(FIN_THREADS) fin_big_out_kernel(const FinArgs a)
{
    extern __shared__ unsigned long long tkeys[];
    double *tval = reinterpret_cast<double *>(tkeys + FIN_TAIL_CAP);
    const int qb = blockIdx.x, tid = threadIdx.x;
    const int cnt = a.fin_valid[qb];
    const unsigned long long *keys = a.eps_list + (size_t)qb * a.eps_cap;
    const double *vals = a.fin_vals + (size_t)qb * a.fin_width;
    __shared__ int s_b1, s_kept;
    if (tid == 0) {
        const float lo = fin_tail_lo(a);
        int l = 0, h = cnt;
        while (l < h) {
            const int mid = (l + h) >> 1;
            if (key_dist(keys[mid]) < lo)
                l = mid + 1;
            else
                h = mid;
        }
        s_b1 = l;
    }
    __syncthreads();
    const int b1 = s_b1, tail = cnt - b1;
    const int width = a.out_width;
    int64_t *oid = a.out_ids + (size_t)qb * width;
    float *odist = a.out_dist + (size_t)qb * width;
    if (tail > FIN_TAIL_CAP) {
        if (tid == 0)
            atomicOr(a.status, KNN_DEV_BAD_SHAPE);
        return;
    }
    for (int i = tid; i < b1; i += blockDim.x) {
        const unsigned long long key = keys[i];
        const float di = key_dist(key);
        oid[i] = (int64_t)key_id(key);
        odist[i] = a.kind == 0 ? di : (float)sqrt((double)di);
    }
    for (int i = tid; i < tail; i += blockDim.x) {
        tkeys[i] = keys[b1 + i];
        tval[i] = vals[b1 + i];
    }
    __syncthreads();
    if (tid == 0) {
        for (int i = 1; i < tail; ++i) {
            const double v = tval[i];
            const unsigned long long k = tkeys[i];
            int j = i - 1;
            while (j >= 0 && (tval[j] > v || (tval[j] == v && key_id(tkeys[j]) > key_id(k)))) {
                tval[j + 1] = tval[j];
                tkeys[j + 1] = tkeys[j];
                --j;
            }
            tval[j + 1] = v;
            tkeys[j + 1] = k;
        }
        int o = 0;
        for (int i = 0; i < tail; ++i)
            if (tval[i] <= (double)a.eps_int) {
                tval[o] = tval[i];
                tkeys[o] = tkeys[i];
                ++o;
            }
        s_kept = o;
    }
    __syncthreads();
    const int kept = b1 + s_kept;
    for (int i = b1 + tid; i < width; i += blockDim.x) {
        int64_t id = -1;
        float dist = KNN_INF;
        if (i < kept) {
            id = (int64_t)key_id(tkeys[i - b1]);
            dist = a.kind == 0 ? (float)tval[i - b1] : (float)sqrt(tval[i - b1]);
        }
        oid[i] = id;
        odist[i] = dist;
    }
    if (tid == 0 && a.out_counts) {
        const int raw = a.eps_count[qb];
        a.out_counts[qb] = raw > a.eps_cap ? raw - (cnt - kept) : kept;
        if (raw > a.eps_cap)
            atomicOr(a.status, KNN_DEV_CAPACITY);
    }
}

// Merge passes needed to sort a list of cap keys from runs of FIN_RUN.
static int fin_merge_passes(int cap)
{
    int passes = 0;
    for (int64_t w = FIN_RUN; w < cap; w *= 2)
        ++passes;
    return passes;
}

void fin_init_attributes()
{
    cudaFuncSetAttribute(fin_rescore_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    cudaFuncSetAttribute(fin_mark_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(fin_out_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(fin_big_out_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         FIN_TAIL_CAP * (sizeof(unsigned long long) + sizeof(double)));
}

int launch_finalize(const FinArgs &a, cudaStream_t st)
{
    const size_t smem_rer =
        ((size_t)3 * (a.rer_row + 2) + (size_t)a.stage_pts * (a.d + 1)) * sizeof(double);
    const int rer_grid = a.rer_cap < 4096 ? a.rer_cap : 4096;
    if (a.k == 0 && a.eps_cap > FIN_SMALL_CAP) {
        int launches = 0;
        // queries on x (up to 2^31 - 1), runs and tiles on y (<= 8192 at 2^24)
        const dim3 runs(a.nq, (a.eps_cap + FIN_RUN - 1) / FIN_RUN);
        fin_run_sort_kernel<<<runs, FIN_RUN_THREADS, 0, st>>>(a);
        ++launches;
        const int passes = fin_merge_passes(a.eps_cap);
        const dim3 tiles(a.nq, (a.eps_cap + FIN_MERGE_TILE - 1) / FIN_MERGE_TILE);
        unsigned long long *src = a.eps_list, *dst = a.eps_tmp;
        for (int p = 0, w = FIN_RUN; p < passes; ++p, w *= 2) {
            fin_merge_kernel<<<tiles, FIN_MERGE_THREADS, 0, st>>>(src, dst, a.eps_count,
                                                                   a.eps_cap, w);
            ++launches;
            unsigned long long *t = src;
            src = dst;
            dst = t;
        }
        if (src != a.eps_list)
            cudaMemcpyAsync(a.eps_list, src, sizeof(unsigned long long) * a.nq * (size_t)a.eps_cap,
                            cudaMemcpyDeviceToDevice, st);
        fin_big_mark_kernel<<<a.nq, FIN_THREADS, 0, st>>>(a);
        fin_rescore_kernel<<<rer_grid, fp64_threads(a.rer_row), smem_rer, st>>>(a);
        fin_big_out_kernel<<<a.nq, FIN_THREADS,
                             FIN_TAIL_CAP * (sizeof(unsigned long long) + sizeof(double)), st>>>(a);
        return launches + 3;
    }
    const size_t smem_mark = (size_t)a.sort_cap * sizeof(unsigned long long);
    const size_t smem_out = (size_t)a.sort_cap * (sizeof(unsigned long long) + sizeof(double));
    fin_mark_kernel<<<a.nq, FIN_THREADS, smem_mark, st>>>(a);
    fin_rescore_kernel<<<rer_grid, fp64_threads(a.rer_row), smem_rer, st>>>(a);
    fin_out_kernel<<<a.nq, FIN_THREADS, smem_out, st>>>(a);
    return 3;
}

// ---------------------------------------------------------------------------
// FP64 pair program: one 32-thread CTA per pair (many pairs run at once)

__global__ void __launch_bounds__(32) pairwise64_kernel(const float *a, const int64_t *a_off,
                                                        const float *b, const int64_t *b_off,
                                                        const int64_t *pa, const int64_t *pb,
                                                        int64_t n, int d, float band, int kind,
                                                        int row, double *out)
{
    extern __shared__ double pbuf[];
    for (int64_t p = blockIdx.x; p < n; p += gridDim.x) {
        const int64_t ia = pa[p], ib = pb[p];
        const int m = (int)(a_off[ia + 1] - a_off[ia]);
        const int nn = (int)(b_off[ib + 1] - b_off[ib]);
        const int r = band_radius(m, nn, band);
        double v = -1.0;
        if (2 * r + 1 <= row)
            v = dp_fp64_cta(a + a_off[ia] * d, m, b + b_off[ib] * d, nn, d, r, kind, pbuf);
        if (threadIdx.x == 0)
            out[p] = v < 0.0 ? v : (kind == 0 ? v : sqrt(v));
        __syncthreads();
    }
}

void launch_pairwise64(const float *a, const int64_t *a_off, const float *b, const int64_t *b_off,
                       const int64_t *pa, const int64_t *pb, int64_t n, int d, float band,
                       int kind, double *out, int row, cudaStream_t st)
{
    const size_t smem = (size_t)3 * (row + 2) * sizeof(double);
    cudaFuncSetAttribute(pairwise64_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         200 * 1024);
    const int blocks = (int)(n < 65536 ? n : 65536);
    pairwise64_kernel<<<blocks > 0 ? blocks : 1, 32, smem, st>>>(a, a_off, b, b_off, pa, pb, n,
                                                                 d, band, kind, row, out);
}

}  // namespace knn
