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
// Three launches: mark (sort, pick entries to re-score), rescore (one thread
// per picked entry, band rows in global scratch), output (final order, cut).
#include "common.cuh"
#include "internal.h"

namespace knn {

constexpr int FIN_THREADS = 128;

// Banded DP in FP64 for one pair, row by row; rows are band offsets
// b = j - i + r in [0, 2r].  kind 0: DTW (sum of squared costs); kind 1: DK^2
// (max of squared costs).  Products and sums are rounded separately (no
// fused multiply-add) and coordinates are accumulated in order, exactly as
// a plain double-precision evaluation of the definition does.
__device__ double dp_fp64(const float *s, int m, const float *t, int n, int d, int r, int kind,
                          double *prev, double *cur)
{
    if (abs(m - n) > r)
        return (double)KNN_INF;
    const int W = 2 * r + 1;
    for (int b = 0; b < W; ++b)
        prev[b] = (double)KNN_INF;
    for (int i = 0; i < m; ++i) {
        for (int b = 0; b < W; ++b) {
            const int j = i + b - r;
            if (j < 0 || j >= n) {
                cur[b] = (double)KNN_INF;
                continue;
            }
            double c = 0.0;
            for (int k = 0; k < d; ++k) {
                const double df =
                    __dsub_rn((double)s[(int64_t)i * d + k], (double)t[(int64_t)j * d + k]);
                c = __dadd_rn(c, __dmul_rn(df, df));
            }
            double v;
            if (i == 0 && j == 0) {
                v = c;
            } else {
                const double left = b > 0 ? cur[b - 1] : (double)KNN_INF;      // (i, j-1)
                const double low = b + 1 < W ? prev[b + 1] : (double)KNN_INF;  // (i-1, j)
                const double diag = prev[b];                                    // (i-1, j-1)
                const double best = fmin(fmin(left, low), diag);
                v = kind == 0 ? __dadd_rn(c, best) : fmax(c, best);
            }
            cur[b] = v;
        }
        double *tmp = prev;
        prev = cur;
        cur = tmp;
    }
    return prev[(n - 1) - (m - 1) + r];
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
    for (int i = tid; i < cnt; i += blockDim.x) {
        const float di = key_dist(keys[i]);
        bool nd = pivot < KNN_INF && di >= pivot * (1.f - w) && di <= pivot * (1.f + w);
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
// 2. rescore: one thread per picked entry

__global__ void fin_rescore_kernel(const FinArgs a)
{
    const int n_rer = min(*a.rer_count, a.rer_cap);
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n_rer; e += gridDim.x * blockDim.x) {
        const int2 it = a.rer_list[e];
        const int qb = it.x, i = it.y;
        const unsigned long long key = a.k > 0 ? a.slots[(size_t)qb * a.kslots + i]
                                               : a.eps_list[(size_t)qb * a.eps_cap + i];
        const uint32_t id = key_id(key);
        const int m = a.q_len[qb];
        const int n = a.db_len_by_id[id];
        const int r = band_radius(m, n, a.band);
        if (2 * r + 1 > a.rer_row) {
            atomicOr(a.status, KNN_DEV_BAD_SHAPE);
            continue;
        }
        double *rows = a.rer_scratch + (size_t)e * 2 * a.rer_row;
        const double v = dp_fp64(a.q + a.q_off[qb], m, a.db + a.db_off_by_id[id], n, a.d, r,
                                 a.kind, rows, rows + a.rer_row);
        a.fin_vals[(size_t)qb * a.fin_width + i] = v;
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

void fin_init_attributes()
{
    cudaFuncSetAttribute(fin_mark_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    cudaFuncSetAttribute(fin_out_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
}

void launch_finalize(const FinArgs &a, cudaStream_t st)
{
    const size_t smem_mark = (size_t)a.sort_cap * sizeof(unsigned long long);
    const size_t smem_out = (size_t)a.sort_cap * (sizeof(unsigned long long) + sizeof(double));
    fin_mark_kernel<<<a.nq, FIN_THREADS, smem_mark, st>>>(a);
    fin_rescore_kernel<<<64, 64, 0, st>>>(a);
    fin_out_kernel<<<a.nq, FIN_THREADS, smem_out, st>>>(a);
}

// ---------------------------------------------------------------------------
// FP64 pair program (thread per pair), band rows in global scratch

__global__ void pairwise64_kernel(const float *a, const int64_t *a_off, const float *b,
                                  const int64_t *b_off, const int64_t *pa, const int64_t *pb,
                                  int64_t n, int d, float band, int kind, double *out,
                                  double *scratch, int row)
{
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t tid = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double *rows = scratch + tid * 2 * row;
    for (int64_t p = tid; p < n; p += stride) {
        const int64_t ia = pa[p], ib = pb[p];
        const int m = (int)(a_off[ia + 1] - a_off[ia]);
        const int nn = (int)(b_off[ib + 1] - b_off[ib]);
        const int r = band_radius(m, nn, band);
        if (2 * r + 1 > row) {
            out[p] = -1.0;
            continue;
        }
        const double v = dp_fp64(a + a_off[ia] * d, m, b + b_off[ib] * d, nn, d, r, kind, rows,
                                 rows + row);
        out[p] = kind == 0 ? v : sqrt(v);
    }
}

void launch_pairwise64(const float *a, const int64_t *a_off, const float *b, const int64_t *b_off,
                       const int64_t *pa, const int64_t *pb, int64_t n, int d, float band,
                       int kind, double *out, double *scratch, int row, int threads_total,
                       cudaStream_t st)
{
    const int tpb = 64;
    const int blocks = threads_total / tpb;
    pairwise64_kernel<<<blocks, tpb, 0, st>>>(a, a_off, b, b_off, pa, pb, n, d, band, kind, out,
                                              scratch, row);
}

}  // namespace knn
