// Subsequence search: a query S of m points against every subsequence
// T[a..b] of one long series T of n points, no band (Section 4.2, Algorithm 3
// with SUB = true, for DK; the same free-start, free-end recursion for DTW),
// and the greedy upper bound of Algorithm 2.
//
// The free-start DP: row 0 of every column starts a match (its value is its
// own cost), rows above follow the DTW (sum) or DK (max) recursion of Section
// 2.1, and the result is the minimum of the last row over all columns, with
// its column (the end b of the best subsequence; the smallest on ties).
//
// Work mapping: one warp per query, a systolic array.  Lane L keeps P query
// rows in registers (rows L*P + e - off, e < P, off = 32P - m, so the last
// row sits at lane 31, slot P-1); the rows below row 0 are virtual, held at
// value 0, which gives row 0 its zero predecessor (the free start).  Step t computes anti-diagonal t: cell e of a lane is (i, t - i), so
// the P cells are independent; a cell needs its own row and the row below at
// step t-1 and the row below at step t-2 (one shuffle each at the lane edge).
// The series streams through: each step a lane loads the one column it sees
// first, held with the others it needs in a ring of P points.  T is copied
// with sentinel points (1e18) on both sides, so cells before the start or
// after the end cost about 1e36 per coordinate and never win.  Cells whose
// value exceeds the caller's threshold are capped just above it: values only
// grow along a path, so such a cell cannot lead to a result within it (for DK
// this is Algorithm 3's sparse visit of the cells of cost <= eps); a result
// above the threshold is reported as +inf.
#include <algorithm>
#include <cmath>
#include <vector>

#include "common.cuh"
#include "runtime.h"

using namespace knn;

namespace {

constexpr int SUB_THREADS = 128;       // four queries per CTA
constexpr int SUB_KC_MAX = 32;         // candidate ends kept per query (k + max(8, k))
constexpr int SUB_KMAX = 16;           // largest k of the k best ends
constexpr int SUB_PMAX = 32;
constexpr int SUB_PAD = 32 * SUB_PMAX + SUB_PMAX + 8;  // sentinel points on each side

struct SubArgs {
    const float *q;           // repacked queries, deff floats per point
    const int64_t *q_off;     // float offset of each query
    const int *q_len;
    const int *q_idx;         // the queries of this launch (one P class)
    int nq;
    const float *t;           // padded series: point k at t + (k + SUB_PAD) * deff
    int64_t n;
    float eps2;               // threshold on cell values (DTW sum, or DK squared)
    int kind;
    float *out;               // greedy: [n_queries] the bound (Euclidean)
    int64_t *out_end;
    int kc;                   // DP: candidate ends kept per query
    float *cand_val;          // DP: [n_queries][kc] FP32 last-row values, ascending
    int64_t *cand_end;        //     and their end columns (-1: none)
    double *val64;            // [n_queries][kc] FP64 values of the candidates
    int k;                    // ends reported per query
    float *out_k;             // [n_queries][k] values (DTW sum, or DK Euclidean)
    int64_t *end_k;           // [n_queries][k] ends (-1: none)
    int *status;              // bit 1: a re-scored match reached the span limit
};

// FP64 re-scoring: the candidate's value may be off by the FP32 rounding of
// a path; it is recomputed in double precision (exact differences of the
// FP32 coordinates, each square added by one fused multiply-add, coordinates
// in order) for every path whose
// value is at most T = v32 (1 + SUB_MARGIN).  A path from start column a to
// end b crosses every column in between and so costs at least the sum (DTW)
// or the max (DK) over those columns of the column's least cell cost; the
// walk back from b stops where that exceeds T, which bounds the first start
// column a0, and the free-start recursion runs over columns [a0, b] only.
constexpr double SUB_MARGIN = 1e-3;
// Candidates re-scored: those within this relative distance of the k-th
// best FP32 value (the FP32 value of a path of L cells is within about
// L * 2^-24 of the exact one; 2e-4 covers paths of some thousands of cells),
// always including the k best.
constexpr float SUB_SELECT = 2e-4f;
constexpr int64_t SUB_SPAN_MAX = 65536;   // columns a re-scored match may span
constexpr int SUB_RS_THREADS = 128;

template <int D, int P, int KIND>
__global__ void __launch_bounds__(SUB_THREADS) subseq_kernel(const SubArgs a)
{
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= a.nq)
        return;  // whole warps only
    const int qi = a.q_idx[warp];
    const int m = a.q_len[qi];
    const int off = 32 * P - m;
    const int base = lane * P - off;  // row of slot 0
    const float *qp = a.q + a.q_off[qi];

    // cap: a cell's value is min(value, cap).  Virtual rows: 0 (values are
    // >= 0, so they stay 0).  Real rows: the float just above the threshold,
    // so a cell above it stays above it, and so does every path through it
    // (values only grow along a path), while values within it are unchanged.
    float qv[P][D], cap[P], cur[P], prv[P];
    const float capv = a.eps2 < KNN_INF ? nextafterf(a.eps2, KNN_INF) : KNN_INF;
#pragma unroll
    for (int e = 0; e < P; ++e) {
        const int i = base + e;
        cap[e] = i >= 0 ? capv : 0.f;
        load_point<D>(qp + (int64_t)(i >= 0 ? i : 0) * D, qv[e]);
        cur[e] = prv[e] = i >= 0 ? KNN_INF : 0.f;
    }
    // ring: the column of cell e at step t is t - base - e, kept in slot
    // (t - e) mod P; fill the slots for steps before 0
    const float *tp = a.t + (int64_t)SUB_PAD * D;
    float xw[P][D];
#pragma unroll
    for (int p = 1; p < P; ++p)
        load_point<D>(tp + (int64_t)(-p - base) * D, xw[P - p]);

    // lane 31 keeps the kc lowest (value, end) pairs of the last row so far,
    // ascending (equal values: the earlier end first), in shared memory; a
    // value enters if it is within eps and below the kc-th kept
    __shared__ float cv_s[SUB_THREADS / 32][SUB_KC_MAX];
    __shared__ long long ce_s[SUB_THREADS / 32][SUB_KC_MAX];
    const int wl = threadIdx.x >> 5;
    const int kc = a.kc;
    const float enter = a.eps2 < KNN_INF ? capv : 1e30f;  // sentinel cells cost ~1e36
    float bound = enter;
    int cnt = 0;
    const int64_t steps = a.n + m - 1;
    for (int64_t t0 = 0; t0 < steps; t0 += P) {
        float lastv[P];  // lane 31: the last row at each step of the block
#pragma unroll
        for (int u = 0; u < P; ++u) {
            const int64_t t = t0 + u;
            load_point<D>(tp + (t - base) * D, xw[u]);
            // the lane below: its top row at steps t-1 and t-2; below lane 0
            // the virtual rows are 0
            float up1 = __shfl_up_sync(KNN_FULL_MASK, cur[P - 1], 1);
            float up2 = __shfl_up_sync(KNN_FULL_MASK, prv[P - 1], 1);
            if (lane == 0)
                up1 = up2 = 0.f;
#pragma unroll
            for (int e = P - 1; e >= 0; --e) {
                const float left = cur[e];
                const float up = e > 0 ? cur[e - 1] : up1;
                const float dg = e > 0 ? prv[e - 1] : up2;
                const float mn = fmin3(left, up, dg);
                const float c = sqdist_acc<D>(qv[e], xw[(u - e + P) % P], 0.f);
                const float v = fminf(KIND == 0 ? c + mn : fmaxf(c, mn), cap[e]);
                prv[e] = cur[e];
                cur[e] = v;
            }
            lastv[u] = cur[P - 1];
        }
        // lane 31, slot P-1 holds the last row, at column t - (m - 1): the
        // block's values enter the list outside the unrolled steps, and only
        // when one of them beats the list (rare once the list is full)
        float bmin = lastv[0];
#pragma unroll
        for (int u = 1; u < P; ++u)
            bmin = fminf(bmin, lastv[u]);
        if (lane == 31 && bmin < bound) {
#pragma unroll
            for (int u = 0; u < P; ++u) {
                const int64_t k = t0 + u - (m - 1);
                const float v = lastv[u];
                if (k >= 0 && k < a.n && v < bound) {
                    int j = cnt < kc ? cnt : kc - 1;
                    while (j > 0 && cv_s[wl][j - 1] > v) {
                        cv_s[wl][j] = cv_s[wl][j - 1];
                        ce_s[wl][j] = ce_s[wl][j - 1];
                        --j;
                    }
                    cv_s[wl][j] = v;
                    ce_s[wl][j] = k;
                    cnt = cnt < kc ? cnt + 1 : kc;
                    bound = cnt == kc ? cv_s[wl][kc - 1] : enter;
                }
            }
        }
    }
    if (lane == 31)
        for (int j = 0; j < kc; ++j) {
            a.cand_val[(int64_t)qi * kc + j] = j < cnt ? cv_s[wl][j] : KNN_INF;
            a.cand_end[(int64_t)qi * kc + j] = j < cnt ? ce_s[wl][j] : -1;
        }
}

// Algorithm 2: the column closest to s_0 (warp-wide argmin, the first on
// ties), then the greedy walk by lane 0 until the last row is reached.
template <int D>
__global__ void __launch_bounds__(SUB_THREADS) subseq_greedy_kernel(const SubArgs a)
{
    const int warp = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (warp >= a.nq)
        return;
    const int qi = a.q_idx[warp];
    const int m = a.q_len[qi];
    const float *qp = a.q + a.q_off[qi];
    const float *tp = a.t + (int64_t)SUB_PAD * D;
    float s0[D];
    load_point<D>(qp, s0);
    float bc = KNN_INF;
    int64_t bj = -1;
    for (int64_t j = lane; j < a.n; j += 32) {
        float x[D];
        load_point<D>(tp + j * D, x);
        const float c = sqdist_acc<D>(s0, x, 0.f);
        if (c < bc) {
            bc = c;
            bj = j;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float oc = __shfl_xor_sync(KNN_FULL_MASK, bc, o);
        const int64_t oj = __shfl_xor_sync(KNN_FULL_MASK, bj, o);
        if (oc < bc || (oc == bc && oj >= 0 && (bj < 0 || oj < bj))) {
            bc = oc;
            bj = oj;
        }
    }
    if (lane != 0)
        return;
    float g = bc;  // squared costs; one square root at the end
    int64_t i = 0, j = bj;
    const float lim = a.eps2;
    while (i != m - 1 && g <= lim) {
        float si[D], sn[D], xj[D], xn[D];
        load_point<D>(qp + (int64_t)i * D, si);
        load_point<D>(qp + (int64_t)(i + 1) * D, sn);
        load_point<D>(tp + j * D, xj);
        const bool more = j + 1 < a.n;
        load_point<D>(tp + (more ? j + 1 : j) * D, xn);
        const float c_up = sqdist_acc<D>(sn, xj, 0.f);
        const float c_diag = more ? sqdist_acc<D>(sn, xn, 0.f) : KNN_INF;
        const float c_right = more ? sqdist_acc<D>(si, xn, 0.f) : KNN_INF;
        float c = c_up;
        int64_t ni = i + 1, nj = j;
        if (c_diag < c) {
            c = c_diag;
            nj = j + 1;
        }
        if (c_right < c) {
            c = c_right;
            ni = i;
            nj = j + 1;
        }
        i = ni;
        j = nj;
        g = fmaxf(g, c);
    }
    a.out[qi] = sqrtf(g);
    a.out_end[qi] = (i == m - 1 && g <= lim) ? j : -1;
}

template <int D>
__device__ __forceinline__ double cost64(const float *x, const float *y)
{
    double c = 0.0;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const double df = __dsub_rn((double)x[k], (double)y[k]);
        c = __fma_rn(df, df, c);
    }
    return c;
}

// One CTA per (candidate, query): the start bound a0, then the free-start
// recursion over columns [a0, b] by anti-diagonals (a thread per row, three
// diagonals in shared memory); writes the value of end b.
template <int D>
__global__ void __launch_bounds__(SUB_RS_THREADS) subseq_rescore_kernel(const SubArgs a)
{
    extern __shared__ double rs[];  // [3][m] anti-diagonals, then [blockDim] column minima
    const int qi = blockIdx.y, tid = threadIdx.x;
    const int64_t slot = (int64_t)qi * a.kc + blockIdx.x;
    const int64_t b = a.cand_end[slot];
    if (b < 0) {
        if (tid == 0)
            a.val64[slot] = (double)KNN_INF;
        return;
    }
    // only candidates that can be among the k best after re-scoring
    const float kth = a.cand_val[(int64_t)qi * a.kc + min(a.k, a.kc) - 1];
    if (blockIdx.x >= a.k && !(a.cand_val[slot] <= kth * (1.f + 2.f * SUB_SELECT))) {
        if (tid == 0)
            a.val64[slot] = (double)KNN_INF;
        return;
    }
    const int m = a.q_len[qi];
    const float *qp = a.q + a.q_off[qi];
    const float *tp = a.t + (int64_t)SUB_PAD * D;
    const double T = (double)a.cand_val[slot] * (1.0 + SUB_MARGIN);
    // column minima in FP32, lowered by their rounding bound ((D + 4) u)
    const double low = 1.0 - (D + 4) * (1.0 / 16777216.0);
    double *colmin = rs + 3 * m;
    __shared__ long long s_a0;
    __shared__ int s_done;
    if (tid == 0) {
        s_a0 = 0;
        s_done = 0;
    }
    double acc = 0.0;  // thread 0: sum of column minima from b back
    for (int64_t jb = b;; jb -= blockDim.x) {
        const int64_t j = jb - tid;
        float cm = KNN_INF;
        if (j >= 0) {
            float y[D];
            load_point<D>(tp + j * D, y);
            for (int i = 0; i < m; ++i) {
                float x[D];
                load_point<D>(qp + (int64_t)i * D, x);
                cm = fminf(cm, sqdist_acc<D>(x, y, 0.f));
            }
        }
        colmin[tid] = (double)cm * low;
        __syncthreads();
        if (tid == 0)
            for (int u = 0; u < (int)blockDim.x && !s_done; ++u) {
                const int64_t jj = jb - u;
                if (jj < 0) {
                    s_a0 = 0;
                    s_done = 1;
                } else if (a.kind == 0 ? (acc = __dadd_rn(acc, colmin[u])) > T : colmin[u] > T) {
                    s_a0 = jj + 1;
                    s_done = 1;
                } else if (b - jj + 1 >= SUB_SPAN_MAX) {
                    s_a0 = jj;
                    s_done = 1;
                    atomicOr(a.status, 1);
                }
            }
        __syncthreads();
        if (s_done)
            break;
    }
    const int64_t a0 = s_a0;
    const int L = (int)(b - a0 + 1);
    double *A = rs, *B = rs + m, *Cn = rs + 2 * m;  // diagonals t-2, t-1, t
    for (int tt = 0; tt <= m + L - 2; ++tt) {
        const int ilo = max(0, tt - L + 1), ihi = min(m - 1, tt);
        for (int i = ilo + tid; i <= ihi; i += blockDim.x) {
            const int jj = tt - i;
            const double c = cost64<D>(qp + (int64_t)i * D, tp + (a0 + jj) * D);
            double pred = 0.0;  // row 0: a match may start in any column
            if (i > 0) {
                const double left = jj >= 1 ? B[i] : (double)KNN_INF;
                const double dg = jj >= 1 ? A[i - 1] : (double)KNN_INF;
                pred = fmin(fmin(left, B[i - 1]), dg);
            }
            Cn[i] = a.kind == 0 ? __dadd_rn(c, pred) : fmax(c, pred);
        }
        __syncthreads();
        double *o = A;
        A = B;
        B = Cn;
        Cn = o;
    }
    if (tid == 0)
        a.val64[slot] = B[m - 1];  // end cell (m-1, b) on the last diagonal
}

// The k best ends of each query by (FP64 value, end), within eps; one warp
// per query (lane 0 orders the kc candidates).
__global__ void subseq_out_kernel(const SubArgs a, int nq)
{
    const int qi = (int)((blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5);
    if (qi >= nq || (threadIdx.x & 31) != 0)
        return;
    double v[SUB_KC_MAX];
    long long e[SUB_KC_MAX];
    int cnt = 0;
    const double lim = (double)a.eps2;
    for (int j = 0; j < a.kc; ++j) {
        const int64_t slot = (int64_t)qi * a.kc + j;
        const double x = a.val64[slot];
        const long long ex = a.cand_end[slot];
        if (ex < 0 || !(x <= lim) || !(x < 1e30))
            continue;
        int p = cnt++;
        while (p > 0 && (v[p - 1] > x || (v[p - 1] == x && e[p - 1] > ex))) {
            v[p] = v[p - 1];
            e[p] = e[p - 1];
            --p;
        }
        v[p] = x;
        e[p] = ex;
    }
    for (int j = 0; j < a.k; ++j) {
        a.out_k[(int64_t)qi * a.k + j] =
            j < cnt ? (a.kind == 0 ? (float)v[j] : (float)sqrt(v[j])) : KNN_INF;
        a.end_k[(int64_t)qi * a.k + j] = j < cnt ? e[j] : -1;
    }
}

template <int D>
void sub_rescore_d(const SubArgs &a, int nq, int max_m, cudaStream_t st)
{
    const size_t smem = (size_t)(3 * max_m + SUB_RS_THREADS) * sizeof(double);
    subseq_rescore_kernel<D><<<dim3(a.kc, nq), SUB_RS_THREADS, smem, st>>>(a);
}

void sub_rescore(const SubArgs &a, int deff, int nq, int max_m, cudaStream_t st)
{
    switch (deff) {
    case 1: sub_rescore_d<1>(a, nq, max_m, st); break;
    case 2: sub_rescore_d<2>(a, nq, max_m, st); break;
    case 3: sub_rescore_d<3>(a, nq, max_m, st); break;
    case 4: sub_rescore_d<4>(a, nq, max_m, st); break;
    case 5: sub_rescore_d<5>(a, nq, max_m, st); break;
    case 6: sub_rescore_d<6>(a, nq, max_m, st); break;
    case 7: sub_rescore_d<7>(a, nq, max_m, st); break;
    case 8: sub_rescore_d<8>(a, nq, max_m, st); break;
    case 16: sub_rescore_d<16>(a, nq, max_m, st); break;
    default: break;
    }
    subseq_out_kernel<<<(nq * 32 + 127) / 128, 128, 0, st>>>(a, nq);
}

// Compiled P per width: registers hold 2 P D + 3 P floats.
int sub_pmax(int deff) { return deff == 1 ? 32 : deff <= 3 ? 16 : deff <= 8 ? 8 : 4; }

template <int D, int P>
void sub_launch_p(const SubArgs &a, cudaStream_t st)
{
    const int blocks = (a.nq * 32 + SUB_THREADS - 1) / SUB_THREADS;
    if (a.kind == 0)
        subseq_kernel<D, P, 0><<<blocks, SUB_THREADS, 0, st>>>(a);
    else
        subseq_kernel<D, P, 1><<<blocks, SUB_THREADS, 0, st>>>(a);
}

template <int D>
void sub_launch_d(const SubArgs &a, int P, bool greedy, cudaStream_t st)
{
    if (greedy) {
        const int blocks = (a.nq * 32 + SUB_THREADS - 1) / SUB_THREADS;
        subseq_greedy_kernel<D><<<blocks, SUB_THREADS, 0, st>>>(a);
        return;
    }
    if constexpr (D == 1) {
        if (P == 32)
            return sub_launch_p<D, 32>(a, st);
    }
    if constexpr (D <= 3) {
        if (P == 16)
            return sub_launch_p<D, 16>(a, st);
    }
    if constexpr (D <= 8) {
        if (P == 8)
            return sub_launch_p<D, 8>(a, st);
    }
    sub_launch_p<D, 4>(a, st);
}

void sub_launch(const SubArgs &a, int deff, int P, bool greedy, cudaStream_t st)
{
    switch (deff) {
    case 1: sub_launch_d<1>(a, P, greedy, st); break;
    case 2: sub_launch_d<2>(a, P, greedy, st); break;
    case 3: sub_launch_d<3>(a, P, greedy, st); break;
    case 4: sub_launch_d<4>(a, P, greedy, st); break;
    case 5: sub_launch_d<5>(a, P, greedy, st); break;
    case 6: sub_launch_d<6>(a, P, greedy, st); break;
    case 7: sub_launch_d<7>(a, P, greedy, st); break;
    case 8: sub_launch_d<8>(a, P, greedy, st); break;
    case 16: sub_launch_d<16>(a, P, greedy, st); break;
    default: break;
    }
}

__global__ void sub_pad_kernel(const float *src, int64_t n, int d, int deff, float *dst)
{
    const int64_t total = (n + 2 * (int64_t)SUB_PAD) * deff;
    for (int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; f < total;
         f += (int64_t)gridDim.x * blockDim.x) {
        const int64_t k = f / deff - SUB_PAD;
        const int j = (int)(f % deff);
        float v;
        if (k < 0 || k >= n)
            v = KNN_DP_SENTINEL;
        else
            v = j < d ? src[k * d + j] : 0.f;
        dst[f] = v;
    }
}

knn_status sub_common(const float *queries, const int64_t *q_offsets, int32_t n_queries,
                      const float *series, int64_t n, int32_t d, int32_t distance, int32_t k,
                      float eps, float *out_dist, int64_t *out_end, void *stream, bool greedy)
{
    if (!queries || !q_offsets || !series || !out_dist || !out_end)
        return set_error(KNN_ERR_INVALID, "NULL argument");
    if (n_queries < 1 || n < 1 || d < 1 || d > 16)
        return set_error(KNN_ERR_INVALID, "need n_queries >= 1, n >= 1, 1 <= d <= 16");
    if (!greedy && distance != KNN_DTW && distance != KNN_DK)
        return set_error(KNN_ERR_INVALID, "distance must be KNN_DTW or KNN_DK");
    if (!(eps >= 0.f))
        return set_error(KNN_ERR_INVALID, "eps must be >= 0 (or +inf)");
    if (!greedy && (k < 1 || k > SUB_KMAX))
        return set_error(KNN_ERR_INVALID, "k must be in [1, 16]");
    if (greedy)
        k = 1;
    const int kc = k + std::max(8, k);
    if (n > ((int64_t)1 << 40))
        return set_error(KNN_ERR_INVALID, "series too long");
    const int deff = deff_for(d);
    cudaStream_t st = (cudaStream_t)stream;
    // query metadata on the host
    std::vector<int64_t> hq(n_queries + 1);
    if (is_device_ptr(q_offsets))
        cudaMemcpy(hq.data(), q_offsets, 8 * (n_queries + 1), cudaMemcpyDeviceToHost);
    else
        std::copy(q_offsets, q_offsets + n_queries + 1, hq.begin());
    if (hq[0] != 0)
        return set_error(KNN_ERR_INVALID, "q_offsets[0] must be 0");
    const int pmax = sub_pmax(deff);
    std::vector<int> len(n_queries), pclass(n_queries);
    std::vector<int64_t> qoff(n_queries);
    int64_t qfloats = 0;
    int max_m = 1;
    for (int i = 0; i < n_queries; ++i) {
        const int64_t m = hq[i + 1] - hq[i];
        if (m < 1)
            return set_error(KNN_ERR_INVALID, "every query needs >= 1 point");
        if (!greedy && m > 32 * pmax)
            return set_error(KNN_ERR_UNSUPPORTED,
                             "query longer than 32 * P_max points for this d (1024 for d = 1, "
                             "512 for d = 2, 3, 256 for 4..8, 128 for 9..16)");
        len[i] = (int)m;
        max_m = std::max(max_m, (int)m);
        int P = 4;
        while (32 * P < m)
            P *= 2;
        pclass[i] = P;
        qoff[i] = qfloats;
        qfloats += (m + 3) / 4 * 4 * deff;
    }
    // device copies: queries (deff floats per point), padded series
    DevBuf qraw, qsrc, qbuf, qo, ql, qidx, traw, tpad, flag;
    knn_status s;
    const int64_t qpts = hq[n_queries];
    const float *qdev = queries;
    if (!is_device_ptr(queries)) {
        if ((s = qraw.ensure(sizeof(float) * qpts * d)))
            return s;
        cudaMemcpyAsync(qraw.p, queries, sizeof(float) * qpts * d, cudaMemcpyHostToDevice, st);
        qdev = qraw.as<float>();
    }
    const float *tdev = series;
    if (!is_device_ptr(series)) {
        if ((s = traw.ensure(sizeof(float) * n * d)))
            return s;
        cudaMemcpyAsync(traw.p, series, sizeof(float) * n * d, cudaMemcpyHostToDevice, st);
        tdev = traw.as<float>();
    }
    if ((s = flag.ensure(sizeof(int))) || (s = qsrc.ensure(8 * (n_queries + 1))) ||
        (s = qbuf.ensure(sizeof(float) * std::max<int64_t>(qfloats, 4))) ||
        (s = qo.ensure(8 * n_queries)) || (s = ql.ensure(4 * n_queries)) ||
        (s = qidx.ensure(4 * n_queries)) ||
        (s = tpad.ensure(sizeof(float) * (n + 2 * (int64_t)SUB_PAD) * deff)))
        return s;
    bool ok = true;
    if ((s = check_finite_dev(qdev, qpts * d, flag.as<int>(), st, &ok)))
        return s;
    if (ok && (s = check_finite_dev(tdev, n * d, flag.as<int>(), st, &ok)))
        return s;
    if (!ok)
        return set_error(KNN_ERR_INVALID, "input contains NaN or Inf");
    cudaMemcpyAsync(qsrc.p, hq.data(), 8 * (n_queries + 1), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(qo.p, qoff.data(), 8 * n_queries, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(ql.p, len.data(), 4 * n_queries, cudaMemcpyHostToDevice, st);
    launch_repack(qdev, qsrc.as<int64_t>(), nullptr, n_queries, d, deff, qo.as<int64_t>(),
                  qbuf.as<float>(), st, false);
    {
        const int64_t total = (n + 2 * (int64_t)SUB_PAD) * deff;
        const int blocks = (int)std::min<int64_t>((total + 255) / 256, 8192);
        sub_pad_kernel<<<blocks, 256, 0, st>>>(tdev, n, d, deff, tpad.as<float>());
    }
    // one launch per P class (queries of similar length)
    std::vector<int> order(n_queries);
    for (int i = 0; i < n_queries; ++i)
        order[i] = i;
    std::stable_sort(order.begin(), order.end(),
                     [&](int x, int y) { return pclass[x] < pclass[y]; });
    cudaMemcpyAsync(qidx.p, order.data(), 4 * n_queries, cudaMemcpyHostToDevice, st);
    DevBuf odev, edev, cval, cend, v64, stat;
    float *out_d = out_dist;
    int64_t *out_e = out_end;
    const int64_t nout = (int64_t)n_queries * k;
    const bool host_out = !is_device_ptr(out_dist) || !is_device_ptr(out_end);
    if (host_out) {
        if ((s = odev.ensure(4 * nout)) || (s = edev.ensure(8 * nout)))
            return s;
        out_d = odev.as<float>();
        out_e = edev.as<int64_t>();
    }
    if (!greedy) {
        const int64_t nc = (int64_t)n_queries * kc;
        if ((s = cval.ensure(4 * nc)) || (s = cend.ensure(8 * nc)) || (s = v64.ensure(8 * nc)) ||
            (s = stat.ensure(sizeof(int))))
            return s;
        cudaMemsetAsync(stat.p, 0, sizeof(int), st);
        if ((size_t)(3 * max_m + SUB_RS_THREADS) * sizeof(double) > 48 * 1024)
            return set_error(KNN_ERR_UNSUPPORTED, "query too long for FP64 re-scoring");
    }
    SubArgs a{};
    a.q = qbuf.as<float>();
    a.q_off = qo.as<int64_t>();
    a.q_len = ql.as<int>();
    a.t = tpad.as<float>();
    a.n = n;
    a.eps2 = std::isinf(eps) ? KNN_INF_HOST : (distance == KNN_DTW && !greedy ? eps : eps * eps);
    a.kind = distance;
    a.out = out_d;
    a.out_end = out_e;
    a.kc = kc;
    a.cand_val = cval.as<float>();
    a.cand_end = cend.as<int64_t>();
    a.val64 = v64.as<double>();
    a.k = k;
    a.out_k = out_d;
    a.end_k = out_e;
    a.status = stat.as<int>();
    for (int b = 0; b < n_queries;) {
        int e = b;
        while (e < n_queries && (greedy || pclass[order[e]] == pclass[order[b]]))
            ++e;
        a.q_idx = qidx.as<int>() + b;
        a.nq = e - b;
        sub_launch(a, deff, pclass[order[b]], greedy, st);
        b = e;
    }
    if (!greedy)
        sub_rescore(a, deff, n_queries, max_m, st);
    if (host_out) {
        cudaMemcpyAsync(out_dist, out_d, 4 * nout, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(out_end, out_e, 8 * nout, cudaMemcpyDeviceToHost, st);
    }
    int span = 0;
    if (!greedy)
        cudaMemcpyAsync(&span, stat.p, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess)
        e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_error(e, "subsequence search");
    if (span)
        return set_error(KNN_ERR_UNSUPPORTED,
                         "a best match may span more than 65,536 columns of the series: exact "
                         "re-scoring is not supported there");
    return KNN_OK;
}

}  // namespace

extern "C" knn_status knn_subseq(const float *queries, const int64_t *q_offsets, int32_t n_queries,
                                 const float *series, int64_t n, int32_t d, int32_t distance,
                                 float eps, float *out_dist, int64_t *out_end, void *stream)
{
    return sub_common(queries, q_offsets, n_queries, series, n, d, distance, 1, eps, out_dist,
                      out_end, stream, false);
}

extern "C" knn_status knn_subseq_k(const float *queries, const int64_t *q_offsets,
                                   int32_t n_queries, const float *series, int64_t n, int32_t d,
                                   int32_t distance, int32_t k, float eps, float *out_dist,
                                   int64_t *out_end, void *stream)
{
    return sub_common(queries, q_offsets, n_queries, series, n, d, distance, k, eps, out_dist,
                      out_end, stream, false);
}

extern "C" knn_status knn_subseq_greedy(const float *queries, const int64_t *q_offsets,
                                        int32_t n_queries, const float *series, int64_t n,
                                        int32_t d, float eps, float *out_ub, int64_t *out_end,
                                        void *stream)
{
    return sub_common(queries, q_offsets, n_queries, series, n, d, KNN_DK, 1, eps, out_ub, out_end,
                      stream, true);
}
