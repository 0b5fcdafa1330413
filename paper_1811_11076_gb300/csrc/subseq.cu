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
    float *out;               // [n_queries] DTW sum, or DK (Euclidean)
    int64_t *out_end;
};

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

    float best = KNN_INF;
    int64_t best_k = -1;
    const int64_t steps = a.n + m - 1;
    for (int64_t t0 = 0; t0 < steps; t0 += P) {
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
            // lane 31, slot P-1 holds the last row, at column t - (m - 1)
            const int64_t k = t - (m - 1);
            if (k >= 0 && k < a.n && cur[P - 1] < best) {
                best = cur[P - 1];
                best_k = k;
            }
        }
    }
    if (lane == 31) {
        const bool found = best <= a.eps2 && best < 1e30f;
        a.out[qi] = found ? (KIND == 0 ? best : sqrtf(best)) : KNN_INF;
        a.out_end[qi] = found ? best_k : -1;
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
                      const float *series, int64_t n, int32_t d, int32_t distance, float eps,
                      float *out_dist, int64_t *out_end, void *stream, bool greedy)
{
    if (!queries || !q_offsets || !series || !out_dist || !out_end)
        return set_error(KNN_ERR_INVALID, "NULL argument");
    if (n_queries < 1 || n < 1 || d < 1 || d > 16)
        return set_error(KNN_ERR_INVALID, "need n_queries >= 1, n >= 1, 1 <= d <= 16");
    if (!greedy && distance != KNN_DTW && distance != KNN_DK)
        return set_error(KNN_ERR_INVALID, "distance must be KNN_DTW or KNN_DK");
    if (!(eps >= 0.f))
        return set_error(KNN_ERR_INVALID, "eps must be >= 0 (or +inf)");
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
    for (int i = 0; i < n_queries; ++i) {
        const int64_t m = hq[i + 1] - hq[i];
        if (m < 1)
            return set_error(KNN_ERR_INVALID, "every query needs >= 1 point");
        if (!greedy && m > 32 * pmax)
            return set_error(KNN_ERR_UNSUPPORTED,
                             "query longer than 32 * P_max points for this d (1024 for d = 1, "
                             "512 for d = 2, 3, 256 for 4..8, 128 for 9..16)");
        len[i] = (int)m;
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
    DevBuf odev, edev;
    float *out_d = out_dist;
    int64_t *out_e = out_end;
    const bool host_out = !is_device_ptr(out_dist) || !is_device_ptr(out_end);
    if (host_out) {
        if ((s = odev.ensure(4 * n_queries)) || (s = edev.ensure(8 * n_queries)))
            return s;
        out_d = odev.as<float>();
        out_e = edev.as<int64_t>();
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
    for (int b = 0; b < n_queries;) {
        int e = b;
        while (e < n_queries && (greedy || pclass[order[e]] == pclass[order[b]]))
            ++e;
        a.q_idx = qidx.as<int>() + b;
        a.nq = e - b;
        sub_launch(a, deff, pclass[order[b]], greedy, st);
        b = e;
    }
    if (host_out) {
        cudaMemcpyAsync(out_dist, out_d, 4 * n_queries, cudaMemcpyDeviceToHost, st);
        cudaMemcpyAsync(out_end, out_e, 8 * n_queries, cudaMemcpyDeviceToHost, st);
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess)
        e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_error(e, "subsequence search");
    return KNN_OK;
}

}  // namespace

extern "C" knn_status knn_subseq(const float *queries, const int64_t *q_offsets, int32_t n_queries,
                                 const float *series, int64_t n, int32_t d, int32_t distance,
                                 float eps, float *out_dist, int64_t *out_end, void *stream)
{
    return sub_common(queries, q_offsets, n_queries, series, n, d, distance, eps, out_dist,
                      out_end, stream, false);
}

extern "C" knn_status knn_subseq_greedy(const float *queries, const int64_t *q_offsets,
                                        int32_t n_queries, const float *series, int64_t n,
                                        int32_t d, float eps, float *out_ub, int64_t *out_end,
                                        void *stream)
{
    return sub_common(queries, q_offsets, n_queries, series, n, d, KNN_DK, eps, out_ub, out_end,
                      stream, true);
}
