// Banded DTW / DK dynamic program over a queue of (query, series) pairs.
//
// Recurrences (Section 2.1; band of Section 2.2), 0-based cells (i, j) with
// |i - j| <= r:
//   DTW: D(i,j) = c(i,j) + min(D(i-1,j), D(i,j-1), D(i-1,j-1)),
//        c = ||q_i - x_j||^2
//   DK:  D(i,j) = max(c(i,j), min(...)) on squared costs; DK = sqrt(D(m-1,n-1))
// (sqrt is monotone, so max/min commute with it exactly).
//
// Work mapping.  A group of G lanes owns one (query, series) pair; a warp
// holds 32/G groups.  Lane lam of a group owns the 2P consecutive band
// diagonals delta = j - i in [lo + 2P*lam, lo + 2P*(lam+1)), lo even and
// <= -r, so G*P >= r+1 lanes-slots cover the band.  Cells are swept by
// anti-diagonals t = i + j; a "step" s computes t = 2s (even diagonals) and
// then t = 2s+1 (odd diagonals).  On one anti-diagonal every cell is
// independent, and a cell needs only its two neighbouring diagonals from
// t-1 (one of them possibly in the adjacent lane: one shuffle per
// anti-diagonal) and its own diagonal from t-2.  So a lane does P
// independent cells per anti-diagonal with no serial chain.
//
// The query rows and series columns a lane touches slide by one per step: a
// ring of U = P+1 points each, refreshed by one load per step, indexed with
// compile-time positions inside a U-times unrolled step loop.  Cells outside
// the band get +inf through the FMA accumulator of their cost (mask 0/inf).
//
// Start and end.  Every pair is swept in whole blocks of U steps, and the
// sweep starts at a step s_start in (-U, 0] chosen so that the end cell
// (m-1, n-1) falls on the last step of a block; the result is then read once
// per block, outside the unrolled loop.  The steps before 0 run over a
// virtual prefix: rows i < 0 and columns j < 0 read a sentinel point of huge
// coordinates, so a cell with both indices negative costs exactly 0 and a
// cell with one negative index costs about 1e36 (or +inf).  The two
// anti-diagonals before the first step start as 0 where both indices are
// negative and +inf elsewhere, so cell (0,0) receives min(...) = 0 from
// (-1,-1) and every real cell receives the same value as in the plain
// recurrence (the prefix can only reach it through (0,0)).
//
// Early abandoning (Section 4, first paragraph; Algorithm 3's empty active
// set for DK): the last two anti-diagonals form a cut of every warping path,
// and costs are non-negative, so their minimum bounds D(m-1,n-1) from below.
// Every U steps the group compares that minimum with the live threshold of
// its query and gives up if it is exceeded.  For DK this is the sparse DK of
// Algorithm 3: a cell above the threshold can never lead to a result below
// it, so the pair is dropped as soon as no cell of the cut is below.
#pragma once

#include "common.cuh"
#include "internal.h"

namespace knn {

constexpr int DP_THREADS = 128;
// WIN kernels: steps between the asynchronous copy of a window piece and its
// first read (the copy's latency hides behind that many steps)
constexpr int DP_WIN_AHEAD = 2;
// Point idx of a series, clamped to [-1, last]: index -1 is the sentinel
// point stored in the chunk before every series and query the DP reads.
template <int D>
__device__ __forceinline__ void load_point_prefix(const float *p, int idx, int last,
                                                  float (&v)[D])
{
    load_point<D>(p + clampi(idx, -1, last) * D, v);
}

// Squared distance of two wide points on packed FP32 pairs: two interleaved
// partial sums (even and odd coordinates), each an FMA chain, joined at the
// end and added to `init` (0, or +inf for an out-of-band slot).  Half the
// instructions of the scalar chain and half its dependent length; the sum has
// at most D/2 + 2 roundings per term, within the (d + 2) u bound.  (Starting
// the even chain at `init` instead saves an add but measured 2.5 % slower at
// d = 16: the scheduler lost more than the instruction.)
template <int D>
__device__ __forceinline__ float sqdist_acc_p2(const float (&a)[D], const float (&b)[D], float init)
{
    static_assert(D % 2 == 0, "pairs of coordinates");
    float2 acc = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < D; k += 2) {
        const float2 t = sub2(make_float2(a[k], a[k + 1]), make_float2(b[k], b[k + 1]));
        acc = __ffma2_rn(t, t, acc);
    }
    return (acc.x + acc.y) + init;
}

// Point cost of the DP: packed pairs from d = 8 on.
template <int D>
__device__ __forceinline__ float dp_cost(const float (&a)[D], const float (&b)[D], float init)
{
    if constexpr (D >= 8 && D % 2 == 0)
        return sqdist_acc_p2<D>(a, b, init);
    else
        return sqdist_acc<D>(a, b, init);
}

// 16-byte asynchronous copy global -> shared (both addresses 16-byte aligned),
// and the wait for every copy this thread has issued.
__device__ __forceinline__ void cp_async16(float *dst_smem, const float *src)
{
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst_smem));
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.wait_all;" ::: "memory");
}
__device__ __forceinline__ void cp_async_commit()
{
    asm volatile("cp.async.commit_group;" ::: "memory");
}
// Wait until at most N of this thread's committed groups are still pending.
template <int N>
__device__ __forceinline__ void cp_async_wait_group()
{
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Rows of the shared-memory window of one lane group (WIN kernels), a power
// of two: the (G-1)P + 1 rows the group's lanes read in one step, the
// DP_WIN_AHEAD rows whose copies are in flight, and one more, so that a copy
// issued in step s never lands on a row that a lane may still read in step
// s - 1 (lanes of a warp meet only at each step's __syncwarp).
__host__ __device__ constexpr int dp_win_rows(int G, int P)
{
    int w = 1;
    while (w < (G - 1) * P + 2 + DP_WIN_AHEAD)
        w <<= 1;
    return w;
}
// Slot of row r (any integer, taken modulo W) in a window: rows P apart sit in
// adjacent slots, so the G lanes of a group, which read rows P apart, hit
// consecutive slots, and with a row stride of an odd number of 16-byte units
// eight such float4 reads fall in distinct bank quads.
template <int P>
__device__ __forceinline__ int dp_win_slot(int r, int wp_mask)
{
    constexpr int LP = (P == 1) ? 0 : (P == 2) ? 1 : (P == 4) ? 2 : (P == 8) ? 3 : 4;
    static_assert((1 << LP) == P, "window path needs P a power of two");
    return (r & (P - 1)) * (wp_mask + 1) + ((r >> LP) & wp_mask);
}
// WIN kernels: the group's newest query row (t - h_0) and series column
// (t + h_{G-1} + P) of step t come in 2*(D/4) float4 pieces, one per lane
// lam < 2*(D/4) (G >= 8 and D <= 16, so a group has lanes enough), copied
// global -> shared asynchronously into their window slots.
template <int D, int P>
__device__ __forceinline__ void dp_win_copy(float *qwin, float *xwin, int wp_mask,
                                            const float *qp, const float *xp, int m, int n,
                                            int lam, int h0, int hT, int t)
{
    constexpr int C = D / 4, RS = D + 4;
    const bool isx = lam >= C;
    const int c = isx ? lam - C : lam;
    const int idx = isx ? t + hT + P : t - h0;
    float *dst = (isx ? xwin : qwin) + dp_win_slot<P>(idx, wp_mask) * RS + 4 * c;
    const float *src = isx ? xp + (int64_t)clampi(idx, -1, n - 1) * D
                           : qp + (int64_t)clampi(idx, -1, m - 1) * D;
    cp_async16(dst, src + 4 * c);
}
// Dynamic shared memory of a WIN kernel CTA: per warp, 32/G groups of two
// windows of dp_win_rows(G, P) rows, the most over the group sizes 8, 16, 32
// (one allocation per kernel whatever G a launch uses).
__host__ __device__ constexpr size_t dp_win_bytes(int D, int P)
{
    size_t rows = 0;
    for (int G = 8; G <= 32; G *= 2) {
        const size_t r = (size_t)(32 / G) * dp_win_rows(G, P);
        rows = r > rows ? r : rows;
    }
    return (size_t)(DP_THREADS / 32) * 2 * rows * (D + 4) * sizeof(float);
}

template <int D, int P, int KIND, bool WIN>
__global__ void __launch_bounds__(DP_THREADS) dp_kernel(const DpArgs a)
{
    constexpr int U = P + 1;
    constexpr int RS = D + 4;  // window row stride in floats (16-byte aligned)
    const int lane = threadIdx.x & 31;
    const int G = a.G;
    const int lam = lane & (G - 1);
    const int gbase = lane & ~(G - 1);
    const unsigned lt_mask = (1u << gbase) - 1u;
    // WIN: the group's windows of the last W query rows and series columns
    extern __shared__ __align__(16) float dwin[];
    const int W = WIN ? dp_win_rows(G, P) : P;
    const int wp_mask = W / P - 1;
    float *qwin = dwin + (size_t)(((threadIdx.x >> 5) * (32 / G) + (lane / G)) * 2 * W) * RS;
    float *xwin = qwin + (size_t)W * RS;
    // WIN: the lanes that copy each step's pieces, and the group's lane mask
    const bool win_loader = WIN && lam < 2 * (D / 4);
    const unsigned grp_mask = G == 32 ? KNN_FULL_MASK : ((1u << G) - 1u) << gbase;

    float qw[U][D], xw[U][D];
    float E[P], O[P], mE[P], mO[P];
#pragma unroll
    for (int e = 0; e < P; ++e) {
        E[e] = O[e] = KNN_INF;
        mE[e] = mO[e] = KNN_INF;
    }
#pragma unroll
    for (int p = 0; p < U; ++p)
#pragma unroll
        for (int k = 0; k < D; ++k) qw[p][k] = xw[p][k] = 0.f;

    const float *qp = a.q;
    const float *xp = a.db;
    int m = 1, n = 1, h = 0, r = 0;
    int s_f = -1, fin_lane = 0, fin_slot = 0, fin_odd = 0;
    int qi = 0, ci = 0, cur_idx = 0;
    bool active = false, done = false;
    int s0 = 0;

    // queue items are taken one per group of the warp per atomic: a pair
    // can run for a long time (long series, high d), so larger grabs would
    // leave a long tail of warps working through their private surplus
    const int grab = 32 / G;
    int wbase = 0, wcur = grab;
    const int n_items = (int)min((int64_t)*a.n_items, a.items_cap);

    unsigned long long st_calls = 0, st_aband = 0, st_cells = 0, st_pruned = 0;

    for (;;) {
        // ---- hand out work to groups that need it (warp-converged) ---------
        for (;;) {
            const bool need = !active && !done;
            const unsigned needy = __ballot_sync(KNN_FULL_MASK, need && lam == 0);
            if (needy == 0)
                break;
            if (wcur >= grab) {
                int b = 0;
                if (lane == 0)
                    b = atomicAdd(a.head, grab);
                wbase = __shfl_sync(KNN_FULL_MASK, b, 0);
                wcur = 0;
            }
            const int avail = grab - wcur;
            const int rank = __popc(needy & lt_mask);
            const int served = min(__popc(needy), avail);
            if (need && rank < avail) {
                const int idx = wbase + wcur + rank;
                if (idx >= n_items) {
                    done = true;
                } else {
                    const int2 it = a.items[idx];
                    const float lb = a.item_lb[idx];
                    const float thr = a.out_pair ? KNN_INF : ld_volatile_f32(a.thr + it.y);
                    const int mm = a.q_len[it.y], nn = a.db_len[it.x];
                    if (abs(mm - nn) > band_radius(mm, nn, a.band)) {
                        // end cell outside the band: distance +inf, nothing to run
                        if (a.out_pair && lam == 0)
                            a.out_pair[idx] = KNN_INF;
                    } else if (lb > thr * a.mu_prune) {
                        st_pruned += (lam == 0);
                    } else {
                        ci = it.x;
                        qi = it.y;
                        cur_idx = idx;
                        m = a.q_len[qi];
                        qp = a.q + a.q_off[qi];
                        n = a.db_len[ci];
                        xp = a.db + a.db_off[ci];
                        r = band_radius(m, n, a.band);
                        const int lo = -(r + (r & 1));
                        h = lo / 2 + P * lam;
                        s_f = (m + n - 2) >> 1;
                        // a whole number of U-step blocks from s0 <= 0 up to s_f
                        const int nsteps = (s_f + 1 + U - 1) / U * U;
                        s0 = s_f - nsteps + 1;
                        // state before step s0: anti-diagonals 2s0-2 (E) and
                        // 2s0-1 (O), all cells with i + j < 0; a cell with both
                        // indices negative is 0, one with a single negative
                        // index (or outside the band) +inf
#pragma unroll
                        for (int e = 0; e < P; ++e) {
                            const int de = lo + 2 * P * lam + 2 * e;
                            mE[e] = (abs(de) <= r) ? 0.f : KNN_INF;
                            mO[e] = (abs(de + 1) <= r) ? 0.f : KNN_INF;
                            const int te = 2 * s0 - 2, to = 2 * s0 - 1;
                            const bool ze = te - de < 0 && te + de < 0;       // 2i, 2j < 0
                            const bool zo = to - de - 1 < 0 && to + de + 1 < 0;
                            E[e] = ze ? mE[e] : KNN_INF;
                            O[e] = zo ? mO[e] : KNN_INF;
                        }
                        const int off = (n - m) - lo;
                        fin_lane = off / (2 * P);
                        fin_slot = (off % (2 * P)) >> 1;
                        fin_odd = off & 1;
#pragma unroll
                        for (int p = 0; p < U; ++p) {
                            load_point_prefix<D>(qp, s0 - h - ((U - p) % U), m - 1, qw[p]);
                            load_point_prefix<D>(xp, s0 + h + p, n - 1, xw[p]);
                        }
                        if constexpr (WIN) {
                            // copies of the previous pair still in flight land
                            // before any lane of the group refills the window
                            cp_async_wait_all();
                            __syncwarp(grp_mask);
                            // the (G-1)P rows and columns before the first step's
                            // newest, in float4 pieces spread over the group, copied
                            // global -> shared asynchronously (no registers, all
                            // copies in flight at once), then the pieces of the
                            // first DP_WIN_AHEAD steps, one commit group each; the
                            // step loop waits for them and its __syncwarp
                            // publishes them to the group
                            const int h0 = lo / 2, hT = lo / 2 + P * (G - 1);
                            const int nf = (G - 1) * P * (D / 4);
                            for (int t = lam; t < nf; t += G) {
                                const int k = t / (D / 4), c = t - k * (D / 4);
                                const int rq = s0 - h0 - (G - 1) * P + k;
                                const int cx = s0 + h0 + P + k;
                                cp_async16(qwin + dp_win_slot<P>(rq, wp_mask) * RS + 4 * c,
                                           qp + (int64_t)clampi(rq, -1, m - 1) * D + 4 * c);
                                cp_async16(xwin + dp_win_slot<P>(cx, wp_mask) * RS + 4 * c,
                                           xp + (int64_t)clampi(cx, -1, n - 1) * D + 4 * c);
                            }
                            cp_async_commit();
#pragma unroll
                            for (int t = 0; t < DP_WIN_AHEAD; ++t) {
                                if (win_loader)
                                    dp_win_copy<D, P>(qwin, xwin, wp_mask, qp, xp, m, n, lam,
                                                      h0, hT, s0 + t);
                                cp_async_commit();
                            }
                        }
                        active = true;
                        st_calls += (lam == 0);
                    }
                }
            }
            wcur += served;
        }
        if (__all_sync(KNN_FULL_MASK, done))
            break;
        // the threshold of this block's abandon test, read now so that the
        // load's latency hides behind the block's steps: thresholds only fall,
        // so a value one block old is still a valid (looser) bound, and the
        // top-k insert keeps the exact k best whatever it is offered
        const float thr_blk = (active && !a.out_pair) ? ld_volatile_f32(a.thr + qi) : KNN_INF;

        // ---- U steps of the wavefront ----------------------------------------
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int s = s0 + u;
            if constexpr (WIN) {
                // the group copies the newest row and column of step
                // s + DP_WIN_AHEAD into its windows (coalesced, asynchronous)
                // and waits for those of this step; each lane then reads its
                // own from shared memory instead of scattered global lines
                const int h0 = h - P * lam, hT = h0 + P * (G - 1);
                if (win_loader)
                    dp_win_copy<D, P>(qwin, xwin, wp_mask, qp, xp, m, n, lam, h0, hT,
                                      s + DP_WIN_AHEAD);
                cp_async_commit();
                cp_async_wait_group<DP_WIN_AHEAD>();
                __syncwarp();
                const float4 *qs =
                    reinterpret_cast<const float4 *>(qwin + dp_win_slot<P>(s - h, wp_mask) * RS);
                const float4 *xs =
                    reinterpret_cast<const float4 *>(xwin + dp_win_slot<P>(s + h + P, wp_mask) * RS);
#pragma unroll
                for (int c = 0; c < D / 4; ++c) {
                    const float4 vq = qs[c], vx = xs[c];
                    qw[u][4 * c] = vq.x; qw[u][4 * c + 1] = vq.y; qw[u][4 * c + 2] = vq.z; qw[u][4 * c + 3] = vq.w;
                    float *xd = xw[(u + P) % U];
                    xd[4 * c] = vx.x; xd[4 * c + 1] = vx.y; xd[4 * c + 2] = vx.z; xd[4 * c + 3] = vx.w;
                }
            } else {
                load_point_prefix<D>(qp, s - h, m - 1, qw[u]);
                load_point_prefix<D>(xp, s + h + P, n - 1, xw[(u + P) % U]);
            }

            float up = __shfl_up_sync(KNN_FULL_MASK, O[P - 1], 1, G);
            up = (lam == 0) ? KNN_INF : up;
#pragma unroll
            for (int e = 0; e < P; ++e) {
                const float c = dp_cost<D>(qw[((u - e) % U + U) % U], xw[(u + e) % U], mE[e]);
                const float left = (e == 0) ? up : O[e - 1];
                const float mn = fmin3(left, O[e], E[e]);
                E[e] = (KIND == 0) ? c + mn : fmaxf(c, mn);
            }
            float dn = __shfl_down_sync(KNN_FULL_MASK, E[0], 1, G);
            dn = (lam == G - 1) ? KNN_INF : dn;
#pragma unroll
            for (int e = 0; e < P; ++e) {
                const float c =
                    dp_cost<D>(qw[((u - e) % U + U) % U], xw[(u + e + 1) % U], mO[e]);
                const float right = (e == P - 1) ? dn : E[e + 1];
                const float mn = fmin3(E[e], right, O[e]);
                O[e] = (KIND == 0) ? c + mn : fmaxf(c, mn);
            }
        }
        s0 += U;

        // the end cell, valid when this block ended on step s_f
        float result = KNN_INF;
#pragma unroll
        for (int e = 0; e < P; ++e)
            if (e == fin_slot)
                result = fin_odd ? O[e] : E[e];

        // ---- finish or abandon (group-wide) ------------------------------------
        const float res = __shfl_sync(KNN_FULL_MASK, result, gbase + fin_lane);
        float mn = KNN_INF;
#pragma unroll
        for (int e = 0; e < P; ++e)
            mn = fminf(mn, fminf(E[e], O[e]));
        for (int o = 1; o < G; o <<= 1)
            mn = fminf(mn, __shfl_xor_sync(KNN_FULL_MASK, mn, o));
        if (active) {
            const float lim = thr_blk * a.mu_keep;
            const bool finished = (s0 - 1 == s_f);
            if (finished) {
                if (lam == 0) {
                    // exact band cells of the m x n matrix
                    long long cells = 0;
                    for (int dlt = -r; dlt <= r; ++dlt) {
                        const int hi = min(m, n - dlt), loi = max(0, -dlt);
                        cells += max(0, hi - loi);
                    }
                    st_cells += cells;
                    if (a.out_pair) {
                        a.out_pair[cur_idx] = res;
                    } else if (res <= lim && res < KNN_INF) {
                        const unsigned long long key = make_key(res, (uint32_t)a.db_id[ci]);
                        if (a.k > 0) {
                            unsigned long long *sl = a.slots + (size_t)qi * a.kslots;
                            topk_insert(sl, a.kslots, key);
                            const unsigned long long kth = ld_volatile_u64(sl + a.k - 1);
                            if (kth != KNN_EMPTY_KEY)
                                atomic_min_pos_float(a.thr + qi, key_dist(kth));
                        } else {
                            const int pos = atomicAdd(a.eps_count + qi, 1);
                            if (pos < a.eps_cap)
                                a.eps_list[(size_t)qi * a.eps_cap + pos] = key;
                        }
                    }
                }
                active = false;
            } else if (mn > lim) {
                if (lam == 0) {
                    st_aband += 1;
                    // exact band cells on the anti-diagonals t = i + j < 2 s0
                    // swept so far (diagonal dlt: rows i with 2i + dlt < 2 s0)
                    long long swept = 0;
                    for (int dlt = -r; dlt <= r; ++dlt) {
                        const int hi = min(m, n - dlt), loi = max(0, -dlt);
                        const int ub = 2 * s0 - dlt;
                        const int ui = ub <= 0 ? 0 : (ub + 1) >> 1;
                        swept += max(0, min(hi, ui) - loi);
                    }
                    st_cells += swept;
                }
                active = false;
            }
        }
    }

    if constexpr (WIN)
        cp_async_wait_all();  // no copy outlives the CTA

    // ---- counters: one atomic per warp per counter --------------------------
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        st_calls += __shfl_xor_sync(KNN_FULL_MASK, st_calls, o);
        st_aband += __shfl_xor_sync(KNN_FULL_MASK, st_aband, o);
        st_cells += __shfl_xor_sync(KNN_FULL_MASK, st_cells, o);
        st_pruned += __shfl_xor_sync(KNN_FULL_MASK, st_pruned, o);
    }
    if (lane == 0 && a.stats) {
        atomicAdd(a.stats + STAT_DP_CALLS, st_calls);
        atomicAdd(a.stats + STAT_DP_ABANDONED, st_aband);
        atomicAdd(a.stats + a.cells_stat, st_cells);
        atomicAdd(a.stats + STAT_LB_PRUNED_LATE, st_pruned);
    }
}

// The shared-memory window pays where a point is wide (d >= 8) and a group
// has enough lanes to load it cooperatively (G >= 8).
template <int D, int P>
constexpr bool dp_has_win()
{
    return D >= 8 && D <= 16 && D % 4 == 0 && (P & (P - 1)) == 0 && P >= 2 && P <= 16;
}

// Resident CTAs per SM of one kernel with the given dynamic shared memory,
// looked up once per kernel (the persistent grid is SMs x this).
template <typename K>
int dp_blocks_for(K kernel, size_t smem)
{
    int blocks = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, DP_THREADS, smem);
    return blocks > 0 ? blocks : 1;
}

template <int D, int P, int KIND, bool WIN>
void dp_launch_one(const DpArgs &a, int n_sm, size_t smem, cudaStream_t st)
{
    static int blocks = 0;
    if (!blocks) {
        if (smem > 48 * 1024) {
            cudaFuncSetAttribute(dp_kernel<D, P, KIND, WIN>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            cudaFuncSetAttribute(dp_kernel<D, P, KIND, WIN>,
                                 cudaFuncAttributePreferredSharedMemoryCarveout,
                                 cudaSharedmemCarveoutMaxShared);
        }
        blocks = dp_blocks_for(dp_kernel<D, P, KIND, WIN>, smem);
    }
    dp_kernel<D, P, KIND, WIN><<<n_sm * blocks, DP_THREADS, smem, st>>>(a);
}

// Launch the variant for the pair shape (the shared-memory window where a
// point is wide and a group has lanes enough to load it); the persistent
// grid is SMs x the resident CTAs of that variant.
template <int D, int P>
bool dp_launch_tpl(const DpArgs &a, int kind, int n_sm, cudaStream_t st)
{
    if constexpr (dp_has_win<D, P>()) {
        if (a.G >= 8) {
            const size_t smem = dp_win_bytes(D, P);
            if (kind == 0)
                dp_launch_one<D, P, 0, true>(a, n_sm, smem, st);
            else
                dp_launch_one<D, P, 1, true>(a, n_sm, smem, st);
            return true;
        }
    }
    if (kind == 0)
        dp_launch_one<D, P, 0, false>(a, n_sm, 0, st);
    else
        dp_launch_one<D, P, 1, false>(a, n_sm, 0, st);
    return true;
}

template <int D, int P>
int dp_occupancy_tpl(int kind)
{
    int blocks = 0;
    if (kind == 0)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, dp_kernel<D, P, 0, false>,
                                                      DP_THREADS, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, dp_kernel<D, P, 1, false>,
                                                      DP_THREADS, 0);
    return blocks;
}

}  // namespace knn
