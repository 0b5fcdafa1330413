// Internal host-side declarations: device argument blocks and launchers.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace knn {

// Thresholds and prune margins live in "internal units": DTW as the sum of
// squared costs, DK as the squared max cost (sqrt is monotone, so order and
// comparisons carry over).  A bound prunes when it exceeds thr * mu_prune; a
// finished distance is kept when it is at most thr * mu_keep.  The margins
// cover FP32 summation drift so that no candidate of the exact FP64 answer
// is ever dropped.
struct Margins {
    float mu_keep;
    float mu_prune;
    float rerank_rel;  // relative width of the FP64 re-scoring band
};

// -- envelope --------------------------------------------------------------
struct EnvArgs {
    const float *q;          // repacked queries
    const int64_t *q_off;    // float offset of each query
    const int *q_len;
    int nq;
    int d;
    float band;
    int n_hi;                // longest series of the bucket (envelope length)
    int radius;              // >= 0: explicit band radius; < 0: from band
    int64_t env_stride;      // floats between consecutive queries' lo arrays
    float *lo;               // [nq][env_stride]
    float *hi;
};
void launch_envelope(const EnvArgs &a, cudaStream_t st);

// -- LB_Box stream ------------------------------------------------------------
struct LbArgs {
    const float *db;           // repacked database
    const int64_t *db_off;     // float offset per (bucket-ordered) series
    const int *db_len;
    int c_begin, c_end;        // series range of this bucket
    const int *q_len;
    int q_first;               // first query of this batch
    int nq;
    float band;
    const float *env_lo, *env_hi;
    int64_t env_stride;
    int env_floats;            // floats of one envelope (chunk padded)
    const float *thr;          // [nq] live thresholds
    float mu_prune;
    const uint32_t *skip;      // [nq][words] bitmap of series already scored (nullable)
    int skip_words;
    int2 *items;               // out: (series, query) survivors
    float *item_lb;            // out: their bounds
    int *n_items;
    int64_t capacity;
    float *out_lb;             // optional: every bound, [nq][n_series] (component API)
    int64_t out_lb_stride;
    unsigned long long *stats; // [STAT_*]
    int *status;
    int single_query_kernel;   // 1: always the warp-per-series kernel
    int qtile;                 // queries per CTA of the multi-query kernel (0: 16)
    int win_chunks;            // > 0: windowed multi-query kernel with windows of this many
                               // chunks; 0: whole envelopes when they fit, else windowed
    const int *q_order;        // multi-query kernels: batch queries in tile order (queries
                               // sorted by length; nullable = batch order)
    int n_lo, n_hi;            // shortest / longest series of the bucket
    float *lbq;                // filter mode: per-CTA survivor queues of the compacting
                               // kernel (nullable: no compaction)
    int compact;               // 0 automatic, 1 never, 2 whenever possible
    int k1, k2;                // compaction checkpoints in chunks (set by the launcher)
    uint32_t fault_wait_spins; // tests only (KNN_FAULT_INJECT=wait): > 0 makes one thread
                               // wait that many polls on a barrier nothing completes
};
// Floats of survivor-queue scratch one LB launch may need for nq queries.
size_t lb_queue_floats(int n_sm, int nq);
void launch_lb(const LbArgs &a, int d, int form, int n_sm, cudaStream_t st);
void lb_init_attributes();

// -- coarse first stage of the LB_Box cascade (segment boxes) ---------------
// Segment width for a database of point width deff whose shortest series has
// min_len points (a power of 4, so that the sqrt(W) scaling of means and
// boxes is exact): wide points take 64-point segments when every series has
// at least four of them (about as tight a filter as 16-point segments at a
// quarter of the segment work and data), else 16; narrow points take 4.
inline int coarse_width(int deff, int min_len)
{
    if (deff < 8)
        return 4;
    return min_len >= 4 * 64 ? 64 : 16;
}
// sqrt(W), exact for the widths above.
inline float coarse_scale(int W) { return W == 64 ? 8.f : W == 16 ? 4.f : 2.f; }
struct SegBoxArgs {
    const float *env_lo, *env_hi;  // [nq][env_stride] envelopes of one bucket
    int64_t env_stride;
    int nq, d;                     // d: point width (deff)
    int W, nseg;                   // segment width, segments of the bucket's longest series
    float scale;                   // sqrt(W)
    float *box_lo, *box_hi;        // out: [nq][box_stride], box_floats used per query
    int64_t box_stride;
    int box_floats;                // nseg * d rounded up to whole chunks
};
struct CoarseArgs {
    const float *sg;               // scaled segment means of the database
    const int64_t *sg_off;         // float offset per series (bucket order)
    const int *db_len;
    int W;
    float inv_w;                   // 1 / W (exact: W is a power of 4)
    int c_begin, c_end;            // series of this bucket
    int n_lo, n_hi;
    const int *q_len;
    const int *q_order;            // batch queries in tile order (nullable)
    int nq;
    float band;
    const float *box_lo, *box_hi;  // scaled segment boxes, [nq][box_stride]
    int64_t box_stride;
    int box_floats;
    int nseg_hi;                   // segments of the bucket's longest series
    int qtile_req;                 // queries per CTA asked for (0: the most that fit)
    float M;                       // largest coordinate magnitude in the database
    const float *thr;
    float mu_prune;
    const uint32_t *skip;          // [nq][skip_words] series already scored (nullable)
    int skip_words;
    int2 *cq;                      // out: (series, query) pairs within their limit
    int *cq_count;                 //   (nullable: no queue)
    int64_t cq_cap;
    float *out_lb;                 // optional: every bound, [nq][out_lb_stride] (component)
    int64_t out_lb_stride;
    unsigned long long *stats;
    int *status;
    uint32_t fault_wait_spins;     // tests only: see LbArgs
    // per-query queue (nullable): pairs of batch query qb go to
    // cq[qb * cq_stride ...], counted in cq_qcount[qb]; else one list
    int *cq_qcount;
    int64_t cq_stride;
};
struct PairLbArgs {
    const int2 *cq;                // (series, query) pairs
    const int *cq_count;
    int64_t cq_cap;
    const int *cq_qcount;          // per-query queue (nullable), see CoarseArgs
    int64_t cq_stride;
    int nq;
    int env_floats;                // floats of one envelope used by the bucket
    const float *db;
    const int64_t *db_off;
    const int *db_len;
    const float *env_lo, *env_hi;  // [nq][env_stride]
    int64_t env_stride;
    const float *thr;
    float mu_prune;
    int2 *items;                   // out: DP queue of the bucket's segment
    float *item_lb;
    int *n_items;
    int64_t capacity;
    unsigned long long *stats;
    int *status;
};
void launch_seg_means(const float *data, const int64_t *off, const int *len, int N, int deff,
                      int W, const int64_t *sg_off, const int64_t *sg_end, float *sg,
                      cudaStream_t st);
void launch_absmax(const float *x, int64_t n, unsigned int *out, cudaStream_t st);
void launch_seg_boxes(const SegBoxArgs &a, cudaStream_t st);
// Queries per coarse CTA whose boxes fit in shared memory (0: none).
int coarse_qtile(int box_floats);
bool launch_lb_coarse(const CoarseArgs &a, int deff, int form, int n_sm, cudaStream_t st);
// Whether the exact stage can take its pairs grouped by query, one query's
// envelope in shared memory per CTA (d' a multiple of 4, envelope small enough).
bool lb_pairs_by_query(int deff, int env_floats);
bool launch_lb_pairs(const PairLbArgs &a, int deff, int form, int n_sm, cudaStream_t st);
void lbc_init_attributes();

// -- greedy upper bound (Algorithm 1) ---------------------------------------
struct GreedyArgs {
    const float *db;
    const int64_t *db_off;
    const int *db_len;
    const int *db_id;
    int c_begin, c_end;
    const float *q;
    const int64_t *q_off;
    const int *q_len;
    int nq;
    float band;
    int k;
    unsigned long long *ub_slots;  // [nq][k] smallest upper bounds (keys)
    float *thr;                    // [nq] threshold, lowered to the k-th bound
    float *out_ub;                 // optional: every bound [nq][stride]
    int64_t out_stride;
    unsigned long long *stats;
};
void launch_greedy(const GreedyArgs &a, int d, int form, cudaStream_t st);

// -- seeded scan: selection of seeds and filtering of survivors -------------
struct SelArgs {
    const float *score;        // [nq][score_stride] ranking score per entry
    const int *cand;           // nullable: series of each entry (else entry c is series c)
    int64_t score_stride;
    float *lb_all;             // [nq][lb_stride] LB_Box per series; seeds are set to -1
                               // (nullable: feasibility from the lengths, seed bound 0)
    int64_t lb_stride;
    const int *q_len;          // with lb_all == nullptr: lengths for the band test
    const int *db_len;
    float band;
    int n;                     // series
    int c_base;                // index of score[0] in bucket order
    int nq;
    int S;                     // seeds per query
    int2 *seed_items;
    float *seed_lb;
    int *n_seed;
    int seed_cap;
    uint32_t *seed_bits;       // nullable: [nq][bits_words] bit per chosen series
    int bits_words;
    unsigned long long *stats;
    int *status;
};
void launch_select(const SelArgs &a, cudaStream_t st);

struct FilterArgs {
    const float *lb_all;
    int64_t lb_stride;
    int c_begin, c_end;
    int nq;
    const float *thr;
    float mu_prune;
    int2 *items;
    float *item_lb;
    int *n_items;
    int64_t capacity;
    unsigned long long *stats;
    int *status;
};
void launch_filter(const FilterArgs &a, int n_sm, cudaStream_t st);

// -- banded dynamic program on the survivor queue ----------------------------
struct DpArgs {
    const int2 *items;
    const float *item_lb;
    const int *n_items;
    int64_t items_cap;         // entries beyond this were never written
    int *head;                 // queue cursor, zero before the launch
    const float *db;
    const int64_t *db_off;
    const int *db_len;
    const int *db_id;
    const float *q;
    const int64_t *q_off;
    const int *q_len;
    float band;
    int G;                     // lanes per candidate (power of two <= 32)
    float *thr;                // [nq] live thresholds (internal units)
    float mu_keep, mu_prune;
    int k;                     // > 0: k-NN
    int kslots;                // slots kept per query (k + rerank spare)
    unsigned long long *slots; // [nq][kslots]
    unsigned long long *eps_list;  // eps-NN: [nq][eps_cap]
    int *eps_count;
    int eps_cap;
    float *out_pair;           // pair mode: result per queue entry, no threshold
    int cells_stat;            // statistics slot receiving the evaluated cells
    unsigned long long *stats;
    int *status;
};
// Returns false if no kernel is compiled for (d, P).  The persistent grid is
// n_sm times the resident CTAs of the variant that runs.
bool launch_dp(const DpArgs &a, int d, int P, int kind, int n_sm, cudaStream_t st);
int dp_block_threads();
// Largest P compiled for this d, and the list of compiled P values.
int dp_num_variants(int d);
int dp_variant_P(int d, int idx);
int dp_max_blocks_per_sm(int d, int P, int kind);

// -- finalise: sort, FP64 re-scoring of the boundary band, output -----------
struct FinArgs {
    int nq;
    int k;
    int kslots;
    unsigned long long *slots;     // k-NN: [nq][kslots], ascending
    unsigned long long *eps_list;  // eps-NN: [nq][eps_cap] (sorted in place)
    unsigned long long *eps_tmp;   // eps_cap > FIN_SMALL_CAP: [nq][eps_cap] merge buffer
    const int *eps_count;
    int eps_cap;
    int kind;
    float band;
    float eps_int;             // eps-NN threshold (internal units)
    float rerank_rel;
    int sort_cap;              // power of two >= every per-query list
    int *fin_valid;            // [nq] scratch
    double *fin_vals;          // [nq][fin_width] scratch
    int fin_width;
    int2 *rer_list;            // (query, position) of entries to re-score
    int *rer_count;
    int rer_cap;
    int rer_row;               // longest band row supported (2r+1)
    int stage_pts;             // points of the two series of an entry staged as
                               // doubles in shared memory (0: none)
    // data for FP64 re-scoring (caller ids -> database rows)
    const float *db;
    const int64_t *db_off_by_id;
    const int *db_len_by_id;
    const float *q;
    const int64_t *q_off;
    const int *q_len;
    int d;
    int64_t *out_ids;          // device
    float *out_dist;
    int64_t *out_counts;       // nullable
    int out_width;
    unsigned long long *stats;
    int *status;
};
// eps-NN lists up to this length are sorted in shared memory; longer ones
// by a merge sort in global memory.
constexpr int FIN_SMALL_CAP = 8192;
// Largest eps-NN capacity per query.
constexpr int64_t FIN_MAX_EPS_CAP = (int64_t)1 << 24;
// Enqueues the finalisation; returns the number of kernels launched.
int launch_finalize(const FinArgs &a, cudaStream_t st);
void fin_init_attributes();

// -- pair programs (no pruning) ----------------------------------------------
// FP64 pair program, one warp per pair; row >= 2r+1 for every pair (r <= 8000).
void launch_pairwise64(const float *a, const int64_t *a_off, const float *b, const int64_t *b_off,
                       const int64_t *pa, const int64_t *pb, int64_t n, int d, float band,
                       int kind, double *out, int row, cudaStream_t st);

// -- small utilities ------------------------------------------------------------
void launch_fill_u64(unsigned long long *p, unsigned long long v, int64_t n, cudaStream_t st);
void launch_fill_f32(float *p, float v, int64_t n, cudaStream_t st);
// Copy series order[c] of `src` (d floats per point, point offsets
// src_off) to dst + dst_off[c] with deff floats per point (extra coordinates
// zero) and zero padding up to the chunk-padded size.  dp_lead: the chunk of
// floats before each series (reserved by the caller's offsets) is filled
// with KNN_DP_SENTINEL, the point the DP reads for negative indices.
// fixed_len > 0: every series has that many points from src_off[s] (the
// series may overlap: windows of one long series).
void launch_repack(const float *src, const int64_t *src_off, const int *order, int nser, int d,
                   int deff, const int64_t *dst_off, float *dst, cudaStream_t st, bool dp_lead,
                   int fixed_len = 0);
// dst[q][id[c]] = src[q][c] for c < n (bucket order -> caller order).
void launch_scatter_by_id(const float *src, const int *db_id, int n, int nq, int64_t src_stride,
                          float *dst, int64_t dst_stride, int out_sqrt, cudaStream_t st);

enum Stat : int {
    STAT_PAIRS = 0,
    STAT_INFEASIBLE,
    STAT_UB_WALKS,
    STAT_SEEDS,
    STAT_LB_PRUNED,
    STAT_LB_PRUNED_LATE,
    STAT_DP_CALLS,
    STAT_DP_ABANDONED,
    STAT_DP_CELLS,
    STAT_RERANKED,
    STAT_SEED_CELLS,
    STAT_LB_POINTS,      // (query, series point) pairs bounded by LB_Box
    STAT_LB_KERNELS,     // bit mask of the LB_Box kernels that ran (knn_stats.lb_kernels)
    STAT_LB_COARSE_PRUNED,  // pairs pruned by the coarse (segment box) stage
    STAT_LB_SEGMENTS,    // (query, series segment) pairs bounded by the coarse stage
    STAT_COUNT
};

// Band radius: r = floor(band * max(m, n)), band >= 1 unconstrained.
__host__ __device__ inline int band_radius(int m, int n, float band)
{
    int L = m > n ? m : n;
    if (band >= 1.0f)
        return L;
    double v = static_cast<double>(band) * static_cast<double>(L);
    int r = static_cast<int>(v);  // v >= 0: truncation is floor
    return r;
}

}  // namespace knn
