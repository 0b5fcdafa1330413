/*
 * knnwarp: exact k-NN / eps-NN scan of multi-dimensional time series under
 * Sakoe-Chiba-banded DTW and the dog-keeper distance DK, for NVIDIA GB300
 * (sm_103a).
 *
 * Method: Bachmann & Freytag, "An Analytical Approach to Improving Time
 * Warping on Multidimensional Time Series" (arXiv 1811.11076).
 *   - DTW and DK definitions: Section 2.1; band: Section 2.2.
 *   - Envelope / LB_Keogh: Section 2.3; LB_Box: Section 3, Eq. 1.
 *   - GDK upper bound: Section 4.1, Algorithm 1.
 *   - Threshold-driven (sparse) DK: Section 4.2, Algorithm 3.
 *   - Nearest-neighbour search with an upper-bound pre-pass: Section 4.3.
 *   - k-NN and eps-NN query semantics: Section 1.
 *
 * Conventions shared by every entry point
 *   - Series are point-major FP32: a series of length n in d dimensions is
 *     n*d consecutive floats (point i, coordinate j at [i*d + j]).  A set of
 *     series is concatenated; offsets[s] .. offsets[s+1] are its points.
 *   - Band: r = floor(band * max(m, n)) for lengths m, n; band >= 1 means no
 *     constraint.  A pair with |m - n| > r has distance +inf and is never
 *     returned.
 *   - Units: DTW is the SUM of squared Euclidean point costs along the best
 *     path (no final root), DK the Euclidean max along the best path.
 *   - Results are ordered by (distance, id) ascending; ids are the caller's
 *     0-based series indices.  k-NN rows with fewer than k finite results are
 *     padded with id -1 and distance +inf.
 *   - Exactness: id sets equal those of an FP64 evaluation; candidates whose
 *     FP32 distance lies within the FP32 error band of the boundary are
 *     re-scored in FP64 on the device before the cut.
 *   - Memory: unless stated otherwise a pointer argument may be host memory
 *     (pageable or pinned) or device memory of the current device; the
 *     library detects the kind and stages host buffers itself.  Callers keep
 *     ownership of everything they pass in.  Library objects (knn_db,
 *     knn_encoder) are owned by the library until their destroy call.
 *   - Streams: `stream` is a cudaStream_t (NULL = legacy default stream).
 *     Every call is synchronous with respect to its outputs: when it returns,
 *     outputs are written and the status is final.
 *   - Errors: every call returns a knn_status; nothing aborts the process,
 *     throws across the boundary or traps on the device.  Invalid arguments
 *     are rejected before any launch.  knn_last_error() gives a
 *     thread-local message for the last failure on the calling thread.
 *   - Thread safety: distinct knn_db objects may be used concurrently; one
 *     knn_db must not be used by two calls at the same time.
 */
#ifndef KNNWARP_H
#define KNNWARP_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KNN_API __attribute__((visibility("default")))

typedef enum { KNN_DTW = 0, KNN_DK = 1 } knn_distance;

typedef enum {
    KNN_OK = 0,
    KNN_ERR_INVALID = 1,     /* bad argument (detected before any launch)        */
    KNN_ERR_OOM = 2,         /* device allocation failed                         */
    KNN_ERR_CUDA = 3,        /* a CUDA call failed                               */
    KNN_ERR_TIMEOUT = 4,     /* a bounded device wait gave up                    */
    KNN_ERR_CAPACITY = 5,    /* eps-NN result larger than eps_capacity; counts
                                bound the sizes (see knn_scan)                   */
    KNN_ERR_UNSUPPORTED = 6  /* configuration not compiled in (e.g. d > 16)     */
} knn_status;

/* How the running threshold is seeded before the pruned scan. */
typedef enum {
    /* Section 4.3: an upper bound for every series from the greedy path of
     * Algorithm 1 (max of costs for DK = GDK; sum of squared costs for DTW);
     * the k-th smallest becomes the initial threshold. */
    KNN_SEED_GREEDY = 0,
    /* Learned proposal: the attached encoder ranks the series by predicted
     * distance, the seed_count best are scored exactly first, and the k-th
     * best exact distance becomes the initial threshold.  Needs an encoder
     * attached to the database (knn_encoder_attach). */
    KNN_SEED_LEARNED = 1,
    /* No pre-pass: the threshold starts at +inf. */
    KNN_SEED_NONE = 2,
    /* LB_Box-ordered proposal: LB_Box is computed for every series first, the
     * seed_count series with the lowest bound are scored exactly, and the
     * k-th best exact distance becomes the threshold against which the rest
     * are filtered (the plain ordering, without an encoder). */
    KNN_SEED_LB = 3
} knn_seed_mode;

typedef struct {
    int32_t k;             /* > 0: k-NN with this k; 0: eps-NN                      */
    float eps;             /* eps-NN radius in output units (ignored for k-NN)      */
    float band;            /* Sakoe-Chiba band as a fraction of max(m, n), > 0       */
    int32_t distance;      /* knn_distance                                           */
    int32_t seed_mode;     /* knn_seed_mode                                          */
    int32_t seed_count;    /* learned seeding: proposals scored exactly first
                              (0 = 4 * k, at least 64)                               */
    int32_t query_batch;   /* queries per launch sequence; 0 = all in one batch      */
    int32_t use_graph;     /* 1 = capture each batch's launch sequence in a CUDA
                              graph and replay it (cached per database and shape)    */
    int64_t eps_capacity;  /* eps-NN: result slots per query, 1 .. 2^24 (above 8,192
                              the lists are sorted in global memory; the scratch
                              is 3 x 8 bytes per slot and query)                     */
    int32_t profile;       /* 1 = time each stage with CUDA events (stats->ms_*);
                              ignored when use_graph = 1                             */
    int32_t reserved;
} knn_params;

/* Counters of one scan (summed over queries).  Cells are DP cells actually
 * evaluated, counted up to the point where a candidate was abandoned. */
typedef struct {
    int64_t pairs;           /* (query, series) pairs considered                 */
    int64_t band_infeasible; /* pairs with |m - n| > r                           */
    int64_t ub_walks;        /* greedy upper-bound walks run                     */
    int64_t seeds;           /* proposals scored exactly before the filter       */
    int64_t seed_cells;      /* DP cells evaluated for the proposals             */
    int64_t lb_pruned;       /* pruned by LB_Box before the DP queue             */
    int64_t lb_pruned_late;  /* pruned by LB_Box at DP start (tighter threshold) */
    int64_t dp_calls;        /* dynamic programs started                         */
    int64_t dp_abandoned;    /* dynamic programs abandoned early                 */
    int64_t dp_cells;        /* band cells of the m x n matrices evaluated: every
                                cell of a finished pair, and the cells on the
                                anti-diagonals swept before an abandoned pair
                                was dropped (lane slots outside the band and
                                the virtual prefix are not counted)              */
    int64_t reranked;        /* candidates re-scored in FP64                     */
    int64_t lb_points;       /* (query, series point) pairs bounded by LB_Box    */
    int64_t launches;        /* kernels launched by the call                     */
    double ms_total;         /* time of the call on the stream                   */
    double ms_seed;          /* profile = 1: threshold seeding (greedy/learned)  */
    double ms_lb;            /* profile = 1: envelopes + LB_Box stream           */
    double ms_dp;            /* profile = 1: banded dynamic programs             */
    double ms_finalize;      /* profile = 1: FP64 re-scoring and output          */
    int64_t lb_kernels;      /* LB_Box kernels that ran, bit mask: 1 one query per
                                pass, 2 whole envelopes, 4 windowed envelopes,
                                8 whole envelopes with compaction, 16 the
                                coarse first stage (segment boxes)             */
    int64_t lb_coarse_pruned; /* pairs pruned by the coarse first stage          */
    int64_t lb_segments;     /* (query, series segment) pairs it bounded         */
} knn_stats;

typedef struct knn_db knn_db;
typedef struct knn_encoder knn_encoder;

/* ---------------------------------------------------------------------- */
/* Database                                                                 */

/* Copy n_series series (concatenated `series`, `offsets` with n_series+1
 * entries in points) into a library-owned device layout: series grouped
 * into length buckets, each series starting on a 16-byte boundary and padded
 * to a whole number of LB chunks.  1 <= d <= 16; every length >= 1. */
KNN_API knn_status knn_db_create(const float *series, const int64_t *offsets,
                                 int64_t n_series, int32_t d, void *stream,
                                 knn_db **out);
/* A database whose series are the windows T[a .. a+m-1] of one long series
 * T (n points, [n][d] point-major, host or device), a = 0, stride,
 * 2 stride, ... up to n - m: series id i starts at point i * stride.  A
 * knn_scan of queries of length m against it is the banded subsequence
 * search (every window of T against the query under the Sakoe-Chiba band of
 * Section 2.2, the whole-match DTW / DK of Section 2.1), with every feature
 * of the scan: k best windows or all within eps, exact order, the LB_Box
 * cascade and early abandoning.  Windows overlap; no exclusion zone is
 * applied (the next best windows are usually neighbours of the best).  The
 * layout stores each window separately: (n - m) / stride + 1 windows of m
 * points.  1 <= m <= 65536, stride >= 1. */
KNN_API knn_status knn_db_create_windows(const float *series, int64_t n, int32_t d, int32_t m,
                                         int32_t stride, void *stream, knn_db **out);
KNN_API knn_status knn_db_destroy(knn_db *db);
/* Number of series and dimensionality. */
KNN_API knn_status knn_db_info(const knn_db *db, int64_t *n_series, int32_t *d,
                               int32_t *n_buckets);

/* ---------------------------------------------------------------------- */
/* Scan                                                                     */

/* Exact k-NN (params->k > 0) or eps-NN (params->k == 0) of n_queries queries
 * against the database (Section 1 semantics; method of Sections 2-4).
 *   queries, q_offsets: as `series`/`offsets` above (q_offsets has
 *     n_queries+1 entries), same d as the database.
 *   k-NN:   out_ids [n_queries][k], out_dist [n_queries][k]; out_counts may
 *           be NULL (else receives the number of finite results per query).
 *   eps-NN: out_ids/out_dist [n_queries][eps_capacity], out_counts
 *           [n_queries] (result sizes).  The result SET is exact; rows are
 *           ordered by the reported distances, which never decrease (FP32,
 *           or FP64 where re-scored near eps), so two results whose exact
 *           distances lie within the FP32 error band of each other may
 *           appear in either order.  If a row holds more results than
 *           eps_capacity the call returns KNN_ERR_CAPACITY: that row's
 *           stored entries are true results (padded with -1 / +inf where
 *           some were dropped at eps) and its count is an upper bound of its
 *           size, above it only by results within the FP32 error band of
 *           eps that could not be stored and re-checked; a retry with that
 *           capacity holds the row.  k-NN rows are in exact order.
 *   stats may be NULL. */
KNN_API knn_status knn_scan(knn_db *db, const float *queries, const int64_t *q_offsets,
                            int32_t n_queries, const knn_params *params,
                            int64_t *out_ids, float *out_dist, int64_t *out_counts,
                            knn_stats *stats, void *stream);

/* One query against series given as a flat array with lengths (the
 * knn_scan(query, db, lengths, d, band, k|eps, distance) form).  k > 0: k-NN
 * (ids/dist hold k entries); k == 0: eps-NN (ids/dist hold n_series
 * entries; *count receives the result size).  Builds a temporary database. */
KNN_API knn_status knn_scan_simple(const float *query, int64_t m, const float *db,
                                   const int64_t *lengths, int64_t n_series, int32_t d,
                                   float band, int32_t k, float eps, int32_t distance,
                                   int64_t *ids, float *dist, int64_t *count);

/* ---------------------------------------------------------------------- */
/* Shape of the banded dynamic program and its autotuner                    */
/*                                                                          */
/* The DP assigns G lanes (a power of two <= 32) to one (query, series)      */
/* pair and P band diagonals to each lane (2P cells per lane per two        */
/* anti-diagonals); G*P >= r+1 must hold.  A shape is chosen per            */
/* (distance, r, n) key, r the band radius and n the longest series of a    */
/* length bucket.  Without tuning, a cost model picks it.  The widest band  */
/* is r <= 32 * P_max - 1 with P_max the largest compiled P: r <= 415 for   */
/* d <= 3, 223 for d = 4..6, 127 for d = 7, 8 and 9..16; wider bands return  */
/* KNN_ERR_UNSUPPORTED.                                                     */

/* Time every compiled shape for each length bucket on the given queries
 * (one full scan per shape, each bucket's DP launch timed with CUDA events)
 * and keep the fastest in `db` for later scans with the same distance,
 * band and query lengths.  cache_path (nullable): a JSON file of previous
 * results (one entry per device name, d and key); keys found there are not
 * re-timed, and the file is rewritten with the new results.  params->k > 0.
 * queries/q_offsets as in knn_scan. */
KNN_API knn_status knn_autotune(knn_db *db, const float *queries, const int64_t *q_offsets,
                                int32_t n_queries, const knn_params *params,
                                const char *cache_path, void *stream);
/* Force the shape for one key (P must be compiled for the database's d). */
KNN_API knn_status knn_set_dp_shape(knn_db *db, int32_t distance, int32_t r, int32_t n,
                                    int32_t P, int32_t G);
/* The shape a scan would use for a key (tuned, forced, or the model's). */
KNN_API knn_status knn_get_dp_shape(knn_db *db, int32_t distance, int32_t r, int32_t n,
                                    int32_t *P, int32_t *G);
/* Compiled P values for dimensionality d: writes up to cap of them to
 * P_list (nullable) and returns how many exist. */
KNN_API int32_t knn_dp_shapes(int32_t d, int32_t *P_list, int32_t cap);

/* Query tile of the LB_Box stream (Section 3, Eq. 1) for one distance: a
 * CTA bounds its 256 series against qtile queries at once (4, 8 or 16; 0 =
 * 16, or the tuned value) so that the database is read once per tile; the
 * coarse first stage of the cascade takes the same tile (at most the number
 * of segment boxes that fit in 100 KB of shared memory).  window_chunks = 0: a CTA stages the tile's whole envelopes in shared
 * memory when they fit (2 * 4 * qtile * padded length * d bytes <= 192 KB)
 * and windows of them otherwise; > 0: always windows of that many chunks of
 * lcm(d', 4) floats (clamped to what fits).  compaction (filter mode with
 * whole envelopes; the early abandoning of Section 4 applied to the bound):
 * 0 = when a CTA walks at least 4 batches of series of at least 16 chunks,
 * 1 = never, 2 = whenever the series have at least 8 chunks.  The result of a
 * scan depends on none of these values.  KNN_ERR_INVALID for other qtile or
 * compaction values or a negative window. */
KNN_API knn_status knn_set_lb_tile(knn_db *db, int32_t distance, int32_t qtile,
                                   int32_t window_chunks, int32_t compaction);
KNN_API knn_status knn_get_lb_tile(knn_db *db, int32_t distance, int32_t *qtile,
                                   int32_t *window_chunks, int32_t *compaction);

/* Coarse first stage of the LB_Box cascade (Section 3, Eq. 1 over segment
 * boxes).  The points of a series are grouped into segments of W consecutive
 * points (W = 4 for d < 8; for d >= 8, 64 when every series of the database
 * has at least 256 points, else 16; partial last segments left out), B_s is
 * the smallest box holding the query envelope's boxes B_j of segment s, and
 *     LB_seg = sum_s W * dist(mean of the segment's points, B_s)^2
 * (form 0; form 1: the max over segments of dist^2) is at most LB_Box, by
 * convexity of the squared distance to a box.  The segment means are built
 * with the database.  In the filtering scan, pairs the coarse bound prunes
 * never reach LB_Box; the others get the exact LB_Box, and only its
 * survivors reach the dynamic program.  coarse = 0 (automatic): used for
 * every bucket whose shortest series has at least 4 segments; 1: never.
 * Results never depend on it.  knn_get_lb_cascade also returns W
 * (segment_width nullable).  KNN_ERR_INVALID for other values. */
KNN_API knn_status knn_set_lb_cascade(knn_db *db, int32_t distance, int32_t coarse);
KNN_API knn_status knn_get_lb_cascade(knn_db *db, int32_t distance, int32_t *coarse,
                                      int32_t *segment_width);

/* ---------------------------------------------------------------------- */
/* Components (each is one step of the scan, exposed for verification and  */
/* for callers who build their own pipelines).  All pointers device memory. */

/* Envelope of one series (Section 2.3; per dimension, Section 3): for
 * i in [0, len) and coordinate j, lo[i*d+j] = min of t[p*d+j] over
 * |p - i| <= r, 0 <= p < n, hi likewise with max; +inf/-inf where the window
 * is empty.  Outputs are [len][d]. */
KNN_API knn_status knn_envelope(const float *t, int64_t n, int32_t d, int64_t r,
                                int64_t len, float *lo, float *hi, void *stream);

/* LB_Box of every database series against the envelope of `query`
 * (Section 3, Eq. 1, with the envelope on the query side; banded DTW is
 * symmetric).  form 0: sum over points of the squared box distance (bounds
 * DTW); form 1: max over points (bounds DK^2).  out_lb[n_series] in the
 * caller's series order; band-infeasible series get +inf. */
KNN_API knn_status knn_lb_box(knn_db *db, const float *query, int64_t m, float band,
                              int32_t form, float *out_lb, void *stream);

/* The coarse bound LB_seg of every database series against `query` (see
 * knn_set_lb_cascade; the same units as knn_lb_box, form 0 or 1), a lower
 * bound of knn_lb_box's value.  out_lb[n_series] in the caller's series
 * order; band-infeasible series get +inf. */
KNN_API knn_status knn_lb_seg(knn_db *db, const float *query, int64_t m, float band,
                              int32_t form, float *out_lb, void *stream);

/* Greedy upper bound of every database series (Section 4.1, Algorithm 1,
 * walked to the end cell): form 0 = GDK (max of Euclidean costs), form 1 =
 * sum of squared costs along the same path (bounds DTW).  out_ub[n_series]
 * in the caller's series order. */
KNN_API knn_status knn_greedy_ub(knn_db *db, const float *query, int64_t m, float band,
                                 int32_t form, float *out_ub, void *stream);

/* Banded DTW / DK of explicit pairs (a[pa[i]], b[pb[i]]) with no pruning
 * (Section 2.1).  a_off/b_off: point offsets (device, int64).  Writes FP32
 * results to out_f32 (nullable) and FP64 results to out_f64 (nullable,
 * computed by a separate FP64 program). */
KNN_API knn_status knn_pairwise(const float *a, const int64_t *a_off, const float *b,
                                const int64_t *b_off, const int64_t *pa, const int64_t *pb,
                                int64_t n_pairs, int32_t d, float band, int32_t distance,
                                float *out_f32, double *out_f64, void *stream);

/* Same FP32 results as knn_pairwise's out_f32, for callers who cannot let
 * the library allocate device memory (their memory belongs to their own
 * allocator, or cudaMalloc/cudaFree, which may synchronise the device, are not
 * acceptable where they call).  The paper has no counterpart: this is an
 * interface for such callers.  Nothing is allocated: the scratch (repacked
 * series, pair queue, results, counters) is one fixed array of about 9.4 MB
 * inside the library, present on every device that loads it until exit.
 * Limits: n_pairs <= 65536; 1 <= n_a, n_b <= 16384 series per set; after
 * padding each series to whole chunks of lcm(d', 4) floats (d' = d, or 16
 * for 9 <= d <= 16), plus one chunk per series, at most 1,048,576 floats
 * per set; max_len (an upper bound
 * on every series length, used to choose the DP shape) <= 65536.  Larger
 * inputs are rejected (KNN_ERR_INVALID for counts, KNN_ERR_CAPACITY for the
 * padded sizes) and nothing is computed.  All pointers are device memory;
 * a_off / b_off have n_a + 1 / n_b + 1 point offsets; out receives n_pairs
 * floats.  The first call on a device looks the array's device address up
 * (cudaGetSymbolAddress) with that device current and keeps it for the life
 * of the process; after the device's primary context is destroyed
 * (cudaDeviceReset) the function must not be called on that device again.
 * Every call shares the array and clears its counters; calls that overlap on
 * the GPU race and must be serialised by the caller.  The call reads its
 * status back and synchronises `stream` before returning, so it cannot be
 * captured into a CUDA graph: on a stream under capture it returns
 * KNN_ERR_INVALID without touching the stream. */
KNN_API knn_status knn_pairwise_noalloc(const float *a, const int64_t *a_off, int64_t n_a,
                                        const float *b, const int64_t *b_off, int64_t n_b,
                                        const int64_t *pa, const int64_t *pb, int64_t n_pairs,
                                        int32_t d, float band, int32_t max_len,
                                        int32_t distance, float *out, void *stream);

/* ---------------------------------------------------------------------- */
/* Subsequence search (Section 4.1 Algorithm 2; Section 4.2 Algorithm 3     */
/* with SUB = true): queries against every subsequence of one long series.  */

/* For each query S (m points) the minimum over all subsequences T[a..b] of
 * the long series T (n points, [n][d] point-major) of DTW(S, T[a..b]) (sum of
 * squared costs, distance = KNN_DTW) or DK(S, T[a..b]) (max of Euclidean
 * costs, KNN_DK), without a band: the free-start, free-end recursion in which
 * every column may start a match and every column may end one.  out_dist
 * [n_queries] receives the value, out_end [n_queries] the end b of the best
 * subsequence (the smallest b on ties).  eps >= 0 (+inf: none): cells whose
 * value exceeds eps (DTW units for DTW, Euclidean for DK) are dropped (values
 * only grow along a path; for DK this is Algorithm 3's sparse visit); a
 * result above eps is reported as +inf with end -1.  queries/q_offsets as
 * in knn_scan; series, queries and outputs may be host or device memory.
 * Exactness: the FP32 sweep keeps the 9 best ends of each query; the best
 * and those within 2e-4 (relative) of it, far beyond the FP32 rounding of
 * a path, are re-scored in FP64 over the columns a path of their value can
 * span (the walk back from b stops where the least cell cost per column,
 * summed for DTW, single for DK, exceeds the FP32 value by 0.1 %), and the
 * best by (FP64 value, end) is reported.  Limits: 1 <= d <= 16; m <= 1024 for d = 1, 512
 * for d = 2, 3, 256 for d = 4..8, 128 for d = 9..16 (else
 * KNN_ERR_UNSUPPORTED); a re-scored match spanning more than 65,536 columns
 * returns KNN_ERR_UNSUPPORTED; coordinates of magnitude well below 1e18
 * (sentinel points of that value pad T).  Synchronises `stream`. */
KNN_API knn_status knn_subseq(const float *queries, const int64_t *q_offsets, int32_t n_queries,
                              const float *series, int64_t n, int32_t d, int32_t distance,
                              float eps, float *out_dist, int64_t *out_end, void *stream);

/* The k best end columns of the same search (1 <= k <= 16): out_dist and
 * out_end are [n_queries][k], ordered by (value, end), padded with +inf / -1
 * where fewer than k ends lie within eps.  The FP32 sweep keeps the
 * k + max(8, k) best ends; the k best and those within 2e-4 of the k-th are
 * re-scored in FP64 as for knn_subseq.  Ends
 * next to the best usually come next (a subsequence and its neighbours match
 * nearly as well); no exclusion zone is applied. */
KNN_API knn_status knn_subseq_k(const float *queries, const int64_t *q_offsets,
                                int32_t n_queries, const float *series, int64_t n, int32_t d,
                                int32_t distance, int32_t k, float eps, float *out_dist,
                                int64_t *out_end, void *stream);

/* Algorithm 2 (greedy dog-keeper for subsequence search): per query the
 * largest Euclidean cost along the greedy walk that starts at row 0 in the
 * column closest to s_0 (the first on ties) and moves to the cheapest of
 * (i+1, j), (i+1, j+1), (i, j+1) until the last row; an upper bound of the
 * subsequence DK.  out_ub [n_queries], out_end [n_queries] (the column where
 * the walk reached the last row).  The walk stops early once the bound
 * exceeds eps; it then reports that bound with end -1.  Arguments and memory
 * as for knn_subseq; no limit on m. */
KNN_API knn_status knn_subseq_greedy(const float *queries, const int64_t *q_offsets,
                                     int32_t n_queries, const float *series, int64_t n, int32_t d,
                                     float eps, float *out_ub, int64_t *out_end, void *stream);

/* ---------------------------------------------------------------------- */
/* Learned proposal: a 1-D convolutional encoder (no counterpart in the     */
/* paper; it generalises the upper-bound pre-pass of Section 4.3).  Three   */
/* convolutions (kernel 5, 64 channels, ReLU), a mean over positions and a  */
/* linear layer map a series to a 64-d embedding; ||e_a - e_b||^2 predicts  */
/* the distance.  Convolutions and their gradients run on BF16 tensor cores */
/* with FP32 accumulation; FP32 master weights, Adam.  The encoder only     */
/* orders the work: scan results never depend on it.                        */

typedef struct {
    int32_t epochs;        /* passes over the training pairs                      */
    int32_t batch_pairs;   /* pairs per optimiser step                            */
    float lr;              /* Adam learning rate                                  */
    int32_t distance;      /* knn_distance of the targets                         */
    float band;            /* band of the target distances                        */
    uint64_t seed;         /* pair sampling and shuffling                         */
} knn_train_params;

typedef struct {
    double first_loss;     /* loss of the first step                              */
    double final_loss;     /* mean loss of the last epoch                         */
    double ms;             /* wall time on the stream                             */
    int64_t pairs;         /* training pairs with a finite distance               */
    int64_t steps;         /* optimiser steps                                     */
} knn_train_stats;

/* Number of parameters (FP32) of the encoder. */
KNN_API int32_t knn_encoder_num_params(void);
/* New encoder for d-dimensional series (1 <= d <= 16), He-normal weights. */
KNN_API knn_status knn_encoder_create(int32_t d, uint64_t seed, knn_encoder **out);
KNN_API knn_status knn_encoder_destroy(knn_encoder *enc);
/* Train on n_pairs random pairs of database series; the target of a pair is
 * log(1 + x) of its banded distance computed by the scan's DP, x = DTW
 * divided by the longer length, or DK^2 (a monotone transform: the ranking
 * is what matters); loss (||e_a - e_b||^2 - target)^2. */
KNN_API knn_status knn_encoder_train(knn_encoder *enc, knn_db *db, int64_t n_pairs,
                                     const knn_train_params *params, knn_train_stats *stats,
                                     void *stream);
/* Embeddings [n][64] (FP32, device) of n series (device, point offsets). */
KNN_API knn_status knn_encoder_embed(knn_encoder *enc, const float *series,
                                     const int64_t *offsets, int64_t n, float *out, void *stream);
/* Embed every database series (BF16, kept by the database) so that scans
 * with seed_mode = KNN_SEED_LEARNED can rank series by predicted distance. */
KNN_API knn_status knn_encoder_attach(knn_db *db, knn_encoder *enc, void *stream);
/* The learned proposal's scores as a scan computes them (a component, for
 * verification): queries are embedded (BF16) and every database series is
 * scored by ||e_q - e_c||^2 from the attached BF16 embeddings, the dot
 * products on the tcgen05 tensor cores with FP32 accumulation.  For each
 * query and each tile of 64 consecutive series of the database's
 * length-sorted order (the caller's order when all series have one length)
 * out_score [n_queries][ceil(n_series / 64)] receives the lowest score and
 * out_series the caller's id of that series (the first on ties).  Outputs:
 * device memory.  KNN_ERR_INVALID without an attached encoder. */
KNN_API knn_status knn_encoder_scores(knn_db *db, const float *queries, const int64_t *q_offsets,
                                      int32_t n_queries, float *out_score, int64_t *out_series,
                                      void *stream);
/* Read (get) and/or replace (set) the FP32 parameters, host arrays of
 * knn_encoder_num_params() floats in the layout W1 [5][16][64], b1, W2
 * [5][64][64], b2, W3 [5][64][64], b3, Wl [64][64] (in x out), bl. */
KNN_API knn_status knn_encoder_params(knn_encoder *enc, float *get, const float *set);
/* Mean loss and its gradient (host, knn_encoder_num_params() floats) for
 * pairs (pa[i], pb[i]) of n_series series (device, point offsets) with
 * targets (host or device). */
KNN_API knn_status knn_encoder_loss_grad(knn_encoder *enc, const float *series,
                                         const int64_t *offsets, int64_t n_series,
                                         const int64_t *pa, const int64_t *pb,
                                         const float *targets, int64_t n_pairs, float *loss,
                                         float *grad, void *stream);
/* Checkpoint: a JSON header line, then FP32 parameters and Adam moments. */
KNN_API knn_status knn_encoder_save(const knn_encoder *enc, const char *path);
KNN_API knn_status knn_encoder_load(const char *path, knn_encoder **out);

/* ---------------------------------------------------------------------- */
/* Diagnostics                                                              */

KNN_API const char *knn_status_string(knn_status s);
/* Thread-local description of the last error on this thread ("" if none). */
KNN_API const char *knn_last_error(void);
/* Library version string. */
KNN_API const char *knn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* KNNWARP_H */
