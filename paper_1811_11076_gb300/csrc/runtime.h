// Host runtime objects: device buffers, the database handle, its workspace.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <map>
#include <string>
#include <tuple>
#include <vector>

#include "../../include/knnwarp.h"
#include "internal.h"

namespace knn {

knn_status set_error(knn_status s, const std::string &msg);
knn_status cuda_error(cudaError_t e, const char *what);
bool is_device_ptr(const void *p);
int deff_for(int d);
Margins margins_for(int kind, int max_path, int d);
void choose_dp_config(int deff, int r, int n, int *P, int *G);
// Sets *ok = false if any of the n floats at dev is NaN or Inf (synchronises st).
knn_status check_finite_dev(const float *dev, int64_t n, int *flag_dev, cudaStream_t st, bool *ok);

// Owning device allocation that only grows.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
    DevBuf() = default;
    DevBuf(const DevBuf &) = delete;
    DevBuf &operator=(const DevBuf &) = delete;
    ~DevBuf() { release(); }
    knn_status ensure(size_t b);
    void release();
    template <class T> T *as() const { return static_cast<T *>(p); }
};

struct Bucket {
    int c_begin, c_end;  // series range in bucket order
    int n_lo, n_hi;      // shortest / longest length
};

// Scratch of the scan, grown on demand and reused across calls.
struct Workspace {
    DevBuf q_raw, q_src_off;            // staged caller queries (host input)
    DevBuf qbuf, q_off, q_len;          // repacked queries of the batch
    DevBuf q_order;                     // batch queries sorted by length (LB tiles)
    DevBuf lbq;                         // LB_Box compaction queues (filter mode)
    DevBuf env_lo, env_hi;
    DevBuf thr, slots, ub_slots;
    DevBuf items, item_lb;
    DevBuf eps_list, eps_count, eps_tmp;
    DevBuf ctrl;                        // counters, status, stats
    DevBuf fin_valid, fin_vals, rer_list, rer_scratch;
    DevBuf out_ids, out_dist, out_counts;
    DevBuf skip;
    DevBuf seed_items, seed_lb, scores, sel, lb_all, qemb, qnorm;
    DevBuf sbox_lo, sbox_hi;            // coarse stage: segment boxes of the queries
    DevBuf cq, cq_count;                // coarse stage: pairs passing it, per bucket
    uint64_t generation = 0;            // bumped whenever a buffer moves
};

// Layout of the control block (ints first, then 64-bit statistics).
constexpr int MAX_SEG = 64;
struct Ctrl {
    int status;
    int rer_count;
    int n_seed;
    int seed_head;
    int seg_count[MAX_SEG];   // survivors appended per DP segment
    int seg_head[MAX_SEG];    // DP queue cursors
    unsigned long long stats[STAT_COUNT];
};

struct GraphKey {
    int nq, k, kind, seed_mode, seed_count;
    float band, eps;
    int64_t eps_cap;
    uint64_t qhash;
    bool operator<(const GraphKey &o) const
    {
        return std::tie(nq, k, kind, seed_mode, seed_count, band, eps, eps_cap, qhash) <
               std::tie(o.nq, o.k, o.kind, o.seed_mode, o.seed_count, o.band, o.eps, o.eps_cap,
                        o.qhash);
    }
};

struct DpChoice {
    int P, G;
};

}  // namespace knn

struct knn_db;
namespace knn {
DpChoice dp_choice(knn_db *db, int kind, int r, int n);
knn_status enc_work(knn_encoder *enc, int B, int L);
// Scores of the best series of each 64-series tile per query
// ([nq][ceil(N/64)], with the series in tile_idx).
knn_status enc_scan_scores(knn_db *db, const float *qbuf, const int64_t *q_off, const int *q_len,
                           int nq, int max_m, void *qemb, float *qnorm, float *scores,
                           int *tile_idx, int *status, cudaStream_t st);
}

struct knn_db {
    int d = 0, deff = 0, N = 0;
    int dev = 0, n_sm = 0;
    int max_len = 0;
    int64_t total_floats = 0;
    knn::DevBuf data, off, len, id, off_by_id, len_by_id;
    std::vector<int> h_len, h_len_by_id;
    std::vector<knn::Bucket> buckets;
    knn::Workspace ws;
    knn_encoder *enc = nullptr;
    knn::DevBuf emb;                      // [N][64] bf16 embeddings (bucket order)
    knn::DevBuf emb_norm;                 // [N] squared norms of the bf16 embeddings
    std::map<knn::GraphKey, cudaGraphExec_t> graphs;
    cudaStream_t cap_stream = nullptr;    // private stream used only to capture graphs
    std::map<std::tuple<int, int, int>, knn::DpChoice> tuned;  // (kind, r, n) -> config
    bool tuning = false;                  // autotuner running: one DP segment per bucket
    int lb_qtile[2] = {0, 0};             // queries per LB pass per distance (0: 16)
    int lb_window[2] = {0, 0};            // LB envelope window in chunks (0: automatic)
    int lb_compact[2] = {0, 0};           // LB compaction: 0 automatic, 1 never, 2 always
    int lb_coarse[2] = {0, 0};            // coarse first LB stage: 0 automatic, 1 never
    knn::DevBuf sg, sg_off;               // scaled segment means per series (bucket order)
    int seg_w = 0;                        // segment width of sg (0: not built)
    float absmax = 0.f;                   // largest coordinate magnitude of the series
    std::vector<double> seg_ms;           // profile: DP time per segment of the last scan
    std::vector<int> seg_first_bucket;    // first bucket of each segment of the last scan
    ~knn_db()
    {
        for (auto &g : graphs)
            cudaGraphExecDestroy(g.second);
        if (cap_stream)
            cudaStreamDestroy(cap_stream);
    }
};
