// knn_scan: batch planning and the launch sequence of the exact scan.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "common.cuh"
#include "runtime.h"

using namespace knn;

namespace {

constexpr int DP_GROUPS = 4;  // DP launches per batch at most (length groups)

struct Segment {
    int b_begin, b_end;  // buckets [b_begin, b_end)
    int P, G;
    int64_t base, cap;   // region of the survivor queue
};

struct Plan {
    int nq = 0;
    std::vector<int> m;
    std::vector<int> order;     // batch queries by length (stable): LB_Box query tiles
    std::vector<int64_t> qoff;  // float offsets of the repacked queries
    int64_t qfloats = 0;
    int max_m = 0;
    int64_t env_stride = 0;
    int64_t box_stride = 0;     // coarse stage: floats of one query's segment boxes
    std::vector<char> coarse;   // per bucket: the coarse first stage runs
    std::vector<Segment> segs;
    std::vector<int> seg_of_bucket;
    int64_t items_cap = 0;
    int k = 0, kslots = 0, width = 0, sort_cap = 0;
    int64_t eps_cap = 0;
    Margins mg{};
    float eps_int = 0.f;
    int rer_row = 0, rer_cap = 0;
    bool seeded = false;
    bool learned = false;       // seeds ranked by the encoder instead of LB_Box
    int S = 0;                  // seeds per query
    DpChoice seed_dp{};
};

// Tests only: KNN_FAULT_INJECT=wait makes the LB_Box launches run one device
// wait that cannot complete, with a limit of 4,096 polls (about a
// millisecond), so that the bounded-wait path reports KNN_ERR_TIMEOUT
// without faulting or hanging the GPU.  Read when the launch is enqueued.
uint32_t fault_wait_spins()
{
    const char *f = getenv("KNN_FAULT_INJECT");
    return f && !strcmp(f, "wait") ? 4096u : 0u;
}

knn_status grow(Workspace &ws, DevBuf &b, size_t bytes)
{
    if (bytes <= b.bytes)
        return KNN_OK;
    ws.generation++;
    return b.ensure(bytes < 256 ? 256 : bytes);
}

int next_pow2i(int v)
{
    int p = 1;
    while (p < v)
        p <<= 1;
    return p;
}

}  // namespace

DpChoice knn::dp_choice(knn_db *db, int kind, int r, int n)
{
    auto it = db->tuned.find(std::make_tuple(kind, r, n));
    if (it != db->tuned.end())
        return it->second;
    DpChoice c;
    choose_dp_config(db->deff, r, n, &c.P, &c.G);
    return c;
}

namespace {

knn_status make_plan(knn_db *db, const std::vector<int64_t> &hq_off, int q0, int nq,
                     const knn_params &p, Plan &pl)
{
    const int CH = chunk_floats(db->deff), PPC = chunk_points(db->deff);
    pl.nq = nq;
    pl.m.resize(nq);
    pl.qoff.resize(nq);
    pl.qfloats = 0;
    pl.max_m = 0;
    for (int i = 0; i < nq; ++i) {
        const int m = (int)(hq_off[q0 + i + 1] - hq_off[q0 + i]);
        pl.m[i] = m;
        pl.qfloats += CH;  // leading chunk: the DP's sentinel point
        pl.qoff[i] = pl.qfloats;
        pl.qfloats += (int64_t)((m + PPC - 1) / PPC) * CH;
        pl.max_m = std::max(pl.max_m, m);
    }
    // LB_Box tiles of queries with similar lengths share the buckets their
    // bands can reach; a tile reaching none of a bucket skips it
    pl.order.resize(nq);
    for (int i = 0; i < nq; ++i)
        pl.order[i] = i;
    std::stable_sort(pl.order.begin(), pl.order.end(),
                     [&](int x, int y) { return pl.m[x] < pl.m[y]; });
    pl.env_stride = 0;
    for (auto &b : db->buckets)
        pl.env_stride = std::max<int64_t>(pl.env_stride, (int64_t)((b.n_hi + PPC - 1) / PPC) * CH);
    if (pl.env_stride * 2 * 4 > 200 * 1024)
        return set_error(KNN_ERR_UNSUPPORTED, "envelope larger than shared memory (length x d)");
    // coarse first stage of the LB_Box cascade: filter mode, buckets whose
    // shortest series has at least 4 whole segments and whose boxes fit
    const bool filter = !(p.k > 0 && p.seed_mode == KNN_SEED_LB);
    pl.coarse.assign(db->buckets.size(), 0);
    pl.box_stride = 0;
    if (filter && db->lb_coarse[p.distance] == 0 && db->seg_w > 0) {
        const int W = db->seg_w;
        for (size_t bi = 0; bi < db->buckets.size(); ++bi) {
            const Bucket &b = db->buckets[bi];
            const int box_floats = std::max(4, (b.n_hi / W + PPC - 1) / PPC * CH);
            if (b.n_lo >= 4 * W && coarse_qtile(box_floats) > 0) {
                pl.coarse[bi] = 1;
                pl.box_stride = std::max<int64_t>(pl.box_stride, box_floats);
            }
        }
    }

    // DP segments: at most DP_GROUPS groups of consecutive buckets with
    // similar series counts, so that every DP launch has enough pairs to
    // fill the GPU; a group's shape covers its widest band (r of its longest
    // bucket).  During tuning every bucket is its own segment.
    pl.segs.clear();
    pl.seg_of_bucket.assign(db->buckets.size(), 0);
    int64_t base = 0;
    const int nb = (int)db->buckets.size();
    const int groups = db->tuning ? nb : std::min(nb, DP_GROUPS);
    int64_t per_group = ((int64_t)db->N + groups - 1) / groups;
    int bi = 0;
    for (int gi = 0; gi < groups && bi < nb; ++gi) {
        Segment sg{};
        sg.b_begin = bi;
        int64_t cnt = 0;
        while (bi < nb && (bi == sg.b_begin || cnt < per_group || gi == groups - 1)) {
            cnt += db->buckets[bi].c_end - db->buckets[bi].c_begin;
            ++bi;
            if (db->tuning)
                break;
        }
        sg.b_end = bi;
        const Bucket &last = db->buckets[bi - 1];
        const int r = band_radius(pl.max_m, last.n_hi, p.band);
        DpChoice c = dp_choice(db, p.distance, r, last.n_hi);
        if (c.P == 0)
            return set_error(KNN_ERR_UNSUPPORTED, "band too wide for the compiled DP variants");
        sg.P = c.P;
        sg.G = c.G;
        sg.cap = (int64_t)nq * cnt;
        for (int b = sg.b_begin; b < sg.b_end; ++b)
            pl.seg_of_bucket[b] = (int)pl.segs.size();
        pl.segs.push_back(sg);
    }
    for (auto &s : pl.segs) {
        s.base = base;
        base += s.cap;
    }
    pl.items_cap = base;

    pl.k = p.k;
    pl.eps_cap = p.k > 0 ? 0 : p.eps_capacity;
    pl.kslots = p.k > 0 ? p.k + std::max(8, p.k / 2) : 0;
    pl.width = p.k > 0 ? p.k : (int)p.eps_capacity;
    if (pl.eps_cap > FIN_MAX_EPS_CAP)
        return set_error(KNN_ERR_UNSUPPORTED, "eps_capacity above 2^24");
    pl.sort_cap = next_pow2i(std::max(pl.kslots, (int)std::min<int64_t>(pl.eps_cap, FIN_SMALL_CAP)));
    pl.mg = margins_for(p.distance, pl.max_m + db->max_len, db->deff);
    pl.eps_int = p.distance == KNN_DK ? p.eps * p.eps : p.eps;
    pl.rer_row = 2 * band_radius(pl.max_m, db->max_len, p.band) + 1;
    if ((size_t)3 * (pl.rer_row + 2) * sizeof(double) > 200 * 1024)
        return set_error(KNN_ERR_UNSUPPORTED, "band too wide for FP64 re-scoring (r > 4000)");
    pl.rer_cap = 1024 + 8 * nq;
    pl.seeded = p.k > 0 && (p.seed_mode == KNN_SEED_LB || p.seed_mode == KNN_SEED_LEARNED);
    pl.learned = pl.seeded && p.seed_mode == KNN_SEED_LEARNED;
    if (pl.seeded) {
        pl.S = p.seed_count > 0 ? p.seed_count : std::max(64, 4 * p.k);
        pl.S = std::max(pl.S, p.k);
        pl.seed_dp = dp_choice(db, p.distance, band_radius(pl.max_m, db->max_len, p.band),
                               db->max_len);
        if (pl.seed_dp.P == 0)
            return set_error(KNN_ERR_UNSUPPORTED, "band too wide for the compiled DP variants");
    }
    return KNN_OK;
}

bool p_learned(const Plan &pl) { return pl.learned; }

knn_status size_workspace(knn_db *db, const Plan &pl)
{
    Workspace &ws = db->ws;
    const int nq = pl.nq;
    knn_status s;
#define G_(buf, bytes)                            \
    if ((s = grow(ws, ws.buf, (size_t)(bytes)))) \
        return s;
    G_(qbuf, sizeof(float) * pl.qfloats);
    G_(q_off, sizeof(int64_t) * nq);
    G_(q_len, sizeof(int) * nq);
    G_(q_order, sizeof(int) * nq);
    if (!(pl.seeded && !pl.learned))
        G_(lbq, sizeof(float) * lb_queue_floats(db->n_sm, nq));
    G_(env_lo, sizeof(float) * nq * pl.env_stride);
    G_(env_hi, sizeof(float) * nq * pl.env_stride);
    G_(thr, sizeof(float) * nq);
    G_(slots, sizeof(unsigned long long) * nq * std::max(pl.kslots, 1));
    G_(ub_slots, sizeof(unsigned long long) * nq * std::max(pl.k, 1));
    G_(items, sizeof(int2) * pl.items_cap);
    if (pl.box_stride > 0) {
        G_(sbox_lo, sizeof(float) * nq * pl.box_stride);
        G_(sbox_hi, sizeof(float) * nq * pl.box_stride);
        G_(cq, sizeof(int2) * pl.items_cap);
        // per bucket: the list's count, then one count per query
        G_(cq_count, sizeof(int) * db->buckets.size() * (nq + 1));
    }
    G_(item_lb, sizeof(float) * pl.items_cap);
    G_(eps_list, sizeof(unsigned long long) * nq * std::max<int64_t>(pl.eps_cap, 1));
    if (pl.eps_cap > FIN_SMALL_CAP)
        G_(eps_tmp, sizeof(unsigned long long) * nq * pl.eps_cap);
    G_(eps_count, sizeof(int) * nq);
    G_(ctrl, sizeof(Ctrl));
    G_(fin_valid, sizeof(int) * nq);
    G_(fin_vals, sizeof(double) * nq * std::max<int64_t>(pl.kslots, pl.eps_cap));
    G_(rer_list, sizeof(int2) * pl.rer_cap);
    G_(out_ids, sizeof(int64_t) * nq * pl.width);
    G_(out_dist, sizeof(float) * nq * pl.width);
    G_(out_counts, sizeof(int64_t) * nq);
    if (pl.seeded && p_learned(pl)) {
        G_(scores, sizeof(float) * nq * (size_t)((db->N + 63) / 64));
        G_(sel, sizeof(int) * nq * (size_t)((db->N + 63) / 64));
        G_(skip, sizeof(uint32_t) * nq * (size_t)((db->N + 31) / 32));
        G_(qemb, sizeof(uint16_t) * nq * 64);
        G_(qnorm, sizeof(float) * nq);
        if ((s = enc_work(db->enc, nq, pl.max_m)))
            return s;
    }
    if (pl.seeded && !pl.learned) {
        G_(lb_all, sizeof(float) * nq * (size_t)db->N);
    }
    if (pl.seeded) {
        G_(seed_items, sizeof(int2) * nq * (size_t)pl.S);
        G_(seed_lb, sizeof(float) * nq * (size_t)pl.S);
    }
#undef G_
    return KNN_OK;
}

DpArgs dp_args(knn_db *db, const Plan &pl, const knn_params &p, const int2 *items,
              const float *item_lb, const int *n_items, int64_t cap, int *head)
{
    Workspace &ws = db->ws;
    Ctrl *ctrl = ws.ctrl.as<Ctrl>();
    DpArgs a{};
    a.items = items;
    a.item_lb = item_lb;
    a.n_items = n_items;
    a.items_cap = cap;
    a.head = head;
    a.db = db->data.as<float>();
    a.db_off = db->off.as<int64_t>();
    a.db_len = db->len.as<int>();
    a.db_id = db->id.as<int>();
    a.q = ws.qbuf.as<float>();
    a.q_off = ws.q_off.as<int64_t>();
    a.q_len = ws.q_len.as<int>();
    a.band = p.band;
    a.thr = ws.thr.as<float>();
    a.mu_keep = pl.mg.mu_keep;
    a.mu_prune = pl.mg.mu_prune;
    a.k = p.k;
    a.kslots = pl.kslots;
    a.slots = ws.slots.as<unsigned long long>();
    a.eps_list = ws.eps_list.as<unsigned long long>();
    a.eps_count = ws.eps_count.as<int>();
    a.eps_cap = (int)pl.eps_cap;
    a.stats = ctrl->stats;
    a.status = &ctrl->status;
    return a;
}

// Optional stage events: [0] start, [1] after the greedy pre-pass, [2] after
// the LB_Box stream, [3] after seed selection and seed programs, [4] after the
// survivor filter, [5] after the DP, [6] after finalise.
struct StageEvents {
    cudaEvent_t ev[7] = {};
    cudaEvent_t seg[MAX_SEG + 1] = {};
    bool live = false;
    void create()
    {
        for (auto &e : ev)
            cudaEventCreate(&e);
        for (auto &e : seg)
            cudaEventCreate(&e);
        live = true;
    }
    ~StageEvents()
    {
        if (!live)
            return;
        for (auto &e : ev)
            cudaEventDestroy(e);
        for (auto &e : seg)
            cudaEventDestroy(e);
    }
};

// The call's two timing events, destroyed on every return path.
struct CallEvents {
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    CallEvents()
    {
        cudaEventCreate(&ev0);
        cudaEventCreate(&ev1);
    }
    ~CallEvents()
    {
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
    }
    CallEvents(const CallEvents &) = delete;
    CallEvents &operator=(const CallEvents &) = delete;
};

// All launches of one batch; capturable (no host synchronisation, no
// pageable copies).  Outputs go to the given device pointers.  Returns the
// number of kernels launched.
int enqueue_batch(knn_db *db, const Plan &pl, const knn_params &p, const float *q_src,
                  const int64_t *q_src_off, int64_t *o_ids, float *o_dist, int64_t *o_counts,
                  cudaStream_t st, StageEvents *sev = nullptr)
{
    int launches = 0;
    if (sev)
        cudaEventRecord(sev->ev[0], st);
    Workspace &ws = db->ws;
    Ctrl *ctrl = ws.ctrl.as<Ctrl>();
    const int nq = pl.nq;
    const int kind = p.distance;
    unsigned long long *stats = ctrl->stats;

    launch_repack(q_src, q_src_off, nullptr, nq, db->d, db->deff, ws.q_off.as<int64_t>(),
                  ws.qbuf.as<float>(), st, true);
    cudaMemsetAsync(&ctrl->rer_count, 0, offsetof(Ctrl, stats) - offsetof(Ctrl, rer_count), st);
    launch_fill_f32(ws.thr.as<float>(), p.k > 0 ? KNN_INF_HOST : pl.eps_int, nq, st);
    launches += 2;
    if (p.k > 0) {
        launch_fill_u64(ws.slots.as<unsigned long long>(), KNN_EMPTY_KEY, (int64_t)nq * pl.kslots,
                        st);
        launch_fill_u64(ws.ub_slots.as<unsigned long long>(), KNN_EMPTY_KEY, (int64_t)nq * pl.k,
                        st);
        launches += 2;
    } else {
        cudaMemsetAsync(ws.eps_count.p, 0, sizeof(int) * nq, st);
    }

    // Section 4.3: upper-bound pre-pass seeds the threshold
    if (p.k > 0 && p.seed_mode == KNN_SEED_GREEDY) {
        for (auto &b : db->buckets) {
            GreedyArgs g{};
            g.db = db->data.as<float>();
            g.db_off = db->off.as<int64_t>();
            g.db_len = db->len.as<int>();
            g.db_id = db->id.as<int>();
            g.c_begin = b.c_begin;
            g.c_end = b.c_end;
            g.q = ws.qbuf.as<float>();
            g.q_off = ws.q_off.as<int64_t>();
            g.q_len = ws.q_len.as<int>();
            g.nq = nq;
            g.band = p.band;
            g.k = p.k;
            g.ub_slots = ws.ub_slots.as<unsigned long long>();
            g.thr = ws.thr.as<float>();
            g.stats = stats;
            launch_greedy(g, db->deff, kind == KNN_DK ? 0 : 1, st);
            ++launches;
        }
    }

    // learned proposal: seeds from the encoder's ranking, scored exactly
    // before the LB_Box stream, so that the stream prunes (and abandons)
    // against the seeded threshold directly
    if (pl.learned) {
        enc_scan_scores(db, ws.qbuf.as<float>(), ws.q_off.as<int64_t>(), ws.q_len.as<int>(), nq,
                        pl.max_m, ws.qemb.p, ws.qnorm.as<float>(), ws.scores.as<float>(),
                        ws.sel.as<int>(), &ctrl->status, st);
        const int tiles = (db->N + 63) / 64;
        SelArgs sa{};
        sa.score = ws.scores.as<float>();
        sa.cand = ws.sel.as<int>();
        sa.score_stride = tiles;
        sa.q_len = ws.q_len.as<int>();
        sa.db_len = db->len.as<int>();
        sa.band = p.band;
        sa.n = tiles;
        sa.nq = nq;
        sa.S = pl.S;
        sa.seed_items = ws.seed_items.as<int2>();
        sa.seed_lb = ws.seed_lb.as<float>();
        sa.n_seed = &ctrl->n_seed;
        sa.seed_cap = nq * pl.S;
        sa.seed_bits = ws.skip.as<uint32_t>();
        sa.bits_words = (db->N + 31) / 32;
        sa.stats = stats;
        sa.status = &ctrl->status;
        cudaMemsetAsync(ws.skip.p, 0, sizeof(uint32_t) * nq * (size_t)sa.bits_words, st);
        launch_select(sa, st);
        DpArgs a = dp_args(db, pl, p, ws.seed_items.as<int2>(), ws.seed_lb.as<float>(),
                           &ctrl->n_seed, (int64_t)nq * pl.S, &ctrl->seed_head);
        a.G = pl.seed_dp.G;
        a.cells_stat = STAT_SEED_CELLS;
        launch_dp(a, db->deff, pl.seed_dp.P, kind, db->n_sm, st);
        launches += 9;
    }
    if (sev)
        cudaEventRecord(sev->ev[1], st);

    // envelope + LB_Box stream per bucket (LB-ordered seeding: store every bound)
    const bool store = pl.seeded && !pl.learned;
    if (pl.box_stride > 0)
        cudaMemsetAsync(ws.cq_count.p, 0, sizeof(int) * db->buckets.size() * (nq + 1), st);
    for (size_t bi = 0; bi < db->buckets.size(); ++bi) {
        const Bucket &b = db->buckets[bi];
        const Segment &sg = pl.segs[pl.seg_of_bucket[bi]];
        const int PPC = chunk_points(db->deff), CH = chunk_floats(db->deff);
        EnvArgs e{};
        e.q = ws.qbuf.as<float>();
        e.q_off = ws.q_off.as<int64_t>();
        e.q_len = ws.q_len.as<int>();
        e.nq = nq;
        e.d = db->deff;
        e.band = p.band;
        e.n_hi = b.n_hi;
        e.radius = -1;
        e.env_stride = pl.env_stride;
        e.lo = ws.env_lo.as<float>();
        e.hi = ws.env_hi.as<float>();
        launch_envelope(e, st);
        if (pl.coarse[bi]) {
            // coarse bound over segment boxes, then the exact LB_Box of the
            // pairs it cannot prune; survivors go to the DP queue
            const int W = db->seg_w;
            const int nseg = b.n_hi / W;
            const int box_floats = std::max(4, (nseg + PPC - 1) / PPC * CH);
            SegBoxArgs sb{};
            sb.env_lo = ws.env_lo.as<float>();
            sb.env_hi = ws.env_hi.as<float>();
            sb.env_stride = pl.env_stride;
            sb.nq = nq;
            sb.d = db->deff;
            sb.W = W;
            sb.nseg = nseg;
            sb.scale = coarse_scale(W);
            sb.box_lo = ws.sbox_lo.as<float>();
            sb.box_hi = ws.sbox_hi.as<float>();
            sb.box_stride = pl.box_stride;
            sb.box_floats = box_floats;
            launch_seg_boxes(sb, st);
            int2 *cq = ws.cq.as<int2>() + (int64_t)nq * b.c_begin;
            int *cq_count = ws.cq_count.as<int>() + bi * (nq + 1);
            const int env_floats = (int)((int64_t)((b.n_hi + PPC - 1) / PPC) * CH);
            // pairs grouped by query when the exact stage can hold one
            // query's envelope in shared memory
            const bool by_query = lb_pairs_by_query(db->deff, env_floats);
            CoarseArgs c{};
            c.sg = db->sg.as<float>();
            c.sg_off = db->sg_off.as<int64_t>();
            c.db_len = db->len.as<int>();
            c.W = W;
            c.inv_w = 1.f / (float)W;
            c.c_begin = b.c_begin;
            c.c_end = b.c_end;
            c.n_lo = b.n_lo;
            c.n_hi = b.n_hi;
            c.q_len = ws.q_len.as<int>();
            c.q_order = ws.q_order.as<int>();
            c.nq = nq;
            c.band = p.band;
            c.box_lo = ws.sbox_lo.as<float>();
            c.box_hi = ws.sbox_hi.as<float>();
            c.box_stride = pl.box_stride;
            c.box_floats = box_floats;
            c.nseg_hi = nseg;
            c.M = db->absmax;
            c.thr = ws.thr.as<float>();
            c.mu_prune = pl.mg.mu_prune;
            if (pl.learned) {
                c.skip = ws.skip.as<uint32_t>();
                c.skip_words = (db->N + 31) / 32;
            }
            c.cq = cq;
            c.cq_count = cq_count;
            c.cq_cap = (int64_t)nq * (b.c_end - b.c_begin);
            if (by_query) {
                c.cq_qcount = cq_count + 1;
                c.cq_stride = b.c_end - b.c_begin;
            }
            c.stats = stats;
            c.status = &ctrl->status;
            c.fault_wait_spins = fault_wait_spins();
            c.qtile_req = db->lb_qtile[kind];
            launch_lb_coarse(c, db->deff, kind, db->n_sm, st);
            PairLbArgs pr{};
            pr.cq = cq;
            pr.cq_count = cq_count;
            pr.cq_cap = c.cq_cap;
            pr.cq_qcount = c.cq_qcount;
            pr.cq_stride = c.cq_stride;
            pr.nq = nq;
            pr.env_floats = env_floats;
            pr.db = db->data.as<float>();
            pr.db_off = db->off.as<int64_t>();
            pr.db_len = db->len.as<int>();
            pr.env_lo = ws.env_lo.as<float>();
            pr.env_hi = ws.env_hi.as<float>();
            pr.env_stride = pl.env_stride;
            pr.thr = ws.thr.as<float>();
            pr.mu_prune = pl.mg.mu_prune;
            pr.items = ws.items.as<int2>() + sg.base;
            pr.item_lb = ws.item_lb.as<float>() + sg.base;
            pr.n_items = &ctrl->seg_count[pl.seg_of_bucket[bi]];
            pr.capacity = sg.cap;
            pr.stats = stats;
            pr.status = &ctrl->status;
            launch_lb_pairs(pr, db->deff, kind, db->n_sm, st);
            launches += 4;
            continue;
        }
        LbArgs l{};
        l.db = db->data.as<float>();
        l.db_off = db->off.as<int64_t>();
        l.db_len = db->len.as<int>();
        l.c_begin = b.c_begin;
        l.c_end = b.c_end;
        l.q_len = ws.q_len.as<int>();
        l.nq = nq;
        l.band = p.band;
        l.env_lo = ws.env_lo.as<float>();
        l.env_hi = ws.env_hi.as<float>();
        l.env_stride = pl.env_stride;
        l.env_floats = (int)((int64_t)((b.n_hi + PPC - 1) / PPC) * CH);
        l.thr = ws.thr.as<float>();
        l.mu_prune = pl.mg.mu_prune;
        l.qtile = db->lb_qtile[kind];
        l.win_chunks = db->lb_window[kind];
        l.q_order = ws.q_order.as<int>();
        l.n_lo = b.n_lo;
        l.n_hi = b.n_hi;
        if (store) {
            l.out_lb = ws.lb_all.as<float>();
            l.out_lb_stride = db->N;
        } else {
            if (pl.learned) {
                l.skip = ws.skip.as<uint32_t>();
                l.skip_words = (db->N + 31) / 32;
            }
            l.lbq = ws.lbq.as<float>();
            l.compact = db->lb_compact[kind];
            l.items = ws.items.as<int2>() + sg.base;
            l.item_lb = ws.item_lb.as<float>() + sg.base;
            l.n_items = &ctrl->seg_count[pl.seg_of_bucket[bi]];
            l.capacity = sg.cap;
        }
        l.stats = stats;
        l.status = &ctrl->status;
        l.fault_wait_spins = fault_wait_spins();
        launch_lb(l, db->deff, kind, db->n_sm, st);
        launches += 2;
    }
    if (sev)
        cudaEventRecord(sev->ev[2], st);

    if (store) {
        // seeds: the S series of lowest LB_Box per query, scored exactly first
        SelArgs sa{};
        sa.score = ws.lb_all.as<float>();
        sa.score_stride = db->N;
        sa.lb_all = ws.lb_all.as<float>();
        sa.lb_stride = db->N;
        sa.n = db->N;
        sa.c_base = 0;
        sa.nq = nq;
        sa.S = pl.S;
        sa.seed_items = ws.seed_items.as<int2>();
        sa.seed_lb = ws.seed_lb.as<float>();
        sa.n_seed = &ctrl->n_seed;
        sa.seed_cap = nq * pl.S;
        sa.stats = stats;
        sa.status = &ctrl->status;
        launch_select(sa, st);
        DpArgs a = dp_args(db, pl, p, ws.seed_items.as<int2>(), ws.seed_lb.as<float>(),
                           &ctrl->n_seed, (int64_t)nq * pl.S, &ctrl->seed_head);
        a.G = pl.seed_dp.G;
        a.cells_stat = STAT_SEED_CELLS;
        launch_dp(a, db->deff, pl.seed_dp.P, kind, db->n_sm, st);
        launches += 2;
    }
    if (sev)
        cudaEventRecord(sev->ev[3], st);
    if (store) {
        for (size_t bi = 0; bi < db->buckets.size(); ++bi) {
            const Bucket &b = db->buckets[bi];
            const Segment &sg = pl.segs[pl.seg_of_bucket[bi]];
            FilterArgs fa{};
            fa.lb_all = ws.lb_all.as<float>();
            fa.lb_stride = db->N;
            fa.c_begin = b.c_begin;
            fa.c_end = b.c_end;
            fa.nq = nq;
            fa.thr = ws.thr.as<float>();
            fa.mu_prune = pl.mg.mu_prune;
            fa.items = ws.items.as<int2>() + sg.base;
            fa.item_lb = ws.item_lb.as<float>() + sg.base;
            fa.n_items = &ctrl->seg_count[pl.seg_of_bucket[bi]];
            fa.capacity = sg.cap;
            fa.stats = stats;
            fa.status = &ctrl->status;
            launch_filter(fa, db->n_sm, st);
            ++launches;
        }
    }
    if (sev)
        cudaEventRecord(sev->ev[4], st);

    // banded DP over each segment's survivors
    for (size_t si = 0; si < pl.segs.size(); ++si) {
        const Segment &sg = pl.segs[si];
        if (sev)
            cudaEventRecord(sev->seg[si], st);
        DpArgs a = dp_args(db, pl, p, ws.items.as<int2>() + sg.base, ws.item_lb.as<float>() + sg.base,
                           &ctrl->seg_count[si], sg.cap, &ctrl->seg_head[si]);
        a.G = sg.G;
        a.cells_stat = STAT_DP_CELLS;
        launch_dp(a, db->deff, sg.P, kind, db->n_sm, st);
        ++launches;
    }
    if (sev) {
        cudaEventRecord(sev->seg[pl.segs.size()], st);
        cudaEventRecord(sev->ev[5], st);
    }

    FinArgs f{};
    f.nq = nq;
    f.k = p.k;
    f.kslots = pl.kslots;
    f.slots = ws.slots.as<unsigned long long>();
    f.eps_list = ws.eps_list.as<unsigned long long>();
    f.eps_tmp = pl.eps_cap > FIN_SMALL_CAP ? ws.eps_tmp.as<unsigned long long>() : nullptr;
    f.eps_count = ws.eps_count.as<int>();
    f.eps_cap = (int)pl.eps_cap;
    f.kind = kind;
    f.band = p.band;
    f.eps_int = pl.eps_int;
    f.rerank_rel = pl.mg.rerank_rel;
    f.sort_cap = pl.sort_cap;
    f.fin_valid = ws.fin_valid.as<int>();
    f.fin_vals = ws.fin_vals.as<double>();
    f.fin_width = std::max<int>(pl.kslots, (int)pl.eps_cap);
    f.rer_list = ws.rer_list.as<int2>();
    f.rer_count = &ctrl->rer_count;
    f.rer_cap = pl.rer_cap;
    f.rer_row = pl.rer_row;
    {
        // stage an entry's query and series as doubles when both fit beside
        // the band rows in 200 KB of shared memory
        const int64_t pts = (int64_t)pl.max_m + db->max_len;
        const size_t bytes =
            ((size_t)3 * (pl.rer_row + 2) + (size_t)pts * (db->deff + 1)) * sizeof(double);
        f.stage_pts = bytes <= 200 * 1024 ? (int)pts : 0;
    }
    f.db = db->data.as<float>();
    f.db_off_by_id = db->off_by_id.as<int64_t>();
    f.db_len_by_id = db->len_by_id.as<int>();
    f.q = ws.qbuf.as<float>();
    f.q_off = ws.q_off.as<int64_t>();
    f.q_len = ws.q_len.as<int>();
    f.d = db->deff;
    f.out_ids = o_ids;
    f.out_dist = o_dist;
    f.out_counts = o_counts;
    f.out_width = pl.width;
    f.stats = stats;
    f.status = &ctrl->status;
    launches += launch_finalize(f, st);
    if (sev)
        cudaEventRecord(sev->ev[6], st);
    return launches;
}

std::map<GraphKey, int> graph_launches;

uint64_t hash_lengths(const std::vector<int> &m)
{
    uint64_t h = 1469598103934665603ull;
    for (int v : m) {
        h ^= (uint64_t)v;
        h *= 1099511628211ull;
    }
    return h;
}

}  // namespace

extern "C" knn_status knn_scan(knn_db *db, const float *queries, const int64_t *q_offsets,
                               int32_t n_queries, const knn_params *params, int64_t *out_ids,
                               float *out_dist, int64_t *out_counts, knn_stats *stats,
                               void *stream)
{
    if (!db || !queries || !q_offsets || !params || !out_ids || !out_dist)
        return set_error(KNN_ERR_INVALID, "NULL argument");
    const knn_params p = *params;
    if (n_queries < 1)
        return set_error(KNN_ERR_INVALID, "n_queries must be >= 1");
    if (p.k < 0)
        return set_error(KNN_ERR_INVALID, "k must be >= 0");
    if (p.k > db->N)
        return set_error(KNN_ERR_INVALID, "k larger than the number of series");
    if (p.k > 1024)
        return set_error(KNN_ERR_UNSUPPORTED, "k above 1024");
    if (!(p.band > 0.f) || !std::isfinite(p.band))
        return set_error(KNN_ERR_INVALID, "band must be a positive finite number");
    if (p.distance != KNN_DTW && p.distance != KNN_DK)
        return set_error(KNN_ERR_INVALID, "unknown distance");
    if (p.k == 0) {
        if (!(p.eps >= 0.f) || !std::isfinite(p.eps))
            return set_error(KNN_ERR_INVALID, "eps must be finite and >= 0");
        if (p.eps_capacity < 1)
            return set_error(KNN_ERR_INVALID, "eps_capacity must be >= 1");
        if (!out_counts)
            return set_error(KNN_ERR_INVALID, "eps-NN needs out_counts");
    }
    if (p.seed_mode < KNN_SEED_GREEDY || p.seed_mode > KNN_SEED_LB)
        return set_error(KNN_ERR_INVALID, "unknown seed_mode");
    if (p.seed_mode == KNN_SEED_LEARNED && !db->enc)
        return set_error(KNN_ERR_INVALID, "learned seeding needs an attached encoder");
    if (p.seed_mode == KNN_SEED_LEARNED && p.k == 0)
        return set_error(KNN_ERR_INVALID, "learned seeding applies to k-NN");
    cudaStream_t st = (cudaStream_t)stream;
    cudaSetDevice(db->dev);

    // query offsets on the host
    std::vector<int64_t> hq(n_queries + 1);
    if (is_device_ptr(q_offsets)) {
        cudaError_t e = cudaMemcpy(hq.data(), q_offsets, sizeof(int64_t) * (n_queries + 1),
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess)
            return cuda_error(e, "copy q_offsets");
    } else {
        memcpy(hq.data(), q_offsets, sizeof(int64_t) * (n_queries + 1));
    }
    if (hq[0] < 0)
        return set_error(KNN_ERR_INVALID, "q_offsets[0] < 0");
    for (int i = 0; i < n_queries; ++i) {
        const int64_t L = hq[i + 1] - hq[i];
        if (L < 1)
            return set_error(KNN_ERR_INVALID, "query " + std::to_string(i) + " has length < 1");
        if (L > 65536)
            return set_error(KNN_ERR_UNSUPPORTED, "query longer than 65536 points");
    }

    Workspace &ws = db->ws;
    knn_status s;
    CallEvents cev;
    cudaEventRecord(cev.ev0, st);

    // queries and their point offsets on the device, relative to hq[0]
    const int64_t qpts = hq[n_queries] - hq[0];
    const bool q_dev = is_device_ptr(queries);
    const bool graph = p.use_graph != 0;
    const float *q_src = queries + hq[0] * db->d;
    if ((s = grow(ws, ws.ctrl, sizeof(Ctrl))))
        return s;
    if (!q_dev || graph) {
        if ((s = grow(ws, ws.q_raw, sizeof(float) * qpts * db->d)))
            return s;
        cudaError_t e = cudaMemcpyAsync(ws.q_raw.p, q_src, sizeof(float) * qpts * db->d,
                                        q_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                                        st);
        if (e != cudaSuccess)
            return cuda_error(e, "copy queries");
        q_src = ws.q_raw.as<float>();
    }
    std::vector<int64_t> rel(n_queries + 1);
    for (int i = 0; i <= n_queries; ++i)
        rel[i] = hq[i] - hq[0];
    if ((s = grow(ws, ws.q_src_off, sizeof(int64_t) * (n_queries + 1))))
        return s;
    {
        bool ok = true;
        cudaError_t e = cudaMemcpyAsync(ws.q_src_off.p, rel.data(),
                                        sizeof(int64_t) * (n_queries + 1), cudaMemcpyHostToDevice,
                                        st);
        if (e != cudaSuccess)
            return cuda_error(e, "copy q offsets");
        if ((s = check_finite_dev(q_src, qpts * db->d, &ws.ctrl.as<Ctrl>()->status, st, &ok)))
            return s;
        if (!ok)
            return set_error(KNN_ERR_INVALID, "queries contain NaN or Inf");
    }
    cudaMemsetAsync(ws.ctrl.p, 0, sizeof(Ctrl), st);

    // batches bounded so that the survivor queue stays below 2^27 entries
    int batch = p.query_batch > 0 ? p.query_batch : n_queries;
    const int64_t max_items = (int64_t)1 << 27;
    batch = (int)std::max<int64_t>(1, std::min<int64_t>(batch, max_items / db->N));
    const int width = p.k > 0 ? p.k : (int)p.eps_capacity;
    const bool out_dev = is_device_ptr(out_ids) && is_device_ptr(out_dist) &&
                         (!out_counts || is_device_ptr(out_counts));

    int64_t launches = 1;  // the finite check
    double stage_ms[4] = {0, 0, 0, 0};
    const bool profile = p.profile != 0 && !graph;
    StageEvents sev;
    if (profile)
        sev.create();
    db->seg_ms.clear();
    db->seg_first_bucket.clear();
    for (int q0 = 0; q0 < n_queries; q0 += batch) {
        const int nq = std::min(batch, n_queries - q0);
        Plan pl;
        if ((s = make_plan(db, hq, q0, nq, p, pl)))
            return s;
        const uint64_t gen0 = ws.generation;
        if ((s = size_workspace(db, pl)))
            return s;
        if (ws.generation != gen0) {
            for (auto &g : db->graphs)
                cudaGraphExecDestroy(g.second);
            db->graphs.clear();
        }
        cudaError_t e = cudaMemcpyAsync(ws.q_off.p, pl.qoff.data(), sizeof(int64_t) * nq,
                                        cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ws.q_len.p, pl.m.data(), sizeof(int) * nq, cudaMemcpyHostToDevice,
                                st);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(ws.q_order.p, pl.order.data(), sizeof(int) * nq,
                                cudaMemcpyHostToDevice, st);
        if (e == cudaSuccess)
            e = cudaStreamSynchronize(st);  // host vectors go out of scope
        if (e != cudaSuccess)
            return cuda_error(e, "upload batch metadata");
        const float *qs = q_src;
        const int64_t *qso = ws.q_src_off.as<int64_t>() + q0;
        int64_t *oi = ws.out_ids.as<int64_t>();
        float *od = ws.out_dist.as<float>();
        int64_t *oc = ws.out_counts.as<int64_t>();
        if (!graph && out_dev) {
            oi = out_ids + (int64_t)q0 * width;
            od = out_dist + (int64_t)q0 * width;
            oc = out_counts ? out_counts + q0 : nullptr;
        }
        if (graph) {
            GraphKey key{nq, p.k, p.distance, p.seed_mode, p.seed_count, p.band, p.eps,
                         p.eps_capacity, hash_lengths(pl.m) ^ ((uint64_t)q0 << 40)};
            auto it = db->graphs.find(key);
            if (it == db->graphs.end()) {
                // capture on a private stream (the caller's may be the legacy
                // default stream, which cannot be captured); replay on the caller's
                if (!db->cap_stream) {
                    e = cudaStreamCreateWithFlags(&db->cap_stream, cudaStreamNonBlocking);
                    if (e != cudaSuccess)
                        return cuda_error(e, "create capture stream");
                }
                cudaGraph_t gph;
                e = cudaStreamBeginCapture(db->cap_stream, cudaStreamCaptureModeThreadLocal);
                if (e != cudaSuccess)
                    return cuda_error(e, "begin capture");
                graph_launches[key] =
                    enqueue_batch(db, pl, p, qs, qso, oi, od, oc, db->cap_stream);
                e = cudaStreamEndCapture(db->cap_stream, &gph);
                if (e != cudaSuccess)
                    return cuda_error(e, "end capture");
                cudaGraphExec_t ex;
                e = cudaGraphInstantiate(&ex, gph, 0);
                cudaGraphDestroy(gph);
                if (e != cudaSuccess)
                    return cuda_error(e, "instantiate graph");
                it = db->graphs.emplace(key, ex).first;
            }
            e = cudaGraphLaunch(it->second, st);
            if (e != cudaSuccess)
                return cuda_error(e, "graph launch");
            launches += graph_launches[key];
        } else {
            launches += enqueue_batch(db, pl, p, qs, qso, oi, od, oc, st, profile ? &sev : nullptr);
            if (profile) {
                e = cudaEventSynchronize(sev.ev[6]);
                if (e != cudaSuccess)
                    return cuda_error(e, "stage events");
                float t[6];
                for (int i = 0; i < 6; ++i)
                    cudaEventElapsedTime(&t[i], sev.ev[i], sev.ev[i + 1]);
                stage_ms[0] += t[0] + t[2];  // seeding: greedy pre-pass, or seeds
                stage_ms[1] += t[1] + t[3];  // envelopes, LB_Box stream, filter
                stage_ms[2] += t[4];         // DP
                stage_ms[3] += t[5];         // finalise
                db->seg_ms.resize(pl.segs.size(), 0.0);
                db->seg_first_bucket.resize(pl.segs.size());
                for (size_t si = 0; si < pl.segs.size(); ++si) {
                    float ms = 0.f;
                    cudaEventElapsedTime(&ms, sev.seg[si], sev.seg[si + 1]);
                    db->seg_ms[si] += ms;
                    db->seg_first_bucket[si] = pl.segs[si].b_begin;
                }
            }
        }
        if (graph || !out_dev) {
            const cudaMemcpyKind k1 = out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
            e = cudaMemcpyAsync(out_ids + (int64_t)q0 * width, oi, sizeof(int64_t) * nq * width, k1,
                                st);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(out_dist + (int64_t)q0 * width, od, sizeof(float) * nq * width,
                                    k1, st);
            if (e == cudaSuccess && out_counts)
                e = cudaMemcpyAsync(out_counts + q0, oc, sizeof(int64_t) * nq, k1, st);
            if (e != cudaSuccess)
                return cuda_error(e, "copy outputs");
        }
        e = cudaGetLastError();
        if (e != cudaSuccess)
            return cuda_error(e, "launch");
    }
    cudaEventRecord(cev.ev1, st);
    Ctrl hc;
    cudaError_t e = cudaMemcpyAsync(&hc, ws.ctrl.p, sizeof(Ctrl), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return cuda_error(e, "scan");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, cev.ev0, cev.ev1);
    if (stats) {
        memset(stats, 0, sizeof(*stats));
        stats->pairs = (int64_t)hc.stats[STAT_PAIRS];
        stats->band_infeasible = (int64_t)hc.stats[STAT_INFEASIBLE];
        stats->ub_walks = (int64_t)hc.stats[STAT_UB_WALKS];
        stats->seeds = (int64_t)hc.stats[STAT_SEEDS];
        stats->seed_cells = (int64_t)hc.stats[STAT_SEED_CELLS];
        stats->lb_pruned = (int64_t)hc.stats[STAT_LB_PRUNED];
        stats->lb_pruned_late = (int64_t)hc.stats[STAT_LB_PRUNED_LATE];
        stats->dp_calls = (int64_t)hc.stats[STAT_DP_CALLS];
        stats->dp_abandoned = (int64_t)hc.stats[STAT_DP_ABANDONED];
        stats->dp_cells = (int64_t)hc.stats[STAT_DP_CELLS];
        stats->reranked = (int64_t)hc.stats[STAT_RERANKED];
        stats->lb_points = (int64_t)hc.stats[STAT_LB_POINTS];
        stats->launches = launches;
        stats->ms_total = ms;
        stats->ms_seed = stage_ms[0];
        stats->ms_lb = stage_ms[1];
        stats->ms_dp = stage_ms[2];
        stats->ms_finalize = stage_ms[3];
        stats->lb_kernels = (int64_t)hc.stats[STAT_LB_KERNELS];
        stats->lb_coarse_pruned = (int64_t)hc.stats[STAT_LB_COARSE_PRUNED];
        stats->lb_segments = (int64_t)hc.stats[STAT_LB_SEGMENTS];
    }
    if (hc.status & KNN_DEV_TIMEOUT)
        return set_error(KNN_ERR_TIMEOUT, "a device wait gave up");
    if (hc.status & KNN_DEV_BAD_SHAPE)
        return set_error(KNN_ERR_UNSUPPORTED, "a kernel received a shape it cannot handle");
    if (hc.status & KNN_DEV_CAPACITY)
        return set_error(KNN_ERR_CAPACITY, p.k == 0 ? "eps-NN result exceeds eps_capacity"
                                                    : "internal capacity exceeded");
    return KNN_OK;
}
