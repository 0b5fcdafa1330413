// Component entry points (envelope, LB_Box, greedy bound, pair programs) and
// the single-query convenience scan.
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "runtime.h"

using namespace knn;

namespace {

// Upload one query as a batch of one into the database workspace.
knn_status stage_one_query(knn_db *db, const float *query, int64_t m, cudaStream_t st,
                           int64_t *env_len_out)
{
    Workspace &ws = db->ws;
    const int CH = chunk_floats(db->deff), PPC = chunk_points(db->deff);
    knn_status s;
    const int64_t qf = (int64_t)((m + PPC - 1) / PPC) * CH;
    if ((s = ws.q_raw.ensure(sizeof(float) * m * db->d)) || (s = ws.q_src_off.ensure(16)) ||
        (s = ws.qbuf.ensure(sizeof(float) * qf)) || (s = ws.q_off.ensure(8)) ||
        (s = ws.q_len.ensure(8)) || (s = ws.ctrl.ensure(sizeof(Ctrl))))
        return s;
    ws.generation++;
    const bool dev = is_device_ptr(query);
    cudaError_t e = cudaMemcpyAsync(ws.q_raw.p, query, sizeof(float) * m * db->d,
                                    dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    const int64_t so[2] = {0, m};
    const int64_t qo = 0;
    const int ml = (int)m;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws.q_src_off.p, so, sizeof(so), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws.q_off.p, &qo, sizeof(qo), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(ws.q_len.p, &ml, sizeof(ml), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return cuda_error(e, "stage query");
    bool ok = true;
    if ((s = check_finite_dev(ws.q_raw.as<float>(), m * db->d, &ws.ctrl.as<Ctrl>()->status, st,
                              &ok)))
        return s;
    if (!ok)
        return set_error(KNN_ERR_INVALID, "query contains NaN or Inf");
    launch_repack(ws.q_raw.as<float>(), ws.q_src_off.as<int64_t>(), nullptr, 1, db->d, db->deff,
                  ws.q_off.as<int64_t>(), ws.qbuf.as<float>(), st, false);
    int64_t env = 0;
    for (auto &b : db->buckets)
        env = std::max<int64_t>(env, (int64_t)((b.n_hi + PPC - 1) / PPC) * CH);
    *env_len_out = env;
    return KNN_OK;
}

}  // namespace

extern "C" knn_status knn_envelope(const float *t, int64_t n, int32_t d, int64_t r, int64_t len,
                                   float *lo, float *hi, void *stream)
{
    if (!t || !lo || !hi)
        return set_error(KNN_ERR_INVALID, "NULL argument");
    if (n < 1 || len < 1 || r < 0 || d < 1 || d > 16)
        return set_error(KNN_ERR_INVALID, "bad shape");
    if (!is_device_ptr(t) || !is_device_ptr(lo) || !is_device_ptr(hi))
        return set_error(KNN_ERR_INVALID, "knn_envelope takes device pointers");
    cudaStream_t st = (cudaStream_t)stream;
    int64_t *dev_off = nullptr;
    int *dev_len = nullptr;
    cudaError_t e = cudaMalloc(&dev_off, 8);
    if (e == cudaSuccess)
        e = cudaMalloc(&dev_len, 4);
    const int64_t zero = 0;
    const int ni = (int)n;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dev_off, &zero, 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(dev_len, &ni, 4, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
        cudaFree(dev_off);
        cudaFree(dev_len);
        return cuda_error(e, "envelope setup");
    }
    EnvArgs a{};
    a.q = t;
    a.q_off = dev_off;
    a.q_len = dev_len;
    a.nq = 1;
    a.d = d;
    a.n_hi = (int)len;
    a.env_stride = len * d;
    a.lo = lo;
    a.hi = hi;
    a.band = -1.f;
    a.radius = (int)r;
    launch_envelope(a, st);
    e = cudaStreamSynchronize(st);
    cudaFree(dev_off);
    cudaFree(dev_len);
    if (e == cudaSuccess)
        e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_error(e, "envelope");
    return KNN_OK;
}

// mode 0: LB_Box (Eq. 1); 1: greedy bound (Algorithm 1); 2: coarse bound
// over segment boxes (the cascade's first stage).
static knn_status bound_common(knn_db *db, const float *query, int64_t m, float band, int32_t form,
                               float *out, void *stream, int mode)
{
    const bool greedy = mode == 1;
    if (!db || !query || !out)
        return set_error(KNN_ERR_INVALID, "NULL argument");
    if (m < 1 || !(band > 0.f) || (form != 0 && form != 1))
        return set_error(KNN_ERR_INVALID, "bad argument");
    if (!is_device_ptr(out))
        return set_error(KNN_ERR_INVALID, "output must be device memory");
    cudaStream_t st = (cudaStream_t)stream;
    Workspace &ws = db->ws;
    int64_t env = 0;
    knn_status s = stage_one_query(db, query, m, st, &env);
    if (s)
        return s;
    if (env * 2 * 4 > 200 * 1024)
        return set_error(KNN_ERR_UNSUPPORTED, "envelope larger than shared memory");
    if ((s = ws.env_lo.ensure(sizeof(float) * env)) || (s = ws.env_hi.ensure(sizeof(float) * env)) ||
        (s = ws.thr.ensure(sizeof(float))) || (s = ws.item_lb.ensure(sizeof(float) * db->N)))
        return s;
    ws.generation++;
    Ctrl *ctrl = ws.ctrl.as<Ctrl>();
    cudaMemsetAsync(ctrl, 0, sizeof(Ctrl), st);
    launch_fill_f32(ws.thr.as<float>(), KNN_INF_HOST, 1, st);
    const int PPC = chunk_points(db->deff), CH = chunk_floats(db->deff);
    float *tmp = ws.item_lb.as<float>();  // bucket-ordered bounds
    for (auto &b : db->buckets) {
        if (greedy) {
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
            g.nq = 1;
            g.band = band;
            g.k = 1;
            g.out_ub = tmp;
            g.out_stride = db->N;
            g.stats = ctrl->stats;
            launch_greedy(g, db->deff, form, st);
        } else {
            EnvArgs e{};
            e.q = ws.qbuf.as<float>();
            e.q_off = ws.q_off.as<int64_t>();
            e.q_len = ws.q_len.as<int>();
            e.nq = 1;
            e.d = db->deff;
            e.band = band;
            e.radius = -1;
            e.n_hi = b.n_hi;
            e.env_stride = env;
            e.lo = ws.env_lo.as<float>();
            e.hi = ws.env_hi.as<float>();
            launch_envelope(e, st);
            if (mode == 2) {
                const int W = db->seg_w, nseg = b.n_hi / W;
                const int box_floats = std::max(4, (nseg + PPC - 1) / PPC * CH);
                if ((s = ws.sbox_lo.ensure(sizeof(float) * box_floats)) ||
                    (s = ws.sbox_hi.ensure(sizeof(float) * box_floats)))
                    return s;
                if (!coarse_qtile(box_floats))
                    return set_error(KNN_ERR_UNSUPPORTED, "segment boxes larger than shared memory");
                SegBoxArgs sb{};
                sb.env_lo = ws.env_lo.as<float>();
                sb.env_hi = ws.env_hi.as<float>();
                sb.env_stride = env;
                sb.nq = 1;
                sb.d = db->deff;
                sb.W = W;
                sb.nseg = nseg;
                sb.scale = coarse_scale(W);
                sb.box_lo = ws.sbox_lo.as<float>();
                sb.box_hi = ws.sbox_hi.as<float>();
                sb.box_stride = box_floats;
                sb.box_floats = box_floats;
                launch_seg_boxes(sb, st);
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
                c.nq = 1;
                c.band = band;
                c.box_lo = ws.sbox_lo.as<float>();
                c.box_hi = ws.sbox_hi.as<float>();
                c.box_stride = box_floats;
                c.box_floats = box_floats;
                c.nseg_hi = nseg;
                c.M = db->absmax;
                c.thr = ws.thr.as<float>();
                c.mu_prune = 1.f;
                c.out_lb = tmp;
                c.out_lb_stride = db->N;
                c.stats = ctrl->stats;
                c.status = &ctrl->status;
                launch_lb_coarse(c, db->deff, form, db->n_sm, st);
                continue;
            }
            LbArgs l{};
            l.db = db->data.as<float>();
            l.db_off = db->off.as<int64_t>();
            l.db_len = db->len.as<int>();
            l.c_begin = b.c_begin;
            l.c_end = b.c_end;
            l.q_len = ws.q_len.as<int>();
            l.nq = 1;
            l.band = band;
            l.env_lo = ws.env_lo.as<float>();
            l.env_hi = ws.env_hi.as<float>();
            l.env_stride = env;
            l.env_floats = (int)((int64_t)((b.n_hi + PPC - 1) / PPC) * CH);
            l.thr = ws.thr.as<float>();
            l.mu_prune = 1.f;
            l.out_lb = tmp;
            l.out_lb_stride = db->N;
            l.stats = ctrl->stats;
            l.status = &ctrl->status;
            l.n_lo = b.n_lo;
            l.n_hi = b.n_hi;
            launch_lb(l, db->deff, form, db->n_sm, st);
        }
    }
    // greedy form 0 keeps squared costs: report GDK itself (Euclidean)
    launch_scatter_by_id(tmp, db->id.as<int>(), db->N, 1, db->N, out, db->N,
                         greedy && form == 0, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess)
        e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_error(e, greedy ? "greedy bound" : mode == 2 ? "lb_seg" : "lb_box");
    int status = 0;
    cudaMemcpy(&status, &ctrl->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (status & KNN_DEV_TIMEOUT)
        return set_error(KNN_ERR_TIMEOUT, "a device wait gave up");
    return KNN_OK;
}

extern "C" knn_status knn_lb_box(knn_db *db, const float *query, int64_t m, float band,
                                 int32_t form, float *out_lb, void *stream)
{
    return bound_common(db, query, m, band, form, out_lb, stream, 0);
}

extern "C" knn_status knn_lb_seg(knn_db *db, const float *query, int64_t m, float band,
                                 int32_t form, float *out_lb, void *stream)
{
    return bound_common(db, query, m, band, form, out_lb, stream, 2);
}

extern "C" knn_status knn_greedy_ub(knn_db *db, const float *query, int64_t m, float band,
                                    int32_t form, float *out_ub, void *stream)
{
    return bound_common(db, query, m, band, form, out_ub, stream, 1);
}

// ---------------------------------------------------------------------------
// pair programs

__global__ void pairs_to_items(const int64_t *pa, const int64_t *pb, int64_t n, int2 *items,
                               float *lb)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x) {
        items[i] = make_int2((int)pb[i], (int)pa[i]);
        lb[i] = 0.f;
    }
}

__global__ void pair_out_kernel(const float *in, int64_t n, int kind, float *out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = kind == 0 ? in[i] : sqrtf(in[i]);
}

extern "C" knn_status knn_pairwise(const float *a, const int64_t *a_off, const float *b,
                                   const int64_t *b_off, const int64_t *pa, const int64_t *pb,
                                   int64_t n_pairs, int32_t d, float band, int32_t distance,
                                   float *out_f32, double *out_f64, void *stream)
{
    if (!a || !a_off || !b || !b_off || !pa || !pb)
        return set_error(KNN_ERR_INVALID, "NULL argument");
    if (n_pairs < 0 || n_pairs > 0x7fffffff || d < 1 || d > 16 || !(band > 0.f) ||
        (distance != 0 && distance != 1))
        return set_error(KNN_ERR_INVALID, "bad argument");
    if (n_pairs == 0)
        return KNN_OK;
    for (const void *p : {(const void *)a, (const void *)a_off, (const void *)b,
                          (const void *)b_off, (const void *)pa, (const void *)pb})
        if (!is_device_ptr(p))
            return set_error(KNN_ERR_INVALID, "knn_pairwise takes device pointers");
    cudaStream_t st = (cudaStream_t)stream;
    // host copies of the index data to size the band and the layout
    std::vector<int64_t> hpa(n_pairs), hpb(n_pairs);
    cudaMemcpy(hpa.data(), pa, 8 * n_pairs, cudaMemcpyDeviceToHost);
    cudaMemcpy(hpb.data(), pb, 8 * n_pairs, cudaMemcpyDeviceToHost);
    int64_t na = 0, nb = 0;
    for (int64_t i = 0; i < n_pairs; ++i) {
        if (hpa[i] < 0 || hpb[i] < 0)
            return set_error(KNN_ERR_INVALID, "negative pair index");
        na = std::max(na, hpa[i] + 1);
        nb = std::max(nb, hpb[i] + 1);
    }
    std::vector<int64_t> hao(na + 1), hbo(nb + 1);
    cudaMemcpy(hao.data(), a_off, 8 * (na + 1), cudaMemcpyDeviceToHost);
    cudaMemcpy(hbo.data(), b_off, 8 * (nb + 1), cudaMemcpyDeviceToHost);
    int max_r = 0;
    int max_n = 1;
    for (int64_t i = 0; i < n_pairs; ++i) {
        const int m = (int)(hao[hpa[i] + 1] - hao[hpa[i]]);
        const int n = (int)(hbo[hpb[i] + 1] - hbo[hpb[i]]);
        if (m < 1 || n < 1)
            return set_error(KNN_ERR_INVALID, "empty series in a pair");
        max_r = std::max(max_r, band_radius(m, n, band));
        max_n = std::max(max_n, std::max(m, n));
    }
    cudaError_t e = cudaSuccess;
    knn_status s;
    if (out_f32) {
        const int deff = deff_for(d);
        const int CH = chunk_floats(deff), PPC = chunk_points(deff);
        std::vector<int64_t> ra(na), rb(nb);
        std::vector<int> la(na), lb(nb), ida(nb);
        int64_t ta = 0, tb = 0;
        for (int64_t i = 0; i < na; ++i) {
            la[i] = (int)(hao[i + 1] - hao[i]);
            ta += CH;  // leading chunk: the DP's sentinel point
            ra[i] = ta;
            ta += (int64_t)((la[i] + PPC - 1) / PPC) * CH;
        }
        for (int64_t i = 0; i < nb; ++i) {
            lb[i] = (int)(hbo[i + 1] - hbo[i]);
            tb += CH;
            rb[i] = tb;
            tb += (int64_t)((lb[i] + PPC - 1) / PPC) * CH;
            ida[i] = (int)i;
        }
        DevBuf A, B, AO, BO, AL, BL, BID, IT, ILB, OUT, CT;
        if ((s = A.ensure(4 * ta)) || (s = B.ensure(4 * tb)) || (s = AO.ensure(8 * na)) ||
            (s = BO.ensure(8 * nb)) || (s = AL.ensure(4 * na)) || (s = BL.ensure(4 * nb)) ||
            (s = BID.ensure(4 * nb)) || (s = IT.ensure(8 * n_pairs)) ||
            (s = ILB.ensure(4 * n_pairs)) || (s = OUT.ensure(4 * n_pairs)) ||
            (s = CT.ensure(sizeof(Ctrl))))
            return s;
        cudaMemcpyAsync(AO.p, ra.data(), 8 * na, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(BO.p, rb.data(), 8 * nb, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(AL.p, la.data(), 4 * na, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(BL.p, lb.data(), 4 * nb, cudaMemcpyHostToDevice, st);
        cudaMemcpyAsync(BID.p, ida.data(), 4 * nb, cudaMemcpyHostToDevice, st);
        cudaMemsetAsync(CT.p, 0, sizeof(Ctrl), st);
        launch_repack(a, a_off, nullptr, (int)na, d, deff, AO.as<int64_t>(), A.as<float>(), st, true);
        launch_repack(b, b_off, nullptr, (int)nb, d, deff, BO.as<int64_t>(), B.as<float>(), st, true);
        pairs_to_items<<<256, 256, 0, st>>>(pa, pb, n_pairs, IT.as<int2>(), ILB.as<float>());
        Ctrl *ct = CT.as<Ctrl>();
        const int np = (int)n_pairs;
        cudaMemcpyAsync(&ct->seg_count[0], &np, 4, cudaMemcpyHostToDevice, st);
        int P = 0, G = 0;
        choose_dp_config(deff, max_r, max_n, &P, &G);
        if (!P)
            return set_error(KNN_ERR_UNSUPPORTED, "band too wide for the compiled DP variants");
        DpArgs x{};
        x.items = IT.as<int2>();
        x.item_lb = ILB.as<float>();
        x.n_items = &ct->seg_count[0];
        x.items_cap = n_pairs;
        x.head = &ct->seg_head[0];
        x.db = B.as<float>();
        x.db_off = BO.as<int64_t>();
        x.db_len = BL.as<int>();
        x.db_id = BID.as<int>();
        x.q = A.as<float>();
        x.q_off = AO.as<int64_t>();
        x.q_len = AL.as<int>();
        x.band = band;
        x.G = G;
        x.mu_keep = 1.f;
        x.mu_prune = 1.f;
        x.out_pair = OUT.as<float>();
        x.cells_stat = STAT_DP_CELLS;
        x.stats = ct->stats;
        x.status = &ct->status;
        int dev = 0, nsm = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
        if (!launch_dp(x, deff, P, distance, nsm, st)) {
            cudaStreamSynchronize(st);
            return set_error(KNN_ERR_UNSUPPORTED, "no DP kernel compiled for this d and shape");
        }
        pair_out_kernel<<<256, 256, 0, st>>>(OUT.as<float>(), n_pairs, distance, out_f32);
        e = cudaStreamSynchronize(st);
        if (e == cudaSuccess)
            e = cudaGetLastError();
        if (e != cudaSuccess)
            return cuda_error(e, "pairwise fp32");
    }
    if (out_f64) {
        const int row = 2 * max_r + 1;
        if ((size_t)3 * (row + 2) * sizeof(double) > 200 * 1024)
            return set_error(KNN_ERR_UNSUPPORTED, "band too wide for the FP64 pair program");
        launch_pairwise64(a, a_off, b, b_off, pa, pb, n_pairs, d, band, distance, out_f64, row,
                          st);
        e = cudaStreamSynchronize(st);
        if (e == cudaSuccess)
            e = cudaGetLastError();
        if (e != cudaSuccess)
            return cuda_error(e, "pairwise fp64");
    }
    return KNN_OK;
}

// ---------------------------------------------------------------------------

extern "C" knn_status knn_scan_simple(const float *query, int64_t m, const float *db_series,
                                      const int64_t *lengths, int64_t n_series, int32_t d,
                                      float band, int32_t k, float eps, int32_t distance,
                                      int64_t *ids, float *dist, int64_t *count)
{
    if (!query || !db_series || !lengths || !ids || !dist)
        return set_error(KNN_ERR_INVALID, "NULL argument");
    if (n_series < 1 || m < 1)
        return set_error(KNN_ERR_INVALID, "bad sizes");
    std::vector<int64_t> hl(n_series);
    if (is_device_ptr(lengths))
        cudaMemcpy(hl.data(), lengths, 8 * n_series, cudaMemcpyDeviceToHost);
    else
        memcpy(hl.data(), lengths, 8 * n_series);
    std::vector<int64_t> off(n_series + 1, 0);
    for (int64_t i = 0; i < n_series; ++i) {
        if (hl[i] < 1)
            return set_error(KNN_ERR_INVALID, "series length < 1");
        off[i + 1] = off[i] + hl[i];
    }
    knn_db *db = nullptr;
    knn_status s = knn_db_create(db_series, off.data(), n_series, d, nullptr, &db);
    if (s)
        return s;
    knn_params p{};
    p.k = k;
    p.eps = eps;
    p.band = band;
    p.distance = distance;
    p.seed_mode = KNN_SEED_GREEDY;
    p.eps_capacity = k > 0 ? 0 : std::min<int64_t>(n_series, 8192);
    int64_t qo[2] = {0, m};
    int64_t cnt = 0;
    s = knn_scan(db, query, qo, 1, &p, ids, dist, &cnt, nullptr, nullptr);
    if (count)
        *count = cnt;
    knn_db_destroy(db);
    return s;
}
