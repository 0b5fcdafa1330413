// C-ABI of the scan library: database layout, scan orchestration, components.
//
// Launch sequence of one query batch (all on the caller's stream, no host
// synchronisation between launches, so the whole sequence can be captured
// into a CUDA graph):
//   repack queries -> init thresholds/slots -> [greedy upper bounds per bucket]
//   -> per bucket: envelope, LB_Box stream (prune + survivor queue)
//   -> DP over the survivor queue -> finalise (FP64 boundary re-scoring, cut)
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/knnwarp.h"
#include "common.cuh"
#include "internal.h"
#include "runtime.h"

using namespace knn;

// ---------------------------------------------------------------------------
// errors

static thread_local std::string g_err;

knn_status knn::set_error(knn_status s, const std::string &msg)
{
    g_err = msg;
    return s;
}

knn_status knn::cuda_error(cudaError_t e, const char *what)
{
    cudaGetLastError();  // clear sticky-free errors
    return set_error(e == cudaErrorMemoryAllocation ? KNN_ERR_OOM : KNN_ERR_CUDA,
                     std::string(what) + ": " + cudaGetErrorString(e));
}

extern "C" const char *knn_status_string(knn_status s)
{
    switch (s) {
    case KNN_OK: return "ok";
    case KNN_ERR_INVALID: return "invalid argument";
    case KNN_ERR_OOM: return "out of device memory";
    case KNN_ERR_CUDA: return "CUDA error";
    case KNN_ERR_TIMEOUT: return "device wait timed out";
    case KNN_ERR_CAPACITY: return "result capacity exceeded";
    case KNN_ERR_UNSUPPORTED: return "unsupported configuration";
    }
    return "unknown status";
}

extern "C" const char *knn_last_error(void) { return g_err.c_str(); }

extern "C" const char *knn_version(void) { return "knnwarp 0.1 (sm_103a)"; }

// ---------------------------------------------------------------------------
// helpers

int knn::deff_for(int d)
{
    if (d >= 1 && d <= 8)
        return d;
    if (d <= 16)
        return 16;
    return 0;
}

bool knn::is_device_ptr(const void *p)
{
    if (!p)
        return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Fault injection for tests (host side, no GPU fault): KNN_FAULT_INJECT=alloc
// fails every device allocation of the library; alloc_after:N lets N more
// allocations succeed (counted from the first allocation that sees this
// value) and fails the ones after.
static bool alloc_fault_injected()
{
    static std::mutex mu;
    static std::string seen;
    static long remaining = 0;
    const char *f = getenv("KNN_FAULT_INJECT");
    std::lock_guard<std::mutex> lk(mu);
    if (!f) {
        seen.clear();
        return false;
    }
    if (!strcmp(f, "alloc"))
        return true;
    if (!strncmp(f, "alloc_after:", 12)) {
        if (seen != f) {
            seen = f;
            remaining = strtol(f + 12, nullptr, 10);
        }
        if (remaining > 0) {
            --remaining;
            return false;
        }
        return true;
    }
    return false;
}

knn_status DevBuf::ensure(size_t b)
{
    if (b <= bytes)
        return KNN_OK;
    release();
    if (alloc_fault_injected())
        return set_error(KNN_ERR_OOM, "allocation failure injected (KNN_FAULT_INJECT)");
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) {
        p = nullptr;
        return cuda_error(e, "cudaMalloc");
    }
    bytes = b;
    return KNN_OK;
}

void DevBuf::release()
{
    if (p)
        cudaFree(p);
    p = nullptr;
    bytes = 0;
}

Margins knn::margins_for(int kind, int max_path, int d)
{
    const double u = std::ldexp(1.0, -24);
    double w;
    if (kind == 0)
        w = 2.0 * (max_path + d + 8) * u;  // DTW: sum along a path of <= m+n-1 cells
    else
        w = 2.0 * (d + 8) * u;             // DK: one cost of d terms, then max/min only
    Margins g;
    g.rerank_rel = (float)w;
    g.mu_keep = (float)(1.0 + w);
    g.mu_prune = (float)(1.0 + 3.0 * w);
    return g;
}

static int next_pow2(int v)
{
    int p = 1;
    while (p < v)
        p <<= 1;
    return p;
}

// Default (P, G) for a band radius r: minimise the modelled lane work
// G * (n + P + 1) * (2P(2d+3) + overhead) subject to G*P >= r+1, G <= 32.
namespace {
// Resident CTAs per SM of the DTW variant (d, P), looked up once.
int dp_blocks_cached(int deff, int P)
{
    static int cache[17][33];
    static bool filled[17][33];
    if (deff < 1 || deff > 16 || P < 1 || P > 32)
        return 1;
    if (!filled[deff][P]) {
        cache[deff][P] = knn::dp_max_blocks_per_sm(deff, P, 0);
        filled[deff][P] = true;
    }
    return cache[deff][P] > 0 ? cache[deff][P] : 1;
}
}  // namespace

void knn::choose_dp_config(int deff, int r, int n, int *P_out, int *G_out)
{
    double best = 1e300;
    int bp = 0, bg = 0;
    const int nv = dp_num_variants(deff);
    for (int v = 0; v < nv; ++v) {
        const int P = dp_variant_P(deff, v);
        int G = next_pow2((r + 1 + P - 1) / P);
        if (G < 1)
            G = 1;
        if (G > 32)
            continue;
        const double per_step = 2.0 * P * (2 * deff + 3) + 16.0 + 2.0 * deff;
        // fewer than 16 resident warps per SM leave latency uncovered: the
        // kernel then runs at about that fraction of its issue rate
        const double warps = (double)dp_blocks_cached(deff, P) * dp_block_threads() / 32.0;
        const double cost = (double)G * (n + P + 1) * per_step / std::min(1.0, std::max(warps, 1.0) / 16.0);
        if (cost < best) {
            best = cost;
            bp = P;
            bg = G;
        }
    }
    *P_out = bp;
    *G_out = bg;
}

// ---------------------------------------------------------------------------
// database

__global__ void check_finite_kernel(const float *p, int64_t n, int *flag)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        if (!isfinite(p[i])) {
            *flag = 1;
            return;
        }
}

knn_status knn::check_finite_dev(const float *dev, int64_t n, int *flag_dev, cudaStream_t st,
                               bool *ok)
{
    cudaError_t e = cudaMemsetAsync(flag_dev, 0, sizeof(int), st);
    if (e != cudaSuccess)
        return cuda_error(e, "cudaMemsetAsync");
    if (n > 0) {
        int64_t b = (n + 255) / 256;
        check_finite_kernel<<<(int)std::min<int64_t>(b, 4096), 256, 0, st>>>(dev, n, flag_dev);
    }
    int h = 0;
    e = cudaMemcpyAsync(&h, flag_dev, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return cuda_error(e, "finite check");
    *ok = h == 0;
    return KNN_OK;
}

// Builds the library layout of N series whose point offsets into `series`
// are hoff[0..N) (hoff[N]: the end of the source points); fixed_len > 0: every
// series has that length (windows may overlap), else series i ends at
// hoff[i+1].  Lengths are validated by the caller.
static knn_status db_build(const float *series, const std::vector<int64_t> &hoff, int N, int32_t d,
                           int max_len, int fixed_len, cudaStream_t st, knn_db **out)
{
    const int64_t n_series = N;
    const int deff = deff_for(d);
    const int CH = chunk_floats(deff), PPC = chunk_points(deff);
    auto len_of = [&](int i) -> int64_t {
        return fixed_len > 0 ? fixed_len : hoff[i + 1] - hoff[i];
    };

    static std::once_flag attr_once;
    std::call_once(attr_once, [] {
        lb_init_attributes();
        fin_init_attributes();
        lbc_init_attributes();
    });
    auto db = new knn_db();
    db->d = d;
    db->deff = deff;
    db->N = N;
    cudaGetDevice(&db->dev);
    cudaDeviceGetAttribute(&db->n_sm, cudaDevAttrMultiProcessorCount, db->dev);
    db->max_len = max_len;

    // length buckets: stable sort by length, a new bucket whenever the length
    // exceeds the bucket's shortest by more than the bucket width
    std::vector<int> order(N);
    for (int i = 0; i < N; ++i)
        order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return len_of(a) < len_of(b);
    });
    db->h_len.resize(N);
    db->h_len_by_id.resize(N);
    std::vector<int64_t> doff(N), doff_by_id(N);
    int64_t total = 0;
    for (int c = 0; c < N; ++c) {
        const int id = order[c];
        const int n = (int)len_of(id);
        db->h_len[c] = n;
        db->h_len_by_id[id] = n;
        total += CH;  // leading chunk: the DP's sentinel point
        doff[c] = total;
        doff_by_id[id] = total;
        total += (int64_t)((n + PPC - 1) / PPC) * CH;
    }
    db->total_floats = total;
    for (int c = 0; c < N;) {
        Bucket b;
        b.c_begin = c;
        b.n_lo = db->h_len[c];
        const int width = std::max(16, b.n_lo / 16);
        while (c < N && db->h_len[c] <= b.n_lo + width)
            ++c;
        b.c_end = c;
        b.n_hi = db->h_len[c - 1];
        db->buckets.push_back(b);
    }

    knn_status s;
    if ((s = db->data.ensure(sizeof(float) * total)) ||
        (s = db->off.ensure(sizeof(int64_t) * N)) || (s = db->len.ensure(sizeof(int) * N)) ||
        (s = db->id.ensure(sizeof(int) * N)) || (s = db->off_by_id.ensure(sizeof(int64_t) * N)) ||
        (s = db->len_by_id.ensure(sizeof(int) * N))) {
        delete db;
        return s;
    }
    cudaError_t e = cudaSuccess;
    auto cpy = [&](void *dst, const void *src, size_t bytes) {
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st);
    };
    cpy(db->off.p, doff.data(), sizeof(int64_t) * N);
    cpy(db->len.p, db->h_len.data(), sizeof(int) * N);
    cpy(db->id.p, order.data(), sizeof(int) * N);
    cpy(db->off_by_id.p, doff_by_id.data(), sizeof(int64_t) * N);
    cpy(db->len_by_id.p, db->h_len_by_id.data(), sizeof(int) * N);

    // source series and offsets on the device
    DevBuf src_stage, off_stage;
    const float *src = series;
    const int64_t npts = hoff[n_series];
    if (!is_device_ptr(series)) {
        if ((s = src_stage.ensure(sizeof(float) * npts * d))) {
            delete db;
            return s;
        }
        cpy(src_stage.p, series, sizeof(float) * npts * d);
        src = (const float *)src_stage.p;
    }
    if ((s = off_stage.ensure(sizeof(int64_t) * (n_series + 1)))) {
        delete db;
        return s;
    }
    cpy(off_stage.p, hoff.data(), sizeof(int64_t) * (n_series + 1));
    if (e != cudaSuccess) {
        delete db;
        return cuda_error(e, "copy database");
    }
    if ((s = db->ws.ctrl.ensure(4096))) {
        delete db;
        return s;
    }
    bool ok = true;
    if ((s = check_finite_dev(src + hoff[0] * d, (npts - hoff[0]) * d, (int *)db->ws.ctrl.p, st, &ok))) {
        delete db;
        return s;
    }
    if (!ok) {
        delete db;
        return set_error(KNN_ERR_INVALID, "database contains NaN or Inf");
    }
    launch_repack(src, (const int64_t *)off_stage.p, (const int *)db->id.p, N, d, deff,
                  (const int64_t *)db->off.p, (float *)db->data.p, st, true, fixed_len);

    // coarse first stage of the LB_Box cascade: scaled segment means of every
    // series (full segments only) and the largest coordinate magnitude
    int min_len = N > 0 ? db->h_len[0] : 0;
    for (int c = 1; c < N; ++c)
        min_len = std::min(min_len, db->h_len[c]);
    const int W = coarse_width(deff, min_len);
    std::vector<int64_t> sg_off(N), sg_end(N);
    int64_t sg_total = 0;
    for (int c = 0; c < N; ++c) {
        const int nseg = db->h_len[c] / W;
        sg_off[c] = sg_total;
        sg_total += (int64_t)((nseg + PPC - 1) / PPC) * CH;
        sg_end[c] = sg_total;
    }
    DevBuf sg_end_dev;
    if ((s = db->sg.ensure(sizeof(float) * std::max<int64_t>(sg_total, 4))) ||
        (s = db->sg_off.ensure(sizeof(int64_t) * N)) ||
        (s = sg_end_dev.ensure(sizeof(int64_t) * N))) {
        delete db;
        return s;
    }
    cpy(db->sg_off.p, sg_off.data(), sizeof(int64_t) * N);
    cpy(sg_end_dev.p, sg_end.data(), sizeof(int64_t) * N);
    if (e != cudaSuccess) {
        delete db;
        return cuda_error(e, "copy segment offsets");
    }
    launch_seg_means((const float *)db->data.p, (const int64_t *)db->off.p,
                     (const int *)db->len.p, N, deff, W, (const int64_t *)db->sg_off.p,
                     (const int64_t *)sg_end_dev.p, (float *)db->sg.p, st);
    unsigned int *amax = reinterpret_cast<unsigned int *>((char *)db->ws.ctrl.p + 256);
    launch_absmax(src + hoff[0] * d, (npts - hoff[0]) * d, amax, st);
    unsigned int amax_bits = 0;
    e = cudaMemcpyAsync(&amax_bits, amax, sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e == cudaSuccess)
        e = cudaGetLastError();
    if (e != cudaSuccess) {
        delete db;
        return cuda_error(e, "repack database");
    }
    memcpy(&db->absmax, &amax_bits, sizeof(float));
    db->seg_w = W;
    *out = db;
    return KNN_OK;
}

extern "C" knn_status knn_db_create(const float *series, const int64_t *offsets, int64_t n_series,
                                    int32_t d, void *stream, knn_db **out)
{
    if (!out)
        return set_error(KNN_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!series || !offsets)
        return set_error(KNN_ERR_INVALID, "series/offsets is NULL");
    if (n_series < 1 || n_series > (int64_t)0x7fffffff)
        return set_error(KNN_ERR_INVALID, "n_series must be in [1, 2^31)");
    if (d < 1 || d > 16)
        return set_error(KNN_ERR_INVALID, "d must be in [1, 16]");
    cudaStream_t st = (cudaStream_t)stream;
    const int deff = deff_for(d);
    const int CH = chunk_floats(deff), PPC = chunk_points(deff);

    std::vector<int64_t> hoff(n_series + 1);
    const bool off_dev = is_device_ptr(offsets);
    if (off_dev) {
        cudaError_t e = cudaMemcpy(hoff.data(), offsets, sizeof(int64_t) * (n_series + 1),
                                   cudaMemcpyDeviceToHost);
        if (e != cudaSuccess)
            return cuda_error(e, "copy offsets");
    } else {
        memcpy(hoff.data(), offsets, sizeof(int64_t) * (n_series + 1));
    }
    if (hoff[0] < 0)
        return set_error(KNN_ERR_INVALID, "offsets[0] < 0");
    int max_len = 0;
    for (int64_t i = 0; i < n_series; ++i) {
        const int64_t L = hoff[i + 1] - hoff[i];
        if (L < 1)
            return set_error(KNN_ERR_INVALID, "series " + std::to_string(i) + " has length < 1");
        if (L > 65536)
            return set_error(KNN_ERR_UNSUPPORTED, "series longer than 65536 points");
        max_len = std::max<int>(max_len, (int)L);
    }
    return db_build(series, hoff, (int)n_series, d, max_len, 0, st, out);
}

extern "C" knn_status knn_db_create_windows(const float *series, int64_t n, int32_t d,
                                            int32_t m, int32_t stride, void *stream,
                                            knn_db **out)
{
    if (!out)
        return set_error(KNN_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!series)
        return set_error(KNN_ERR_INVALID, "series is NULL");
    if (d < 1 || d > 16)
        return set_error(KNN_ERR_INVALID, "d must be in [1, 16]");
    if (m < 1 || n < m || stride < 1)
        return set_error(KNN_ERR_INVALID, "need 1 <= m <= n and stride >= 1");
    if (m > 65536)
        return set_error(KNN_ERR_UNSUPPORTED, "windows longer than 65536 points");
    const int64_t N = (n - m) / stride + 1;
    if (N > (int64_t)0x7fffffff)
        return set_error(KNN_ERR_INVALID, "more than 2^31 - 1 windows");
    std::vector<int64_t> hoff(N + 1);
    for (int64_t i = 0; i < N; ++i)
        hoff[i] = i * stride;
    hoff[N] = n;
    return db_build(series, hoff, (int)N, d, m, m, (cudaStream_t)stream, out);
}

extern "C" knn_status knn_db_destroy(knn_db *db)
{
    if (!db)
        return set_error(KNN_ERR_INVALID, "db is NULL");
    cudaDeviceSynchronize();
    delete db;
    return KNN_OK;
}

extern "C" knn_status knn_db_info(const knn_db *db, int64_t *n_series, int32_t *d,
                                  int32_t *n_buckets)
{
    if (!db)
        return set_error(KNN_ERR_INVALID, "db is NULL");
    if (n_series)
        *n_series = db->N;
    if (d)
        *d = db->d;
    if (n_buckets)
        *n_buckets = (int32_t)db->buckets.size();
    return KNN_OK;
}
