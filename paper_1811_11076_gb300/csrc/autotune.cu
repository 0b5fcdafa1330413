// Autotuner for the shape of the banded DP: P band cells per lane and G lanes
// per (query, series) pair, chosen per (distance, band radius, length) key.
//
// Every length bucket of the database has its own key.  For each key the
// compiled P values are tried with the smallest G that covers the band
// (G*P >= r+1) and with twice that G; the whole scan is run on the given
// queries with one DP launch per bucket, each launch timed with CUDA events,
// and the fastest shape per key is kept in the database handle (later scans
// use it).  Results can be cached in a small JSON file keyed by the device
// name and the dimensionality.
#include <algorithm>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "runtime.h"

using namespace knn;

namespace {

struct Key {
    int kind, r, n;
};

int next_pow2(int v)
{
    int p = 1;
    while (p < v)
        p <<= 1;
    return p;
}

std::vector<DpChoice> candidates(int deff, int r)
{
    std::vector<DpChoice> out;
    const int nv = dp_num_variants(deff);
    for (int v = 0; v < nv; ++v) {
        const int P = dp_variant_P(deff, v);
        const int G = next_pow2((r + 1 + P - 1) / P);
        if (G <= 32)
            out.push_back({P, G});
        if (2 * G <= 32)
            out.push_back({P, 2 * G});
    }
    return out;
}

std::string device_name(int dev)
{
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess)
        return "unknown";
    return prop.name;
}

// One entry per line:
// {"device": "...", "d": 3, "kind": 0, "r": 25, "n": 256, "P": 13, "G": 2, "ms": 1.5}
void load_cache(const char *path, const std::string &dev, int deff,
                std::map<std::tuple<int, int, int>, DpChoice> &out)
{
    FILE *f = fopen(path, "r");
    if (!f)
        return;
    char line[512];
    while (fgets(line, sizeof line, f)) {
        const char *dp = strstr(line, "\"device\": \"");
        if (!dp)
            continue;
        dp += 11;
        const char *de = strchr(dp, '"');
        if (!de || std::string(dp, de) != dev)
            continue;
        int d = 0, kind = 0, r = 0, n = 0, P = 0, G = 0;
        const char *rest = strstr(de, "\"d\":");
        if (!rest || sscanf(rest, "\"d\": %d, \"kind\": %d, \"r\": %d, \"n\": %d, \"P\": %d, \"G\": %d",
                            &d, &kind, &r, &n, &P, &G) != 6)
            continue;
        if (d != deff)
            continue;
        bool compiled = false;
        for (int v = 0; v < dp_num_variants(deff); ++v)
            compiled |= dp_variant_P(deff, v) == P;
        if (compiled && G >= 1 && G <= 32 && (G & (G - 1)) == 0 && G * P >= r + 1)
            out[std::make_tuple(kind, r, n)] = {P, G};
    }
    fclose(f);
}

void save_cache(const char *path, const std::string &dev, int deff,
                const std::map<std::tuple<int, int, int>, DpChoice> &tuned,
                const std::map<std::tuple<int, int, int>, double> &ms)
{
    // keep other devices' / dimensionalities' lines, replace ours
    std::vector<std::string> keep;
    if (FILE *f = fopen(path, "r")) {
        char line[512];
        while (fgets(line, sizeof line, f)) {
            if (!strstr(line, "\"device\""))
                continue;
            std::string l(line);
            char probe[160];
            snprintf(probe, sizeof probe, "\"device\": \"%s\", \"d\": %d,", dev.c_str(), deff);
            if (l.find(probe) == std::string::npos) {
                while (!l.empty() && (l.back() == '\n' || l.back() == ','))
                    l.pop_back();
                keep.push_back(l);
            }
        }
        fclose(f);
    }
    for (auto &kv : tuned) {
        char buf[320];
        auto it = ms.find(kv.first);
        snprintf(buf, sizeof buf,
                 "{\"device\": \"%s\", \"d\": %d, \"kind\": %d, \"r\": %d, \"n\": %d, \"P\": %d, "
                 "\"G\": %d, \"ms\": %.4f}",
                 dev.c_str(), deff, std::get<0>(kv.first), std::get<1>(kv.first),
                 std::get<2>(kv.first), kv.second.P, kv.second.G,
                 it == ms.end() ? -1.0 : it->second);
        keep.push_back(buf);
    }
    const std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f)
        return;
    fprintf(f, "{\"dp_shapes\": [\n");
    for (size_t i = 0; i < keep.size(); ++i)
        fprintf(f, "%s%s\n", keep[i].c_str(), i + 1 < keep.size() ? "," : "");
    fprintf(f, "]}\n");
    fclose(f);
    rename(tmp.c_str(), path);
}

}  // namespace

extern "C" knn_status knn_autotune(knn_db *db, const float *queries, const int64_t *q_offsets,
                                   int32_t n_queries, const knn_params *params,
                                   const char *cache_path, void *stream)
{
    if (!db || !queries || !q_offsets || !params)
        return set_error(KNN_ERR_INVALID, "NULL argument");
    if (n_queries < 1 || params->k < 1)
        return set_error(KNN_ERR_INVALID, "autotune needs k-NN parameters and >= 1 query");
    const std::string dev = device_name(db->dev);
    std::vector<int64_t> hq(n_queries + 1);
    if (is_device_ptr(q_offsets))
        cudaMemcpy(hq.data(), q_offsets, 8 * (n_queries + 1), cudaMemcpyDeviceToHost);
    else
        memcpy(hq.data(), q_offsets, 8 * (n_queries + 1));
    int max_m = 0;
    for (int i = 0; i < n_queries; ++i)
        max_m = std::max<int>(max_m, (int)(hq[i + 1] - hq[i]));
    std::vector<Key> keys;
    for (auto &b : db->buckets)
        keys.push_back({params->distance, band_radius(max_m, b.n_hi, params->band), b.n_hi});
    std::map<std::tuple<int, int, int>, DpChoice> cached;
    if (cache_path)
        load_cache(cache_path, dev, db->deff, cached);
    bool all_cached = true;
    for (auto &k : keys)
        all_cached &= cached.count(std::make_tuple(k.kind, k.r, k.n)) > 0;
    if (all_cached) {
        for (auto &kv : cached)
            db->tuned[kv.first] = kv.second;
        return KNN_OK;
    }
    std::vector<std::vector<DpChoice>> cand(keys.size());
    size_t trials = 0;
    for (size_t b = 0; b < keys.size(); ++b) {
        cand[b] = candidates(db->deff, keys[b].r);
        trials = std::max(trials, cand[b].size());
    }
    knn_params p = *params;
    p.profile = 1;
    p.use_graph = 0;
    const int width = p.k;
    std::vector<int64_t> ids((size_t)n_queries * width);
    std::vector<float> dist((size_t)n_queries * width);
    std::vector<double> best(keys.size(), 1e300);
    std::vector<DpChoice> best_c(keys.size());
    auto saved = db->tuned;
    db->tuning = true;
    knn_status s = KNN_OK;
    // trial 0 warms the caches and the workspace; its times are discarded
    for (size_t t = 0; t <= trials && !s; ++t) {
        const size_t ti = t == 0 ? 0 : t - 1;
        for (size_t b = 0; b < keys.size(); ++b)
            db->tuned[std::make_tuple(keys[b].kind, keys[b].r, keys[b].n)] =
                cand[b][std::min(ti, cand[b].size() - 1)];
        s = knn_scan(db, queries, q_offsets, n_queries, &p, ids.data(), dist.data(), nullptr,
                     nullptr, stream);
        if (s || t == 0)
            continue;
        for (size_t si = 0; si < db->seg_ms.size(); ++si) {
            const int b = db->seg_first_bucket[si];
            if (ti < cand[b].size() && db->seg_ms[si] < best[b]) {
                best[b] = db->seg_ms[si];
                best_c[b] = cand[b][ti];
            }
        }
    }
    db->tuning = false;
    db->tuned = saved;
    if (s)
        return s;
    std::map<std::tuple<int, int, int>, double> ms;
    for (size_t b = 0; b < keys.size(); ++b) {
        const auto key = std::make_tuple(keys[b].kind, keys[b].r, keys[b].n);
        if (best[b] < 1e300) {
            db->tuned[key] = best_c[b];
            ms[key] = best[b];
        }
    }
    for (auto &kv : cached)
        if (!db->tuned.count(kv.first))
            db->tuned[kv.first] = kv.second;
    // queries per LB_Box pass: time the LB stage with each tile
    if (n_queries >= 8) {
        double best_lb = 1e300;
        int best_q = 0;
        for (int qt : {16, 8, 4}) {
            db->lb_qtile[p.distance] = qt;
            knn_stats st{};
            double tot = 0.0;
            for (int rep = 0; rep < 2 && !s; ++rep) {
                s = knn_scan(db, queries, q_offsets, n_queries, &p, ids.data(), dist.data(),
                             nullptr, &st, stream);
                if (rep == 1)
                    tot = st.ms_lb;
            }
            if (s)
                break;
            if (tot < best_lb) {
                best_lb = tot;
                best_q = qt;
            }
        }
        db->lb_qtile[p.distance] = best_q;
        if (s)
            return s;
    }
    if (cache_path)
        save_cache(cache_path, dev, db->deff, db->tuned, ms);
    return KNN_OK;
}

extern "C" knn_status knn_set_dp_shape(knn_db *db, int32_t distance, int32_t r, int32_t n,
                                       int32_t P, int32_t G)
{
    if (!db)
        return set_error(KNN_ERR_INVALID, "db is NULL");
    bool compiled = false;
    for (int v = 0; v < dp_num_variants(db->deff); ++v)
        compiled |= dp_variant_P(db->deff, v) == P;
    if (!compiled)
        return set_error(KNN_ERR_UNSUPPORTED, "P not compiled for this dimensionality");
    if (G < 1 || G > 32 || (G & (G - 1)) || G * P < r + 1)
        return set_error(KNN_ERR_INVALID, "G must be a power of two <= 32 with G*P >= r+1");
    db->tuned[std::make_tuple((int)distance, (int)r, (int)n)] = {P, G};
    return KNN_OK;
}

extern "C" knn_status knn_get_dp_shape(knn_db *db, int32_t distance, int32_t r, int32_t n,
                                       int32_t *P, int32_t *G)
{
    if (!db || !P || !G)
        return set_error(KNN_ERR_INVALID, "NULL argument");
    DpChoice c = dp_choice(db, distance, r, n);
    *P = c.P;
    *G = c.G;
    return c.P ? KNN_OK : set_error(KNN_ERR_UNSUPPORTED, "no compiled shape covers the band");
}

extern "C" knn_status knn_set_lb_tile(knn_db *db, int32_t distance, int32_t qtile,
                                      int32_t window_chunks, int32_t compaction)
{
    if (!db)
        return set_error(KNN_ERR_INVALID, "db is NULL");
    if (distance != KNN_DTW && distance != KNN_DK)
        return set_error(KNN_ERR_INVALID, "distance must be KNN_DTW or KNN_DK");
    if (qtile != 0 && qtile != 4 && qtile != 8 && qtile != 16)
        return set_error(KNN_ERR_INVALID, "qtile must be 0, 4, 8 or 16");
    if (window_chunks < 0)
        return set_error(KNN_ERR_INVALID, "window_chunks must be >= 0");
    if (compaction < 0 || compaction > 2)
        return set_error(KNN_ERR_INVALID, "compaction must be 0, 1 or 2");
    db->lb_qtile[distance] = qtile;
    db->lb_window[distance] = window_chunks;
    db->lb_compact[distance] = compaction;
    return KNN_OK;
}

extern "C" knn_status knn_get_lb_tile(knn_db *db, int32_t distance, int32_t *qtile,
                                      int32_t *window_chunks, int32_t *compaction)
{
    if (!db || !qtile || !window_chunks || !compaction)
        return set_error(KNN_ERR_INVALID, "NULL argument");
    if (distance != KNN_DTW && distance != KNN_DK)
        return set_error(KNN_ERR_INVALID, "distance must be KNN_DTW or KNN_DK");
    *qtile = db->lb_qtile[distance];
    *window_chunks = db->lb_window[distance];
    *compaction = db->lb_compact[distance];
    return KNN_OK;
}

extern "C" knn_status knn_set_lb_cascade(knn_db *db, int32_t distance, int32_t coarse)
{
    if (!db)
        return set_error(KNN_ERR_INVALID, "db is NULL");
    if (distance != KNN_DTW && distance != KNN_DK)
        return set_error(KNN_ERR_INVALID, "distance must be KNN_DTW or KNN_DK");
    if (coarse != 0 && coarse != 1)
        return set_error(KNN_ERR_INVALID, "coarse must be 0 (automatic) or 1 (never)");
    db->lb_coarse[distance] = coarse;
    return KNN_OK;
}

extern "C" knn_status knn_get_lb_cascade(knn_db *db, int32_t distance, int32_t *coarse,
                                         int32_t *segment_width)
{
    if (!db || !coarse)
        return set_error(KNN_ERR_INVALID, "NULL argument");
    if (distance != KNN_DTW && distance != KNN_DK)
        return set_error(KNN_ERR_INVALID, "distance must be KNN_DTW or KNN_DK");
    *coarse = db->lb_coarse[distance];
    if (segment_width)
        *segment_width = db->seg_w;
    return KNN_OK;
}

extern "C" int32_t knn_dp_shapes(int32_t d, int32_t *P_list, int32_t cap)
{
    const int deff = deff_for(d);
    const int nv = deff ? dp_num_variants(deff) : 0;
    for (int v = 0; v < nv && v < cap; ++v)
        if (P_list)
            P_list[v] = dp_variant_P(deff, v);
    return nv;
}
