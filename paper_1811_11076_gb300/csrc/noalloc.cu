// knn_pairwise_noalloc: the FP32 pair programs of knn_pairwise without any
// device allocation.
//
// Some callers cannot let this library call cudaMalloc: an application whose
// device memory is owned by its own allocator or memory pool, or a
// latency-critical loop in which cudaMalloc / cudaFree (which may synchronise
// the whole device) are not acceptable.  This entry point takes the caller's
// inputs and outputs as they are and keeps everything else it needs — the
// repacked series, the work queue of pairs, the per-pair results and the
// control block of counters — in one file-scope __device__ array of fixed
// size, declared below.  Every GPU that loads the library holds that array
// (about 9.4 MB) until the process exits.
//
// The array is shared by every call on a device and keeps the last call's
// contents; each call clears what must start at zero (the control block).
// Calls that overlap on the GPU (two streams, two host threads) race on the
// array and must be serialised by the caller.
//
// Host code may not use the array's name as a device address (in host code
// it is only a stand-in).  The first call on each device, with that device
// current, looks the address up once with cudaGetSymbolAddress and caches it;
// because of that set-up, make the first call on a device before capturing
// any stream.
#include <mutex>

#include "common.cuh"
#include "runtime.h"

using namespace knn;

namespace {

constexpr int64_t NA_MAX_PAIRS = 65536;
constexpr int64_t NA_MAX_SERIES = 16384;       // per set (a and b)
constexpr int64_t NA_MAX_FLOATS = 1 << 20;     // per set, after repacking

constexpr size_t align256(size_t v) { return (v + 255) / 256 * 256; }
constexpr size_t OFF_CTRL = 0;
constexpr size_t OFF_A = align256(OFF_CTRL + sizeof(Ctrl));
constexpr size_t OFF_B = align256(OFF_A + sizeof(float) * NA_MAX_FLOATS);
constexpr size_t OFF_AOFF = align256(OFF_B + sizeof(float) * NA_MAX_FLOATS);
constexpr size_t OFF_ALEN = align256(OFF_AOFF + sizeof(int64_t) * NA_MAX_SERIES);
constexpr size_t OFF_BOFF = align256(OFF_ALEN + sizeof(int) * NA_MAX_SERIES);
constexpr size_t OFF_BLEN = align256(OFF_BOFF + sizeof(int64_t) * NA_MAX_SERIES);
constexpr size_t OFF_BID = align256(OFF_BLEN + sizeof(int) * NA_MAX_SERIES);
constexpr size_t OFF_ITEMS = align256(OFF_BID + sizeof(int) * NA_MAX_SERIES);
constexpr size_t OFF_ILB = align256(OFF_ITEMS + sizeof(int2) * NA_MAX_PAIRS);
constexpr size_t OFF_RES = align256(OFF_ILB + sizeof(float) * NA_MAX_PAIRS);
constexpr size_t NA_BYTES = align256(OFF_RES + sizeof(float) * NA_MAX_PAIRS);

enum : int { NA_BAD_LENGTH = 8, NA_BAD_INDEX = 16, NA_TOO_LARGE = 32 };

}  // namespace

// The scratch of knn_pairwise_noalloc (see the top of this file).
static __device__ __align__(256) unsigned char knn_noalloc_scratch[NA_BYTES];

namespace {

struct NaPtrs {
    Ctrl *ctrl;
    float *a, *b;
    int64_t *a_off, *b_off;
    int *a_len, *b_len, *b_id;
    int2 *items;
    float *ilb, *res;
};

NaPtrs carve(unsigned char *base)
{
    NaPtrs p;
    p.ctrl = reinterpret_cast<Ctrl *>(base + OFF_CTRL);
    p.a = reinterpret_cast<float *>(base + OFF_A);
    p.b = reinterpret_cast<float *>(base + OFF_B);
    p.a_off = reinterpret_cast<int64_t *>(base + OFF_AOFF);
    p.a_len = reinterpret_cast<int *>(base + OFF_ALEN);
    p.b_off = reinterpret_cast<int64_t *>(base + OFF_BOFF);
    p.b_len = reinterpret_cast<int *>(base + OFF_BLEN);
    p.b_id = reinterpret_cast<int *>(base + OFF_BID);
    p.items = reinterpret_cast<int2 *>(base + OFF_ITEMS);
    p.ilb = reinterpret_cast<float *>(base + OFF_ILB);
    p.res = reinterpret_cast<float *>(base + OFF_RES);
    return p;
}

// Device address of the scratch array on the current device, looked up once
// per device ordinal and kept for the life of the process.  The address
// belongs to the device's primary context: an application that destroys that
// context (cudaDeviceReset) must not call knn_pairwise_noalloc on the device
// afterwards, since the array may then live elsewhere.
knn_status scratch_base(unsigned char **out)
{
    static std::mutex mu;
    static unsigned char *cache[64] = {};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess)
        return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64)
        return set_error(KNN_ERR_UNSUPPORTED, "device ordinal above 63");
    std::lock_guard<std::mutex> lk(mu);
    if (!cache[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, knn_noalloc_scratch);
        if (e != cudaSuccess)
            return cuda_error(e, "cudaGetSymbolAddress(knn_noalloc_scratch)");
        cache[dev] = static_cast<unsigned char *>(p);
    }
    *out = cache[dev];
    return KNN_OK;
}

// Repacked offsets of one set: exclusive prefix sum of the chunk-padded
// sizes, computed by one block; flags bad lengths and overflow.
__device__ void na_offsets(const int64_t *off, int n, int max_len, int ppc, int chf,
                           int64_t *roff, int *rlen, int *flag, int64_t *total_out)
{
    __shared__ int64_t part[1024];
    const int T = blockDim.x, t = threadIdx.x;
    const int per = (n + T - 1) / T;
    const int s0 = min(n, t * per), s1 = min(n, s0 + per);
    int64_t sum = 0;
    for (int s = s0; s < s1; ++s) {
        const int64_t L = off[s + 1] - off[s];
        if (L < 1 || L > max_len)
            atomicOr(flag, NA_BAD_LENGTH);
        const int64_t Lc = L < 1 ? 1 : (L > max_len ? max_len : L);
        sum += chf + (Lc + ppc - 1) / ppc * chf;  // sentinel chunk + the series
    }
    part[t] = sum;
    __syncthreads();
    if (t == 0) {
        int64_t acc = 0;
        for (int i = 0; i < T; ++i) {
            const int64_t v = part[i];
            part[i] = acc;
            acc += v;
        }
        *total_out = acc;
    }
    __syncthreads();
    int64_t acc = part[t];
    for (int s = s0; s < s1; ++s) {
        const int64_t L = off[s + 1] - off[s];
        const int64_t Lc = L < 1 ? 1 : (L > max_len ? max_len : L);
        acc += chf;  // leading chunk: the DP's sentinel point
        roff[s] = acc;
        rlen[s] = (int)Lc;
        acc += (Lc + ppc - 1) / ppc * chf;
    }
}

__global__ void __launch_bounds__(1024) na_prepare_kernel(NaPtrs p, const int64_t *a_off, int n_a,
                                                          const int64_t *b_off, int n_b,
                                                          const int64_t *pa, const int64_t *pb,
                                                          int n_pairs, int max_len, int deff)
{
    __shared__ int64_t tot_a, tot_b;
    __shared__ int flag;
    // clear the control block: counters, cursors, status and statistics
    int *c = reinterpret_cast<int *>(p.ctrl);
    for (int i = threadIdx.x; i < (int)(sizeof(Ctrl) / sizeof(int)); i += blockDim.x)
        c[i] = 0;
    if (threadIdx.x == 0)
        flag = 0;
    __syncthreads();
    const int chf = chunk_floats(deff), ppc = chunk_points(deff);
    na_offsets(a_off, n_a, max_len, ppc, chf, p.a_off, p.a_len, &flag, &tot_a);
    __syncthreads();
    na_offsets(b_off, n_b, max_len, ppc, chf, p.b_off, p.b_len, &flag, &tot_b);
    for (int i = threadIdx.x; i < n_b; i += blockDim.x)
        p.b_id[i] = i;
    for (int i = threadIdx.x; i < n_pairs; i += blockDim.x)
        if (pa[i] < 0 || pa[i] >= n_a || pb[i] < 0 || pb[i] >= n_b)
            atomicOr(&flag, NA_BAD_INDEX);
    __syncthreads();
    if (threadIdx.x == 0) {
        int f = flag;
        if (tot_a > NA_MAX_FLOATS || tot_b > NA_MAX_FLOATS)
            f |= NA_TOO_LARGE;
        p.ctrl->status = f;
        p.ctrl->seg_count[0] = f ? 0 : n_pairs;  // nothing to do after an error
    }
}

// Warp per series (a first, then b); pair list.  Does nothing after an error.
__global__ void na_fill_kernel(NaPtrs p, const float *a, const int64_t *a_off, int n_a,
                               const float *b, const int64_t *b_off, int n_b, const int64_t *pa,
                               const int64_t *pb, int n_pairs, int d, int deff)
{
    if (p.ctrl->status)
        return;
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nw = (gridDim.x * blockDim.x) >> 5;
    const int chf = chunk_floats(deff), ppc = chunk_points(deff);
    for (int s = warp; s < n_a + n_b; s += nw) {
        const bool is_a = s < n_a;
        const int t = is_a ? s : s - n_a;
        const float *src = is_a ? a + a_off[t] * d : b + b_off[t] * d;
        const int n = is_a ? p.a_len[t] : p.b_len[t];
        float *dst = is_a ? p.a + p.a_off[t] : p.b + p.b_off[t];
        const int64_t total = (int64_t)((n + ppc - 1) / ppc) * chf;
        for (int f = lane; f < chf; f += 32)
            dst[f - chf] = KNN_DP_SENTINEL;
        for (int64_t f = lane; f < total; f += 32) {
            const int64_t i = f / deff;
            const int j = (int)(f - i * deff);
            dst[f] = (i < n && j < d) ? src[i * d + j] : 0.f;
        }
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pairs; i += gridDim.x * blockDim.x) {
        p.items[i] = make_int2((int)pb[i], (int)pa[i]);
        p.ilb[i] = 0.f;
    }
}

__global__ void na_out_kernel(NaPtrs p, int n_pairs, int kind, float *out)
{
    if (p.ctrl->status)
        return;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pairs; i += gridDim.x * blockDim.x)
        out[i] = kind == 0 ? p.res[i] : sqrtf(p.res[i]);
}

}  // namespace

extern "C" knn_status knn_pairwise_noalloc(const float *a, const int64_t *a_off, int64_t n_a,
                                           const float *b, const int64_t *b_off, int64_t n_b,
                                           const int64_t *pa, const int64_t *pb, int64_t n_pairs,
                                           int32_t d, float band, int32_t max_len,
                                           int32_t distance, float *out, void *stream)
{
    if (!a || !a_off || !b || !b_off || !pa || !pb || !out)
        return set_error(KNN_ERR_INVALID, "NULL argument");
    if (d < 1 || d > 16 || !(band > 0.f) || (distance != 0 && distance != 1))
        return set_error(KNN_ERR_INVALID, "bad d, band or distance");
    if (n_pairs < 0 || n_pairs > NA_MAX_PAIRS)
        return set_error(KNN_ERR_INVALID, "n_pairs must be in [0, 65536] for knn_pairwise_noalloc");
    if (n_a < 1 || n_a > NA_MAX_SERIES || n_b < 1 || n_b > NA_MAX_SERIES)
        return set_error(KNN_ERR_INVALID,
                         "n_a and n_b must be in [1, 16384] for knn_pairwise_noalloc");
    if (max_len < 1 || max_len > 65536)
        return set_error(KNN_ERR_INVALID, "max_len must be in [1, 65536]");
    if (n_pairs == 0)
        return KNN_OK;
    const int deff = deff_for(d);
    int P = 0, G = 0;
    choose_dp_config(deff, band_radius(max_len, max_len, band), max_len, &P, &G);
    if (!P)
        return set_error(KNN_ERR_UNSUPPORTED, "band too wide for the compiled DP variants");
    cudaStream_t st = (cudaStream_t)stream;
    // the call reads its status back and synchronises the stream, which a
    // stream under capture does not allow: refuse before touching it
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaError_t e = cudaStreamIsCapturing(st, &cap);
    if (e != cudaSuccess)
        return cuda_error(e, "cudaStreamIsCapturing");
    if (cap != cudaStreamCaptureStatusNone)
        return set_error(KNN_ERR_INVALID,
                         "knn_pairwise_noalloc cannot run while the stream is being captured");
    unsigned char *base = nullptr;
    knn_status s = scratch_base(&base);
    if (s)
        return s;
    const NaPtrs p = carve(base);
    cudaGetLastError();  // an earlier, unrelated launch error is not this call's
    na_prepare_kernel<<<1, 1024, 0, st>>>(p, a_off, (int)n_a, b_off, (int)n_b, pa, pb,
                                          (int)n_pairs, max_len, deff);
    na_fill_kernel<<<512, 256, 0, st>>>(p, a, a_off, (int)n_a, b, b_off, (int)n_b, pa, pb,
                                        (int)n_pairs, d, deff);
    DpArgs x{};
    x.items = p.items;
    x.item_lb = p.ilb;
    x.n_items = &p.ctrl->seg_count[0];
    x.items_cap = n_pairs;
    x.head = &p.ctrl->seg_head[0];
    x.db = p.b;
    x.db_off = p.b_off;
    x.db_len = p.b_len;
    x.db_id = p.b_id;
    x.q = p.a;
    x.q_off = p.a_off;
    x.q_len = p.a_len;
    x.band = band;
    x.G = G;
    x.mu_keep = 1.f;
    x.mu_prune = 1.f;
    x.out_pair = p.res;
    x.cells_stat = STAT_DP_CELLS;
    x.stats = p.ctrl->stats;
    x.status = &p.ctrl->status;
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (!launch_dp(x, deff, P, distance, nsm, st)) {
        cudaStreamSynchronize(st);  // retire the two launches already enqueued
        return set_error(KNN_ERR_UNSUPPORTED, "no DP kernel compiled for this d and shape");
    }
    na_out_kernel<<<256, 256, 0, st>>>(p, (int)n_pairs, distance, out);
    int status = 0;
    e = cudaMemcpyAsync(&status, &p.ctrl->status, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e == cudaSuccess)
        e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_error(e, "knn_pairwise_noalloc");
    if (status & NA_BAD_LENGTH)
        return set_error(KNN_ERR_INVALID, "a series is empty or longer than max_len");
    if (status & NA_BAD_INDEX)
        return set_error(KNN_ERR_INVALID, "a pair index is outside its set");
    if (status & NA_TOO_LARGE)
        return set_error(KNN_ERR_CAPACITY,
                         "series exceed the fixed scratch (1,048,576 floats per set after "
                         "padding each series to whole chunks, plus one chunk per series)");
    if (status)
        return set_error(KNN_ERR_CUDA, "device status set by the DP kernel");
    return KNN_OK;
}
