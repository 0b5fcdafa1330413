// Small device utilities: fills, repacking into the chunked layout, scatter.
#include "common.cuh"
#include "internal.h"

namespace knn {

__global__ void fill_u64_kernel(unsigned long long *p, unsigned long long v, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

__global__ void fill_f32_kernel(float *p, float v, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

static int blocks_for(int64_t n, int threads)
{
    int64_t b = (n + threads - 1) / threads;
    if (b > 4096)
        b = 4096;
    return b < 1 ? 1 : (int)b;
}

void launch_fill_u64(unsigned long long *p, unsigned long long v, int64_t n, cudaStream_t st)
{
    if (n > 0)
        fill_u64_kernel<<<blocks_for(n, 256), 256, 0, st>>>(p, v, n);
}

void launch_fill_f32(float *p, float v, int64_t n, cudaStream_t st)
{
    if (n > 0)
        fill_f32_kernel<<<blocks_for(n, 256), 256, 0, st>>>(p, v, n);
}

// One CTA per series (grid-stride over the series in x); when there are few
// series, blockIdx.y splits each series' floats over gridDim.y CTAs.
__global__ void repack_kernel(const float *src, const int64_t *src_off, const int *order, int nser,
                              int d, int deff, const int64_t *dst_off, float *dst, int lead,
                              int fixed_len)
{
    const int ppc = chunk_floats(deff) / deff;  // host guarantees deff is a compiled width
    const int chf = chunk_floats(deff);
    const int t0 = blockIdx.y * blockDim.x + threadIdx.x;
    const int tstride = gridDim.y * blockDim.x;
    for (int c = blockIdx.x; c < nser; c += gridDim.x) {
        const int s = order ? order[c] : c;
        const int64_t b = src_off[s];
        const int n = fixed_len > 0 ? fixed_len : (int)(src_off[s + 1] - b);
        const int64_t total = (int64_t)((n + ppc - 1) / ppc) * chf;
        const float *sp = src + b * d;
        float *dp = dst + dst_off[c];
        for (int f = t0; f < lead; f += tstride)
            dp[f - lead] = KNN_DP_SENTINEL;
        for (int64_t f = t0; f < total; f += tstride) {
            const int64_t i = f / deff;
            const int j = (int)(f - i * deff);
            dp[f] = (i < n && j < d) ? sp[i * d + j] : 0.f;
        }
    }
}

void launch_repack(const float *src, const int64_t *src_off, const int *order, int nser, int d,
                   int deff, const int64_t *dst_off, float *dst, cudaStream_t st, bool dp_lead,
                   int fixed_len)
{
    if (nser <= 0)
        return;
    const int bx = nser < 8192 ? nser : 8192;
    const int by = nser >= 1024 ? 1 : (1024 / nser < 64 ? 1024 / nser : 64);
    repack_kernel<<<dim3(bx, by), 256, 0, st>>>(src, src_off, order, nser, d, deff, dst_off, dst,
                                                dp_lead ? chunk_floats(deff) : 0, fixed_len);
}

__global__ void scatter_kernel(const float *src, const int *db_id, int n, int64_t src_stride,
                               float *dst, int64_t dst_stride, int out_sqrt)
{
    const int q = blockIdx.y;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        float v = src[(int64_t)q * src_stride + c];
        if (out_sqrt)
            v = sqrtf(v);
        dst[(int64_t)q * dst_stride + db_id[c]] = v;
    }
}

void launch_scatter_by_id(const float *src, const int *db_id, int n, int nq, int64_t src_stride,
                          float *dst, int64_t dst_stride, int out_sqrt, cudaStream_t st)
{
    dim3 grid(blocks_for(n, 256) > 1024 ? 1024 : blocks_for(n, 256), nq);
    scatter_kernel<<<grid, 256, 0, st>>>(src, db_id, n, src_stride, dst, dst_stride, out_sqrt);
}

}  // namespace knn
