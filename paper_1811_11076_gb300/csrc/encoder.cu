// Learned proposal: encoder kernels (BF16 tensor cores, FP32 accumulation),
// training (pair distances from the scan's own DP as targets, Adam), and the
// embedding of the database.  See encoder.cuh for the network.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "common.cuh"
#include "encoder.cuh"
#include "runtime.h"

using namespace knn;

// ---------------------------------------------------------------------------
// tensor-core primitive: D = A (16x16, row) * B (16x8, col) + D, BF16 in, FP32 acc

namespace knn {

__device__ __forceinline__ void mma_16816(float (&c)[4], const uint32_t (&a)[4],
                                          const uint32_t (&b)[2])
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ uint32_t pack2(__nv_bfloat16 lo, __nv_bfloat16 hi)
{
    return (uint32_t)__bfloat16_as_ushort(lo) | ((uint32_t)__bfloat16_as_ushort(hi) << 16);
}

__device__ __forceinline__ uint32_t ld32(const __nv_bfloat16 *p)
{
    return *reinterpret_cast<const uint32_t *>(p);
}

}  // namespace knn

namespace {

constexpr int TILE_T = 64;  // positions per conv tile

struct ConvArgs {
    const __nv_bfloat16 *in;     // [B][L][CIN]
    const __nv_bfloat16 *w;      // [64][5*CIN] (output channel major, k = tap*CIN + ci)
    const float *bias;           // [64] (forward)
    const __nv_bfloat16 *aprev;  // [B][L][64] (backward-data: ReLU mask)
    __nv_bfloat16 *out;          // [B][L][64]
    const int *len;              // [B]
    int B, L, tiles_per_series;
};

// Convolution (kernel 5, same padding) as an implicit GEMM: rows = 64
// positions of one series, columns = 64 output channels, K = 5*CIN.
// EPI 0: + bias, ReLU (forward).  EPI 1: times (aprev > 0) (backward-data:
// the input is dZ of the layer, the weights are flipped and transposed).
// Positions beyond a series' length are written as zero.
template <int CIN, int EPI>
__global__ void __launch_bounds__(128) conv_mma_kernel(const ConvArgs a)
{
    constexpr int KT = ENC_K * CIN;
    constexpr int XS = CIN + 8;   // padded row strides (bank-conflict free fragments)
    constexpr int WS = KT + 8;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __nv_bfloat16 *Ws = reinterpret_cast<__nv_bfloat16 *>(smem_raw);
    __nv_bfloat16 *Xs = Ws + 64 * WS;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t4 = lane & 3;

    for (int i = tid; i < 64 * KT / 2; i += blockDim.x) {
        const int n = (2 * i) / KT, k = (2 * i) % KT;
        *reinterpret_cast<uint32_t *>(&Ws[n * WS + k]) = ld32(a.w + (size_t)n * KT + k);
    }
    const int ntiles = a.B * a.tiles_per_series;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int b = tile / a.tiles_per_series;
        const int t0 = (tile % a.tiles_per_series) * TILE_T;
        const int len = a.len[b];
        __syncthreads();  // previous tile done with Xs (and Ws loaded)
        for (int i = tid; i < (TILE_T + 4) * CIN / 2; i += blockDim.x) {
            const int p = (2 * i) / CIN, ci = (2 * i) % CIN;
            const int pos = t0 - 2 + p;
            uint32_t v = 0;
            if (pos >= 0 && pos < len)
                v = ld32(a.in + ((size_t)b * a.L + pos) * CIN + ci);
            *reinterpret_cast<uint32_t *>(&Xs[p * XS + ci]) = v;
        }
        __syncthreads();
        float acc[8][4];
#pragma unroll
        for (int nt = 0; nt < 8; ++nt)
#pragma unroll
            for (int q = 0; q < 4; ++q)
                acc[nt][q] = 0.f;
        const int r0 = warp * 16 + g;
#pragma unroll
        for (int ks = 0; ks < KT / 16; ++ks) {
            const int tap = (ks * 16) / CIN, ci0 = (ks * 16) % CIN;
            uint32_t af[4];
            af[0] = ld32(&Xs[(r0 + tap) * XS + ci0 + 2 * t4]);
            af[1] = ld32(&Xs[(r0 + 8 + tap) * XS + ci0 + 2 * t4]);
            af[2] = ld32(&Xs[(r0 + tap) * XS + ci0 + 2 * t4 + 8]);
            af[3] = ld32(&Xs[(r0 + 8 + tap) * XS + ci0 + 2 * t4 + 8]);
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                uint32_t bf[2];
                bf[0] = ld32(&Ws[(nt * 8 + g) * WS + ks * 16 + 2 * t4]);
                bf[1] = ld32(&Ws[(nt * 8 + g) * WS + ks * 16 + 2 * t4 + 8]);
                mma_16816(acc[nt], af, bf);
            }
        }
#pragma unroll
        for (int half = 0; half < 2; ++half) {
            const int t = t0 + r0 + 8 * half;
            if (t >= a.L)
                continue;
            const bool valid = t < len;
            __nv_bfloat16 *o = a.out + ((size_t)b * a.L + t) * ENC_C;
#pragma unroll
            for (int nt = 0; nt < 8; ++nt) {
                const int co = nt * 8 + 2 * t4;
                float v0 = acc[nt][2 * half], v1 = acc[nt][2 * half + 1];
                if (EPI == 0) {
                    v0 = fmaxf(v0 + a.bias[co], 0.f);
                    v1 = fmaxf(v1 + a.bias[co + 1], 0.f);
                } else {
                    const __nv_bfloat16 *ap = a.aprev + ((size_t)b * a.L + t) * ENC_C + co;
                    v0 = __bfloat162float(ap[0]) > 0.f ? v0 : 0.f;
                    v1 = __bfloat162float(ap[1]) > 0.f ? v1 : 0.f;
                }
                if (!valid)
                    v0 = v1 = 0.f;
                *reinterpret_cast<uint32_t *>(o + co) =
                    pack2(__float2bfloat16_rn(v0), __float2bfloat16_rn(v1));
            }
        }
    }
}

struct WgradArgs {
    const __nv_bfloat16 *x;   // [B][L][CIN] layer input
    const __nv_bfloat16 *dz;  // [B][L][64] gradient of the pre-activation
    const int *len;
    int B, L, tiles_per_series;
    float *dw;                // [5][CIN][64] (accumulated atomically)
    float *db;                // [64]
};

// Weight gradient: dW[(tap, ci)][co] = sum over positions t of
// x[t + tap - 2][ci] * dz[t][co]; rows (tap, ci) x columns co, reduction
// over positions (K).  Warp w owns column tile w for every row tile.
template <int CIN>
__global__ void __launch_bounds__(256) wgrad_mma_kernel(const WgradArgs a)
{
    constexpr int MT = ENC_K * CIN / 16;
    constexpr int XS = CIN + 8;
    constexpr int DS = ENC_C + 8;
    __shared__ __align__(16) __nv_bfloat16 Xs[(TILE_T + 4) * XS];
    __shared__ __align__(16) __nv_bfloat16 Ds[TILE_T * DS];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int g = lane >> 2, t4 = lane & 3;
    float acc[MT][4];
#pragma unroll
    for (int j = 0; j < MT; ++j)
#pragma unroll
        for (int q = 0; q < 4; ++q)
            acc[j][q] = 0.f;
    float dbacc = 0.f;
    const int ntiles = a.B * a.tiles_per_series;
    for (int tile = blockIdx.x; tile < ntiles; tile += gridDim.x) {
        const int b = tile / a.tiles_per_series;
        const int t0 = (tile % a.tiles_per_series) * TILE_T;
        const int len = a.len[b];
        __syncthreads();
        for (int i = tid; i < (TILE_T + 4) * CIN / 2; i += blockDim.x) {
            const int p = (2 * i) / CIN, ci = (2 * i) % CIN;
            const int pos = t0 - 2 + p;
            uint32_t v = 0;
            if (pos >= 0 && pos < len)
                v = ld32(a.x + ((size_t)b * a.L + pos) * CIN + ci);
            *reinterpret_cast<uint32_t *>(&Xs[p * XS + ci]) = v;
        }
        for (int i = tid; i < TILE_T * ENC_C / 2; i += blockDim.x) {
            const int p = (2 * i) / ENC_C, c = (2 * i) % ENC_C;
            const int pos = t0 + p;
            uint32_t v = 0;
            if (pos < len)
                v = ld32(a.dz + ((size_t)b * a.L + pos) * ENC_C + c);
            *reinterpret_cast<uint32_t *>(&Ds[p * DS + c]) = v;
        }
        __syncthreads();
        if (tid < ENC_C)
            for (int p = 0; p < TILE_T; ++p)
                dbacc += __bfloat162float(Ds[p * DS + tid]);
#pragma unroll
        for (int kk = 0; kk < TILE_T / 16; ++kk) {
            const int p0 = kk * 16 + 2 * t4;
            uint32_t bf[2];
            bf[0] = pack2(Ds[p0 * DS + warp * 8 + g], Ds[(p0 + 1) * DS + warp * 8 + g]);
            bf[1] = pack2(Ds[(p0 + 8) * DS + warp * 8 + g], Ds[(p0 + 9) * DS + warp * 8 + g]);
#pragma unroll
            for (int j = 0; j < MT; ++j) {
                const int tap = (j * 16) / CIN, ci0 = (j * 16) % CIN;
                uint32_t af[4];
                af[0] = pack2(Xs[(p0 + tap) * XS + ci0 + g], Xs[(p0 + 1 + tap) * XS + ci0 + g]);
                af[1] = pack2(Xs[(p0 + tap) * XS + ci0 + g + 8],
                              Xs[(p0 + 1 + tap) * XS + ci0 + g + 8]);
                af[2] = pack2(Xs[(p0 + 8 + tap) * XS + ci0 + g],
                              Xs[(p0 + 9 + tap) * XS + ci0 + g]);
                af[3] = pack2(Xs[(p0 + 8 + tap) * XS + ci0 + g + 8],
                              Xs[(p0 + 9 + tap) * XS + ci0 + g + 8]);
                mma_16816(acc[j], af, bf);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < MT; ++j) {
        const int row = j * 16 + g;  // = tap*CIN + ci
        const int co = warp * 8 + 2 * t4;
        atomicAdd(a.dw + (size_t)row * ENC_C + co, acc[j][0]);
        atomicAdd(a.dw + (size_t)row * ENC_C + co + 1, acc[j][1]);
        atomicAdd(a.dw + (size_t)(row + 8) * ENC_C + co, acc[j][2]);
        atomicAdd(a.dw + (size_t)(row + 8) * ENC_C + co + 1, acc[j][3]);
    }
    if (tid < ENC_C)
        atomicAdd(a.db + tid, dbacc);
}

// Input of the network: series rows (any layout with a float offset, a
// point stride and a length per series) rounded to BF16, [B][L][16].
__global__ void gather_input_kernel(const float *src, const int64_t *off, int stride,
                                    const int *len, const int *idx, int d, int B, int L,
                                    float in_scale, __nv_bfloat16 *x0, int *len_out)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)B * L * ENC_CIN;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(e / ((int64_t)L * ENC_CIN));
        const int rem = (int)(e - (int64_t)b * L * ENC_CIN);
        const int t = rem / ENC_CIN, c = rem % ENC_CIN;
        const int s = idx ? idx[b] : b;
        const int n = len[s];
        float v = 0.f;
        if (t < n && c < d)
            v = src[off[s] + (int64_t)t * stride + c] * in_scale;
        x0[e] = __float2bfloat16_rn(v);
        if (rem == 0)
            len_out[b] = min(n, L);
    }
}

// Mean over valid positions and the linear layer; one block (64 threads) per series.
__global__ void pool_linear_kernel(const __nv_bfloat16 *a3, const int *len, int L,
                                   const float *params, float *h, float *e)
{
    __shared__ float hs[ENC_C];
    const int b = blockIdx.x, c = threadIdx.x;
    const int n = len[b];
    float s = 0.f;
    for (int t = 0; t < n; ++t)
        s += __bfloat162float(a3[((size_t)b * L + t) * ENC_C + c]);
    s /= (float)max(n, 1);
    hs[c] = s;
    if (h)
        h[(size_t)b * ENC_C + c] = s;
    __syncthreads();
    const float *wl = params + ENC_OFF_WL;
    float o = params[ENC_OFF_BL + c];
    for (int i = 0; i < ENC_C; ++i)
        o = __fmaf_rn(hs[i], wl[i * ENC_E + c], o);
    e[(size_t)b * ENC_E + c] = o;
}

// Loss (pred - target)^2, pred = ||e_a - e_b||^2, mean over pairs; de for both sides.
__global__ void loss_kernel(const float *e, const int *pa, const int *pb, const float *target,
                            int n_pairs, float *de, float *loss)
{
    const int p = blockIdx.x * (blockDim.x / 64) + threadIdx.x / 64;
    const int c = threadIdx.x & 63;
    const bool valid = p < n_pairs;  // every thread reaches the barrier below
    const int ia = valid ? pa[p] : 0, ib = valid ? pb[p] : 0;
    const float diff = valid ? e[(size_t)ia * ENC_E + c] - e[(size_t)ib * ENC_E + c] : 0.f;
    float sq = diff * diff;
    // reduce over the 64 lanes of this pair (two warps)
    __shared__ float red[8][2];
    for (int o = 16; o > 0; o >>= 1)
        sq += __shfl_xor_sync(KNN_FULL_MASK, sq, o);
    const int slot = (threadIdx.x / 64) % 8;
    if ((threadIdx.x & 31) == 0)
        red[slot][(threadIdx.x >> 5) & 1] = sq;
    __syncthreads();
    if (!valid)
        return;
    const float pred = red[slot][0] + red[slot][1];
    const float r = pred - target[p];
    const float gsc = 2.f * r / (float)n_pairs;
    atomicAdd(de + (size_t)ia * ENC_E + c, gsc * 2.f * diff);
    atomicAdd(de + (size_t)ib * ENC_E + c, -gsc * 2.f * diff);
    if (c == 0)
        atomicAdd(loss, r * r / (float)n_pairs);
}

// Backward of the linear layer and the mean: dh = de Wl^T, dZ3 = (dh / n) where
// a3 > 0; gradients of Wl and bl accumulated over the batch.
__global__ void pool_linear_bwd_kernel(const __nv_bfloat16 *a3, const int *len, int L,
                                       const float *params, const float *de, __nv_bfloat16 *dz3)
{
    __shared__ float des[ENC_E];
    const int b = blockIdx.x, c = threadIdx.x;
    des[c] = de[(size_t)b * ENC_E + c];
    __syncthreads();
    const float *wl = params + ENC_OFF_WL;
    float dh = 0.f;
    for (int o = 0; o < ENC_E; ++o)
        dh = __fmaf_rn(des[o], wl[c * ENC_E + o], dh);
    const int n = len[b];
    const float v = dh / (float)max(n, 1);
    for (int t = 0; t < L; ++t) {
        const size_t at = ((size_t)b * L + t) * ENC_C + c;
        const float z = (t < n && __bfloat162float(a3[at]) > 0.f) ? v : 0.f;
        dz3[at] = __float2bfloat16_rn(z);
    }
}

// dWl[i][o] = sum_b h[b][i] de[b][o]; dbl[o] = sum_b de[b][o].  Block per i.
__global__ void linear_wgrad_kernel(const float *h, const float *de, int B, float *grad)
{
    const int i = blockIdx.x, o = threadIdx.x;
    float s = 0.f, sb = 0.f;
    for (int b = 0; b < B; ++b) {
        const float d = de[(size_t)b * ENC_E + o];
        s = __fmaf_rn(h[(size_t)b * ENC_C + i], d, s);
        if (i == 0)
            sb += d;
    }
    grad[ENC_OFF_WL + i * ENC_E + o] += s;
    if (i == 0)
        grad[ENC_OFF_BL + o] += sb;
}

// FP32 masters -> BF16 layouts: forward [co][tap*CIN + ci]; backward-data
// (layers 2, 3) [ci][tap'*64 + co] with tap' = 4 - tap.
__global__ void weights_to_bf16_kernel(const float *params, __nv_bfloat16 *w1f, __nv_bfloat16 *w2f,
                                       __nv_bfloat16 *w3f, __nv_bfloat16 *w2d, __nv_bfloat16 *w3d)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < ENC_K * ENC_CIN * ENC_C) {
        const int tap = i / (ENC_CIN * ENC_C), ci = (i / ENC_C) % ENC_CIN, co = i % ENC_C;
        w1f[co * (ENC_K * ENC_CIN) + tap * ENC_CIN + ci] = __float2bfloat16_rn(params[ENC_OFF_W1 + i]);
    }
    if (i < ENC_K * ENC_C * ENC_C) {
        const int tap = i / (ENC_C * ENC_C), ci = (i / ENC_C) % ENC_C, co = i % ENC_C;
        const __nv_bfloat16 v2 = __float2bfloat16_rn(params[ENC_OFF_W2 + i]);
        const __nv_bfloat16 v3 = __float2bfloat16_rn(params[ENC_OFF_W3 + i]);
        w2f[co * (ENC_K * ENC_C) + tap * ENC_C + ci] = v2;
        w3f[co * (ENC_K * ENC_C) + tap * ENC_C + ci] = v3;
        w2d[ci * (ENC_K * ENC_C) + (ENC_K - 1 - tap) * ENC_C + co] = v2;
        w3d[ci * (ENC_K * ENC_C) + (ENC_K - 1 - tap) * ENC_C + co] = v3;
    }
}

__global__ void adam_kernel(float *w, const float *gr, float *m, float *v, int n, float lr,
                            float b1, float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const float g = gr[i];
    const float mi = b1 * m[i] + (1.f - b1) * g;
    const float vi = b2 * v[i] + (1.f - b2) * g * g;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

__global__ void emb_to_bf16_kernel(const float *e, const int *dst_index, int B,
                                   __nv_bfloat16 *out, float *norm_out)
{
    const int b = blockIdx.x, c = threadIdx.x;
    const __nv_bfloat16 v = __float2bfloat16_rn(e[(size_t)b * ENC_E + c]);
    const int dst = dst_index ? dst_index[b] : b;
    out[(size_t)dst * ENC_E + c] = v;
    float f = __bfloat162float(v);
    float s = f * f;
    for (int o = 16; o > 0; o >>= 1)
        s += __shfl_xor_sync(KNN_FULL_MASK, s, o);
    __shared__ float part[2];
    if ((c & 31) == 0)
        part[c >> 5] = s;
    __syncthreads();
    if (c == 0 && norm_out)
        norm_out[dst] = part[0] + part[1];
}

__global__ void pair_targets_kernel(const float *raw, const int *la, const int *lb,
                                    const int2 *items, int n, int kind, float *target)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float v = raw[i];
        const int m = la[items[i].y], nn = lb[items[i].x];
        // log(1 + DTW / longer length) or log(1 + DK^2): monotone in the
        // distance (ranking is what the proposal needs) and of moderate range
        target[i] = kind == 0 ? log1pf(v / (float)max(m, nn)) : log1pf(v);
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host side

struct knn_encoder {
    int d = 0;
    int dev = 0;
    int64_t step = 0;
    float in_scale = 1.f;  // inputs are multiplied by this before the first layer
    DevBuf params, grad, m, v;
    DevBuf w1f, w2f, w3f, w2d, w3d;
    // work buffers for a forward/backward batch
    DevBuf x0, a1, a2, a3, dz, dz2, lenb, idx, h, e, de, loss, pairs_a, pairs_b, tgt;
    int cap_B = 0, cap_L = 0;
};

namespace knn {

static knn_status enc_alloc_params(knn_encoder *enc)
{
    knn_status s;
    if ((s = enc->params.ensure(sizeof(float) * ENC_NPARAM)) ||
        (s = enc->grad.ensure(sizeof(float) * ENC_NPARAM)) ||
        (s = enc->m.ensure(sizeof(float) * ENC_NPARAM)) ||
        (s = enc->v.ensure(sizeof(float) * ENC_NPARAM)) ||
        (s = enc->w1f.ensure(2 * ENC_K * ENC_CIN * ENC_C)) ||
        (s = enc->w2f.ensure(2 * ENC_K * ENC_C * ENC_C)) ||
        (s = enc->w3f.ensure(2 * ENC_K * ENC_C * ENC_C)) ||
        (s = enc->w2d.ensure(2 * ENC_K * ENC_C * ENC_C)) ||
        (s = enc->w3d.ensure(2 * ENC_K * ENC_C * ENC_C)))
        return s;
    return KNN_OK;
}

knn_status enc_work(knn_encoder *enc, int B, int L)
{
    if (B <= enc->cap_B && L <= enc->cap_L)
        return KNN_OK;
    B = std::max(B, enc->cap_B);
    L = std::max((L + TILE_T - 1) / TILE_T * TILE_T, enc->cap_L);
    const size_t act = (size_t)B * L * ENC_C * 2;
    knn_status s;
    if ((s = enc->x0.ensure((size_t)B * L * ENC_CIN * 2)) || (s = enc->a1.ensure(act)) ||
        (s = enc->a2.ensure(act)) || (s = enc->a3.ensure(act)) || (s = enc->dz.ensure(act)) ||
        (s = enc->dz2.ensure(act)) || (s = enc->lenb.ensure(4 * (size_t)B)) ||
        (s = enc->idx.ensure(4 * (size_t)B)) || (s = enc->h.ensure(4 * (size_t)B * ENC_C)) ||
        (s = enc->e.ensure(4 * (size_t)B * ENC_E)) || (s = enc->de.ensure(4 * (size_t)B * ENC_E)) ||
        (s = enc->loss.ensure(16)))
        return s;
    enc->cap_B = B;
    enc->cap_L = L;
    return KNN_OK;
}

static void enc_weights_bf16(knn_encoder *enc, cudaStream_t st)
{
    weights_to_bf16_kernel<<<(ENC_K * ENC_C * ENC_C + 255) / 256, 256, 0, st>>>(
        enc->params.as<float>(), enc->w1f.as<__nv_bfloat16>(), enc->w2f.as<__nv_bfloat16>(),
        enc->w3f.as<__nv_bfloat16>(), enc->w2d.as<__nv_bfloat16>(), enc->w3d.as<__nv_bfloat16>());
}

static int conv_grid(int ntiles, int n_sm)
{
    return std::max(1, std::min(ntiles, n_sm * 4));
}

template <int CIN, int EPI>
static void conv_launch(const ConvArgs &a, int n_sm, cudaStream_t st)
{
    const size_t smem = (size_t)2 * (64 * (ENC_K * CIN + 8) + (TILE_T + 4) * (CIN + 8));
    conv_mma_kernel<CIN, EPI>
        <<<conv_grid(a.B * a.tiles_per_series, n_sm), 128, smem, st>>>(a);
}

// Forward pass for B series from a row source (float offset, point stride,
// length per series, optional index list).  Leaves x0, a1..a3, h, e filled.
knn_status enc_forward(knn_encoder *enc, const float *src, const int64_t *off, int stride,
                       const int *len, const int *idx, int d, int B, int L, int n_sm,
                       cudaStream_t st)
{
    knn_status s = enc_work(enc, B, L);
    if (s)
        return s;
    const int Lp = (L + TILE_T - 1) / TILE_T * TILE_T;
    const int64_t tot = (int64_t)B * Lp * ENC_CIN;
    gather_input_kernel<<<(int)std::min<int64_t>((tot + 255) / 256, 8192), 256, 0, st>>>(
        src, off, stride, len, idx, d, B, Lp, enc->in_scale, enc->x0.as<__nv_bfloat16>(),
        enc->lenb.as<int>());
    ConvArgs c{};
    c.len = enc->lenb.as<int>();
    c.B = B;
    c.L = Lp;
    c.tiles_per_series = Lp / TILE_T;
    c.in = enc->x0.as<__nv_bfloat16>();
    c.w = enc->w1f.as<__nv_bfloat16>();
    c.bias = enc->params.as<float>() + ENC_OFF_B1;
    c.out = enc->a1.as<__nv_bfloat16>();
    conv_launch<ENC_CIN, 0>(c, n_sm, st);
    c.in = enc->a1.as<__nv_bfloat16>();
    c.w = enc->w2f.as<__nv_bfloat16>();
    c.bias = enc->params.as<float>() + ENC_OFF_B2;
    c.out = enc->a2.as<__nv_bfloat16>();
    conv_launch<ENC_C, 0>(c, n_sm, st);
    c.in = enc->a2.as<__nv_bfloat16>();
    c.w = enc->w3f.as<__nv_bfloat16>();
    c.bias = enc->params.as<float>() + ENC_OFF_B3;
    c.out = enc->a3.as<__nv_bfloat16>();
    conv_launch<ENC_C, 0>(c, n_sm, st);
    pool_linear_kernel<<<B, ENC_C, 0, st>>>(enc->a3.as<__nv_bfloat16>(), enc->lenb.as<int>(), Lp,
                                            enc->params.as<float>(), enc->h.as<float>(),
                                            enc->e.as<float>());
    return KNN_OK;
}

// Loss and gradient (into enc->grad, which is zeroed first) for pairs of the
// B series of the last forward pass.
static void enc_backward(knn_encoder *enc, const int *pa, const int *pb, const float *tgt,
                         int n_pairs, int B, int L, int n_sm, cudaStream_t st)
{
    const int Lp = (L + TILE_T - 1) / TILE_T * TILE_T;
    cudaMemsetAsync(enc->grad.p, 0, sizeof(float) * ENC_NPARAM, st);
    cudaMemsetAsync(enc->de.p, 0, sizeof(float) * B * ENC_E, st);
    cudaMemsetAsync(enc->loss.p, 0, 4, st);
    loss_kernel<<<(n_pairs + 7) / 8, 512, 0, st>>>(enc->e.as<float>(), pa, pb, tgt, n_pairs,
                                                   enc->de.as<float>(), enc->loss.as<float>());
    float *gr = enc->grad.as<float>();
    linear_wgrad_kernel<<<ENC_C, ENC_E, 0, st>>>(enc->h.as<float>(), enc->de.as<float>(), B, gr);
    pool_linear_bwd_kernel<<<B, ENC_C, 0, st>>>(enc->a3.as<__nv_bfloat16>(), enc->lenb.as<int>(),
                                                Lp, enc->params.as<float>(), enc->de.as<float>(),
                                                enc->dz.as<__nv_bfloat16>());
    const int tps = Lp / TILE_T;
    const int wg = std::max(1, std::min(B * tps, n_sm * 2));
    WgradArgs w{};
    w.len = enc->lenb.as<int>();
    w.B = B;
    w.L = Lp;
    w.tiles_per_series = tps;
    // layer 3
    w.x = enc->a2.as<__nv_bfloat16>();
    w.dz = enc->dz.as<__nv_bfloat16>();
    w.dw = gr + ENC_OFF_W3;
    w.db = gr + ENC_OFF_B3;
    wgrad_mma_kernel<ENC_C><<<wg, 256, 0, st>>>(w);
    ConvArgs c{};
    c.len = enc->lenb.as<int>();
    c.B = B;
    c.L = Lp;
    c.tiles_per_series = tps;
    c.in = enc->dz.as<__nv_bfloat16>();
    c.w = enc->w3d.as<__nv_bfloat16>();
    c.aprev = enc->a2.as<__nv_bfloat16>();
    c.out = enc->dz2.as<__nv_bfloat16>();
    conv_launch<ENC_C, 1>(c, n_sm, st);
    // layer 2
    w.x = enc->a1.as<__nv_bfloat16>();
    w.dz = enc->dz2.as<__nv_bfloat16>();
    w.dw = gr + ENC_OFF_W2;
    w.db = gr + ENC_OFF_B2;
    wgrad_mma_kernel<ENC_C><<<wg, 256, 0, st>>>(w);
    c.in = enc->dz2.as<__nv_bfloat16>();
    c.w = enc->w2d.as<__nv_bfloat16>();
    c.aprev = enc->a1.as<__nv_bfloat16>();
    c.out = enc->dz.as<__nv_bfloat16>();
    conv_launch<ENC_C, 1>(c, n_sm, st);
    // layer 1
    w.x = enc->x0.as<__nv_bfloat16>();
    w.dz = enc->dz.as<__nv_bfloat16>();
    w.dw = gr + ENC_OFF_W1;
    w.db = gr + ENC_OFF_B1;
    wgrad_mma_kernel<ENC_CIN><<<wg, 256, 0, st>>>(w);
}

knn_status enc_score(knn_encoder *enc, const __nv_bfloat16 *eq, const float *nq2, int nq,
                     const __nv_bfloat16 *ec, const float *nc2, int n, float *score,
                     int *tile_idx, int64_t stride, int *status, cudaStream_t st)
{
    (void)enc;
    launch_score_tc(eq, nq2, nq, ec, nc2, n, score, tile_idx, stride, status, st);
    return KNN_OK;
}

void enc_emb_bf16(const float *e, const int *dst_index, int B, __nv_bfloat16 *out, float *norm,
                  cudaStream_t st)
{
    emb_to_bf16_kernel<<<B, ENC_E, 0, st>>>(e, dst_index, B, out, norm);
}

void enc_init_attributes()
{
    cudaFuncSetAttribute(conv_mma_kernel<ENC_CIN, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         96 * 1024);
    cudaFuncSetAttribute(conv_mma_kernel<ENC_C, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         96 * 1024);
    cudaFuncSetAttribute(conv_mma_kernel<ENC_C, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         96 * 1024);
}

// Scan side: embed the batch's queries (repacked rows), then score every
// series of the database: score[q][c] = ||e_q - e_c||^2 (bucket order).
knn_status enc_scan_scores(knn_db *db, const float *qbuf, const int64_t *q_off, const int *q_len,
                           int nq, int max_m, void *qemb_v, float *qnorm, float *scores,
                           int *tile_idx, int *status, cudaStream_t st)
{
    __nv_bfloat16 *qemb = static_cast<__nv_bfloat16 *>(qemb_v);
    knn_encoder *enc = db->enc;
    knn_status s = enc_forward(enc, qbuf, q_off, db->deff, q_len, nullptr, db->d, nq, max_m,
                               db->n_sm, st);
    if (s)
        return s;
    enc_emb_bf16(enc->e.as<float>(), nullptr, nq, qemb, qnorm, st);
    return enc_score(enc, qemb, qnorm, nq, db->emb.as<__nv_bfloat16>(), db->emb_norm.as<float>(),
                     db->N, scores, tile_idx, (db->N + 63) / 64, status, st);
}

}  // namespace knn

// ---------------------------------------------------------------------------
// C-ABI

static uint64_t splitmix(uint64_t &x)
{
    uint64_t z = (x += 0x9e3779b97f4a7c15ull);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

static double uniform01(uint64_t &x) { return ((splitmix(x) >> 11) + 0.5) * (1.0 / 9007199254740992.0); }

extern "C" int32_t knn_encoder_num_params(void) { return ENC_NPARAM; }

extern "C" knn_status knn_encoder_create(int32_t d, uint64_t seed, knn_encoder **out)
{
    if (!out)
        return set_error(KNN_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (d < 1 || d > 16)
        return set_error(KNN_ERR_INVALID, "d must be in [1, 16]");
    static std::once_flag attr_once;
    std::call_once(attr_once, [] { enc_init_attributes(); });
    auto enc = new knn_encoder();
    enc->d = d;
    cudaGetDevice(&enc->dev);
    knn_status s = enc_alloc_params(enc);
    if (s) {
        delete enc;
        return s;
    }
    // He-normal initialisation (fan-in), zero biases; Box-Muller on splitmix64
    std::vector<float> p(ENC_NPARAM, 0.f);
    uint64_t st = seed ^ 0x5eedull;
    auto fill = [&](int off, int count, int fan_in) {
        const double sd = std::sqrt(2.0 / fan_in);
        for (int i = 0; i < count; ++i) {
            const double u1 = uniform01(st), u2 = uniform01(st);
            p[off + i] = (float)(sd * std::sqrt(-2.0 * std::log(u1)) * std::cos(6.283185307179586 * u2));
        }
    };
    fill(ENC_OFF_W1, ENC_K * ENC_CIN * ENC_C, ENC_K * d);
    fill(ENC_OFF_W2, ENC_K * ENC_C * ENC_C, ENC_K * ENC_C);
    fill(ENC_OFF_W3, ENC_K * ENC_C * ENC_C, ENC_K * ENC_C);
    fill(ENC_OFF_WL, ENC_C * ENC_E, ENC_C);
    for (int i = 0; i < ENC_C * ENC_E; ++i)
        p[ENC_OFF_WL + i] *= 0.1f;  // start with small embeddings
    // coordinates beyond d never carry data: keep their weights at zero
    for (int tap = 0; tap < ENC_K; ++tap)
        for (int ci = d; ci < ENC_CIN; ++ci)
            for (int co = 0; co < ENC_C; ++co)
                p[ENC_OFF_W1 + (tap * ENC_CIN + ci) * ENC_C + co] = 0.f;
    cudaError_t e = cudaMemcpy(enc->params.p, p.data(), sizeof(float) * ENC_NPARAM,
                               cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemset(enc->m.p, 0, sizeof(float) * ENC_NPARAM);
    if (e == cudaSuccess)
        e = cudaMemset(enc->v.p, 0, sizeof(float) * ENC_NPARAM);
    if (e != cudaSuccess) {
        delete enc;
        return cuda_error(e, "encoder init");
    }
    enc_weights_bf16(enc, nullptr);
    e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        delete enc;
        return cuda_error(e, "encoder init");
    }
    *out = enc;
    return KNN_OK;
}

extern "C" knn_status knn_encoder_destroy(knn_encoder *enc)
{
    if (!enc)
        return set_error(KNN_ERR_INVALID, "encoder is NULL");
    cudaDeviceSynchronize();
    delete enc;
    return KNN_OK;
}

extern "C" knn_status knn_encoder_params(knn_encoder *enc, float *get, const float *set)
{
    if (!enc)
        return set_error(KNN_ERR_INVALID, "encoder is NULL");
    cudaError_t e = cudaSuccess;
    if (set) {
        e = cudaMemcpy(enc->params.p, set, sizeof(float) * ENC_NPARAM, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) {
            enc_weights_bf16(enc, nullptr);
            e = cudaDeviceSynchronize();
        }
    }
    if (e == cudaSuccess && get)
        e = cudaMemcpy(get, enc->params.p, sizeof(float) * ENC_NPARAM, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess)
        return cuda_error(e, "encoder params");
    return KNN_OK;
}

// Series given point-major (d floats per point) with point offsets: the
// device arrays a forward pass needs (float offsets, lengths).
static knn_status raw_rows(const int64_t *offsets, int64_t n, int d, DevBuf &foff, DevBuf &len,
                           int *max_len)
{
    std::vector<int64_t> ho(n + 1);
    if (is_device_ptr(offsets))
        cudaMemcpy(ho.data(), offsets, 8 * (n + 1), cudaMemcpyDeviceToHost);
    else
        memcpy(ho.data(), offsets, 8 * (n + 1));
    std::vector<int64_t> fo(n);
    std::vector<int> ln(n);
    int mx = 0;
    for (int64_t i = 0; i < n; ++i) {
        const int64_t L = ho[i + 1] - ho[i];
        if (L < 1 || L > 65536)
            return set_error(KNN_ERR_INVALID, "series length must be in [1, 65536]");
        fo[i] = ho[i] * d;
        ln[i] = (int)L;
        mx = std::max(mx, (int)L);
    }
    knn_status s;
    if ((s = foff.ensure(8 * n)) || (s = len.ensure(4 * n)))
        return s;
    cudaMemcpy(foff.p, fo.data(), 8 * n, cudaMemcpyHostToDevice);
    cudaMemcpy(len.p, ln.data(), 4 * n, cudaMemcpyHostToDevice);
    *max_len = mx;
    return KNN_OK;
}

static int sm_count(int dev)
{
    int n = 0;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

extern "C" knn_status knn_encoder_embed(knn_encoder *enc, const float *series,
                                        const int64_t *offsets, int64_t n, float *out,
                                        void *stream)
{
    if (!enc || !series || !offsets || !out)
        return set_error(KNN_ERR_INVALID, "NULL argument");
    if (n < 1)
        return set_error(KNN_ERR_INVALID, "n must be >= 1");
    if (!is_device_ptr(series) || !is_device_ptr(out))
        return set_error(KNN_ERR_INVALID, "series and out must be device memory");
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf foff, len;
    int mx = 0;
    knn_status s = raw_rows(offsets, n, enc->d, foff, len, &mx);
    if (s)
        return s;
    const int nsm = sm_count(enc->dev);
    const int chunk = std::max(1, (int)std::min<int64_t>(n, (int64_t)(1 << 21) / std::max(mx, 1)));
    std::vector<int> idx(chunk);
    DevBuf didx;
    if ((s = didx.ensure(4 * (size_t)chunk)))
        return s;
    for (int64_t b0 = 0; b0 < n; b0 += chunk) {
        const int B = (int)std::min<int64_t>(chunk, n - b0);
        for (int i = 0; i < B; ++i)
            idx[i] = (int)(b0 + i);
        cudaMemcpyAsync(didx.p, idx.data(), 4 * B, cudaMemcpyHostToDevice, st);
        if ((s = enc_forward(enc, series, foff.as<int64_t>(), enc->d, len.as<int>(),
                             didx.as<int>(), enc->d, B, mx, nsm, st)))
            return s;
        cudaMemcpyAsync(out + b0 * ENC_E, enc->e.p, sizeof(float) * B * ENC_E,
                        cudaMemcpyDeviceToDevice, st);
        cudaStreamSynchronize(st);
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess)
        e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_error(e, "encoder embed");
    return KNN_OK;
}

extern "C" knn_status knn_encoder_loss_grad(knn_encoder *enc, const float *series,
                                            const int64_t *offsets, int64_t n_series,
                                            const int64_t *pa, const int64_t *pb,
                                            const float *targets, int64_t n_pairs, float *loss,
                                            float *grad, void *stream)
{
    if (!enc || !series || !offsets || !pa || !pb || !targets || !loss || !grad)
        return set_error(KNN_ERR_INVALID, "NULL argument");
    if (n_series < 1 || n_series > 65536 || n_pairs < 1 || n_pairs > (1 << 22))
        return set_error(KNN_ERR_INVALID, "bad sizes");
    if (!is_device_ptr(series))
        return set_error(KNN_ERR_INVALID, "series must be device memory");
    cudaStream_t st = (cudaStream_t)stream;
    DevBuf foff, len, dpa, dpb, dt;
    int mx = 0;
    knn_status s = raw_rows(offsets, n_series, enc->d, foff, len, &mx);
    if (s)
        return s;
    std::vector<int64_t> h64(n_pairs);
    std::vector<int> ia(n_pairs), ib(n_pairs);
    auto fetch = [&](const int64_t *p, std::vector<int> &out) {
        if (is_device_ptr(p))
            cudaMemcpy(h64.data(), p, 8 * n_pairs, cudaMemcpyDeviceToHost);
        else
            memcpy(h64.data(), p, 8 * n_pairs);
        for (int64_t i = 0; i < n_pairs; ++i)
            out[i] = (int)h64[i];
    };
    fetch(pa, ia);
    fetch(pb, ib);
    for (int64_t i = 0; i < n_pairs; ++i)
        if (ia[i] < 0 || ia[i] >= n_series || ib[i] < 0 || ib[i] >= n_series)
            return set_error(KNN_ERR_INVALID, "pair index out of range");
    if ((s = dpa.ensure(4 * n_pairs)) || (s = dpb.ensure(4 * n_pairs)) || (s = dt.ensure(4 * n_pairs)))
        return s;
    cudaMemcpy(dpa.p, ia.data(), 4 * n_pairs, cudaMemcpyHostToDevice);
    cudaMemcpy(dpb.p, ib.data(), 4 * n_pairs, cudaMemcpyHostToDevice);
    cudaMemcpy(dt.p, targets, 4 * n_pairs,
               is_device_ptr(targets) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice);
    const int nsm = sm_count(enc->dev);
    if ((s = enc_forward(enc, series, foff.as<int64_t>(), enc->d, len.as<int>(), nullptr, enc->d,
                         (int)n_series, mx, nsm, st)))
        return s;
    enc_backward(enc, dpa.as<int>(), dpb.as<int>(), dt.as<float>(), (int)n_pairs, (int)n_series,
                 mx, nsm, st);
    cudaError_t e = cudaMemcpyAsync(loss, enc->loss.p, 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(grad, enc->grad.p, sizeof(float) * ENC_NPARAM, cudaMemcpyDeviceToHost,
                            st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e == cudaSuccess)
        e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_error(e, "encoder loss_grad");
    return KNN_OK;
}

extern "C" knn_status knn_encoder_train(knn_encoder *enc, knn_db *db, int64_t n_pairs,
                                        const knn_train_params *tp, knn_train_stats *stats,
                                        void *stream)
{
    if (!enc || !db || !tp)
        return set_error(KNN_ERR_INVALID, "NULL argument");
    if (enc->d != db->d)
        return set_error(KNN_ERR_INVALID, "encoder and database dimensionality differ");
    if (n_pairs < 1 || n_pairs > (1 << 24) || tp->epochs < 1 || tp->batch_pairs < 1 ||
        !(tp->lr > 0.f) || !(tp->band > 0.f) || (tp->distance != 0 && tp->distance != 1))
        return set_error(KNN_ERR_INVALID, "bad training parameters");
    cudaStream_t st = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventRecord(e0, st);
    // input scale from the database's spread, fixed at the first training call
    uint64_t rng = tp->seed ^ 0x7a1eull;
    const int N = db->N;
    if (enc->step == 0) {
        const int64_t ns = std::min<int64_t>(db->total_floats, 1 << 20);
        std::vector<float> sample(ns);
        cudaMemcpy(sample.data(), db->data.p, 4 * ns, cudaMemcpyDeviceToHost);
        double sum = 0, sq = 0;
        int64_t cnt = 0;
        // zeros are padding, the 1e18 values the DP's sentinel chunks
        for (float v : sample)
            if (v != 0.f && fabsf(v) < 0.5f * KNN_DP_SENTINEL) {
                sum += v;
                sq += (double)v * v;
                ++cnt;
            }
        const double var = cnt > 1 ? sq / cnt - (sum / cnt) * (sum / cnt) : 1.0;
        enc->in_scale = (float)(1.0 / std::sqrt(std::max(var, 1e-12)));
    }
    // pairs, seeded: half uniformly random, half "near": for an anchor the
    // nearest (by the exact distance) of MINE random candidates, so that the
    // ranking of close series is learned and not only the bulk of far ones
    constexpr int MINE = 16;
    const int64_t n_near = N > MINE ? n_pairs / 2 : 0;
    const int64_t n_rand = n_pairs - n_near;
    const int64_t n_dp = n_near * MINE + n_rand;
    std::vector<int2> items(n_dp);
    for (int64_t i = 0; i < n_near; ++i) {
        const int a = (int)(splitmix(rng) % (uint64_t)N);
        for (int j = 0; j < MINE; ++j) {
            int b;
            do {
                b = (int)(splitmix(rng) % (uint64_t)N);
            } while (b == a);
            items[i * MINE + j] = make_int2(b, a);  // (series, "query") as the DP expects
        }
    }
    for (int64_t i = 0; i < n_rand; ++i) {
        int a, b;
        do {
            a = (int)(splitmix(rng) % (uint64_t)N);
            b = (int)(splitmix(rng) % (uint64_t)N);
        } while (a == b && N > 1);
        items[n_near * MINE + i] = make_int2(b, a);
    }
    DevBuf ditems, dlb, draw, dtgt, ctl, bidx, bpa, bpb, btgt;
    knn_status s;
    if ((s = ditems.ensure(sizeof(int2) * n_dp)) || (s = dlb.ensure(4 * n_dp)) ||
        (s = draw.ensure(4 * n_dp)) || (s = dtgt.ensure(4 * n_dp)) ||
        (s = ctl.ensure(sizeof(Ctrl))))
        return s;
    cudaMemcpyAsync(ditems.p, items.data(), sizeof(int2) * n_dp, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(dlb.p, 0, 4 * n_dp, st);
    cudaMemsetAsync(ctl.p, 0, sizeof(Ctrl), st);
    const int np = (int)n_dp;
    Ctrl *ct = ctl.as<Ctrl>();
    cudaMemcpyAsync(&ct->seg_count[0], &np, 4, cudaMemcpyHostToDevice, st);
    // targets from the scan's own DP (pair mode, no threshold)
    int P = 0, G = 0;
    const int r_all = band_radius(db->max_len, db->max_len, tp->band);
    choose_dp_config(db->deff, r_all, db->max_len, &P, &G);
    if (!P)
        return set_error(KNN_ERR_UNSUPPORTED, "band too wide for the compiled DP variants");
    DpArgs x{};
    x.items = ditems.as<int2>();
    x.item_lb = dlb.as<float>();
    x.n_items = &ct->seg_count[0];
    x.items_cap = n_dp;
    x.head = &ct->seg_head[0];
    x.db = db->data.as<float>();
    x.db_off = db->off.as<int64_t>();
    x.db_len = db->len.as<int>();
    x.db_id = db->id.as<int>();
    x.q = db->data.as<float>();
    x.q_off = db->off.as<int64_t>();
    x.q_len = db->len.as<int>();
    x.band = tp->band;
    x.G = G;
    x.mu_keep = 1.f;
    x.mu_prune = 1.f;
    x.out_pair = draw.as<float>();
    x.cells_stat = STAT_DP_CELLS;
    x.stats = ct->stats;
    x.status = &ct->status;
    launch_dp(x, db->deff, P, tp->distance, db->n_sm, st);
    pair_targets_kernel<<<256, 256, 0, st>>>(draw.as<float>(), db->len.as<int>(), db->len.as<int>(),
                                             ditems.as<int2>(), np, tp->distance,
                                             dtgt.as<float>());
    std::vector<float> hall(n_dp);
    cudaMemcpyAsync(hall.data(), dtgt.p, 4 * n_dp, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess)
        return cuda_error(e, "training targets");
    // keep, per anchor, its nearest candidate; then the random pairs
    std::vector<int2> chosen;
    std::vector<float> htgt;
    chosen.reserve(n_pairs);
    htgt.reserve(n_pairs);
    for (int64_t i = 0; i < n_near; ++i) {
        int64_t best = -1;
        for (int j = 0; j < MINE; ++j) {
            const int64_t t = i * MINE + j;
            if (std::isfinite(hall[t]) && (best < 0 || hall[t] < hall[best]))
                best = t;
        }
        if (best >= 0) {
            chosen.push_back(items[best]);
            htgt.push_back(hall[best]);
        }
    }
    for (int64_t i = 0; i < n_rand; ++i) {
        chosen.push_back(items[n_near * MINE + i]);
        htgt.push_back(hall[n_near * MINE + i]);
    }
    items.swap(chosen);
    n_pairs = (int64_t)items.size();
    // pairs with an unreachable end cell carry no target: drop them
    std::vector<int64_t> keep;
    keep.reserve(n_pairs);
    for (int64_t i = 0; i < n_pairs; ++i)
        if (std::isfinite(htgt[i]))
            keep.push_back(i);
    if (keep.empty())
        return set_error(KNN_ERR_INVALID, "no training pair has a finite distance");
    const int BP = std::min<int>(tp->batch_pairs, (int)keep.size());
    const int L = db->max_len;
    if ((s = bidx.ensure(4 * (size_t)2 * BP)) || (s = bpa.ensure(4 * (size_t)BP)) ||
        (s = bpb.ensure(4 * (size_t)BP)) || (s = btgt.ensure(4 * (size_t)BP)))
        return s;
    std::vector<int> hpa(BP), hpb(BP);
    for (int i = 0; i < BP; ++i) {
        hpa[i] = i;
        hpb[i] = BP + i;
    }
    cudaMemcpyAsync(bpa.p, hpa.data(), 4 * BP, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(bpb.p, hpb.data(), 4 * BP, cudaMemcpyHostToDevice, st);
    std::vector<int> hidx(2 * BP);
    std::vector<float> hbt(BP);
    double first_loss = -1.0, last_loss = 0.0;
    int64_t steps = 0;
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    for (int ep = 0; ep < tp->epochs; ++ep) {
        // shuffle (Fisher-Yates on the seeded generator)
        for (int64_t i = (int64_t)keep.size() - 1; i > 0; --i)
            std::swap(keep[i], keep[splitmix(rng) % (uint64_t)(i + 1)]);
        double ep_loss = 0.0;
        int ep_batches = 0;
        for (size_t b0 = 0; b0 + BP <= keep.size(); b0 += BP) {
            for (int i = 0; i < BP; ++i) {
                const int2 it = items[keep[b0 + i]];
                hidx[i] = it.y;
                hidx[BP + i] = it.x;
                hbt[i] = htgt[keep[b0 + i]];
            }
            cudaMemcpyAsync(bidx.p, hidx.data(), 4 * 2 * BP, cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(btgt.p, hbt.data(), 4 * BP, cudaMemcpyHostToDevice, st);
            if ((s = enc_forward(enc, db->data.as<float>(), db->off.as<int64_t>(), db->deff,
                                 db->len.as<int>(), bidx.as<int>(), db->d, 2 * BP, L, db->n_sm,
                                 st)))
                return s;
            enc_backward(enc, bpa.as<int>(), bpb.as<int>(), btgt.as<float>(), BP, 2 * BP, L,
                         db->n_sm, st);
            ++enc->step;
            ++steps;
            const float c1 = 1.f - std::pow(b1, (float)enc->step);
            const float c2 = 1.f - std::pow(b2, (float)enc->step);
            adam_kernel<<<(ENC_NPARAM + 255) / 256, 256, 0, st>>>(
                enc->params.as<float>(), enc->grad.as<float>(), enc->m.as<float>(),
                enc->v.as<float>(), ENC_NPARAM, tp->lr, b1, b2, eps, c1, c2);
            enc_weights_bf16(enc, st);
            float l = 0.f;
            cudaMemcpyAsync(&l, enc->loss.p, 4, cudaMemcpyDeviceToHost, st);
            cudaStreamSynchronize(st);  // host buffers are reused next batch
            if (first_loss < 0)
                first_loss = l;
            ep_loss += l;
            ++ep_batches;
        }
        last_loss = ep_batches ? ep_loss / ep_batches : 0.0;
    }
    cudaEventRecord(e1, st);
    e = cudaStreamSynchronize(st);
    if (e == cudaSuccess)
        e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_error(e, "encoder training");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (stats) {
        stats->first_loss = first_loss;
        stats->final_loss = last_loss;
        stats->ms = ms;
        stats->pairs = (int64_t)keep.size();
        stats->steps = steps;
    }
    return KNN_OK;
}

// caller ids of the winners of each (query, tile): tile_idx is in the
// database's length-sorted order
__global__ void score_ids_kernel(const float *score, const int *tile_idx, const int *db_id,
                                 int64_t total, float *out_score, int64_t *out_series)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int c = tile_idx[i];
        out_score[i] = c >= 0 ? score[i] : KNN_INF;
        out_series[i] = c >= 0 ? (int64_t)db_id[c] : -1;
    }
}

extern "C" knn_status knn_encoder_scores(knn_db *db, const float *queries,
                                         const int64_t *q_offsets, int32_t n_queries,
                                         float *out_score, int64_t *out_series, void *stream)
{
    if (!db || !queries || !q_offsets || !out_score || !out_series)
        return set_error(KNN_ERR_INVALID, "NULL argument");
    if (!db->enc)
        return set_error(KNN_ERR_INVALID, "no encoder attached to the database");
    if (n_queries < 1)
        return set_error(KNN_ERR_INVALID, "n_queries must be >= 1");
    if (!is_device_ptr(out_score) || !is_device_ptr(out_series))
        return set_error(KNN_ERR_INVALID, "outputs must be device memory");
    cudaStream_t st = (cudaStream_t)stream;
    std::vector<int64_t> hq(n_queries + 1);
    if (is_device_ptr(q_offsets))
        cudaMemcpy(hq.data(), q_offsets, 8 * (n_queries + 1), cudaMemcpyDeviceToHost);
    else
        std::copy(q_offsets, q_offsets + n_queries + 1, hq.begin());
    const int CH = chunk_floats(db->deff), PPC = chunk_points(db->deff);
    std::vector<int64_t> rel(n_queries + 1), qoff(n_queries);
    std::vector<int> len(n_queries);
    int64_t qfloats = 0;
    int max_m = 1;
    for (int i = 0; i < n_queries; ++i) {
        const int64_t m = hq[i + 1] - hq[i];
        if (m < 1 || m > 65536)
            return set_error(KNN_ERR_INVALID, "query lengths must be in [1, 65536]");
        len[i] = (int)m;
        max_m = std::max(max_m, (int)m);
        qfloats += CH;  // leading chunk, as in the scan's layout
        qoff[i] = qfloats;
        qfloats += (m + PPC - 1) / PPC * CH;
    }
    for (int i = 0; i <= n_queries; ++i)
        rel[i] = hq[i] - hq[0];
    const int64_t tiles = (db->N + 63) / 64;
    const int64_t npts = hq[n_queries] - hq[0];
    DevBuf qraw, src_off, qbuf, qo, ql, qemb, qnorm, scores, idx, status;
    knn_status s;
    if ((s = qraw.ensure(sizeof(float) * npts * db->d)) || (s = src_off.ensure(8 * (n_queries + 1))) ||
        (s = qbuf.ensure(sizeof(float) * qfloats)) || (s = qo.ensure(8 * n_queries)) ||
        (s = ql.ensure(4 * n_queries)) || (s = qemb.ensure(2 * 64 * n_queries)) ||
        (s = qnorm.ensure(4 * n_queries)) || (s = scores.ensure(4 * n_queries * tiles)) ||
        (s = idx.ensure(4 * n_queries * tiles)) || (s = status.ensure(sizeof(int))))
        return s;
    const float *src = queries + hq[0] * db->d;
    cudaMemcpyAsync(qraw.p, src, sizeof(float) * npts * db->d,
                    is_device_ptr(queries) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(src_off.p, rel.data(), 8 * (n_queries + 1), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(qo.p, qoff.data(), 8 * n_queries, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(ql.p, len.data(), 4 * n_queries, cudaMemcpyHostToDevice, st);
    cudaMemsetAsync(status.p, 0, sizeof(int), st);
    launch_repack(qraw.as<float>(), src_off.as<int64_t>(), nullptr, n_queries, db->d, db->deff,
                  qo.as<int64_t>(), qbuf.as<float>(), st, true);
    if ((s = enc_work(db->enc, n_queries, max_m)))
        return s;
    if ((s = enc_scan_scores(db, qbuf.as<float>(), qo.as<int64_t>(), ql.as<int>(), n_queries,
                             max_m, qemb.p, qnorm.as<float>(), scores.as<float>(), idx.as<int>(),
                             status.as<int>(), st)))
        return s;
    const int64_t total = (int64_t)n_queries * tiles;
    score_ids_kernel<<<(int)std::min<int64_t>((total + 255) / 256, 4096), 256, 0, st>>>(
        scores.as<float>(), idx.as<int>(), db->id.as<int>(), total, out_score, out_series);
    int hs = 0;
    cudaMemcpyAsync(&hs, status.p, sizeof(int), cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess)
        e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_error(e, "encoder scores");
    if (hs & KNN_DEV_TIMEOUT)
        return set_error(KNN_ERR_TIMEOUT, "a device wait gave up");
    return KNN_OK;
}

extern "C" knn_status knn_encoder_attach(knn_db *db, knn_encoder *enc, void *stream)
{
    if (!db || !enc)
        return set_error(KNN_ERR_INVALID, "NULL argument");
    if (enc->d != db->d)
        return set_error(KNN_ERR_INVALID, "encoder and database dimensionality differ");
    cudaStream_t st = (cudaStream_t)stream;
    knn_status s;
    if ((s = db->emb.ensure(sizeof(__nv_bfloat16) * (size_t)db->N * ENC_E)) ||
        (s = db->emb_norm.ensure(sizeof(float) * (size_t)db->N)))
        return s;
    const int chunk = std::max(1, std::min(db->N, (1 << 21) / std::max(db->max_len, 1)));
    DevBuf didx;
    if ((s = didx.ensure(4 * (size_t)chunk)))
        return s;
    std::vector<int> idx(chunk);
    for (int b0 = 0; b0 < db->N; b0 += chunk) {
        const int B = std::min(chunk, db->N - b0);
        for (int i = 0; i < B; ++i)
            idx[i] = b0 + i;  // bucket order: embeddings stored in bucket order
        cudaMemcpyAsync(didx.p, idx.data(), 4 * B, cudaMemcpyHostToDevice, st);
        if ((s = enc_forward(enc, db->data.as<float>(), db->off.as<int64_t>(), db->deff,
                             db->len.as<int>(), didx.as<int>(), db->d, B, db->max_len, db->n_sm,
                             st)))
            return s;
        enc_emb_bf16(enc->e.as<float>(), didx.as<int>(), B, db->emb.as<__nv_bfloat16>(),
                     db->emb_norm.as<float>(), st);
        cudaStreamSynchronize(st);
    }
    cudaError_t e = cudaStreamSynchronize(st);
    if (e == cudaSuccess)
        e = cudaGetLastError();
    if (e != cudaSuccess)
        return cuda_error(e, "encoder attach");
    db->enc = enc;
    for (auto &g : db->graphs)
        cudaGraphExecDestroy(g.second);
    db->graphs.clear();
    return KNN_OK;
}

extern "C" knn_status knn_encoder_save(const knn_encoder *enc, const char *path)
{
    if (!enc || !path)
        return set_error(KNN_ERR_INVALID, "NULL argument");
    std::vector<float> p(ENC_NPARAM), m(ENC_NPARAM), v(ENC_NPARAM);
    cudaMemcpy(p.data(), enc->params.p, 4 * ENC_NPARAM, cudaMemcpyDeviceToHost);
    cudaMemcpy(m.data(), enc->m.p, 4 * ENC_NPARAM, cudaMemcpyDeviceToHost);
    cudaMemcpy(v.data(), enc->v.p, 4 * ENC_NPARAM, cudaMemcpyDeviceToHost);
    FILE *f = fopen(path, "wb");
    if (!f)
        return set_error(KNN_ERR_INVALID, std::string("cannot write ") + path);
    // JSON header line, then little-endian float32 params, Adam m, Adam v
    fprintf(f, "{\"format\": \"knnwarp-encoder\", \"version\": 1, \"d\": %d, \"params\": %d, "
               "\"step\": %lld, \"in_scale\": %.9g}\n",
            enc->d, ENC_NPARAM, (long long)enc->step, (double)enc->in_scale);
    fwrite(p.data(), 4, ENC_NPARAM, f);
    fwrite(m.data(), 4, ENC_NPARAM, f);
    fwrite(v.data(), 4, ENC_NPARAM, f);
    fclose(f);
    return KNN_OK;
}

extern "C" knn_status knn_encoder_load(const char *path, knn_encoder **out)
{
    if (!path || !out)
        return set_error(KNN_ERR_INVALID, "NULL argument");
    *out = nullptr;
    FILE *f = fopen(path, "rb");
    if (!f)
        return set_error(KNN_ERR_INVALID, std::string("cannot read ") + path);
    char line[512];
    if (!fgets(line, sizeof line, f)) {
        fclose(f);
        return set_error(KNN_ERR_INVALID, "empty encoder file");
    }
    int d = 0, np = 0;
    long long step = 0;
    double in_scale = 1.0;
    if (!strstr(line, "knnwarp-encoder") ||
        sscanf(strstr(line, "\"d\":"), "\"d\": %d, \"params\": %d, \"step\": %lld, \"in_scale\": %lf",
               &d, &np, &step, &in_scale) != 4 ||
        np != ENC_NPARAM) {
        fclose(f);
        return set_error(KNN_ERR_INVALID, "not an encoder file of this version");
    }
    std::vector<float> p(ENC_NPARAM), m(ENC_NPARAM), v(ENC_NPARAM);
    const bool ok = fread(p.data(), 4, ENC_NPARAM, f) == (size_t)ENC_NPARAM &&
                    fread(m.data(), 4, ENC_NPARAM, f) == (size_t)ENC_NPARAM &&
                    fread(v.data(), 4, ENC_NPARAM, f) == (size_t)ENC_NPARAM;
    fclose(f);
    if (!ok)
        return set_error(KNN_ERR_INVALID, "truncated encoder file");
    knn_encoder *enc = nullptr;
    knn_status s = knn_encoder_create(d, 0, &enc);
    if (s)
        return s;
    cudaMemcpy(enc->params.p, p.data(), 4 * ENC_NPARAM, cudaMemcpyHostToDevice);
    cudaMemcpy(enc->m.p, m.data(), 4 * ENC_NPARAM, cudaMemcpyHostToDevice);
    cudaMemcpy(enc->v.p, v.data(), 4 * ENC_NPARAM, cudaMemcpyHostToDevice);
    enc->step = step;
    enc->in_scale = (float)in_scale;
    enc_weights_bf16(enc, nullptr);
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        knn_encoder_destroy(enc);
        return cuda_error(e, "encoder load");
    }
    *out = enc;
    return KNN_OK;
}
