// Device-side helpers shared by the scan kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define KNN_FULL_MASK 0xffffffffu
#define KNN_INF __int_as_float(0x7f800000)
#define KNN_INF_HOST (__builtin_huge_valf())
#define KNN_EMPTY_KEY 0xffffffffffffffffull

// Status bits written by kernels into the per-call device status word.
enum : int {
    KNN_DEV_OK = 0,
    KNN_DEV_TIMEOUT = 1,     // a bounded wait (mbarrier / queue) gave up
    KNN_DEV_CAPACITY = 2,    // an eps-NN list overflowed
    KNN_DEV_BAD_SHAPE = 4,   // a launch received a shape it cannot handle
};

// Coordinate of the sentinel point stored before every series and query the
// DP reads (the chunk of floats before its first point): a row or column
// index below 0 reads it, so a cell with both indices negative costs 0 and a
// cell with one negative index about 1e36 per coordinate.
#define KNN_DP_SENTINEL 1e18f

// Upper limit on polling iterations of any device-side wait; with the
// backoff below this is of the order of a second.
#define KNN_SPIN_LIMIT (1u << 22)

namespace knn {

// Floats per LB chunk: the smallest multiple of both the point size and one
// float4, so that a chunk holds whole points and whole 16-byte vectors.
__host__ __device__ constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }
__host__ __device__ constexpr int chunk_floats(int d) { return d / gcd_c(d, 4) * 4; }
__host__ __device__ constexpr int chunk_points(int d) { return chunk_floats(d) / d; }

__device__ __forceinline__ int clampi(int v, int lo, int hi) { return min(max(v, lo), hi); }

// Load one D-dimensional point with the widest aligned vector the layout
// allows.  Every series starts on a 16-byte boundary, so point i starts on a
// (4*D*i mod 16)-aligned address: float4 when D%4==0, float2 when D%2==0.
template <int D>
__device__ __forceinline__ void load_point(const float *__restrict__ p, float (&v)[D])
{
    if constexpr (D % 4 == 0) {
#pragma unroll
        for (int k = 0; k < D; k += 4) {
            float4 t = __ldg(reinterpret_cast<const float4 *>(p + k));
            v[k] = t.x; v[k + 1] = t.y; v[k + 2] = t.z; v[k + 3] = t.w;
        }
    } else if constexpr (D % 2 == 0) {
#pragma unroll
        for (int k = 0; k < D; k += 2) {
            float2 t = __ldg(reinterpret_cast<const float2 *>(p + k));
            v[k] = t.x; v[k + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int k = 0; k < D; ++k) v[k] = __ldg(p + k);
    }
}

// min(a, b, c) in one instruction (three-input PTX min, sm_100 and later).
__device__ __forceinline__ float fmin3(float a, float b, float c)
{
    float d;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// max(a, b, c) in one instruction (three-input PTX max, sm_100 and later).
__device__ __forceinline__ float fmax3(float a, float b, float c)
{
    float d;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
    return d;
}

// Distance of x to the interval [l, u] (l <= u, or l = +inf / u = -inf for
// an empty window): the positive one of l - x and x - u, else 0.  Equal to
// x - clamp(x, l, u) in magnitude bit for bit (the same single rounded
// subtraction), with one three-input max instead of a max and a min.
__device__ __forceinline__ float box_gap(float x, float l, float u)
{
    return fmax3(l - x, x - u, 0.f);
}

// a - b on both lanes of a packed pair, one rounding each (b * -1 is exact,
// so the fused form rounds exactly like a subtraction).  Packed FP32 pairs
// (sm_100 and later) halve the instructions issued per coordinate.
__device__ __forceinline__ float2 sub2(float2 a, float2 b)
{
    return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
}

// Squared Euclidean distance, accumulated on top of `init` with FMAs in
// coordinate order.  init = +inf masks a cell out of the band.
template <int D>
__device__ __forceinline__ float sqdist_acc(const float (&a)[D], const float (&b)[D], float init)
{
    float acc = init;
#pragma unroll
    for (int k = 0; k < D; ++k) {
        const float t = a[k] - b[k];
        acc = __fmaf_rn(t, t, acc);
    }
    return acc;
}

// (distance, id) packed so that unsigned 64-bit order is (distance, id)
// order; distances are non-negative floats whose bit patterns sort like the
// values.
__device__ __forceinline__ unsigned long long make_key(float dist, uint32_t id)
{
    return (static_cast<unsigned long long>(__float_as_uint(dist)) << 32) | id;
}
__device__ __forceinline__ float key_dist(unsigned long long key)
{
    return __uint_as_float(static_cast<uint32_t>(key >> 32));
}
__device__ __forceinline__ uint32_t key_id(unsigned long long key)
{
    return static_cast<uint32_t>(key & 0xffffffffu);
}

__device__ __forceinline__ unsigned long long ld_volatile_u64(const unsigned long long *p)
{
    return *reinterpret_cast<const volatile unsigned long long *>(p);
}
__device__ __forceinline__ float ld_volatile_f32(const float *p)
{
    return *reinterpret_cast<const volatile float *>(p);
}

// Lock-free insertion of `key` into the `len` smallest keys kept ascending
// in slots[0..len).  Each slot is swapped atomically with the carried key
// (atomicMin keeps the smaller, the larger travels on), so every key that
// falls off the end is larger than all keys left behind.  A key equal to a
// slot's content is already present and stops (no duplicates).  Returns
// true if the key was kept.
__device__ __forceinline__ bool topk_insert(unsigned long long *slots, int len,
                                            unsigned long long key)
{
    if (key >= ld_volatile_u64(slots + len - 1))
        return false;
    unsigned long long carry = key;
    for (int s = 0; s < len; ++s) {
        unsigned long long old = atomicMin(slots + s, carry);
        if (old == carry)
            return true;  // already present
        if (old == KNN_EMPTY_KEY)
            return true;  // took an empty slot
        carry = old > carry ? old : carry;
    }
    return carry != key;
}

// Non-negative floats order like their bit patterns: atomicMin on the bits.
__device__ __forceinline__ void atomic_min_pos_float(float *addr, float v)
{
    atomicMin(reinterpret_cast<unsigned int *>(addr), __float_as_uint(v));
}

}  // namespace knn
