// kc_device.cuh -- device helpers shared by the library's kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace kc {

// ---- packed float pairs (two fp32 lanes in one 64-bit register pair) ----

__device__ __forceinline__ uint64_t pk(float a, float b)
{
    uint64_t r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}

__device__ __forceinline__ float2 upk(uint64_t v)
{
    float2 r;
    asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
    return r;
}

// (a.x - b.x, a.y - b.y), each correctly rounded.
__device__ __forceinline__ uint64_t sub2(uint64_t a, uint64_t b)
{
    uint64_t r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}

// (a.x*b.x + c.x, a.y*b.y + c.y), each fused (one rounding).
__device__ __forceinline__ uint64_t fma2(uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

__device__ __forceinline__ float max3f(float a, float b, float c)
{
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Squared distance from a sample to a box, float.  px[a] = (x_a, -x_a),
// bx[a] = (lo_a, -hi_a): one packed subtraction gives (lo_a - x_a, x_a - hi_a),
// whose maximum with 0 is the distance to the interval along a (exactly the
// |x_a - mid{lo_a, x_a, hi_a}| of Section 3.1, up to the subtraction's
// rounding).  Squares accumulate in two interleaved fused chains.
template <int D>
__device__ __forceinline__ float box_dist_f32(const uint64_t *px, const uint64_t *bx)
{
    uint64_t acc = 0;
#pragma unroll
    for (int a = 0; a + 1 < D; a += 2) {
        const float2 t0 = upk(sub2(bx[a], px[a]));
        const float2 t1 = upk(sub2(bx[a + 1], px[a + 1]));
        const uint64_t m = pk(max3f(t0.x, t0.y, 0.f), max3f(t1.x, t1.y, 0.f));
        acc = fma2(m, m, acc);
    }
    float2 s = upk(acc);
    if (D & 1) {
        const float2 t = upk(sub2(bx[D - 1], px[D - 1]));
        const float m = max3f(t.x, t.y, 0.f);
        s.x = fmaf(m, m, s.x);
    }
    return s.x + s.y;
}

// Squared distance between a sample and a point, float.  px[a/2] = (x_a, x_{a+1}),
// cx likewise; two interleaved fused chains (same rounding count as above).
template <int D>
__device__ __forceinline__ float pt_dist_f32(const uint64_t *px, const uint64_t *cx)
{
    uint64_t acc = 0;
#pragma unroll
    for (int p = 0; p < D / 2; ++p) {
        const uint64_t t = sub2(px[p], cx[p]);
        acc = fma2(t, t, acc);
    }
    float2 s = upk(acc);
    if (D & 1) {
        const float2 xl = upk(px[D / 2]);
        const float2 cl = upk(cx[D / 2]);
        const float t = xl.x - cl.x;
        s.x = fmaf(t, t, s.x);
    }
    return s.x + s.y;
}

// ---- double evaluation in attribute order, no contraction ----

__device__ __forceinline__ double mid3d(double l, double x, double h)
{
    return x < l ? l : (x > h ? h : x);
}

// ---- ordered keys: (value, position) packed so that a larger key is a
// larger value, and among equal values a smaller position. ----

__device__ __forceinline__ unsigned long long key_max(float v, uint32_t pos)
{
    return ((unsigned long long)__float_as_uint(v) << 32) | (unsigned long long)(0xFFFFFFFFu - pos);
}
__device__ __forceinline__ float key_val(unsigned long long k) { return __uint_as_float((uint32_t)(k >> 32)); }
__device__ __forceinline__ uint32_t key_pos(unsigned long long k) { return 0xFFFFFFFFu - (uint32_t)k; }

// Order-preserving map of a float to uint32 (for min/max of signed floats).
__device__ __forceinline__ uint32_t ord_f32(float v)
{
    const uint32_t u = __float_as_uint(v);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float unord_f32(uint32_t u)
{
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7FFFFFFFu) : ~u);
}
__device__ __forceinline__ uint64_t ord_f64(double v)
{
    const uint64_t u = (uint64_t)__double_as_longlong(v);
    return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
}
__device__ __forceinline__ double unord_f64(uint64_t u)
{
    return __longlong_as_double((long long)((u & 0x8000000000000000ull) ? (u & 0x7FFFFFFFFFFFFFFFull) : ~u));
}

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// Work item w of a list batch -> (node, first entry); see ListBatch.
__device__ __forceinline__ void list_item(const int64_t *__restrict__ tile_prefix, int B, int64_t w, int tile,
                                          int *b_out, int64_t *start_out)
{
    int lo = 0, hi = B;   // largest b with tile_prefix[b] <= w
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (tile_prefix[mid] <= w) lo = mid;
        else hi = mid;
    }
    *b_out = lo;
    *start_out = (int64_t)(w - tile_prefix[lo]) * tile;
}

}  // namespace kc
