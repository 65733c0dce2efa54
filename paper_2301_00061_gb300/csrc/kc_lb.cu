// kc_lb.cu -- node lower bound beta(M) = max_s min_k beta_s^k(M^k)
// (Section 3.1, Eqs. 9-11 with the closed-form minimiser mid{lo, x, hi}).
//
// One persistent launch evaluates a batch of B nodes: the node boxes are staged
// once per CTA in shared memory, every sample is read from HBM once per batch
// (coalesced 64/128-bit loads of the attribute-major copy), and each thread
// keeps ST samples in registers while it sweeps all B nodes.  The max over
// samples is tracked per warp in shared memory as a packed (value, position)
// key; a warp only reduces with shuffles when one of its lanes beats the
// warp's running best.  One partial per CTA and node goes to global scratch
// and a second small kernel reduces them (deterministic: the largest value,
// the smallest position on ties).
#include <cuda_runtime.h>

#include <atomic>

#include "kc_device.cuh"
#include "kc_internal.cuh"

namespace kc {

namespace {

template <int ST>
__device__ __forceinline__ void load_row(const float *__restrict__ p, float (&v)[ST])
{
    if constexpr (ST == 4) {
        const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
        v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
    } else if constexpr (ST == 2) {
        const float2 q = __ldg(reinterpret_cast<const float2 *>(p));
        v[0] = q.x; v[1] = q.y;
    } else {
        v[0] = __ldg(p);
    }
}

// D packed (lo, -hi) pairs of one box from shared memory into registers.
template <int D>
__device__ __forceinline__ void load_box(const uint64_t *p, uint64_t (&bx)[D])
{
    if constexpr ((D % 2) == 0) {
#pragma unroll
        for (int a = 0; a < D; a += 2) {
            const ulonglong2 q = *reinterpret_cast<const ulonglong2 *>(p + a);
            bx[a] = q.x;
            bx[a + 1] = q.y;
        }
    } else {
#pragma unroll
        for (int a = 0; a < D; ++a) bx[a] = p[a];
    }
}

// Every node's running maximum over one thread's ST samples px (packed
// (x, -x) per attribute; when not `full`, samples s0 + j >= n are ignored),
// merged into the warp's keys mine[b] (value bits, ~position): a warp
// reduces with shuffles only when one of its lanes may beat the warp's best.
template <int D, int K, int ST>
__device__ __forceinline__ void eval_nodes(const uint64_t (&px)[ST][D], bool full, int64_t s0, int64_t n,
                                           const uint64_t *sbox, int B, unsigned long long *mine, int lane)
{
    constexpr int KD = K * D;
    for (int b = 0; b < B; ++b) {
        const uint64_t *bb = sbox + (size_t)b * KD;
        float best[ST];
#pragma unroll
        for (int j = 0; j < ST; ++j) best[j] = __int_as_float(0x7f800000);
#pragma unroll
        for (int k = 0; k < K; ++k) {
            uint64_t bx[D];
            load_box<D>(bb + k * D, bx);
#pragma unroll
            for (int j = 0; j < ST; ++j) best[j] = fminf(best[j], box_dist_f32<D>(px[j], bx));
        }
        if (!full) {
#pragma unroll
            for (int j = 0; j < ST; ++j)
                if (s0 + j >= n) best[j] = -1.f;
        }
        float m = best[0];
#pragma unroll
        for (int j = 1; j < ST; ++j) m = fmaxf(m, best[j]);
        const unsigned long long cur = mine[b];
        const bool maybe = m >= key_val(cur);
        if (__any_sync(0xffffffffu, maybe)) {
            unsigned long long key = 0ull;
            if (maybe) {
                int jm = 0;
#pragma unroll
                for (int j = ST - 1; j >= 0; --j)
                    if (best[j] == m) jm = j;
                key = key_max(m, (uint32_t)(s0 + jm));
            }
            key = warp_max_u64(key);
            if (lane == 0 && key > cur) mine[b] = key;
            __syncwarp();
        }
    }
}

// Float lower bound, compile-time D and K.  Shared memory: B*K*D packed
// boxes + (warps x B) running-best keys.
template <int D, int K, int ST>
__global__ void __launch_bounds__(kThreads, 2)
lb_f32_fast(const float *__restrict__ X, int64_t ld, int64_t n, const float *__restrict__ lo,
            const float *__restrict__ hi, int B, unsigned long long *__restrict__ part)
{
    constexpr int KD = K * D;
    constexpr int NW = kThreads / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *sbox = reinterpret_cast<uint64_t *>(smem);
    unsigned long long *wbest = reinterpret_cast<unsigned long long *>(sbox + (size_t)B * KD);
    for (int i = threadIdx.x; i < B * KD; i += kThreads) sbox[i] = pk(lo[i], -hi[i]);
    for (int i = threadIdx.x; i < NW * B; i += kThreads) wbest[i] = 0ull;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    unsigned long long *mine = wbest + (threadIdx.x >> 5) * B;
    const int64_t tile = (int64_t)kThreads * ST;
    for (int64_t base = (int64_t)blockIdx.x * tile; base < n; base += (int64_t)gridDim.x * tile) {
        const int64_t s0 = base + (int64_t)threadIdx.x * ST;
        const bool full = s0 + ST <= n;
        uint64_t px[ST][D];
        if (full) {
#pragma unroll
            for (int a = 0; a < D; ++a) {
                float v[ST];
                load_row<ST>(X + (size_t)a * ld + s0, v);
#pragma unroll
                for (int j = 0; j < ST; ++j) px[j][a] = pk(v[j], -v[j]);
            }
        } else {
#pragma unroll
            for (int a = 0; a < D; ++a)
#pragma unroll
                for (int j = 0; j < ST; ++j) {
                    const float v = (s0 + j < n) ? X[(size_t)a * ld + s0 + j] : 0.f;
                    px[j][a] = pk(v, -v);
                }
        }
        eval_nodes<D, K, ST>(px, full, s0, n, sbox, B, mine, lane);
    }
    __syncthreads();
    for (int b = threadIdx.x; b < B; b += kThreads) {
        unsigned long long m = 0ull;
        for (int w = 0; w < NW; ++w) {
            const unsigned long long v = wbest[w * B + b];
            m = v > m ? v : m;
        }
        part[(size_t)blockIdx.x * B + b] = m;
    }
}

// Float lower bound for any D <= DMAX and K (runtime).  Boxes are staged with
// D padded to an even count by (0, -0) pairs, which add exactly zero.
template <int DMAX>
__global__ void __launch_bounds__(kThreads)
lb_f32_generic(const float *__restrict__ X, int64_t ld, int64_t n, const float *__restrict__ lo,
               const float *__restrict__ hi, int B, int K, int D, unsigned long long *__restrict__ part)
{
    constexpr int NW = kThreads / 32;
    const int Dp = (D + 1) & ~1;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *sbox = reinterpret_cast<uint64_t *>(smem);                        // [B][K][Dp]
    unsigned long long *wbest = reinterpret_cast<unsigned long long *>(sbox + (size_t)B * K * Dp);
    for (int i = threadIdx.x; i < B * K * Dp; i += kThreads) {
        const int a = i % Dp, bk = i / Dp;
        sbox[i] = a < D ? pk(lo[(size_t)bk * D + a], -hi[(size_t)bk * D + a]) : pk(0.f, -0.f);
    }
    for (int i = threadIdx.x; i < NW * B; i += kThreads) wbest[i] = 0ull;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    unsigned long long *mine = wbest + (threadIdx.x >> 5) * B;
    for (int64_t s = (int64_t)blockIdx.x * kThreads + threadIdx.x; s - threadIdx.x < n;
         s += (int64_t)gridDim.x * kThreads) {
        const bool valid = s < n;
        uint64_t px[DMAX];
#pragma unroll
        for (int a = 0; a < DMAX; ++a) {
            const float v = (valid && a < D) ? X[(size_t)a * ld + s] : 0.f;
            px[a] = pk(v, -v);
        }
        for (int b = 0; b < B; ++b) {
            float best = __int_as_float(0x7f800000);
            for (int k = 0; k < K; ++k) {
                const uint64_t *bx = sbox + ((size_t)b * K + k) * Dp;
                uint64_t acc = 0;
#pragma unroll
                for (int a = 0; a < DMAX; a += 2) {
                    if (a < Dp) {
                        const float2 t0 = upk(sub2(bx[a], px[a]));
                        const float2 t1 = upk(sub2(bx[a + 1], px[a + 1]));
                        const uint64_t m = pk(max3f(t0.x, t0.y, 0.f), max3f(t1.x, t1.y, 0.f));
                        acc = fma2(m, m, acc);
                    }
                }
                const float2 sacc = upk(acc);
                best = fminf(best, sacc.x + sacc.y);
            }
            const float m = valid ? best : -1.f;
            const unsigned long long cur = mine[b];
            const bool maybe = m >= key_val(cur);
            if (__any_sync(0xffffffffu, maybe)) {
                unsigned long long key = maybe ? key_max(m, (uint32_t)s) : 0ull;
                key = warp_max_u64(key);
                if (lane == 0 && key > cur) mine[b] = key;
                __syncwarp();
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < B; b += kThreads) {
        unsigned long long m = 0ull;
        for (int w = 0; w < NW; ++w) {
            const unsigned long long v = wbest[w * B + b];
            m = v > m ? v : m;
        }
        part[(size_t)blockIdx.x * B + b] = m;
    }
}

// Double lower bound: mid{lo, x, hi}, d = x - mid, acc = acc + d*d in attribute
// order with separate roundings -- the serial evaluation, bit for bit.
template <int DMAX>
__global__ void __launch_bounds__(kThreads)
lb_f64(const double *__restrict__ X, int64_t ld, int64_t n, const double *__restrict__ lo,
       const double *__restrict__ hi, int B, int K, int D, double *__restrict__ pval,
       uint32_t *__restrict__ ppos)
{
    constexpr int NW = kThreads / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    double *slo = reinterpret_cast<double *>(smem);
    double *shi = slo + (size_t)B * K * D;
    double *wval = shi + (size_t)B * K * D;                       // [NW][B]
    uint32_t *wpos = reinterpret_cast<uint32_t *>(wval + NW * B); // [NW][B]
    for (int i = threadIdx.x; i < B * K * D; i += kThreads) { slo[i] = lo[i]; shi[i] = hi[i]; }
    for (int i = threadIdx.x; i < NW * B; i += kThreads) { wval[i] = -1.0; wpos[i] = 0xFFFFFFFFu; }
    __syncthreads();

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t s = (int64_t)blockIdx.x * kThreads + threadIdx.x; s - threadIdx.x < n;
         s += (int64_t)gridDim.x * kThreads) {
        const bool valid = s < n;
        double x[DMAX];
#pragma unroll
        for (int a = 0; a < DMAX; ++a) x[a] = (valid && a < D) ? X[(size_t)a * ld + s] : 0.0;
        for (int b = 0; b < B; ++b) {
            double best = __longlong_as_double(0x7ff0000000000000ll);
            for (int k = 0; k < K; ++k) {
                const double *l = slo + ((size_t)b * K + k) * D, *h = shi + ((size_t)b * K + k) * D;
                double acc = 0.0;
#pragma unroll
                for (int a = 0; a < DMAX; ++a) {
                    if (a < D) {
                        const double mu = mid3d(l[a], x[a], h[a]);
                        const double d = __dsub_rn(x[a], mu);
                        acc = __dadd_rn(acc, __dmul_rn(d, d));
                    }
                }
                if (acc < best) best = acc;
            }
            const double m = valid ? best : -1.0;
            const double cur = wval[w * B + b];
            const bool maybe = m >= cur && m >= 0.0;
            if (__any_sync(0xffffffffu, maybe)) {
                double v = maybe ? m : -1.0;
                uint32_t p = maybe ? (uint32_t)s : 0xFFFFFFFFu;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
                    const uint32_t p2 = __shfl_xor_sync(0xffffffffu, p, o);
                    if (v2 > v || (v2 == v && p2 < p)) { v = v2; p = p2; }
                }
                if (lane == 0 && (v > cur || (v == cur && p < wpos[w * B + b]))) {
                    wval[w * B + b] = v;
                    wpos[w * B + b] = p;
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < B; b += kThreads) {
        double v = -1.0;
        uint32_t p = 0xFFFFFFFFu;
        for (int q = 0; q < NW; ++q) {
            const double v2 = wval[q * B + b];
            const uint32_t p2 = wpos[q * B + b];
            if (v2 > v || (v2 == v && p2 < p)) { v = v2; p = p2; }
        }
        pval[(size_t)blockIdx.x * B + b] = v;
        ppos[(size_t)blockIdx.x * B + b] = p;
    }
}

// Exact refinement of float-data lower bounds: each node comes with a float
// threshold below which no sample can attain the double maximum (from the
// float pass and its error bound); samples at or above it are re-evaluated in
// double in attribute order (mid{lo,x,hi}, separate multiply and add), so the
// node's value equals a serial double evaluation over all samples.
template <int DMAX>
__global__ void __launch_bounds__(kThreads)
lb_refine_f32(const float *__restrict__ X, int64_t ld, int64_t n, const float *__restrict__ lo,
              const float *__restrict__ hi, int B, int K, int D, const float *__restrict__ thr,
              double *__restrict__ pval, uint32_t *__restrict__ ppos)
{
    constexpr int NW = kThreads / 32;
    const int Dp = (D + 1) & ~1;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *sbox = reinterpret_cast<uint64_t *>(smem);                       // [B][K][Dp] (lo, -hi)
    float *sthr = reinterpret_cast<float *>(sbox + (size_t)B * K * Dp);
    double *wval = reinterpret_cast<double *>(sthr + ((B + 1) & ~1));          // [NW][B]
    uint32_t *wpos = reinterpret_cast<uint32_t *>(wval + NW * B);
    for (int i = threadIdx.x; i < B * K * Dp; i += kThreads) {
        const int a = i % Dp, bk = i / Dp;
        sbox[i] = a < D ? pk(lo[(size_t)bk * D + a], -hi[(size_t)bk * D + a]) : pk(0.f, -0.f);
    }
    for (int i = threadIdx.x; i < B; i += kThreads) sthr[i] = thr[i];
    for (int i = threadIdx.x; i < NW * B; i += kThreads) { wval[i] = -1.0; wpos[i] = 0xFFFFFFFFu; }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t s = (int64_t)blockIdx.x * kThreads + threadIdx.x; s - threadIdx.x < n;
         s += (int64_t)gridDim.x * kThreads) {
        const bool valid = s < n;
        uint64_t px[DMAX];
#pragma unroll
        for (int a = 0; a < DMAX; ++a) {
            const float v = (valid && a < D) ? X[(size_t)a * ld + s] : 0.f;
            px[a] = pk(v, -v);
        }
        for (int b = 0; b < B; ++b) {
            float best = __int_as_float(0x7f800000);
            for (int k = 0; k < K; ++k) {
                const uint64_t *bx = sbox + ((size_t)b * K + k) * Dp;
                uint64_t acc = 0;
#pragma unroll
                for (int a = 0; a < DMAX; a += 2)
                    if (a < Dp) {
                        const float2 t0 = upk(sub2(bx[a], px[a]));
                        const float2 t1 = upk(sub2(bx[a + 1], px[a + 1]));
                        const uint64_t m = pk(max3f(t0.x, t0.y, 0.f), max3f(t1.x, t1.y, 0.f));
                        acc = fma2(m, m, acc);
                    }
                const float2 sacc = upk(acc);
                best = fminf(best, sacc.x + sacc.y);
            }
            const bool cand = valid && best >= sthr[b];
            double e = -1.0;
            if (cand) {
                e = __longlong_as_double(0x7ff0000000000000ll);
                for (int k = 0; k < K; ++k) {
                    double acc = 0.0;
#pragma unroll
                    for (int a = 0; a < DMAX; ++a)
                        if (a < D) {
                            const double x = (double)upk(px[a]).x;
                            const double l = (double)lo[((size_t)b * K + k) * D + a];
                            const double h = (double)hi[((size_t)b * K + k) * D + a];
                            const double d = __dsub_rn(x, mid3d(l, x, h));
                            acc = __dadd_rn(acc, __dmul_rn(d, d));
                        }
                    if (acc < e) e = acc;
                }
            }
            const double cur = wval[w * B + b];
            const bool maybe = cand && e >= cur;
            if (__any_sync(0xffffffffu, maybe)) {
                double v = maybe ? e : -1.0;
                uint32_t p = maybe ? (uint32_t)s : 0xFFFFFFFFu;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
                    const uint32_t p2 = __shfl_xor_sync(0xffffffffu, p, o);
                    if (v2 > v || (v2 == v && p2 < p)) { v = v2; p = p2; }
                }
                if (lane == 0 && (v > cur || (v == cur && p < wpos[w * B + b]))) {
                    wval[w * B + b] = v;
                    wpos[w * B + b] = p;
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    for (int b = threadIdx.x; b < B; b += kThreads) {
        double v = -1.0;
        uint32_t p = 0xFFFFFFFFu;
        for (int q = 0; q < NW; ++q) {
            const double v2 = wval[q * B + b];
            const uint32_t p2 = wpos[q * B + b];
            if (v2 > v || (v2 == v && p2 < p)) { v = v2; p = p2; }
        }
        pval[(size_t)blockIdx.x * B + b] = v;
        ppos[(size_t)blockIdx.x * B + b] = p;
    }
}

__global__ void lb_finalize_f32(const unsigned long long *__restrict__ part, int nparts, int B,
                                const uint32_t *__restrict__ ids, double defl, double slack,
                                double *__restrict__ lb, double *__restrict__ lb_raw,
                                int64_t *__restrict__ arg)
{
    const int b = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= B) return;
    unsigned long long m = 0ull;
    for (int p = lane; p < nparts; p += 32) {
        const unsigned long long v = part[(size_t)p * B + b];
        m = v > m ? v : m;
    }
    m = warp_max_u64(m);
    if (lane == 0) {
        const double raw = m ? (double)key_val(m) : 0.0;
        if (lb_raw) lb_raw[b] = raw;
        if (lb) lb[b] = fmax(0.0, __dsub_rd(__dmul_rd(raw, defl), slack));
        if (arg) {
            const int64_t pos = m ? (int64_t)key_pos(m) : -1;
            arg[b] = (pos < 0 || !ids) ? pos : (int64_t)ids[pos];
        }
    }
}

__global__ void lb_finalize_f64(const double *__restrict__ pval, const uint32_t *__restrict__ ppos,
                                int nparts, int B, const uint32_t *__restrict__ ids, double defl,
                                double slack, double *__restrict__ lb, double *__restrict__ lb_raw,
                                int64_t *__restrict__ arg)
{
    const int b = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (b >= B) return;
    double v = -1.0;
    uint32_t p = 0xFFFFFFFFu;
    for (int q = lane; q < nparts; q += 32) {
        const double v2 = pval[(size_t)q * B + b];
        const uint32_t p2 = ppos[(size_t)q * B + b];
        if (v2 > v || (v2 == v && p2 < p)) { v = v2; p = p2; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
        const uint32_t p2 = __shfl_xor_sync(0xffffffffu, p, o);
        if (v2 > v || (v2 == v && p2 < p)) { v = v2; p = p2; }
    }
    if (lane == 0) {
        const bool none = v < 0.0;
        const double raw = none ? 0.0 : v;
        if (lb_raw) lb_raw[b] = raw;
        if (lb) lb[b] = fmax(0.0, __dsub_rd(__dmul_rd(raw, defl), slack));
        if (arg) arg[b] = none ? -1 : (ids ? (int64_t)ids[p] : (int64_t)p);
    }
}

// ---------------------------------------------------------------- dispatch

using FastFn = void (*)(const float *, int64_t, int64_t, const float *, const float *, int,
                        unsigned long long *);

struct FastEntry {
    int D, K, ST;
    FastFn fn;
};

// Shapes of the measured workloads get compile-time kernels; others use the
// generic ones.
const FastEntry kFast[] = {
    {2, 3, 4, lb_f32_fast<2, 3, 4>}, {2, 3, 2, lb_f32_fast<2, 3, 2>},
    {2, 4, 4, lb_f32_fast<2, 4, 4>}, {2, 4, 2, lb_f32_fast<2, 4, 2>},
    {3, 3, 4, lb_f32_fast<3, 3, 4>}, {3, 3, 2, lb_f32_fast<3, 3, 2>},
    {4, 3, 4, lb_f32_fast<4, 3, 4>}, {4, 3, 2, lb_f32_fast<4, 3, 2>},
    {8, 5, 4, lb_f32_fast<8, 5, 4>}, {8, 5, 2, lb_f32_fast<8, 5, 2>},
};

template <typename F>
kc_status prep_kernel(kc_ctx *c, F fn, size_t smem, int *grid, int64_t tiles)
{
    if (smem > 48 * 1024)
        KC_CUDA(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    KC_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem));
    if (per_sm < 1) return set_err(c, KC_EINTERNAL, "lower-bound kernel does not fit (smem %zu)", smem);
    int64_t g = (int64_t)per_sm * c->num_sms;
    if (g > tiles) g = tiles;
    *grid = (int)(g < 1 ? 1 : g);
    return KC_OK;
}

}  // namespace

kc_status launch_lower_bounds_view(kc_ctx *c, const View &v, const void *lo, const void *hi, int B,
                                   double *lb, double *lb_raw, int64_t *arg, int st_override)
{
    return launch_lower_bounds_cfg(c, v, lo, hi, B, lb, lb_raw, arg, st_override, 0);
}

kc_status launch_lower_bounds_cfg(kc_ctx *c, const View &v, const void *lo, const void *hi, int B, double *lb,
                                  double *lb_raw, int64_t *arg, int st_override, int chunk_override)
{
    if (B <= 0) return KC_OK;
    const int D = c->D, K = c->K;
    const double defl = deflate_factor(c->dt, D), slack = underflow_slack(c->dt, D);
    const size_t smem_cap = c->smem_optin > 0 ? c->smem_optin : 48 * 1024;
    const int NW = kThreads / 32;
    if (c->dt == KC_F32) {
        const FastFn *fast = nullptr;
        int st = st_override > 0 ? st_override : (c->lb_st > 0 ? c->lb_st : 4);
        for (const auto &e : kFast)
            if (e.D == D && e.K == K && e.ST == st) fast = &e.fn;
        const int Dp = fast ? D : ((D + 1) & ~1);
        const size_t per_node = (size_t)K * Dp * 8 + NW * 8;
        // chunk the node batch so two CTAs fit per SM where possible
        int chunk = (int)std::min<size_t>((size_t)B, (smem_cap / 2 > per_node ? (smem_cap / 2) / per_node : 1));
        const int chunk_pref = chunk_override > 0 ? chunk_override : c->lb_chunk;
        if (chunk_pref > 0 && chunk_pref < chunk) chunk = chunk_pref;
        if (chunk < 1) chunk = 1;
        for (int b0 = 0; b0 < B; b0 += chunk) {
            const int nb = std::min(chunk, B - b0);
            const size_t smem = per_node * nb;
            const float *l = static_cast<const float *>(lo) + (size_t)b0 * K * D;
            const float *h = static_cast<const float *>(hi) + (size_t)b0 * K * D;
            int grid = 1;
            if (fast) {
                const int64_t tiles = (v.n + (int64_t)kThreads * st - 1) / ((int64_t)kThreads * st);
                KC_TRY(prep_kernel(c, *fast, smem, &grid, tiles));
                KC_TRY(ensure(c, c->part, (size_t)grid * nb * 8));
                if (v.n > 0)
                    (*fast)<<<grid, kThreads, smem, c->stream>>>(
                        static_cast<const float *>(v.X), v.ld, v.n, l, h, nb,
                        static_cast<unsigned long long *>(c->part.p));
            } else {
                const int64_t tiles = (v.n + kThreads - 1) / kThreads;
                auto g = D <= 16 ? lb_f32_generic<16> : (D <= 64 ? lb_f32_generic<64> : lb_f32_generic<128>);
                KC_TRY(prep_kernel(c, g, smem, &grid, tiles));
                KC_TRY(ensure(c, c->part, (size_t)grid * nb * 8));
                if (v.n > 0)
                    g<<<grid, kThreads, smem, c->stream>>>(static_cast<const float *>(v.X), v.ld, v.n, l, h, nb, K, D,
                                                           static_cast<unsigned long long *>(c->part.p));
            }
            if (v.n > 0) KC_TRY(after_launch(c, "lower bound"));
            const int nparts = v.n > 0 ? grid : 0;
            lb_finalize_f32<<<(nb + 3) / 4, 128, 0, c->stream>>>(
                static_cast<const unsigned long long *>(c->part.p), nparts, nb, v.ids, defl, slack,
                lb ? lb + b0 : nullptr, lb_raw ? lb_raw + b0 : nullptr, arg ? arg + b0 : nullptr);
            KC_TRY(after_launch(c, "lower bound finalize"));
        }
    } else {
        const size_t per_node = (size_t)K * D * 16 + NW * 12;
        int chunk = (int)std::min<size_t>((size_t)B, (smem_cap / 2 > per_node ? (smem_cap / 2) / per_node : 1));
        if (chunk < 1) chunk = 1;
        for (int b0 = 0; b0 < B; b0 += chunk) {
            const int nb = std::min(chunk, B - b0);
            const size_t smem = per_node * nb;
            const double *l = static_cast<const double *>(lo) + (size_t)b0 * K * D;
            const double *h = static_cast<const double *>(hi) + (size_t)b0 * K * D;
            const int64_t tiles = (v.n + kThreads - 1) / kThreads;
            int grid = 1;
            auto g = D <= 16 ? lb_f64<16> : (D <= 64 ? lb_f64<64> : lb_f64<128>);
            KC_TRY(prep_kernel(c, g, smem, &grid, tiles));
            KC_TRY(ensure(c, c->part, (size_t)grid * nb * 12));
            double *pval = static_cast<double *>(c->part.p);
            uint32_t *ppos = reinterpret_cast<uint32_t *>(pval + (size_t)grid * nb);
            if (v.n > 0) {
                g<<<grid, kThreads, smem, c->stream>>>(static_cast<const double *>(v.X), v.ld, v.n, l, h, nb, K, D, pval,
                                                       ppos);
                KC_TRY(after_launch(c, "lower bound f64"));
            }
            lb_finalize_f64<<<(nb + 3) / 4, 128, 0, c->stream>>>(
                pval, ppos, v.n > 0 ? grid : 0, nb, v.ids, defl, slack, lb ? lb + b0 : nullptr,
                lb_raw ? lb_raw + b0 : nullptr, arg ? arg + b0 : nullptr);
            KC_TRY(after_launch(c, "lower bound finalize f64"));
        }
    }
    return KC_OK;
}

kc_status launch_lower_bounds(kc_ctx *c, const void *lo, const void *hi, int B, double *lb,
                              double *lb_raw, int64_t *argmax)
{
    return launch_lower_bounds_view(c, full_view(c), lo, hi, B, lb, lb_raw, argmax, 0);
}

// Double-precision refinement of float-data lower bounds (see lb_refine_f32):
// raw[b] is the float pass's value of node b; lb_out gets the certified bound
// from the serial double value, lb_exact_out (nullable) that double value.
kc_status launch_lower_bounds_refine(kc_ctx *c, const View &v, const void *lo, const void *hi, int B,
                                     const double *raw_host, double *lb_out, double *lb_exact_out, int64_t *arg)
{
    if (B <= 0) return KC_OK;
    if (c->dt != KC_F32) return set_err(c, KC_EINTERNAL, "refinement is for float data");
    const int D = c->D, K = c->K, NW = kThreads / 32, Dp = (D + 1) & ~1;
    const double gam = gamma_n(f32_roundings(D), kU32) + 2 * gamma_n(f64_roundings(D), kU64) + 1e-15;
    std::vector<float> thr(B);
    for (int b = 0; b < B; ++b) {
        double t = raw_host[b] / (1.0 + gam) * (1.0 - gam) * (1.0 - 1e-6) - 1e-37;
        float f = (float)t;
        if ((double)f > t) f = nextafterf(f, -1.f);
        thr[b] = t > 0 ? f : -1.f;
    }
    const size_t smem_cap = c->smem_optin > 0 ? c->smem_optin : 48 * 1024;
    const size_t per_node = (size_t)K * Dp * 8 + 4 + (size_t)NW * 12;
    const int chunk = (int)std::max<size_t>(1, std::min<size_t>((size_t)B, (smem_cap / 2) / per_node));
    const double defl = deflate_factor(KC_F64, D), slack = underflow_slack(KC_F64, D);
    for (int b0 = 0; b0 < B; b0 += chunk) {
        const int nb = std::min(chunk, B - b0);
        const size_t smem = (size_t)K * Dp * 8 * nb + (size_t)((nb + 1) & ~1) * 4 + (size_t)NW * 12 * nb;
        const int64_t tiles = (v.n + kThreads - 1) / kThreads;
        int grid = 1;
        auto kern = D <= 16 ? lb_refine_f32<16> : (D <= 64 ? lb_refine_f32<64> : lb_refine_f32<128>);
        KC_TRY(prep_kernel(c, kern, smem, &grid, tiles));
        const size_t thr_off = 0, part_off = 256 + (size_t)nb * 4;
        KC_TRY(ensure(c, c->part, part_off + (size_t)grid * nb * 12 + 256));
        char *pbuf = static_cast<char *>(c->part.p);
        float *dthr = reinterpret_cast<float *>(pbuf + thr_off);
        double *pval = reinterpret_cast<double *>(pbuf + ((part_off + 15) & ~(size_t)15));
        uint32_t *ppos = reinterpret_cast<uint32_t *>(pval + (size_t)grid * nb);
        KC_CUDA(c, cudaMemcpyAsync(dthr, thr.data() + b0, (size_t)nb * 4, cudaMemcpyHostToDevice, c->stream));
        const float *l = static_cast<const float *>(lo) + (size_t)b0 * K * D;
        const float *h = static_cast<const float *>(hi) + (size_t)b0 * K * D;
        if (v.n > 0) {
            kern<<<grid, kThreads, smem, c->stream>>>(static_cast<const float *>(v.X), v.ld, v.n, l, h, nb, K, D, dthr,
                                                      pval, ppos);
            KC_TRY(after_launch(c, "lower bound refinement"));
        }
        lb_finalize_f64<<<(nb + 3) / 4, 128, 0, c->stream>>>(pval, ppos, v.n > 0 ? grid : 0, nb, v.ids, defl, slack,
                                                             lb_out + b0, lb_exact_out ? lb_exact_out + b0 : nullptr,
                                                             arg ? arg + b0 : nullptr);
        KC_TRY(after_launch(c, "lower bound refinement finalize"));
        if (b0 + chunk < B) KC_CUDA(c, cudaStreamSynchronize(c->stream));   // thr upload reuses the buffer
    }
    return KC_OK;
}

// Times the float lower-bound kernel's launch shapes on the given node batch
// (samples per thread x node chunk: occupancy against extra sample passes)
// and keeps the fastest in the context.  Untimed work for the caller.
kc_status autotune_lower_bounds(kc_ctx *c, const void *lo, const void *hi, int B, double *lb_scratch, int *st_out,
                                int *chunk_out, float *ms_out)
{
    *st_out = 0;
    *chunk_out = 0;
    if (c->dt != KC_F32 || B <= 0) return KC_OK;
    const View v = full_view(c);
    const int chunks[4] = {B, (B + 1) / 2, (B + 2) / 3, (B + 3) / 4};
    const int sts[2] = {4, 2};
    cudaEvent_t e0, e1;
    KC_CUDA(c, cudaEventCreate(&e0));
    KC_CUDA(c, cudaEventCreate(&e1));
    float best = 3.4e38f;
    int bst = 4, bch = 0;
    kc_status st = KC_OK;
    for (int si = 0; si < 2 && st == KC_OK; ++si)
        for (int ci = 0; ci < 4 && st == KC_OK; ++ci) {
            const int ch = chunks[ci];
            if (ci > 0 && ch == chunks[ci - 1]) continue;
            st = launch_lower_bounds_cfg(c, v, lo, hi, B, lb_scratch, nullptr, nullptr, sts[si], ch);
            if (st != KC_OK) break;
            cudaEventRecord(e0, c->stream);
            for (int r = 0; r < 3 && st == KC_OK; ++r)
                st = launch_lower_bounds_cfg(c, v, lo, hi, B, lb_scratch, nullptr, nullptr, sts[si], ch);
            cudaEventRecord(e1, c->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) { st = set_err(c, KC_ECUDA, "autotune: event sync failed"); break; }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            ms /= 3.f;
            if (ms < best) { best = ms; bst = sts[si]; bch = ch; }
        }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != KC_OK) return st;
    c->lb_st = bst;
    c->lb_chunk = bch;
    *st_out = bst;
    *chunk_out = bch;
    *ms_out = best;
    return KC_OK;
}

}  // namespace kc

// ------------------------------------------------------------------------
// kc_lower_bounds_noalloc: the float lower-bound kernel with its per-CTA
// partial results in a fixed device array instead of a context's buffers.
// Nothing here allocates; see include/kc.h for who needs this.

namespace kc {
namespace {

constexpr int kNoAllocMaxCtas = 512;      // partial slots per node
constexpr int kNoAllocChunk = 256;        // nodes per launch
constexpr int kNoAllocMaxNodes = 4096;    // nodes per call
constexpr int kNoAllocMaxDevices = 64;

// One CTA's best key per node of the current chunk: 512 x 256 x 8 bytes = 1 MiB,
// held by every GPU that loads the library until the process exits.
static __device__ __align__(256) unsigned long long g_noalloc_partials[kNoAllocMaxCtas * kNoAllocChunk];

std::atomic<void *> g_noalloc_ptr[kNoAllocMaxDevices];

}  // namespace
}  // namespace kc

extern "C" kc_status kc_lower_bounds_noalloc(const float *X, int64_t N, int64_t ld, int32_t D, int32_t K,
                                             const float *lo, const float *hi, int32_t B, double *lb_out,
                                             double *lb_raw_out, int64_t *argmax_out, void *stream)
{
    using namespace kc;
    if (!X || !lo || !hi || !lb_out) return KC_EINVAL;
    if (K < 1 || K > kMaxK || D < 1 || D > kMaxD || N < 0 || ld < N || N > 4294967294ll) return KC_EINVAL;
    if (B < 0 || B > kNoAllocMaxNodes) return KC_EINVAL;   // more nodes than the fixed scratch is sized for
    if (B == 0) return KC_OK;
    // An error already pending in this thread belongs to earlier work: report
    // it without clearing it (cudaPeekAtLastError) and launch nothing.
    if (cudaPeekAtLastError() != cudaSuccess) return KC_ECUDA;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) return KC_ECUDA;
    // Every array must be device memory of the current GPU: a host array
    // would make the kernels read or write through a host address.
    // cudaPointerGetAttributes allocates nothing.
    {
        const void *args[6] = {X, lo, hi, lb_out, lb_raw_out, argmax_out};
        for (const void *p : args) {
            if (!p) continue;
            cudaPointerAttributes a;
            if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
                cudaGetLastError();   // the error this query just raised
                return KC_EINVAL;
            }
            if ((a.type != cudaMemoryTypeDevice && a.type != cudaMemoryTypeManaged) || a.device != dev)
                return KC_EINVAL;
        }
    }
    // The host-side name of a __device__ array is not a device address: look
    // the address up once per device, with that device current.
    void *scratch = g_noalloc_ptr[dev].load();
    if (!scratch) {
        if (cudaGetSymbolAddress(&scratch, g_noalloc_partials) != cudaSuccess || !scratch) return KC_ECUDA;
        g_noalloc_ptr[dev].store(scratch);
    }
    int sms = 0, optin = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
        return KC_ECUDA;
    const int NW = kThreads / 32;
    const double defl = deflate_factor(KC_F32, D), slack = underflow_slack(KC_F32, D);
    const bool aligned = ((uintptr_t)X % 16 == 0) && (ld % 4 == 0);
    FastFn fast = nullptr;
    for (const auto &e : kFast)
        if (aligned && e.D == D && e.K == K && e.ST == 4) fast = e.fn;
    const int Dp = fast ? D : ((D + 1) & ~1);
    const size_t per_node = (size_t)K * Dp * 8 + NW * 8;
    int chunk = (int)std::min<size_t>(kNoAllocChunk, (size_t)optin / per_node);
    if (chunk < 1) return KC_EINVAL;
    unsigned long long *part = static_cast<unsigned long long *>(scratch);
    for (int b0 = 0; b0 < B; b0 += chunk) {
        const int nb = std::min(chunk, B - b0);
        const size_t smem = per_node * nb;
        const float *l = lo + (size_t)b0 * K * D, *h = hi + (size_t)b0 * K * D;
        int per_sm = 0, grid = 1;
        if (fast) {
            if (smem > 48 * 1024 &&
                cudaFuncSetAttribute(fast, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                return KC_ECUDA;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fast, kThreads, smem) != cudaSuccess)
                return KC_ECUDA;
        } else {
            auto g = D <= 16 ? lb_f32_generic<16> : (D <= 64 ? lb_f32_generic<64> : lb_f32_generic<128>);
            if (smem > 48 * 1024 &&
                cudaFuncSetAttribute(g, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
                return KC_ECUDA;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, g, kThreads, smem) != cudaSuccess)
                return KC_ECUDA;
        }
        if (per_sm < 1) return KC_EINVAL;
        const int64_t tile = (int64_t)kThreads * (fast ? 4 : 1);
        const int64_t tiles = (N + tile - 1) / tile;
        grid = (int)std::max<int64_t>(1, std::min<int64_t>({(int64_t)per_sm * sms, tiles, (int64_t)kNoAllocMaxCtas}));
        if (N > 0) {
            if (fast)
                fast<<<grid, kThreads, smem, st>>>(X, ld, N, l, h, nb, part);
            else
                (D <= 16 ? lb_f32_generic<16> : (D <= 64 ? lb_f32_generic<64> : lb_f32_generic<128>))
                    <<<grid, kThreads, smem, st>>>(X, ld, N, l, h, nb, K, D, part);
            if (cudaGetLastError() != cudaSuccess) return KC_ECUDA;
        }
        lb_finalize_f32<<<(nb + 3) / 4, 128, 0, st>>>(part, N > 0 ? grid : 0, nb, nullptr, defl, slack, lb_out + b0,
                                                      lb_raw_out ? lb_raw_out + b0 : nullptr,
                                                      argmax_out ? argmax_out + b0 : nullptr);
        if (cudaGetLastError() != cudaSuccess) return KC_ECUDA;
    }
    return KC_OK;
}
