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
                if (D <= 16) {
                    KC_TRY(prep_kernel(c, lb_f32_generic<16>, smem, &grid, tiles));
                    KC_TRY(ensure(c, c->part, (size_t)grid * nb * 8));
                    if (v.n > 0)
                        lb_f32_generic<16><<<grid, kThreads, smem, c->stream>>>(
                            static_cast<const float *>(v.X), v.ld, v.n, l, h, nb, K, D,
                            static_cast<unsigned long long *>(c->part.p));
                } else {
                    KC_TRY(prep_kernel(c, lb_f32_generic<64>, smem, &grid, tiles));
                    KC_TRY(ensure(c, c->part, (size_t)grid * nb * 8));
                    if (v.n > 0)
                        lb_f32_generic<64><<<grid, kThreads, smem, c->stream>>>(
                            static_cast<const float *>(v.X), v.ld, v.n, l, h, nb, K, D,
                            static_cast<unsigned long long *>(c->part.p));
                }
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
            if (D <= 16) {
                KC_TRY(prep_kernel(c, lb_f64<16>, smem, &grid, tiles));
            } else {
                KC_TRY(prep_kernel(c, lb_f64<64>, smem, &grid, tiles));
            }
            KC_TRY(ensure(c, c->part, (size_t)grid * nb * 12));
            double *pval = static_cast<double *>(c->part.p);
            uint32_t *ppos = reinterpret_cast<uint32_t *>(pval + (size_t)grid * nb);
            if (v.n > 0) {
                if (D <= 16)
                    lb_f64<16><<<grid, kThreads, smem, c->stream>>>(static_cast<const double *>(v.X), v.ld,
                                                                    v.n, l, h, nb, K, D, pval, ppos);
                else
                    lb_f64<64><<<grid, kThreads, smem, c->stream>>>(static_cast<const double *>(v.X), v.ld,
                                                                    v.n, l, h, nb, K, D, pval, ppos);
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

}  // namespace kc
