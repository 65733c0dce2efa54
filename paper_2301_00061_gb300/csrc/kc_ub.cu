// kc_ub.cu -- objective of Eq. 1 at center sets on samples: the upper bound
// alpha(M) of Eq. 12, the farthest-point queries of Algorithm 2, and the final
// double-precision certificate.
//
// Float data take two streaming passes.  The screen pass evaluates every
// sample against S center sets in float (packed f32x2 subtract / fused
// multiply-add) and keeps each set's maximum.  Every float value lies within
// a relative Gamma of the double value, so only samples whose float value
// reaches max * (1 - Gamma) / (1 + Gamma) can attain the double maximum; the
// exact pass re-evaluates just those in double, in attribute order without
// contraction (bit-identical to a serial double evaluation), and reduces
// (value, position) with the smallest position on ties.  Double data take
// the exact pass over every sample.
#include <cuda_runtime.h>

#include "kc_device.cuh"
#include "kc_internal.cuh"

namespace kc {

namespace {

// Center coordinates of S*Kc centers as packed float pairs [S*Kc][Dh].
__global__ void gather_pairs_f32(const float *__restrict__ X, int64_t ld, int D, int Dh,
                                 const int64_t *__restrict__ centers, int SK, uint64_t *__restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < SK * Dh; i += gridDim.x * blockDim.x) {
        const int sk = i / Dh, p = i % Dh;
        const int64_t c = centers[sk];
        const int a0 = 2 * p, a1 = 2 * p + 1;
        const float x0 = X[(size_t)a0 * ld + c];
        const float x1 = a1 < D ? X[(size_t)a1 * ld + c] : 0.f;
        out[i] = pk(x0, x1);
    }
}

// Center coordinates given as points [S*Kc][D] -> packed float pairs [S*Kc][Dh].
__global__ void pack_pairs_f32(const float *__restrict__ pts, int D, int Dh, int SK, uint64_t *__restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < SK * Dh; i += gridDim.x * blockDim.x) {
        const int sk = i / Dh, p = i % Dh;
        const int a0 = 2 * p, a1 = 2 * p + 1;
        out[i] = pk(pts[(size_t)sk * D + a0], a1 < D ? pts[(size_t)sk * D + a1] : 0.f);
    }
}

// Float screen: per set, the maximum over samples of min_k ||x - c_k||^2.
template <int DH>
__global__ void __launch_bounds__(kThreads)
obj_screen_f32(const float *__restrict__ X, int64_t ld, int64_t n, int D, const uint64_t *__restrict__ gsets,
               int S, int Kc, int Dh, unsigned long long *__restrict__ part)
{
    constexpr int NW = kThreads / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *sset = reinterpret_cast<uint64_t *>(smem);
    unsigned long long *wbest = reinterpret_cast<unsigned long long *>(sset + (size_t)S * Kc * Dh);
    for (int i = threadIdx.x; i < S * Kc * Dh; i += kThreads) sset[i] = gsets[i];
    for (int i = threadIdx.x; i < NW * S; i += kThreads) wbest[i] = 0ull;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    unsigned long long *mine = wbest + (threadIdx.x >> 5) * S;
    for (int64_t s = (int64_t)blockIdx.x * kThreads + threadIdx.x; s - threadIdx.x < n;
         s += (int64_t)gridDim.x * kThreads) {
        const bool valid = s < n;
        uint64_t px[DH];
#pragma unroll
        for (int p = 0; p < DH; ++p) {
            const int a0 = 2 * p, a1 = 2 * p + 1;
            const float x0 = (valid && a0 < D) ? X[(size_t)a0 * ld + s] : 0.f;
            const float x1 = (valid && a1 < D) ? X[(size_t)a1 * ld + s] : 0.f;
            px[p] = pk(x0, x1);
        }
        for (int q = 0; q < S; ++q) {
            float best = __int_as_float(0x7f800000);
            for (int k = 0; k < Kc; ++k) {
                const uint64_t *cx = sset + ((size_t)q * Kc + k) * Dh;
                uint64_t acc = 0;
#pragma unroll
                for (int p = 0; p < DH; ++p)
                    if (p < Dh) {
                        const uint64_t t = sub2(px[p], cx[p]);
                        acc = fma2(t, t, acc);
                    }
                const float2 r = upk(acc);
                best = fminf(best, r.x + r.y);
            }
            const float m = valid ? best : -1.f;
            const unsigned long long cur = mine[q];
            const bool maybe = m >= key_val(cur);
            if (__any_sync(0xffffffffu, maybe)) {
                unsigned long long key = maybe ? key_max(m, (uint32_t)s) : 0ull;
                key = warp_max_u64(key);
                if (lane == 0 && key > cur) mine[q] = key;
                __syncwarp();
            }
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < S; q += kThreads) {
        unsigned long long m = 0ull;
        for (int w = 0; w < NW; ++w) {
            const unsigned long long v = wbest[w * S + q];
            m = v > m ? v : m;
        }
        part[(size_t)blockIdx.x * S + q] = m;
    }
}

// Per set: threshold for the exact pass from the screen maximum, or +inf when
// the screen already proves the value is >= alpha_cut (the set is skipped).
__global__ void obj_threshold(const unsigned long long *__restrict__ part, int nparts, int S, double gam,
                              double alpha_cut, float *__restrict__ thr, double *__restrict__ val)
{
    const int q = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (q >= S) return;
    unsigned long long m = 0ull;
    for (int p = lane; p < nparts; p += 32) {
        const unsigned long long v = part[(size_t)p * S + q];
        m = v > m ? v : m;
    }
    m = warp_max_u64(m);
    if (lane == 0) {
        const double raw = m ? (double)key_val(m) : 0.0;
        const double low = __ddiv_rd(raw, 1.0 + gam);   // <= the exact maximum
        if (low >= alpha_cut) {
            thr[q] = __int_as_float(0x7f800000);
            val[q] = __longlong_as_double(0x7ff0000000000000ll);
        } else {
            double t = __dmul_rd(__dmul_rd(low, 1.0 - gam), 1.0 - 1e-6) - 1e-37;
            thr[q] = t > 0.0 ? __double2float_rd(t) : -1.0f;
        }
    }
}

// Exact pass over float data: candidates (float value >= thr) in double.
template <int DH>
__global__ void __launch_bounds__(kThreads)
obj_exact_f32(const float *__restrict__ X, int64_t ld, int64_t n, int D, const uint64_t *__restrict__ gsets,
              int S, int Kc, int Dh, const float *__restrict__ thr, double *__restrict__ pval,
              uint32_t *__restrict__ ppos)
{
    constexpr int NW = kThreads / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *sset = reinterpret_cast<uint64_t *>(smem);
    float *sthr = reinterpret_cast<float *>(sset + (size_t)S * Kc * Dh);
    double *wval = reinterpret_cast<double *>(sthr + ((S + 1) & ~1));
    uint32_t *wpos = reinterpret_cast<uint32_t *>(wval + NW * S);
    for (int i = threadIdx.x; i < S * Kc * Dh; i += kThreads) sset[i] = gsets[i];
    for (int i = threadIdx.x; i < S; i += kThreads) sthr[i] = thr[i];
    for (int i = threadIdx.x; i < NW * S; i += kThreads) { wval[i] = -1.0; wpos[i] = 0xFFFFFFFFu; }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t s = (int64_t)blockIdx.x * kThreads + threadIdx.x; s - threadIdx.x < n;
         s += (int64_t)gridDim.x * kThreads) {
        const bool valid = s < n;
        uint64_t px[DH];
#pragma unroll
        for (int p = 0; p < DH; ++p) {
            const int a0 = 2 * p, a1 = 2 * p + 1;
            const float x0 = (valid && a0 < D) ? X[(size_t)a0 * ld + s] : 0.f;
            const float x1 = (valid && a1 < D) ? X[(size_t)a1 * ld + s] : 0.f;
            px[p] = pk(x0, x1);
        }
        for (int q = 0; q < S; ++q) {
            const float tq = sthr[q];
            if (tq == __int_as_float(0x7f800000)) continue;   // uniform across the block
            float best = __int_as_float(0x7f800000);
            for (int k = 0; k < Kc; ++k) {
                const uint64_t *cx = sset + ((size_t)q * Kc + k) * Dh;
                uint64_t acc = 0;
#pragma unroll
                for (int p = 0; p < DH; ++p)
                    if (p < Dh) {
                        const uint64_t t = sub2(px[p], cx[p]);
                        acc = fma2(t, t, acc);
                    }
                const float2 r = upk(acc);
                best = fminf(best, r.x + r.y);
            }
            const bool cand = valid && best >= tq;
            double e = -1.0;
            if (cand) {
                e = __longlong_as_double(0x7ff0000000000000ll);
                for (int k = 0; k < Kc; ++k) {
                    const uint64_t *cx = sset + ((size_t)q * Kc + k) * Dh;
                    double acc = 0.0;
#pragma unroll
                    for (int p = 0; p < DH; ++p) {
                        if (p < Dh) {
                            const float2 xv = upk(px[p]), cv = upk(cx[p]);
                            double d = __dsub_rn((double)xv.x, (double)cv.x);
                            acc = __dadd_rn(acc, __dmul_rn(d, d));
                            if (2 * p + 1 < D) {
                                d = __dsub_rn((double)xv.y, (double)cv.y);
                                acc = __dadd_rn(acc, __dmul_rn(d, d));
                            }
                        }
                    }
                    if (acc < e) e = acc;
                }
            }
            const double cur = wval[w * S + q];
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
                if (lane == 0 && (v > cur || (v == cur && p < wpos[w * S + q]))) {
                    wval[w * S + q] = v;
                    wpos[w * S + q] = p;
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < S; q += kThreads) {
        double v = -1.0;
        uint32_t p = 0xFFFFFFFFu;
        for (int r = 0; r < NW; ++r) {
            const double v2 = wval[r * S + q];
            const uint32_t p2 = wpos[r * S + q];
            if (v2 > v || (v2 == v && p2 < p)) { v = v2; p = p2; }
        }
        pval[(size_t)blockIdx.x * S + q] = v;
        ppos[(size_t)blockIdx.x * S + q] = p;
    }
}

// Exact pass over double data (every sample).  Centers are read from the
// full dataset by index.
template <int DMAX>
__global__ void __launch_bounds__(kThreads)
obj_exact_f64(const double *__restrict__ X, int64_t ld, int64_t n, int D, const double *__restrict__ Xfull,
              int64_t ldf, const int64_t *__restrict__ centers, const double *__restrict__ pts, int S, int Kc,
              double *__restrict__ pval, uint32_t *__restrict__ ppos)
{
    // centers by sample index from Xfull, or (pts != NULL) as points [S*Kc][D]
    constexpr int NW = kThreads / 32;
    extern __shared__ __align__(16) unsigned char smem[];
    double *sc = reinterpret_cast<double *>(smem);                 // [S][Kc][D]
    double *wval = sc + (size_t)S * Kc * D;
    uint32_t *wpos = reinterpret_cast<uint32_t *>(wval + NW * S);
    for (int i = threadIdx.x; i < S * Kc * D; i += kThreads) {
        const int a = i % D, sk = i / D;
        sc[i] = pts ? pts[(size_t)sk * D + a] : Xfull[(size_t)a * ldf + centers[sk]];
    }
    for (int i = threadIdx.x; i < NW * S; i += kThreads) { wval[i] = -1.0; wpos[i] = 0xFFFFFFFFu; }
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int64_t s = (int64_t)blockIdx.x * kThreads + threadIdx.x; s - threadIdx.x < n;
         s += (int64_t)gridDim.x * kThreads) {
        const bool valid = s < n;
        double x[DMAX];
#pragma unroll
        for (int a = 0; a < DMAX; ++a) x[a] = (valid && a < D) ? X[(size_t)a * ld + s] : 0.0;
        for (int q = 0; q < S; ++q) {
            double e = __longlong_as_double(0x7ff0000000000000ll);
            for (int k = 0; k < Kc; ++k) {
                const double *c = sc + ((size_t)q * Kc + k) * D;
                double acc = 0.0;
#pragma unroll
                for (int a = 0; a < DMAX; ++a)
                    if (a < D) {
                        const double d = __dsub_rn(x[a], c[a]);
                        acc = __dadd_rn(acc, __dmul_rn(d, d));
                    }
                if (acc < e) e = acc;
            }
            const double m = valid ? e : -1.0;
            const double cur = wval[w * S + q];
            const bool maybe = valid && m >= cur;
            if (__any_sync(0xffffffffu, maybe)) {
                double v = maybe ? m : -1.0;
                uint32_t p = maybe ? (uint32_t)s : 0xFFFFFFFFu;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const double v2 = __shfl_xor_sync(0xffffffffu, v, o);
                    const uint32_t p2 = __shfl_xor_sync(0xffffffffu, p, o);
                    if (v2 > v || (v2 == v && p2 < p)) { v = v2; p = p2; }
                }
                if (lane == 0 && (v > cur || (v == cur && p < wpos[w * S + q]))) {
                    wval[w * S + q] = v;
                    wpos[w * S + q] = p;
                }
                __syncwarp();
            }
        }
    }
    __syncthreads();
    for (int q = threadIdx.x; q < S; q += kThreads) {
        double v = -1.0;
        uint32_t p = 0xFFFFFFFFu;
        for (int r = 0; r < NW; ++r) {
            const double v2 = wval[r * S + q];
            const uint32_t p2 = wpos[r * S + q];
            if (v2 > v || (v2 == v && p2 < p)) { v = v2; p = p2; }
        }
        pval[(size_t)blockIdx.x * S + q] = v;
        ppos[(size_t)blockIdx.x * S + q] = p;
    }
}

// (value, position) partials -> value and sample index per set.  Sets marked
// skipped (thr = +inf) keep val = +inf and arg = -1.
__global__ void obj_finalize(const double *__restrict__ pval, const uint32_t *__restrict__ ppos, int nparts,
                             int S, const uint32_t *__restrict__ ids, const float *__restrict__ thr,
                             double *__restrict__ val, int64_t *__restrict__ arg)
{
    const int q = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (q >= S) return;
    if (thr && thr[q] == __int_as_float(0x7f800000)) {
        if (lane == 0 && arg) arg[q] = -1;
        return;
    }
    double v = -1.0;
    uint32_t p = 0xFFFFFFFFu;
    for (int r = lane; r < nparts; r += 32) {
        const double v2 = pval[(size_t)r * S + q];
        const uint32_t p2 = ppos[(size_t)r * S + q];
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
        val[q] = none ? 0.0 : v;
        if (arg) arg[q] = none ? -1 : (ids ? (int64_t)ids[p] : (int64_t)p);
    }
}

template <typename F>
kc_status grid_for(kc_ctx *c, F fn, size_t smem, int64_t n, int *grid)
{
    if (smem > 48 * 1024)
        KC_CUDA(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    KC_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem));
    if (per_sm < 1) return set_err(c, KC_EINTERNAL, "objective kernel does not fit (smem %zu)", smem);
    int64_t g = (int64_t)per_sm * c->num_sms;
    const int64_t tiles = (n + kThreads - 1) / kThreads;
    if (g > tiles) g = tiles;
    *grid = (int)(g < 1 ? 1 : g);
    return KC_OK;
}

// The float-screen error bound Gamma between a float-evaluated distance and
// its double evaluation (both relative to the exact value).
double screen_gamma(int D)
{
    return gamma_n(f32_roundings(D), kU32) + 2 * gamma_n(f64_roundings(D), kU64) + 1e-15;
}

kc_status objective_chunk(kc_ctx *c, const View &v, const int64_t *centers, int S, int Kc,
                          double alpha_cut, double *val, int64_t *arg, const void *pts)
{
    const int D = c->D;
    const int NW = kThreads / 32;
    if (c->dt == KC_F32) {
        const int Dh = (D + 1) / 2;
        const size_t sets_bytes = (size_t)S * Kc * Dh * 8;
        // work layout: [pairs][thr][keys/partials]
        const size_t off_thr = (sets_bytes + 255) & ~(size_t)255;
        const size_t off_part = (off_thr + (size_t)S * 4 + 255) & ~(size_t)255;
        const size_t smem1 = sets_bytes + (size_t)NW * S * 8;
        const size_t smem2 = sets_bytes + (size_t)((S + 1) & ~1) * 4 + (size_t)NW * S * 12;
        int g1 = 1, g2 = 1;
        auto k1 = Dh <= 4 ? obj_screen_f32<4>
                          : (Dh <= 8 ? obj_screen_f32<8> : (Dh <= 32 ? obj_screen_f32<32> : obj_screen_f32<64>));
        auto k2 = Dh <= 4 ? obj_exact_f32<4>
                          : (Dh <= 8 ? obj_exact_f32<8> : (Dh <= 32 ? obj_exact_f32<32> : obj_exact_f32<64>));
        KC_TRY(grid_for(c, k1, smem1, v.n, &g1));
        KC_TRY(grid_for(c, k2, smem2, v.n, &g2));
        const int gmax = g1 > g2 ? g1 : g2;
        KC_TRY(ensure(c, c->work, off_part + (size_t)gmax * S * 12 + 64));
        char *w = static_cast<char *>(c->work.p);
        uint64_t *pairs = reinterpret_cast<uint64_t *>(w);
        float *thr = reinterpret_cast<float *>(w + off_thr);
        if (pts)
            pack_pairs_f32<<<(S * Kc * Dh + 255) / 256, 256, 0, c->stream>>>(static_cast<const float *>(pts), D, Dh,
                                                                             S * Kc, pairs);
        else
            gather_pairs_f32<<<(S * Kc * Dh + 255) / 256, 256, 0, c->stream>>>(
                static_cast<const float *>(c->X), c->ldx, D, Dh, centers, S * Kc, pairs);
        KC_TRY(after_launch(c, "gather centers"));
        unsigned long long *keys = reinterpret_cast<unsigned long long *>(w + off_part);
        if (v.n > 0) {
            k1<<<g1, kThreads, smem1, c->stream>>>(static_cast<const float *>(v.X), v.ld, v.n, D, pairs, S,
                                                   Kc, Dh, keys);
            KC_TRY(after_launch(c, "objective screen"));
        }
        obj_threshold<<<(S + 3) / 4, 128, 0, c->stream>>>(keys, v.n > 0 ? g1 : 0, S, screen_gamma(D),
                                                          alpha_cut, thr, val);
        KC_TRY(after_launch(c, "objective threshold"));
        double *pval = reinterpret_cast<double *>(w + off_part);
        uint32_t *ppos = reinterpret_cast<uint32_t *>(pval + (size_t)g2 * S);
        if (v.n > 0) {
            k2<<<g2, kThreads, smem2, c->stream>>>(static_cast<const float *>(v.X), v.ld, v.n, D, pairs, S,
                                                   Kc, Dh, thr, pval, ppos);
            KC_TRY(after_launch(c, "objective exact"));
        }
        obj_finalize<<<(S + 3) / 4, 128, 0, c->stream>>>(pval, ppos, v.n > 0 ? g2 : 0, S, v.ids, thr, val, arg);
        KC_TRY(after_launch(c, "objective finalize"));
    } else {
        const size_t smem = (size_t)S * Kc * D * 8 + (size_t)NW * S * 12;
        int g = 1;
        auto k = D <= 8 ? obj_exact_f64<8>
                        : (D <= 16 ? obj_exact_f64<16> : (D <= 64 ? obj_exact_f64<64> : obj_exact_f64<128>));
        KC_TRY(grid_for(c, k, smem, v.n, &g));
        KC_TRY(ensure(c, c->work, (size_t)g * S * 12 + 64));
        double *pval = static_cast<double *>(c->work.p);
        uint32_t *ppos = reinterpret_cast<uint32_t *>(pval + (size_t)g * S);
        if (v.n > 0) {
            k<<<g, kThreads, smem, c->stream>>>(static_cast<const double *>(v.X), v.ld, v.n, D,
                                                static_cast<const double *>(c->X), c->ldx, centers,
                                                static_cast<const double *>(pts), S, Kc, pval, ppos);
            KC_TRY(after_launch(c, "objective f64"));
        }
        obj_finalize<<<(S + 3) / 4, 128, 0, c->stream>>>(pval, ppos, v.n > 0 ? g : 0, S, v.ids, nullptr, val,
                                                         arg);
        KC_TRY(after_launch(c, "objective finalize"));
    }
    return KC_OK;
}

}  // namespace

kc_status launch_objective(kc_ctx *c, const View &v, const int64_t *centers, int S, int Kc,
                           double alpha_cut, double *val, int64_t *arg, const void *pts)
{
    if (S <= 0) return KC_OK;
    const int D = c->D;
    const size_t cap = (c->smem_optin > 0 ? c->smem_optin : 48 * 1024) / 2;
    const size_t per_set = c->dt == KC_F32 ? (size_t)Kc * ((D + 1) / 2) * 8 + 4 + 12 * 8
                                           : (size_t)Kc * D * 8 + 12 * 8;
    int chunk = (int)std::max<size_t>(1, cap / per_set);
    for (int s0 = 0; s0 < S; s0 += chunk) {
        const int ns = std::min(chunk, S - s0);
        KC_TRY(objective_chunk(c, v, centers ? centers + (size_t)s0 * Kc : nullptr, ns, Kc, alpha_cut, val + s0,
                               arg ? arg + s0 : nullptr,
                               pts ? static_cast<const char *>(pts) + (size_t)s0 * Kc * D * c->esize : nullptr));
    }
    return KC_OK;
}

}  // namespace kc
