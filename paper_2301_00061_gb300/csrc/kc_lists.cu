// kc_lists.cu -- per-node sample lists (Section 4.2: a sample redundant in a
// node for both the lower bound and the upper bound stays redundant in all of
// its descendants, so the descendants only need the node's surviving samples).
//
// Every kernel here works on work items (node b, offset into b's list): the
// CTA gathers that slice of sample ids and their coordinates, and evaluates it
// against node b only.  Keys name samples by their id, so ties still go to the
// smallest sample index.
//   seg_lb_f32        lower bound of each node over its list (float, certified)
//   seg_refine_f32    exact double re-evaluation of the samples that can attain it
//   seg_obj_screen / seg_obj_exact   objective of a candidate set over a list
//   seg_filter_f32    the surviving samples of a tightened node -> new list
// (float data, D <= 8: the shapes the tightening kernels take).
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "kc_device.cuh"
#include "kc_internal.cuh"

namespace kc {

namespace {

constexpr int kLT = 1024;   // list entries per work item (block of 256 threads)
constexpr int kListMaxD = 8;

// Float clamp distance over runtime D (pairs padded with (0, -0), which add 0).
template <int DMAX>
__device__ __forceinline__ float box_dist_rt(const uint64_t *px, const uint64_t *bx, int Dp)
{
    uint64_t acc = 0;
#pragma unroll
    for (int a = 0; a < DMAX; a += 2)
        if (a < Dp) {
            const float2 t0 = upk(sub2(bx[a], px[a]));
            const float2 t1 = upk(sub2(bx[a + 1], px[a + 1]));
            const uint64_t m = pk(max3f(t0.x, t0.y, 0.f), max3f(t1.x, t1.y, 0.f));
            acc = fma2(m, m, acc);
        }
    const float2 s = upk(acc);
    return s.x + s.y;
}

__device__ __forceinline__ unsigned long long block_max_u64(unsigned long long v, unsigned long long *red)
{
    v = warp_max_u64(v);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) red[w] = v;
    __syncthreads();
    unsigned long long r = 0ull;
    if (threadIdx.x == 0)
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r = red[i] > r ? red[i] : r;
    __syncthreads();
    return r;
}

// Lower bound of every node of a group over one tile of the group's list
// (float, packed key); the tile's samples stay in registers across the nodes.
template <int DMAX>
__global__ void __launch_bounds__(256)
seg_lb_f32(const float *__restrict__ X, int64_t ld, ListBatch L, const float *__restrict__ lo,
           const float *__restrict__ hi, int K, int D, unsigned long long *__restrict__ keys)
{
    constexpr int kPer = kLT / 256;   // samples per thread
    __shared__ unsigned long long red[8];
    __shared__ uint64_t sbox[kMaxK * DMAX];
    const int Dp = (D + 1) & ~1;
    for (int64_t w = blockIdx.x; w < L.W; w += gridDim.x) {
        int g;
        int64_t st;
        list_item(L.tile_prefix, L.B, w, kLT, &g, &st);
        const int64_t ng = L.seg_n[g];
        const int tn = (int)((ng - st) < (int64_t)kLT ? (ng - st) : (int64_t)kLT);
        const uint32_t *ids = L.pool + L.seg_off[g] + st;
        uint64_t px[kPer][DMAX];
        uint32_t pid[kPer];
#pragma unroll
        for (int q = 0; q < kPer; ++q) {
            const int j = threadIdx.x + q * 256;
            pid[q] = j < tn ? ids[j] : 0u;
#pragma unroll
            for (int a = 0; a < DMAX; ++a) {
                const float v = (j < tn && a < D) ? X[(size_t)a * ld + pid[q]] : 0.f;
                px[q][a] = pk(v, -v);
            }
        }
        const int n0 = L.node_start ? L.node_start[g] : g, n1 = L.node_start ? L.node_start[g + 1] : g + 1;
        for (int b = n0; b < n1; ++b) {
            for (int i = threadIdx.x; i < K * Dp; i += blockDim.x) {
                const int k = i / Dp, a = i % Dp;
                const size_t o = ((size_t)b * K + k) * D + a;
                sbox[i] = a < D ? pk(lo[o], -hi[o]) : pk(0.f, -0.f);
            }
            __syncthreads();
            unsigned long long best = 0ull;
#pragma unroll
            for (int q = 0; q < kPer; ++q)
                if (threadIdx.x + q * 256 < tn) {
                    float bmin = __int_as_float(0x7f800000);
                    for (int k = 0; k < K; ++k) bmin = fminf(bmin, box_dist_rt<DMAX>(px[q], sbox + k * Dp, Dp));
                    const unsigned long long key = key_max(bmin, pid[q]);
                    best = key > best ? key : best;
                }
            best = block_max_u64(best, red);   // ends with a barrier: sbox may be rewritten
            if (threadIdx.x == 0 && best) atomicMax(&keys[b], best);
        }
    }
}

// Exact double value of the lower bound of node b over the samples of its list
// whose float value reaches thr[b] (value only: ordered 64-bit max).
template <int DMAX>
__global__ void __launch_bounds__(256)
seg_refine_f32(const float *__restrict__ X, int64_t ld, ListBatch L, const float *__restrict__ lo,
               const float *__restrict__ hi, int K, int D, const float *__restrict__ thr,
               unsigned long long *__restrict__ vmax, const unsigned long long *__restrict__ vfound,
               unsigned *__restrict__ wid)
{
    // vfound NULL: the ordered double maximum into vmax; otherwise a second
    // pass over the same samples: the smallest id whose double value equals
    // vfound[b] into wid[b] (the sample attaining the refined bound)
    __shared__ uint64_t sbox[kMaxK * DMAX];
    const int Dp = (D + 1) & ~1;
    for (int64_t w = blockIdx.x; w < L.W; w += gridDim.x) {
        int b;
        int64_t st;
        list_item(L.tile_prefix, L.B, w, kLT, &b, &st);
        const int64_t nb = L.seg_n[b];
        const int tn = (int)((nb - st) < (int64_t)kLT ? (nb - st) : (int64_t)kLT);
        const uint32_t *ids = L.pool + L.seg_off[b] + st;
        for (int i = threadIdx.x; i < K * Dp; i += blockDim.x) {
            const int k = i / Dp, a = i % Dp;
            const size_t o = ((size_t)b * K + k) * D + a;
            sbox[i] = a < D ? pk(lo[o], -hi[o]) : pk(0.f, -0.f);
        }
        __syncthreads();
        const float t = thr[b];
        for (int j = threadIdx.x; j < tn; j += blockDim.x) {
            const uint32_t id = ids[j];
            uint64_t px[DMAX];
#pragma unroll
            for (int a = 0; a < DMAX; ++a) {
                const float v = a < D ? X[(size_t)a * ld + id] : 0.f;
                px[a] = pk(v, -v);
            }
            float bmin = __int_as_float(0x7f800000);
            for (int k = 0; k < K; ++k) bmin = fminf(bmin, box_dist_rt<DMAX>(px, sbox + k * Dp, Dp));
            if (bmin >= t) {
                double e = __longlong_as_double(0x7ff0000000000000ll);
                for (int k = 0; k < K; ++k) {
                    double acc = 0.0;
                    for (int a = 0; a < D; ++a) {
                        const double x = (double)upk(px[a]).x;
                        const size_t o = ((size_t)b * K + k) * D + a;
                        const double d = __dsub_rn(x, mid3d((double)lo[o], x, (double)hi[o]));
                        acc = __dadd_rn(acc, __dmul_rn(d, d));
                    }
                    if (acc < e) e = acc;
                }
                if (!vfound) atomicMax(&vmax[b], ord_f64(e));
                else if (ord_f64(e) == vfound[b]) atomicMin(&wid[b], id);
            }
        }
        __syncthreads();
    }
}

__global__ void wid_finalize(const unsigned *__restrict__ wid, const unsigned long long *__restrict__ v, int B,
                             int64_t *__restrict__ wit)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    wit[b] = (v[b] && wid[b] != 0xFFFFFFFFu) ? (int64_t)wid[b] : -1;
}

// Objective screen: float max over node b's list of min_k ||x - c_k||^2.
template <int DMAX>
__global__ void __launch_bounds__(256)
seg_obj_screen(const float *__restrict__ X, int64_t ld, ListBatch L, const float *__restrict__ Xf, int64_t ldf,
               const int64_t *__restrict__ centers, int K, int D, unsigned long long *__restrict__ keys)
{
    __shared__ unsigned long long red[8];
    __shared__ float sc[kMaxK * DMAX];
    for (int64_t w = blockIdx.x; w < L.W; w += gridDim.x) {
        int b;
        int64_t st;
        list_item(L.tile_prefix, L.B, w, kLT, &b, &st);
        const int64_t nb = L.seg_n[b];
        const int tn = (int)((nb - st) < (int64_t)kLT ? (nb - st) : (int64_t)kLT);
        const uint32_t *ids = L.pool + L.seg_off[b] + st;
        for (int i = threadIdx.x; i < K * D; i += blockDim.x)
            sc[i] = Xf[(size_t)(i % D) * ldf + centers[(size_t)b * K + i / D]];
        __syncthreads();
        unsigned long long best = 0ull;
        for (int j = threadIdx.x; j < tn; j += blockDim.x) {
            const uint32_t id = ids[j];
            float x[DMAX];
#pragma unroll
            for (int a = 0; a < DMAX; ++a) x[a] = a < D ? X[(size_t)a * ld + id] : 0.f;
            float q = __int_as_float(0x7f800000);
            for (int k = 0; k < K; ++k) {
                float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
                for (int a = 0; a < DMAX; a += 2) {
                    if (a < D) { const float t = x[a] - sc[k * D + a]; acc0 = fmaf(t, t, acc0); }
                    if (a + 1 < D) { const float t = x[a + 1] - sc[k * D + a + 1]; acc1 = fmaf(t, t, acc1); }
                }
                q = fminf(q, acc0 + acc1);
            }
            const unsigned long long key = key_max(q, id);
            best = key > best ? key : best;
        }
        best = block_max_u64(best, red);
        if (threadIdx.x == 0 && best) atomicMax(&keys[b], best);
    }
}

// Objective exact pass: double value of the samples whose float value reaches thr[b].
template <int DMAX>
__global__ void __launch_bounds__(256)
seg_obj_exact(const float *__restrict__ X, int64_t ld, ListBatch L, const float *__restrict__ Xf, int64_t ldf,
              const int64_t *__restrict__ centers, int K, int D, const float *__restrict__ thr,
              unsigned long long *__restrict__ vmax)
{
    __shared__ float sc[kMaxK * DMAX];
    for (int64_t w = blockIdx.x; w < L.W; w += gridDim.x) {
        int b;
        int64_t st;
        list_item(L.tile_prefix, L.B, w, kLT, &b, &st);
        const float t = thr[b];
        if (t == __int_as_float(0x7f800000)) continue;   // uniform: the set is skipped
        const int64_t nb = L.seg_n[b];
        const int tn = (int)((nb - st) < (int64_t)kLT ? (nb - st) : (int64_t)kLT);
        const uint32_t *ids = L.pool + L.seg_off[b] + st;
        __syncthreads();
        for (int i = threadIdx.x; i < K * D; i += blockDim.x)
            sc[i] = Xf[(size_t)(i % D) * ldf + centers[(size_t)b * K + i / D]];
        __syncthreads();
        for (int j = threadIdx.x; j < tn; j += blockDim.x) {
            const uint32_t id = ids[j];
            float x[DMAX];
#pragma unroll
            for (int a = 0; a < DMAX; ++a) x[a] = a < D ? X[(size_t)a * ld + id] : 0.f;
            float q = __int_as_float(0x7f800000);
            for (int k = 0; k < K; ++k) {
                float acc0 = 0.f, acc1 = 0.f;
#pragma unroll
                for (int a = 0; a < DMAX; a += 2) {
                    if (a < D) { const float tt = x[a] - sc[k * D + a]; acc0 = fmaf(tt, tt, acc0); }
                    if (a + 1 < D) { const float tt = x[a + 1] - sc[k * D + a + 1]; acc1 = fmaf(tt, tt, acc1); }
                }
                q = fminf(q, acc0 + acc1);
            }
            if (q >= t) {
                double e = __longlong_as_double(0x7ff0000000000000ll);
                for (int k = 0; k < K; ++k) {
                    double acc = 0.0;
                    for (int a = 0; a < D; ++a) {
                        const double d = __dsub_rn((double)x[a], (double)sc[k * D + a]);
                        acc = __dadd_rn(acc, __dmul_rn(d, d));
                    }
                    if (acc < e) e = acc;
                }
                atomicMax(&vmax[b], ord_f64(e));
            }
        }
    }
}

// Surviving samples of node b after its tightening: a sample is dropped when it
// is redundant for the lower bound (farthest-corner value proved below beta_b)
// and for the upper bound (outside every box, or some representative of each
// box that holds it proved farther than alpha).  Output: appended to the
// node's region out_pool[out_off[b] ...], count in out_n[b] (unordered tiles);
// out_off[b] < 0 (or out_pool NULL) counts node b's survivors without writing;
// with out_cap, entries at positions >= out_cap[b] are counted, not written.
// With ckeys, the lower bounds of node b's two children over the surviving
// samples come out of the same pass: child 0 has hi[cvar[b]] = csplit[2b],
// child 1 has lo[cvar[b]] = csplit[2b + 1], all other bounds as node b's boxes
// (packed keys ckeys[2b], ckeys[2b + 1]).
template <int DMAX>
__global__ void __launch_bounds__(256)
seg_filter_f32(const float *__restrict__ X, int64_t ld, ListBatch L, const float *__restrict__ lo,
               const float *__restrict__ hi, int K, int D, const float *__restrict__ beta_dn, float infl, float slack,
               float t_alpha, const float *__restrict__ repx, const int *__restrict__ nreps, int RM,
               const int *__restrict__ rmap, uint32_t *__restrict__ out_pool, const int64_t *__restrict__ out_off,
               const int64_t *__restrict__ out_cap, unsigned long long *__restrict__ out_n,
               const int *__restrict__ cvar, const float *__restrict__ csplit, unsigned long long *__restrict__ ckeys)
{
    // out_pool NULL: count the surviving samples only
    __shared__ uint64_t sbox[kMaxK * DMAX];
    __shared__ float sl[kMaxK * DMAX], sh[kMaxK * DMAX];
    __shared__ unsigned long long red[8];
    __shared__ int snr[kMaxK];
    // the node's representatives as packed coordinate pairs [K][RM][Dp / 2]
    extern __shared__ uint64_t srep[];
    const int Dp = (D + 1) & ~1, H = Dp / 2;
    const int lane = threadIdx.x & 31;
    for (int64_t w = blockIdx.x; w < L.W; w += gridDim.x) {
        int b;
        int64_t st;
        list_item(L.tile_prefix, L.B, w, kLT, &b, &st);
        const int64_t nb = L.seg_n[b];
        const int tn = (int)((nb - st) < (int64_t)kLT ? (nb - st) : (int64_t)kLT);
        const uint32_t *ids = L.pool + L.seg_off[b] + st;
        __syncthreads();   // the previous item's readers of the boxes are done
        for (int i = threadIdx.x; i < K * Dp; i += blockDim.x) {
            const int k = i / Dp, a = i % Dp;
            const size_t o = ((size_t)b * K + k) * D + a;
            sbox[i] = a < D ? pk(lo[o], -hi[o]) : pk(0.f, -0.f);
            if (a < D) { sl[k * D + a] = lo[o]; sh[k * D + a] = hi[o]; }
        }
        const size_t rb = rmap ? (size_t)rmap[b] : (size_t)b;   // row of the node's representatives
        for (int k = threadIdx.x; k < K; k += blockDim.x) snr[k] = nreps ? nreps[rb * K + k] : 0;
        if (nreps)
            for (int i = threadIdx.x; i < K * RM * H; i += blockDim.x) {
                const int k = i / (RM * H), r = (i / H) % RM, p = i % H;
                const float *c = repx + ((rb * K + k) * RM + r) * D;
                if (r < nreps[rb * K + k]) srep[i] = pk(c[2 * p], 2 * p + 1 < D ? c[2 * p + 1] : 0.f);
            }
        __syncthreads();
        const float bth = beta_dn[b];
        // the children's split: box ks, attribute as_, at (cm | cs)
        const int cv = ckeys ? cvar[b] : 0, ks = cv / D, as_ = cv % D;
        const float cm = ckeys ? csplit[2 * b] : 0.f, cs = ckeys ? csplit[2 * b + 1] : 0.f;
        unsigned long long best0 = 0ull, best1 = 0ull;
        for (int j0 = 0; j0 < tn; j0 += blockDim.x) {
            const int j = j0 + threadIdx.x;
            bool keep = false;
            uint32_t id = 0;
            if (j < tn) {
                id = ids[j];
                float x[DMAX];
                uint64_t px[DMAX];
#pragma unroll
                for (int a = 0; a < DMAX; ++a) {
                    x[a] = a < D ? X[(size_t)a * ld + id] : 0.f;
                    px[a] = pk(x[a], -x[a]);
                }
                // lower-bound redundancy: alpha_s(M) < beta (Eq. 13), proved in float
                float as = __int_as_float(0x7f800000);
                for (int k = 0; k < K; ++k) {
                    uint64_t acc = 0;
#pragma unroll
                    for (int a = 0; a < DMAX; a += 2)
                        if (a < Dp) {
                            const float2 t0 = upk(sub2(sbox[k * Dp + a], px[a]));
                            const float2 t1 = upk(sub2(sbox[k * Dp + a + 1], px[a + 1]));
                            const uint64_t m = pk(fmaxf(fabsf(t0.x), fabsf(t0.y)), fmaxf(fabsf(t1.x), fabsf(t1.y)));
                            acc = fma2(m, m, acc);
                        }
                    const float2 s2 = upk(acc);
                    as = fminf(as, s2.x + s2.y);
                }
                const bool lbred = __fadd_ru(__fmul_ru(as, infl), slack) < bth;
                // the upper-bound test only matters for lower-bound redundant samples
                bool ubred = lbred;
                uint64_t pxx[DMAX / 2];
#pragma unroll
                for (int p = 0; p < DMAX / 2; ++p) pxx[p] = pk(x[2 * p], x[2 * p + 1]);
                for (int k = 0; k < K && ubred; ++k) {
                    bool inb = true;
                    for (int a = 0; a < D; ++a)
                        if (x[a] < sl[k * D + a] || x[a] > sh[k * D + a]) inb = false;
                    if (!inb) continue;
                    bool excl = false;
                    const int nr = snr[k];
                    const uint64_t *ck = srep + (size_t)k * RM * H;
                    // chunks of 4 representatives decided by their largest distance
                    // (a short last chunk repeats the last representative)
                    for (int r0 = 0; r0 < nr && !excl; r0 += 4) {
                        float d[4];
#pragma unroll
                        for (int u = 0; u < 4; ++u) {
                            const uint64_t *cr = ck + (size_t)(r0 + u < nr ? r0 + u : nr - 1) * H;
                            // squared distance: even attributes in .x, odd in .y, each
                            // a fused chain in attribute order (zero padding adds 0)
                            uint64_t acc = 0;
#pragma unroll
                            for (int p = 0; p < DMAX / 2; ++p)
                                if (p < H) {
                                    const uint64_t t = sub2(pxx[p], cr[p]);
                                    acc = fma2(t, t, acc);
                                }
                            const float2 s2 = upk(acc);
                            d[u] = s2.x + s2.y;
                        }
                        if (fmaxf(fmaxf(d[0], d[1]), fmaxf(d[2], d[3])) > t_alpha) excl = true;
                    }
                    if (!excl) ubred = false;
                }
                keep = !(lbred && ubred);
                if (keep && ckeys) {
                    // children's bounds over the surviving samples (the closed form
                    // of Section 3.1 in the same float evaluation as seg_lb_f32)
                    float other = __int_as_float(0x7f800000);
                    for (int k = 0; k < K; ++k)
                        if (k != ks) other = fminf(other, box_dist_rt<DMAX>(px, sbox + k * Dp, Dp));
                    uint64_t cb[DMAX];
#pragma unroll
                    for (int a = 0; a < DMAX; ++a)
                        cb[a] = a == as_ ? pk(sl[ks * D + as_], -cm) : (a < Dp ? sbox[ks * Dp + a] : pk(0.f, -0.f));
                    const float d0 = box_dist_rt<DMAX>(px, cb, Dp);
#pragma unroll
                    for (int a = 0; a < DMAX; ++a)
                        if (a == as_) cb[a] = pk(cs, -sh[ks * D + as_]);
                    const float d1 = box_dist_rt<DMAX>(px, cb, Dp);
                    const unsigned long long k0 = key_max(fminf(other, d0), id), k1 = key_max(fminf(other, d1), id);
                    best0 = k0 > best0 ? k0 : best0;
                    best1 = k1 > best1 ? k1 : best1;
                }
            }
            // one reservation per warp (no block barrier): lane 0 claims the
            // warp's surviving entries, the others write behind it in lane order
            const unsigned bal = __ballot_sync(0xffffffffu, keep);
            if (bal) {
                unsigned long long base = 0ull;
                if (lane == 0) base = atomicAdd(&out_n[b], (unsigned long long)__popc(bal));
                base = __shfl_sync(0xffffffffu, base, 0);
                const int64_t pos = (int64_t)(base + __popc(bal & ((1u << lane) - 1u)));
                if (keep && out_pool && out_off[b] >= 0 && (!out_cap || pos < out_cap[b]))
                    out_pool[out_off[b] + pos] = id;
            }
        }
        if (ckeys) {
            best0 = block_max_u64(best0, red);
            best1 = block_max_u64(best1, red);
            if (threadIdx.x == 0) {
                if (best0) atomicMax(&ckeys[2 * b], best0);
                if (best1) atomicMax(&ckeys[2 * b + 1], best1);
            }
        }
    }
}

__global__ void iota_kernel(uint32_t *p, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = (uint32_t)i;
}

__global__ void keys_finalize(const unsigned long long *__restrict__ keys, int B, double defl, double slack,
                              double *__restrict__ lb, double *__restrict__ raw, int64_t *__restrict__ arg)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const unsigned long long m = keys[b];
    const double r = m ? (double)key_val(m) : 0.0;
    if (raw) raw[b] = r;
    if (lb) lb[b] = fmax(0.0, __dsub_rd(__dmul_rd(r, defl), slack));
    if (arg) arg[b] = m ? (int64_t)key_pos(m) : -1;
}

__global__ void vmax_finalize(const unsigned long long *__restrict__ v, int B, double defl, double slack,
                              double *__restrict__ out, const float *__restrict__ thr)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    if (thr && thr[b] == __int_as_float(0x7f800000)) { out[b] = __longlong_as_double(0x7ff0000000000000ll); return; }
    const double e = v[b] ? unord_f64(v[b]) : 0.0;
    out[b] = defl < 1.0 ? fmax(0.0, __dsub_rd(__dmul_rd(e, defl), slack)) : e;
}

__global__ void screen_threshold(const unsigned long long *__restrict__ keys, int B, double gam, double alpha_cut,
                                 float *__restrict__ thr)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    const double raw = keys[b] ? (double)key_val(keys[b]) : 0.0;
    const double low = __ddiv_rd(raw, 1.0 + gam);
    if (low >= alpha_cut) { thr[b] = __int_as_float(0x7f800000); return; }
    const double t = __dmul_rd(__dmul_rd(low, 1.0 - gam), 1.0 - 1e-6) - 1e-37;
    thr[b] = t > 0.0 ? __double2float_rd(t) : -1.0f;
}

int grid_items(const kc_ctx *c, int64_t W) { return (int)std::max<int64_t>(1, std::min<int64_t>(W, c->num_sms * 8)); }

}  // namespace

int list_tile() { return kLT; }

kc_status launch_iota(kc_ctx *c, uint32_t *p, int64_t n)
{
    iota_kernel<<<c->num_sms * 8, 256, 0, c->stream>>>(p, n);
    return after_launch(c, "list iota");
}

// keys [B] (device scratch, zeroed here) -> lb, raw, arg (device).
kc_status launch_seg_lb(kc_ctx *c, const ListBatch &L, const void *lo, const void *hi, int B, unsigned long long *keys,
                        double *lb, double *raw, int64_t *arg)
{
    if (c->D > kListMaxD) return set_err(c, KC_EINVAL, "list kernels: D <= %d (got %d)", kListMaxD, c->D);
    if (B <= 0) return KC_OK;
    KC_CUDA(c, cudaMemsetAsync(keys, 0, (size_t)B * 8, c->stream));
    if (L.W > 0) {
        const int g = grid_items(c, L.W);
        seg_lb_f32<8><<<g, 256, 0, c->stream>>>(static_cast<const float *>(c->X), c->ldx, L,
                                                static_cast<const float *>(lo), static_cast<const float *>(hi), c->K,
                                                c->D, keys);
        KC_TRY(after_launch(c, "list lower bound"));
    }
    keys_finalize<<<(B + 127) / 128, 128, 0, c->stream>>>(keys, B, deflate_factor(KC_F32, c->D),
                                                          underflow_slack(KC_F32, c->D), lb, raw, arg);
    return after_launch(c, "list lower bound finalize");
}

// raw_host [B]: the float bounds being refined (host); thr [B] float and
// vmax [B] device scratch; out [B] certified double bounds (device).  Samples
// whose float value is below a threshold derived from raw (with the float and
// double error bounds) cannot attain the maximum and are skipped.
kc_status launch_seg_refine(kc_ctx *c, const ListBatch &L, const void *lo, const void *hi, int B, const double *raw_host,
                            float *thr_dev, unsigned long long *vmax, double *out, unsigned *wid, int64_t *wit)
{
    if (c->D > kListMaxD) return set_err(c, KC_EINVAL, "list kernels: D <= %d (got %d)", kListMaxD, c->D);
    if (B <= 0) return KC_OK;
    const double gam = gamma_n(f32_roundings(c->D), kU32) + 2 * gamma_n(f64_roundings(c->D), kU64) + 1e-15;
    std::vector<float> thr(B);
    for (int b = 0; b < B; ++b) {
        const double t = raw_host[b] / (1.0 + gam) * (1.0 - gam) * (1.0 - 1e-6) - 1e-37;
        float f = (float)t;
        if ((double)f > t) f = nextafterf(f, -1.f);
        thr[b] = t > 0 ? f : -1.f;
    }
    KC_CUDA(c, cudaMemcpyAsync(thr_dev, thr.data(), (size_t)B * 4, cudaMemcpyHostToDevice, c->stream));
    KC_CUDA(c, cudaMemsetAsync(vmax, 0, (size_t)B * 8, c->stream));
    if (L.W > 0) {
        const int g = grid_items(c, L.W);
        seg_refine_f32<8><<<g, 256, 0, c->stream>>>(static_cast<const float *>(c->X), c->ldx, L,
                                                    static_cast<const float *>(lo), static_cast<const float *>(hi),
                                                    c->K, c->D, thr_dev, vmax, nullptr, nullptr);
        KC_TRY(after_launch(c, "list refinement"));
    }
    vmax_finalize<<<(B + 127) / 128, 128, 0, c->stream>>>(vmax, B, deflate_factor(KC_F64, c->D),
                                                          underflow_slack(KC_F64, c->D), out, nullptr);
    KC_TRY(after_launch(c, "list refinement finalize"));
    if (wit) {
        // the sample attaining each refined value (a second pass over the lists)
        KC_CUDA(c, cudaMemsetAsync(wid, 0xFF, (size_t)B * 4, c->stream));
        if (L.W > 0) {
            const int g = grid_items(c, L.W);
            seg_refine_f32<8><<<g, 256, 0, c->stream>>>(static_cast<const float *>(c->X), c->ldx, L,
                                                        static_cast<const float *>(lo), static_cast<const float *>(hi),
                                                        c->K, c->D, thr_dev, nullptr, vmax, wid);
            KC_TRY(after_launch(c, "list refinement witness"));
        }
        wid_finalize<<<(B + 127) / 128, 128, 0, c->stream>>>(wid, vmax, B, wit);
        KC_TRY(after_launch(c, "list refinement witness finalize"));
    }
    return KC_OK;
}

// Objective of B candidate sets (centers [B][K] ids, device), each over its own
// list; sets proved >= alpha_cut by the float screen get +inf.  keys, vmax:
// device scratch [B]; thr: device scratch [B] floats; val: device [B].
kc_status launch_seg_objective(kc_ctx *c, const ListBatch &L, const int64_t *centers, int B, double alpha_cut,
                               unsigned long long *keys, unsigned long long *vmax, float *thr, double *val)
{
    if (c->D > kListMaxD) return set_err(c, KC_EINVAL, "list kernels: D <= %d (got %d)", kListMaxD, c->D);
    if (B <= 0) return KC_OK;
    KC_CUDA(c, cudaMemsetAsync(keys, 0, (size_t)B * 8, c->stream));
    KC_CUDA(c, cudaMemsetAsync(vmax, 0, (size_t)B * 8, c->stream));
    const float *X = static_cast<const float *>(c->X);
    const int g = grid_items(c, L.W);
    if (L.W > 0) {
        seg_obj_screen<8><<<g, 256, 0, c->stream>>>(X, c->ldx, L, X, c->ldx, centers, c->K, c->D, keys);
        KC_TRY(after_launch(c, "list objective screen"));
    }
    const double gam = gamma_n(f32_roundings(c->D), kU32) + 2 * gamma_n(f64_roundings(c->D), kU64) + 1e-15;
    screen_threshold<<<(B + 127) / 128, 128, 0, c->stream>>>(keys, B, gam, alpha_cut, thr);
    KC_TRY(after_launch(c, "list objective threshold"));
    if (L.W > 0) {
        seg_obj_exact<8><<<g, 256, 0, c->stream>>>(X, c->ldx, L, X, c->ldx, centers, c->K, c->D, thr, vmax);
        KC_TRY(after_launch(c, "list objective exact"));
    }
    vmax_finalize<<<(B + 127) / 128, 128, 0, c->stream>>>(vmax, B, 1.0, 0.0, val, thr);
    return after_launch(c, "list objective finalize");
}

kc_status launch_seg_filter(kc_ctx *c, const ListBatch &L, const void *lo, const void *hi, int B,
                            const float *beta_dn_dev, double alpha, const void *repx, const int *nreps, int RM,
                            const int *rmap, uint32_t *out_pool, const int64_t *out_off, const int64_t *out_cap,
                            unsigned long long *out_n, const int *cvar, const float *csplit,
                            unsigned long long *ckeys, double *child_lb, double *child_raw, int64_t *child_arg)
{
    if (c->D > kListMaxD) return set_err(c, KC_EINVAL, "list kernels: D <= %d (got %d)", kListMaxD, c->D);
    if (B <= 0) return KC_OK;
    KC_CUDA(c, cudaMemsetAsync(out_n, 0, (size_t)B * 8, c->stream));
    if (ckeys) KC_CUDA(c, cudaMemsetAsync(ckeys, 0, (size_t)2 * B * 8, c->stream));
    const double g = gamma_n(f32_roundings(c->D), kU32);
    float infl = (float)(1.0 / (1.0 - g));
    if ((double)infl < 1.0 / (1.0 - g)) infl = nextafterf(infl, 2.f);
    const float slack = (float)((c->D + 2) * 1.401298464324817e-45);
    float defl = (float)(1.0 - g);
    if ((double)defl > 1.0 - g) defl = nextafterf(defl, 0.f);
    float aup = (float)alpha;
    if ((double)aup < alpha) aup = nextafterf(aup, 3.4e38f);
    float t_alpha = (float)(((double)aup + (double)slack) / (double)defl * (1.0 + 1e-6));
    if ((double)t_alpha < ((double)aup + (double)slack) / (double)defl * (1.0 + 1e-6)) t_alpha = nextafterf(t_alpha, 3.4e38f);
    const int gr = grid_items(c, L.W);
    const size_t srep = nreps ? (size_t)c->K * RM * (((c->D + 1) & ~1) / 2) * 8 : 0;
    if (srep > 48 * 1024)
        KC_CUDA(c, cudaFuncSetAttribute(seg_filter_f32<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)srep));
    seg_filter_f32<8><<<gr, 256, srep, c->stream>>>(static_cast<const float *>(c->X), c->ldx, L,
                                                 static_cast<const float *>(lo), static_cast<const float *>(hi), c->K,
                                                 c->D, beta_dn_dev, infl, slack, t_alpha,
                                                 static_cast<const float *>(repx), nreps, RM, rmap, out_pool, out_off,
                                                 out_cap, out_n, cvar, csplit, ckeys);
    KC_TRY(after_launch(c, "list filter"));
    if (ckeys) {
        keys_finalize<<<(2 * B + 127) / 128, 128, 0, c->stream>>>(ckeys, 2 * B, deflate_factor(KC_F32, c->D),
                                                                  underflow_slack(KC_F32, c->D), child_lb, child_raw,
                                                                  child_arg);
        KC_TRY(after_launch(c, "list filter: children's bounds"));
    }
    return KC_OK;
}

}  // namespace kc
