// kc_wide.cu -- cluster assignment and bounds tightening (Section 4.1,
// Algorithms 3-4) for float data of any shape up to K = 16 clusters and
// D = 128 attributes (the compile-time kernels of kc_visit.cu cover the small
// shapes).  Same decisions, same proofs of float exclusions, same outputs.
//
// Layout of the work: a CTA stages a tile of samples in shared memory (packed
// (x, -x) pairs) and then evaluates one node at a time with all its threads;
// the node's boxes and its accumulators (extreme keys, bounding boxes,
// counts, candidate keys) live in shared memory, sized at launch from K and
// D, so no thread holds K x D values in registers.  Accumulators are updated
// with shared-memory atomics, each preceded by a plain read that skips the
// atomic when it cannot change the value, and merged into the global ones
// once per (tile, node).
#include <cuda_runtime.h>

#include <vector>

#include "kc_device.cuh"
#include "kc_internal.cuh"

namespace kc {

namespace {

constexpr int kWT = 256;   // threads of the wide kernels

// Float clamp distance of a staged sample to box k of a node, runtime D
// (pairs of attributes in two interleaved fused chains, as box_dist_f32).
__device__ __forceinline__ float wide_box_dist(const uint64_t *tp, int tile, int j, const uint64_t *bx, int D)
{
    uint64_t acc = 0;
    int a = 0;
    for (; a + 1 < D; a += 2) {
        const float2 t0 = upk(sub2(bx[a], tp[(size_t)a * tile + j]));
        const float2 t1 = upk(sub2(bx[a + 1], tp[(size_t)(a + 1) * tile + j]));
        const uint64_t m = pk(max3f(t0.x, t0.y, 0.f), max3f(t1.x, t1.y, 0.f));
        acc = fma2(m, m, acc);
    }
    float2 s = upk(acc);
    if (a < D) {
        const float2 t = upk(sub2(bx[a], tp[(size_t)a * tile + j]));
        const float m = max3f(t.x, t.y, 0.f);
        s.x = fmaf(m, m, s.x);
    }
    return s.x + s.y;
}

// Float squared distance of a staged sample to a point c (runtime D), in the
// rounding pattern of pt_dist_f32: pairs (x_a - c_a, x_{a+1} - c_{a+1}) into
// two fused chains, an odd last attribute into the first chain.
__device__ __forceinline__ float wide_pt_dist(const uint64_t *tp, int tile, int j, const float *c, int D)
{
    uint64_t acc = 0;
    int a = 0;
    for (; a + 1 < D; a += 2) {
        const float x0 = upk(tp[(size_t)a * tile + j]).x, x1 = upk(tp[(size_t)(a + 1) * tile + j]).x;
        const uint64_t t = sub2(pk(x0, x1), pk(c[a], c[a + 1]));
        acc = fma2(t, t, acc);
    }
    float2 s = upk(acc);
    if (a < D) {
        const float t = upk(tp[(size_t)a * tile + j]).x - c[a];
        s.x = fmaf(t, t, s.x);
    }
    return s.x + s.y;
}

__device__ __forceinline__ void smax_u64(unsigned long long *p, unsigned long long v)
{
    if (v > *p) atomicMax(p, v);
}
__device__ __forceinline__ void smax_u32(unsigned *p, unsigned v)
{
    if (v > *p) atomicMax(p, v);
}
__device__ __forceinline__ void smin_u32(unsigned *p, unsigned v)
{
    if (v < *p) atomicMin(p, v);
}

__device__ __forceinline__ unsigned long long wkey_max(float v, uint32_t p)
{
    return ((unsigned long long)ord_f32(v) << 32) | (unsigned long long)(0xFFFFFFFFu - p);
}
__device__ __forceinline__ unsigned long long wkey_min(float v, uint32_t p)
{
    return ((unsigned long long)(~ord_f32(v)) << 32) | (unsigned long long)(0xFFFFFFFFu - p);
}

// A tile of samples -> shared memory as packed (x, -x) pairs [D][tile];
// tids != NULL: gathered by sample id (list mode), else rows base .. base + tn.
__device__ __forceinline__ void wide_stage(const float *__restrict__ X, int64_t ld, int D, int tile, int tn,
                                           int64_t base, const uint32_t *tids, uint64_t *tp)
{
    for (int i = threadIdx.x; i < D * tile; i += kWT) {
        const int a = i / tile, j = i - a * tile;
        float v = 0.f;
        if (j < tn) v = tids ? X[(size_t)a * ld + tids[j]] : X[(size_t)a * ld + base + j];
        tp[i] = pk(v, -v);
    }
}

// ------------------------------------------------------------------ pass A
// Per node: the certified lower bound's key of the input boxes, the center-
// based assignment (Lemma 1) and, per cluster, the arg-extremes of every
// attribute over the assigned samples (float keys as in kc_visit.cu).
// Shared memory: tile [D][tile] u64 | boxes [K][D] u64 | amax, amin [K][D] u64
// | lbkey u64 | flag.

// Directions after the attributes (the representatives' pair directions):
// direction q of ndir is attribute pair q / 2 (pairs a < b in lexicographic
// order, a in pa, b in pb), as x_a + x_b (q even) or x_a - x_b (q odd), in float.
struct WideDirs {
    int ndir;
    const signed char *pa, *pb;   // shared memory [ndir / 2]
    unsigned long long *sdmax, *sdmin;
    unsigned long long *__restrict__ dmax, *__restrict__ dmin;   // global [B][K][ndir]
};

__device__ __forceinline__ void wide_a_node(const uint64_t *tp, int tile, int tn, const uint32_t *tids, int64_t base,
                            const float *__restrict__ lo, const float *__restrict__ hi, int b, int K, int D,
                            const Margins &mg, uint64_t *sbx, unsigned long long *samax,
                            unsigned long long *samin, unsigned long long *slb, unsigned *sflag,
                            unsigned long long *__restrict__ lbkey, unsigned long long *__restrict__ amax,
                            unsigned long long *__restrict__ amin, unsigned *__restrict__ flags, const WideDirs &dv)
{
    const int KD = K * D, KQ = K * dv.ndir;
    __syncthreads();   // the previous node's readers are done
    for (int i = threadIdx.x; i < KD; i += kWT) {
        const size_t o = (size_t)b * KD + i;
        sbx[i] = pk(lo[o], -hi[o]);
        samax[i] = 0ull;
        samin[i] = 0ull;
    }
    for (int i = threadIdx.x; i < KQ; i += kWT) {
        dv.sdmax[i] = 0ull;
        dv.sdmin[i] = 0ull;
    }
    if (threadIdx.x == 0) {
        *slb = 0ull;
        *sflag = 0u;
    }
    __syncthreads();
    unsigned long long best = 0ull;
    bool infeasible = false;
    for (int j = threadIdx.x; j < tn; j += kWT) {
        const uint32_t pos = tids ? tids[j] : (uint32_t)(base + j);
        float bmin = 0.f;
        int left = 0, k1 = -1;
        for (int k = 0; k < K; ++k) {
            const float v = wide_box_dist(tp, tile, j, sbx + (size_t)k * D, D);
            bmin = (k == 0 || v < bmin) ? v : bmin;
            if (!(v > mg.t_alpha)) { ++left; k1 = k; }
        }
        const unsigned long long key = wkey_max(bmin, pos);
        best = key > best ? key : best;
        if (left == 0) infeasible = true;
        if (left == 1) {
            for (int a = 0; a < D; ++a) {
                const float x = upk(tp[(size_t)a * tile + j]).x;
                smax_u64(&samax[k1 * D + a], wkey_max(x, pos));
                smax_u64(&samin[k1 * D + a], wkey_min(x, pos));
            }
            for (int q = 0; q < dv.ndir; ++q) {
                const float xa = upk(tp[(size_t)dv.pa[q >> 1] * tile + j]).x;
                const float xb = upk(tp[(size_t)dv.pb[q >> 1] * tile + j]).x;
                const float v = (q & 1) ? xa - xb : xa + xb;
                smax_u64(&dv.sdmax[k1 * dv.ndir + q], wkey_max(v, pos));
                smax_u64(&dv.sdmin[k1 * dv.ndir + q], wkey_min(v, pos));
            }
        }
    }
    best = warp_max_u64(best);
    if ((threadIdx.x & 31) == 0 && best) smax_u64(slb, best);
    if (__any_sync(0xffffffffu, infeasible) && (threadIdx.x & 31) == 0) atomicOr(sflag, 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < KD; i += kWT) {
        const size_t o = (size_t)b * KD + i;
        if (samax[i]) atomicMax(&amax[o], samax[i]);
        if (samin[i]) atomicMax(&amin[o], samin[i]);
    }
    for (int i = threadIdx.x; i < KQ; i += kWT) {
        const size_t o = (size_t)b * KQ + i;
        if (dv.sdmax[i]) atomicMax(&dv.dmax[o], dv.sdmax[i]);
        if (dv.sdmin[i]) atomicMax(&dv.dmin[o], dv.sdmin[i]);
    }
    if (threadIdx.x == 0) {
        if (*slb) atomicMax(&lbkey[b], *slb);
        if (*sflag) atomicOr(&flags[b], 1u);
    }
}

__global__ void __launch_bounds__(kWT, 2)
wide_a_kernel(const float *__restrict__ X, int64_t ld, int64_t n, int tile, ListBatch L, int B, int K, int D,
              const float *__restrict__ lo, const float *__restrict__ hi, Margins mg,
              unsigned long long *__restrict__ lbkey, unsigned long long *__restrict__ amax,
              unsigned long long *__restrict__ amin, unsigned *__restrict__ flags, int ndir,
              unsigned long long *__restrict__ dmax, unsigned long long *__restrict__ dmin)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int KD = K * D, KQ = K * ndir;
    uint64_t *tp = reinterpret_cast<uint64_t *>(smem);
    uint64_t *sbx = tp + (size_t)D * tile;
    unsigned long long *samax = reinterpret_cast<unsigned long long *>(sbx + KD), *samin = samax + KD;
    unsigned long long *sdmax = samin + KD, *sdmin = sdmax + KQ, *slb = sdmin + KQ;
    unsigned *sflag = reinterpret_cast<unsigned *>(slb + 1);
    signed char *pa = reinterpret_cast<signed char *>(sflag + 2), *pb = pa + 16;
    uint32_t *tids = reinterpret_cast<uint32_t *>(pa + 32);
    if (threadIdx.x == 0) {
        // the attribute pairs a < b in lexicographic order
        int p = 0;
        for (int a = 0; a < D && p < ndir / 2; ++a)
            for (int c = a + 1; c < D && p < ndir / 2; ++c, ++p) {
                pa[p] = (signed char)a;
                pb[p] = (signed char)c;
            }
    }
    const WideDirs dv{ndir, pa, pb, sdmax, sdmin, dmax, dmin};
    if (L.pool) {
        for (int64_t w = blockIdx.x; w < L.W; w += gridDim.x) {
            int g;
            int64_t st;
            list_item(L.tile_prefix, L.B, w, tile, &g, &st);
            const int64_t ng = L.seg_n[g];
            const int tn = (int)((ng - st) < (int64_t)tile ? (ng - st) : (int64_t)tile);
            __syncthreads();
            for (int j = threadIdx.x; j < tn; j += kWT) tids[j] = L.pool[L.seg_off[g] + st + j];
            __syncthreads();
            wide_stage(X, ld, D, tile, tn, 0, tids, tp);
            const int n0 = L.node_start ? L.node_start[g] : g, n1 = L.node_start ? L.node_start[g + 1] : g + 1;
            for (int b = n0; b < n1; ++b)
                wide_a_node(tp, tile, tn, tids, 0, lo, hi, b, K, D, mg, sbx, samax, samin, slb, sflag, lbkey, amax,
                            amin, flags, dv);
        }
    } else {
        for (int64_t base = (int64_t)blockIdx.x * tile; base < n; base += (int64_t)gridDim.x * tile) {
            const int tn = (int)((n - base) < (int64_t)tile ? (n - base) : (int64_t)tile);
            __syncthreads();
            wide_stage(X, ld, D, tile, tn, base, nullptr, tp);
            for (int b = 0; b < B; ++b)
                wide_a_node(tp, tile, tn, nullptr, base, lo, hi, b, K, D, mg, sbx, samax, samin, slb, sflag, lbkey,
                            amax, amin, flags, dv);
        }
    }
}

// ------------------------------------------------------------------ pass B
// Per node: sample-based assignment (Lemma 2) of the samples the center-
// based rule left open, ball-based tightening and "centers on samples"
// (Algorithm 4): |S_+^k|, the bounding box of S_+^k, the bounding box of the
// sample-based assigned samples and the candidate closest to the midpoint of
// the box-BT box.  Shared memory: tile [D][tile] u64 | input boxes [K][D] u64
// | box-BT lo, hi, mid [K][D] f32 | smax, smin, jmax, jmin [K][D] u32 |
// counts [K] u64 | cand [K] u64 | nr [K] int | flag.

struct WideB {
    const float *blo, *bhi, *repx;
    const int *nreps, *allhave;
    const int64_t *seeds;
    int RM;
    unsigned long long *cnt, *cand;
    unsigned *smax, *smin, *jmax, *jmin, *flags;
};

__device__ __forceinline__ void wide_b_node(const uint64_t *tp, int tile, int tn, const uint32_t *tids, const uint32_t *ids,
                            int64_t base, const float *__restrict__ lo, const float *__restrict__ hi, int b, int K,
                            int D, const Margins &mg, unsigned char *ns, const WideB &p)
{
    const int KD = K * D;
    uint64_t *sbx = reinterpret_cast<uint64_t *>(ns);
    float *sl = reinterpret_cast<float *>(sbx + KD), *sh = sl + KD, *smid = sh + KD;
    unsigned *s_smax = reinterpret_cast<unsigned *>(smid + KD), *s_smin = s_smax + KD;
    unsigned *s_jmax = s_smin + KD, *s_jmin = s_jmax + KD;
    unsigned long long *scnt = reinterpret_cast<unsigned long long *>(
        (reinterpret_cast<uintptr_t>(s_jmin + KD) + 7) & ~(uintptr_t)7);
    unsigned long long *scand = scnt + K;
    int *snr = reinterpret_cast<int *>(scand + K);
    unsigned *sflag = reinterpret_cast<unsigned *>(snr + K);
    __syncthreads();
    for (int i = threadIdx.x; i < KD; i += kWT) {
        const size_t o = (size_t)b * KD + i;
        sbx[i] = pk(lo[o], -hi[o]);
        const float lv = p.blo[o], hv = p.bhi[o];
        sl[i] = lv;
        sh[i] = hv;
        smid[i] = (float)(0.5 * ((double)lv + (double)hv));
        s_smax[i] = 0u;
        s_smin[i] = ~0u;
        s_jmax[i] = 0u;
        s_jmin[i] = ~0u;
    }
    for (int k = threadIdx.x; k < K; k += kWT) {
        scnt[k] = 0ull;
        scand[k] = 0ull;
        snr[k] = p.nreps[(size_t)b * K + k];
    }
    if (threadIdx.x == 0) *sflag = 0u;
    __syncthreads();
    const bool have = p.allhave[b] != 0;
    const float *rxb = p.repx + (size_t)b * K * p.RM * D;
    bool infeasible = false;
    for (int j = threadIdx.x; j < tn; j += kWT) {
        const uint32_t pos = tids ? tids[j] : (uint32_t)(base + j);
        // clusters the center-based rule leaves open
        int left = 0;
        if (have)
            for (int k = 0; k < K; ++k)
                if (!(wide_box_dist(tp, tile, j, sbx + (size_t)k * D, D) > mg.t_alpha)) ++left;
        bool open = false;
        if (have && left >= 2) {
            const int64_t id = tids ? (int64_t)tids[j] : (ids ? (int64_t)ids[base + j] : base + j);
            bool is_seed = false;
            for (int k = 0; k < K; ++k)
                if (p.seeds && p.seeds[k] == id) is_seed = true;
            open = !is_seed;
        }
        int left4 = 0, k4 = -1;
        for (int k = 0; k < K; ++k) {
            bool inb = true;
            for (int a = 0; a < D && inb; ++a) {
                const float x = upk(tp[(size_t)a * tile + j]).x;
                if (x < sl[k * D + a] || x > sh[k * D + a]) inb = false;
            }
            if (!open && !inb) continue;
            // distances to the representatives of cluster k
            bool far4 = false, far1 = false;
            for (int r = 0; r < snr[k]; ++r) {
                const float d = wide_pt_dist(tp, tile, j, rxb + ((size_t)k * p.RM + r) * D, D);
                if (d > mg.t_four) far4 = true;
                if (d > mg.t_alpha) far1 = true;
            }
            if (open && !far4) { ++left4; k4 = k; }
            if (inb && !far1) {
                // ball-based tightening and centers on samples
                atomicAdd(&scnt[k], 1ull);
                for (int a = 0; a < D; ++a) {
                    const unsigned v = ord_f32(upk(tp[(size_t)a * tile + j]).x);
                    smax_u32(&s_smax[k * D + a], v);
                    smin_u32(&s_smin[k * D + a], v);
                }
                const float dm = wide_pt_dist(tp, tile, j, smid + (size_t)k * D, D);
                smax_u64(&scand[k], wkey_min(dm, pos));
            }
        }
        if (open) {
            // sample-based assignment (Algorithm 3, Lemma 2)
            if (left4 == 0) infeasible = true;
            if (left4 == 1)
                for (int a = 0; a < D; ++a) {
                    const unsigned v = ord_f32(upk(tp[(size_t)a * tile + j]).x);
                    smax_u32(&s_jmax[k4 * D + a], v);
                    smin_u32(&s_jmin[k4 * D + a], v);
                }
        }
    }
    if (__any_sync(0xffffffffu, infeasible) && (threadIdx.x & 31) == 0) atomicOr(sflag, 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < KD; i += kWT) {
        const size_t o = (size_t)b * KD + i;
        if (s_smax[i] != 0u) atomicMax(&p.smax[o], s_smax[i]);
        if (s_smin[i] != ~0u) atomicMin(&p.smin[o], s_smin[i]);
        if (s_jmax[i] != 0u) atomicMax(&p.jmax[o], s_jmax[i]);
        if (s_jmin[i] != ~0u) atomicMin(&p.jmin[o], s_jmin[i]);
    }
    for (int k = threadIdx.x; k < K; k += kWT) {
        const size_t o = (size_t)b * K + k;
        if (scnt[k]) atomicAdd(&p.cnt[o], scnt[k]);
        if (scand[k]) atomicMax(&p.cand[o], scand[k]);
    }
    if (threadIdx.x == 0 && *sflag) atomicOr(&p.flags[b], 1u);
}

__global__ void __launch_bounds__(kWT, 2)
wide_b_kernel(const float *__restrict__ X, int64_t ld, int64_t n, int tile, ListBatch L, int B, int K, int D,
              const float *__restrict__ lo, const float *__restrict__ hi, Margins mg, const uint32_t *__restrict__ ids,
              WideB p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *tp = reinterpret_cast<uint64_t *>(smem);
    unsigned char *ns = reinterpret_cast<unsigned char *>(tp + (size_t)D * tile);
    const size_t node_bytes = ((size_t)K * D * (8 + 12 + 16) + 16 + (size_t)K * 20 + 8 + 15) & ~(size_t)15;
    uint32_t *tids = reinterpret_cast<uint32_t *>(ns + node_bytes);
    if (L.pool) {
        for (int64_t w = blockIdx.x; w < L.W; w += gridDim.x) {
            int g;
            int64_t st;
            list_item(L.tile_prefix, L.B, w, tile, &g, &st);
            const int64_t ng = L.seg_n[g];
            const int tn = (int)((ng - st) < (int64_t)tile ? (ng - st) : (int64_t)tile);
            __syncthreads();
            for (int j = threadIdx.x; j < tn; j += kWT) tids[j] = L.pool[L.seg_off[g] + st + j];
            __syncthreads();
            wide_stage(X, ld, D, tile, tn, 0, tids, tp);
            const int n0 = L.node_start ? L.node_start[g] : g, n1 = L.node_start ? L.node_start[g + 1] : g + 1;
            for (int b = n0; b < n1; ++b) wide_b_node(tp, tile, tn, tids, nullptr, 0, lo, hi, b, K, D, mg, ns, p);
        }
    } else {
        for (int64_t base = (int64_t)blockIdx.x * tile; base < n; base += (int64_t)gridDim.x * tile) {
            const int tn = (int)((n - base) < (int64_t)tile ? (n - base) : (int64_t)tile);
            __syncthreads();
            wide_stage(X, ld, D, tile, tn, base, nullptr, tp);
            for (int b = 0; b < B; ++b) wide_b_node(tp, tile, tn, nullptr, ids, base, lo, hi, b, K, D, mg, ns, p);
        }
    }
}

// ------------------------------------------------- every-sample step B
// The step-A sets J_A^k of node b: the samples whose center-based rule
// leaves exactly the cluster k (Lemma 1, the float decisions of pass A) and
// the seed of k.  jpool == NULL: counts |J_A^k| into jcnt [B][K]; otherwise
// writes view positions at jpool[joff[b][k] + slot], slot taken from jcnt
// (reset to 0 before), one atomic per warp and cluster.
__global__ void __launch_bounds__(kWT)
jall_kernel(const float *__restrict__ X, int64_t ld, int64_t n, int tile, int B, int K, int D,
            const float *__restrict__ lo, const float *__restrict__ hi, Margins mg, const uint32_t *__restrict__ ids,
            const int64_t *__restrict__ seeds, unsigned long long *__restrict__ jcnt,
            const int64_t *__restrict__ joff, uint32_t *__restrict__ jpool)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *tp = reinterpret_cast<uint64_t *>(smem);
    uint64_t *sbx = tp + (size_t)D * tile;   // [K][D] boxes of the current node
    const int KD = K * D, lane = threadIdx.x & 31;
    for (int64_t base = (int64_t)blockIdx.x * tile; base < n; base += (int64_t)gridDim.x * tile) {
        const int tn = (int)((n - base) < (int64_t)tile ? (n - base) : (int64_t)tile);
        __syncthreads();
        wide_stage(X, ld, D, tile, tn, base, nullptr, tp);
        for (int b = 0; b < B; ++b) {
            __syncthreads();
            for (int i = threadIdx.x; i < KD; i += kWT) sbx[i] = pk(lo[(size_t)b * KD + i], -hi[(size_t)b * KD + i]);
            __syncthreads();
            for (int j = threadIdx.x; j < tn; j += kWT) {
                const int64_t pos = base + j, id = ids ? (int64_t)ids[pos] : pos;
                int kk = -1;
                if (seeds)
                    for (int k = 0; k < K; ++k)
                        if (seeds[k] == id) kk = k;
                if (kk < 0) {
                    int left = 0, k1 = -1;
                    for (int k = 0; k < K; ++k)
                        if (!(wide_box_dist(tp, tile, j, sbx + (size_t)k * D, D) > mg.t_alpha)) { ++left; k1 = k; }
                    if (left == 1) kk = k1;
                }
                // lanes of a warp with the same cluster share one atomic
                const unsigned grp = __match_any_sync(__activemask(), kk);
                const int leader = __ffs(grp) - 1, rank = __popc(grp & ((1u << lane) - 1u));
                unsigned long long slot = 0ull;
                const size_t o = (size_t)b * K + (kk < 0 ? 0 : kk);
                if (kk >= 0 && lane == leader) slot = atomicAdd(&jcnt[o], (unsigned long long)__popc(grp));
                slot = __shfl_sync(grp, slot, leader);
                // the counting pass took the same decisions; the bound keeps a
                // write inside its set regardless
                const int64_t at = joff ? joff[o] + (int64_t)slot + rank : 0;
                if (kk >= 0 && jpool && at < joff[o + 1]) jpool[at] = (uint32_t)pos;
            }
        }
    }
}

// Step B of node b = blockIdx.y against every sample of J_A^k (Algorithm 3's
// sample-based assignment and Algorithm 4's ball test without a budget): one
// view sample per thread (kWT per CTA, blockIdx.x), the lists J_A^k streamed
// through shared memory kJC points at a time.  A sample's scan of cluster k
// stops once it is decided (some point proved farther than 4 alpha, or than
// alpha when only the ball test needs k); the CTA stops when all are.
// Distances and decisions as in wide_b_node; chunks of 4 points are decided
// by their largest distance.
constexpr int kJC = 256;
constexpr int kAllMaxD = 16;

// wide_pt_dist with the sample in registers as coordinate pairs (xp[p] =
// (x_2p, x_2p+1), zero beyond D; xlast = x_{D-1}): the same pairs, chains
// and order.
template <int DM>
struct RegSample {
    uint64_t xp[DM / 2];
    float xlast;
};

template <int DM>
__device__ __forceinline__ float reg_pt_dist(const RegSample<DM> &x, const float *c, int D)
{
    uint64_t acc = 0;
#pragma unroll
    for (int p = 0; p < DM / 2; ++p)
        if (2 * p + 1 < D) {
            const uint64_t t = sub2(x.xp[p], pk(c[2 * p], c[2 * p + 1]));
            acc = fma2(t, t, acc);
        }
    float2 s = upk(acc);
    if (D & 1) {
        const float t = x.xlast - c[D - 1];
        s.x = fmaf(t, t, s.x);
    }
    return s.x + s.y;
}

template <int DM>   // D <= DM (2, 4, 8 or 16): the unrolled width of the distance scans
__global__ void __launch_bounds__(kWT)
ball_all_kernel(const float *__restrict__ X, int64_t ld, int64_t n, int K, int D, const float *__restrict__ lo,
                const float *__restrict__ hi, Margins mg, const uint32_t *__restrict__ ids,
                const int64_t *__restrict__ joff, const uint32_t *__restrict__ jpool, WideB p)
{
    extern __shared__ __align__(16) unsigned char smem[];
    const int KD = K * D, b = blockIdx.y;
    uint64_t *tp = reinterpret_cast<uint64_t *>(smem);                  // [D][kWT] staged samples
    uint64_t *sbx = tp + (size_t)D * kWT;                                 // [K][D] input boxes
    float *sl = reinterpret_cast<float *>(sbx + KD), *sh = sl + KD, *smid = sh + KD;   // box-BT boxes
    float *chunk = smid + KD;                                             // [kJC][D]
    unsigned *s_smax = reinterpret_cast<unsigned *>(chunk + (size_t)kJC * D), *s_smin = s_smax + KD;
    unsigned *s_jmax = s_smin + KD, *s_jmin = s_jmax + KD;
    unsigned long long *scnt = reinterpret_cast<unsigned long long *>(
        (reinterpret_cast<uintptr_t>(s_jmin + KD) + 7) & ~(uintptr_t)7);
    unsigned long long *scand = scnt + K;
    unsigned *sflag = reinterpret_cast<unsigned *>(scand + K);
    const int64_t base = (int64_t)blockIdx.x * kWT;
    const int tn = (int)((n - base) < (int64_t)kWT ? (n - base) : (int64_t)kWT);
    wide_stage(X, ld, D, kWT, tn, base, nullptr, tp);
    for (int i = threadIdx.x; i < KD; i += kWT) {
        const size_t o = (size_t)b * KD + i;
        sbx[i] = pk(lo[o], -hi[o]);
        const float lv = p.blo[o], hv = p.bhi[o];
        sl[i] = lv;
        sh[i] = hv;
        smid[i] = (float)(0.5 * ((double)lv + (double)hv));
        s_smax[i] = 0u;
        s_smin[i] = ~0u;
        s_jmax[i] = 0u;
        s_jmin[i] = ~0u;
    }
    for (int k = threadIdx.x; k < K; k += kWT) {
        scnt[k] = 0ull;
        scand[k] = 0ull;
    }
    if (threadIdx.x == 0) *sflag = 0u;
    __syncthreads();
    const int j = threadIdx.x;
    const bool valid = j < tn, have = p.allhave[b] != 0;
    const uint32_t pos = (uint32_t)(base + j);
    // clusters the center-based rule leaves open; an open sample that is not
    // a seed gets the sample-based rule
    bool open = false;
    if (valid && have) {
        int left = 0;
        for (int k = 0; k < K; ++k)
            if (!(wide_box_dist(tp, kWT, j, sbx + (size_t)k * D, D) > mg.t_alpha)) ++left;
        if (left >= 2) {
            const int64_t id = ids ? (int64_t)ids[base + j] : base + j;
            bool is_seed = false;
            for (int k = 0; k < K; ++k)
                if (p.seeds && p.seeds[k] == id) is_seed = true;
            open = !is_seed;
        }
    }
    // the thread's sample in registers for the distance scans
    RegSample<DM> xr;
    xr.xlast = upk(tp[(size_t)(D - 1) * kWT + j]).x;
#pragma unroll
    for (int p = 0; p < DM / 2; ++p)
        xr.xp[p] = pk(2 * p < D ? upk(tp[(size_t)(2 * p) * kWT + j]).x : 0.f,
                      2 * p + 1 < D ? upk(tp[(size_t)(2 * p + 1) * kWT + j]).x : 0.f);
    int left4 = 0, k4 = -1;
    bool infeasible = false;
    for (int k = 0; k < K; ++k) {
        bool inb = valid;
        for (int a = 0; a < D && inb; ++a) {
            const float x = upk(tp[(size_t)a * kWT + j]).x;
            if (x < sl[k * D + a] || x > sh[k * D + a]) inb = false;
        }
        const bool need = open || inb;
        if (!__syncthreads_or(need)) continue;
        bool far4 = false, far1 = false, done = !need;
        const int64_t q1 = joff[(size_t)b * K + k + 1];
        for (int64_t q0 = joff[(size_t)b * K + k]; q0 < q1; q0 += kJC) {
            const int cn = (int)((q1 - q0) < kJC ? (q1 - q0) : kJC);
            for (int i = threadIdx.x; i < cn * D; i += kWT) {
                const int r = i / D, a = i - r * D;
                chunk[i] = X[(size_t)a * ld + jpool[q0 + r]];
            }
            __syncthreads();
            if (!done) {
                for (int r0 = 0; r0 < cn; r0 += 4) {
                    float d[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u)
                        d[u] = reg_pt_dist(xr, chunk + (size_t)(r0 + u < cn ? r0 + u : cn - 1) * D, D);
                    const float m = fmaxf(fmaxf(d[0], d[1]), fmaxf(d[2], d[3]));
                    if (m > mg.t_alpha) {
                        far1 = true;
                        if (m > mg.t_four) { far4 = true; break; }
                        if (!open) break;
                    }
                }
                done = far4 || (far1 && !open);
            }
            // the barrier before the next chunk overwrites the buffer
            if (!__syncthreads_or(!done)) break;
        }
        if (open && !far4) { ++left4; k4 = k; }
        if (inb && !far1) {
            // ball-based tightening and centers on samples
            atomicAdd(&scnt[k], 1ull);
            for (int a = 0; a < D; ++a) {
                const unsigned v = ord_f32(upk(tp[(size_t)a * kWT + j]).x);
                smax_u32(&s_smax[k * D + a], v);
                smin_u32(&s_smin[k * D + a], v);
            }
            const float dm = wide_pt_dist(tp, kWT, j, smid + (size_t)k * D, D);
            smax_u64(&scand[k], wkey_min(dm, pos));
        }
    }
    if (open) {
        // sample-based assignment (Algorithm 3, Lemma 2)
        if (left4 == 0) infeasible = true;
        if (left4 == 1)
            for (int a = 0; a < D; ++a) {
                const unsigned v = ord_f32(upk(tp[(size_t)a * kWT + j]).x);
                smax_u32(&s_jmax[k4 * D + a], v);
                smin_u32(&s_jmin[k4 * D + a], v);
            }
    }
    if (infeasible) atomicOr(sflag, 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < KD; i += kWT) {
        const size_t o = (size_t)b * KD + i;
        if (s_smax[i] != 0u) atomicMax(&p.smax[o], s_smax[i]);
        if (s_smin[i] != ~0u) atomicMin(&p.smin[o], s_smin[i]);
        if (s_jmax[i] != 0u) atomicMax(&p.jmax[o], s_jmax[i]);
        if (s_jmin[i] != ~0u) atomicMin(&p.jmin[o], s_jmin[i]);
    }
    for (int k = threadIdx.x; k < K; k += kWT) {
        const size_t o = (size_t)b * K + k;
        if (scnt[k]) atomicAdd(&p.cnt[o], scnt[k]);
        if (scand[k]) atomicMax(&p.cand[o], scand[k]);
    }
    if (threadIdx.x == 0 && *sflag) atomicOr(&p.flags[b], 1u);
}

}  // namespace

size_t wide_b_node_bytes(int K, int D)
{
    return ((size_t)K * D * (8 + 12 + 16) + 16 + (size_t)K * 20 + 8 + 15) & ~(size_t)15;
}

// Pass A and pass B of the wide path on the context's stream; the caller
// (tighten_common in kc_visit.cu) owns the workspace and the finalize kernels.
kc_status launch_wide_a(kc_ctx *c, const View &v, const ListBatch *L, const float *lo, const float *hi, int B,
                        const Margins &mg, unsigned long long *lbkey, unsigned long long *amax,
                        unsigned long long *amin, unsigned *flags, int ndir, unsigned long long *dmax,
                        unsigned long long *dmin)
{
    const int K = c->K, D = c->D, KD = K * D;
    if (ndir > 32) return set_err(c, KC_EINTERNAL, "wide tightening: at most 16 attribute pairs");
    // a list batch is laid out in list_tile() entries per work item
    const int tile = L ? list_tile()
                       : (int)std::max<int64_t>(64, std::min<int64_t>(1024, (48 * 1024) / (8 * (int64_t)D)) / 32 * 32);
    const size_t smem = (size_t)D * tile * 8 + (size_t)KD * 24 + (size_t)K * ndir * 16 + 16 + 32 + (size_t)tile * 4 +
                        16;
    if (smem > 48 * 1024)
        KC_CUDA(c, cudaFuncSetAttribute(wide_a_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    KC_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wide_a_kernel, kWT, smem));
    if (per_sm < 1) return set_err(c, KC_EINTERNAL, "wide tightening pass A does not fit (smem %zu)", smem);
    ListBatch Lz;
    const int64_t work = L ? L->W : (v.n + tile - 1) / tile;
    if (work <= 0) return KC_OK;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(work, (int64_t)per_sm * c->num_sms));
    wide_a_kernel<<<grid, kWT, smem, c->stream>>>(static_cast<const float *>(v.X), v.ld, v.n, tile, L ? *L : Lz, B,
                                                  K, D, lo, hi, mg, lbkey, amax, amin, flags, ndir, dmax, dmin);
    return after_launch(c, "tighten pass A (wide)");
}

kc_status launch_wide_b(kc_ctx *c, const View &v, const ListBatch *L, const float *lo, const float *hi, int B,
                        const Margins &mg, const float *blo, const float *bhi, const float *repx, const int *nreps,
                        const int *allhave, const int64_t *seeds, int RM, unsigned long long *cnt,
                        unsigned long long *cand, unsigned *smax, unsigned *smin, unsigned *jmax, unsigned *jmin,
                        unsigned *flags)
{
    const int K = c->K, D = c->D;
    // a list batch is laid out in list_tile() entries per work item
    const int tile = L ? list_tile()
                       : (int)std::max<int64_t>(64, std::min<int64_t>(1024, (48 * 1024) / (8 * (int64_t)D)) / 32 * 32);
    const size_t smem = (size_t)D * tile * 8 + wide_b_node_bytes(K, D) + (size_t)tile * 4 + 16;
    if (smem > 48 * 1024)
        KC_CUDA(c, cudaFuncSetAttribute(wide_b_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    KC_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, wide_b_kernel, kWT, smem));
    if (per_sm < 1) return set_err(c, KC_EINTERNAL, "wide tightening pass B does not fit (smem %zu)", smem);
    ListBatch Lz;
    const int64_t work = L ? L->W : (v.n + tile - 1) / tile;
    if (work <= 0) return KC_OK;
    const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(work, (int64_t)per_sm * c->num_sms));
    WideB p{blo, bhi, repx, nreps, allhave, seeds, RM, cnt, cand, smax, smin, jmax, jmin, flags};
    wide_b_kernel<<<grid, kWT, smem, c->stream>>>(static_cast<const float *>(v.X), v.ld, v.n, tile, L ? *L : Lz, B, K,
                                                  D, lo, hi, mg, L ? nullptr : v.ids, p);
    return after_launch(c, "tighten pass B (wide)");
}

kc_status launch_wide_ball_all(kc_ctx *c, const View &v, const float *lo, const float *hi, int B, const Margins &mg,
                               const float *blo, const float *bhi, const int *allhave, const int64_t *seeds,
                               unsigned long long *cnt, unsigned long long *cand, unsigned *smax, unsigned *smin,
                               unsigned *jmax, unsigned *jmin, unsigned *flags, VisitScratch *vs)
{
    const int K = c->K, D = c->D;
    if (v.n <= 0 || B <= 0) return KC_OK;
    if (v.n > (int64_t)UINT32_MAX) return set_err(c, KC_EINVAL, "every-sample tightening: at most 2^32 - 1 samples");
    const size_t BK = (size_t)B * K;
    // counts, then offsets (host prefix), then the lists
    const size_t o_off = (BK * 8 + 255) & ~(size_t)255, o_pool = o_off + (((BK + 1) * 8 + 255) & ~(size_t)255);
    KC_TRY(ensure(c, vs->jbuf, o_pool));
    unsigned long long *jcnt = static_cast<unsigned long long *>(vs->jbuf.p);
    const int tile = (int)std::max<int64_t>(64, std::min<int64_t>(1024, (48 * 1024) / (8 * (int64_t)D)) / 32 * 32);
    const size_t smemJ = (size_t)D * tile * 8 + (size_t)K * D * 8;
    if (smemJ > 48 * 1024)
        KC_CUDA(c, cudaFuncSetAttribute(jall_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemJ));
    int per_sm = 0;
    KC_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, jall_kernel, kWT, smemJ));
    if (per_sm < 1) return set_err(c, KC_EINTERNAL, "every-sample tightening: list kernel does not fit");
    const int gJ = (int)std::max<int64_t>(1, std::min<int64_t>((v.n + tile - 1) / tile, (int64_t)per_sm * c->num_sms));
    const float *X = static_cast<const float *>(v.X);
    KC_CUDA(c, cudaMemsetAsync(jcnt, 0, BK * 8, c->stream));
    jall_kernel<<<gJ, kWT, smemJ, c->stream>>>(X, v.ld, v.n, tile, B, K, D, lo, hi, mg, v.ids, seeds, jcnt, nullptr,
                                                nullptr);
    KC_TRY(after_launch(c, "every-sample tightening: set sizes"));
    std::vector<unsigned long long> hc(BK);
    std::vector<int64_t> ho(BK + 1);
    KC_CUDA(c, cudaMemcpyAsync(hc.data(), jcnt, BK * 8, cudaMemcpyDeviceToHost, c->stream));
    KC_CUDA(c, cudaStreamSynchronize(c->stream));
    ho[0] = 0;
    for (size_t i = 0; i < BK; ++i) ho[i + 1] = ho[i] + (int64_t)hc[i];
    KC_TRY(ensure(c, vs->jbuf, o_pool + (size_t)std::max<int64_t>(1, ho[BK]) * 4));
    jcnt = static_cast<unsigned long long *>(vs->jbuf.p);
    int64_t *joff = reinterpret_cast<int64_t *>(static_cast<char *>(vs->jbuf.p) + o_off);
    uint32_t *jpool = reinterpret_cast<uint32_t *>(static_cast<char *>(vs->jbuf.p) + o_pool);
    KC_CUDA(c, cudaMemcpyAsync(joff, ho.data(), (BK + 1) * 8, cudaMemcpyHostToDevice, c->stream));
    KC_CUDA(c, cudaMemsetAsync(jcnt, 0, BK * 8, c->stream));
    jall_kernel<<<gJ, kWT, smemJ, c->stream>>>(X, v.ld, v.n, tile, B, K, D, lo, hi, mg, v.ids, seeds, jcnt, joff,
                                                jpool);
    KC_TRY(after_launch(c, "every-sample tightening: sets"));
    // the tiled pass
    const size_t KD = (size_t)K * D;
    const size_t smemB = (size_t)D * kWT * 8 + KD * 8 + KD * 12 + (size_t)kJC * D * 4 + KD * 16 + 8 + (size_t)K * 16 + 8;
    if ((v.n + kWT - 1) / kWT > (int64_t)INT32_MAX || B > 65535)
        return set_err(c, KC_EINVAL, "every-sample tightening: grid too large");
    if (D > kAllMaxD) return set_err(c, KC_EINVAL, "every-sample tightening: D <= %d", kAllMaxD);
    const dim3 grid((unsigned)((v.n + kWT - 1) / kWT), (unsigned)B);
    WideB p{blo, bhi, nullptr, nullptr, allhave, seeds, 0, cnt, cand, smax, smin, jmax, jmin, flags};
    auto kern = D <= 2 ? ball_all_kernel<2> : D <= 4 ? ball_all_kernel<4> : D <= 8 ? ball_all_kernel<8>
                                                                              : ball_all_kernel<16>;
    if (smemB > 48 * 1024)
        KC_CUDA(c, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smemB));
    kern<<<grid, kWT, smemB, c->stream>>>(X, v.ld, v.n, K, D, lo, hi, mg, v.ids, joff, jpool, p);
    // keep the host vectors alive until the copies they feed have run
    KC_CUDA(c, cudaStreamSynchronize(c->stream));
    return after_launch(c, "every-sample tightening: tiled pass");
}

}  // namespace kc
