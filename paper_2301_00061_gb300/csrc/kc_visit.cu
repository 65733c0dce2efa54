// kc_visit.cu -- cluster assignment and bounds tightening of a batch of nodes
// (Section 4.1, Algorithms 3 and 4) and sample reduction (Section 4.2,
// Algorithm 5).
//
// Layout of the work: each CTA stages a tile of samples in shared memory;
// each warp takes one node at a time and sweeps the whole tile with per-lane
// register accumulators, then reduces them across the warp once per (node,
// tile) and merges them into global accumulators with atomics.  Extremes that
// must also name a sample (the representatives) are (value, position) keys:
// packed into 64 bits and merged with 64-bit atomics for float data; for
// double data (two words) the kernels run as one CTA whose warps own disjoint
// nodes, and the owning lane merges them without atomics.
//
// Float data take every exclusion only where the float evaluation proves it:
// a distance d evaluated as d' satisfies d' (1 - g) <= d <= d' / (1 - g), so
//   d > t is proved by  RD(d' * (1 - g)) - slack > RU(t),
// and a sample is kept in a ball unless the same test proves it is outside.
// Double data decide exactly as a serial double evaluation.
#include <cuda_runtime.h>

#include "kc_device.cuh"
#include "kc_internal.cuh"

namespace kc {

namespace {

constexpr int NWV = kThreads / 32;

// ------------------------------------------------------------------- keys

template <typename T>
struct Key;

template <>
struct Key<float> {
    using K = unsigned long long;
    __device__ static K none() { return 0ull; }
    __device__ static K max_of(float v, uint32_t p) { return ((K)ord_f32(v) << 32) | (K)(0xFFFFFFFFu - p); }
    __device__ static K min_of(float v, uint32_t p) { return ((K)(~ord_f32(v)) << 32) | (K)(0xFFFFFFFFu - p); }
    __device__ static bool gt(const K &a, const K &b) { return a > b; }
    __device__ static bool is_none(const K &a) { return a == 0ull; }
    __device__ static K shfl(const K &a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
    __device__ static float vmax(const K &k) { return unord_f32((uint32_t)(k >> 32)); }
    __device__ static float vmin(const K &k) { return unord_f32(~(uint32_t)(k >> 32)); }
    __device__ static uint32_t pos(const K &k) { return 0xFFFFFFFFu - (uint32_t)k; }
    __device__ static void atomic_max(K *p, const K &v, unsigned *) { atomicMax(p, v); }
};

struct K128 {
    unsigned long long hi, lo;
};

template <>
struct Key<double> {
    using K = K128;
    __device__ static K none() { return K{0ull, 0ull}; }
    __device__ static K max_of(double v, uint32_t p) { return K{ord_f64(v), 0xFFFFFFFFull - p}; }
    __device__ static K min_of(double v, uint32_t p) { return K{~ord_f64(v), 0xFFFFFFFFull - p}; }
    __device__ static bool gt(const K &a, const K &b) { return a.hi > b.hi || (a.hi == b.hi && a.lo > b.lo); }
    __device__ static bool is_none(const K &a) { return a.hi == 0ull && a.lo == 0ull; }
    __device__ static K shfl(const K &a, int o)
    {
        return K{__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o)};
    }
    __device__ static double vmax(const K &k) { return unord_f64(k.hi); }
    __device__ static double vmin(const K &k) { return unord_f64(~k.hi); }
    __device__ static uint32_t pos(const K &k) { return (uint32_t)(0xFFFFFFFFull - k.lo); }
    // Double keys do not fit one 64-bit atomic.  The double-data kernels run
    // as a single CTA in which node b belongs to warp b % 8 alone, so lane 0
    // of that warp is the only writer of the node's keys: a plain
    // read-compare-write merge is race-free there.
    __device__ static void atomic_max(K *p, const K &v, unsigned *)
    {
        const K cur = *p;
        if (gt(v, cur)) *p = v;
    }
};

template <typename T>
__device__ __forceinline__ typename Key<T>::K kmax(const typename Key<T>::K &a, const typename Key<T>::K &b)
{
    return Key<T>::gt(a, b) ? a : b;
}

template <typename T>
__device__ __forceinline__ typename Key<T>::K warp_kmax(typename Key<T>::K v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = kmax<T>(v, Key<T>::shfl(v, o));
    return v;
}

// values as order-preserving unsigned integers (no position)
template <typename T>
using OrdT = typename std::conditional<sizeof(T) == 4, unsigned, unsigned long long>::type;
__device__ __forceinline__ float from_ord(unsigned u) { return unord_f32(u); }
__device__ __forceinline__ double from_ord(unsigned long long u) { return unord_f64(u); }

// ---------------------------------------------------- distance primitives

// Float clamp distance with padded compile-time DM (pairs beyond D add 0).
template <int DM>
__device__ __forceinline__ float box_dist_pad(const uint64_t *px, const uint64_t *bx)
{
    return box_dist_f32<DM>(px, bx);
}

// Double clamp distance in attribute order (the serial evaluation).
template <int DM>
__device__ __forceinline__ double box_dist_f64(const double *x, const double *lo, const double *hi, int D)
{
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < DM; ++a)
        if (a < D) {
            const double mu = mid3d(lo[a], x[a], hi[a]);
            const double d = __dsub_rn(x[a], mu);
            acc = __dadd_rn(acc, __dmul_rn(d, d));
        }
    return acc;
}

template <int DM>
__device__ __forceinline__ double pt_dist_f64(const double *x, const double *c, int D)
{
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < DM; ++a)
        if (a < D) {
            const double d = __dsub_rn(x[a], c[a]);
            acc = __dadd_rn(acc, __dmul_rn(d, d));
        }
    return acc;
}

// Farthest-corner distance (Eq. 13) for one box, float: per attribute
// max(|lo - x|, |x - hi|), squared and summed in the same two chains.
template <int DM>
__device__ __forceinline__ float corner_dist_f32(const uint64_t *px, const uint64_t *bx)
{
    uint64_t acc = 0;
#pragma unroll
    for (int a = 0; a + 1 < DM; a += 2) {
        const float2 t0 = upk(sub2(bx[a], px[a]));
        const float2 t1 = upk(sub2(bx[a + 1], px[a + 1]));
        const uint64_t m = pk(fmaxf(fabsf(t0.x), fabsf(t0.y)), fmaxf(fabsf(t1.x), fabsf(t1.y)));
        acc = fma2(m, m, acc);
    }
    float2 s = upk(acc);
    if (DM & 1) {
        const float2 t = upk(sub2(bx[DM - 1], px[DM - 1]));
        const float m = fmaxf(fabsf(t.x), fabsf(t.y));
        s.x = fmaf(m, m, s.x);
    }
    return s.x + s.y;
}

template <int DM>
__device__ __forceinline__ double corner_dist_f64(const double *x, const double *lo, const double *hi, int D)
{
    double acc = 0.0;
#pragma unroll
    for (int a = 0; a < DM; ++a)
        if (a < D) {
            const double mu = (fabs(__dsub_rn(lo[a], x[a])) > fabs(__dsub_rn(hi[a], x[a]))) ? lo[a] : hi[a];
            const double d = __dsub_rn(x[a], mu);
            acc = __dadd_rn(acc, __dmul_rn(d, d));
        }
    return acc;
}

// Proof helpers for float evaluations (see the file comment).
__device__ __forceinline__ bool proved_gt(float dhat, float defl, float slack, float t_up)
{
    return __fsub_rd(__fmul_rd(dhat, defl), slack) > t_up;
}
__device__ __forceinline__ bool proved_lt(float dhat, float infl, float slack, float t_dn)
{
    return __fadd_ru(__fmul_ru(dhat, infl), slack) < t_dn;
}


// ------------------------------------------------------------ pass A
//
// pass_a_node: one warp's share of one node over a staged tile of samples
// (j = j0, j0 + step, ... < tn).  Keys name a sample by tids[j] when the tile
// was gathered from a list of sample ids, else by its position base + j.

// Float data keep the node's arg-extreme keys in the warp's shared-memory
// slot sk, updated with atomics that a plain read skips when they cannot
// change the value, and merged into global memory at the end of the node:
// per cluster and attribute (max, min) at sk [K][D][2], then, with ndir > 0,
// per cluster and pair direction at sk [2KD + (k ndir + q) 2] -- the keys of
// x_a + x_b and x_a - x_b (added in float) for the first ndir / 2 attribute
// pairs a < b in lexicographic order, merged into dmax / dmin [B][K][ndir].
// Double data keep the attribute keys in registers (no directions).
struct WarpKeys {
    int ndir;
    unsigned long long *sk;
    unsigned long long *__restrict__ dmax, *__restrict__ dmin;
};

// u64 words of a warp's key slot
__host__ __device__ constexpr int warp_key_words(int K, int D, int ndir) { return 2 * K * D + 2 * K * ndir; }

// Raise the float key at `slot` (max) and `slot + 1` (min) by value v of the
// sample at position pos.  A key's high word is the ordered value, so a 32-bit
// read of it decides all but the ties; the stored keys only grow, so a stale
// read can only cost an atomic that changes nothing.
__device__ __forceinline__ void raise_keys(unsigned long long *slot, float v, uint32_t pos)
{
    const uint32_t o = ord_f32(v);
    const uint32_t *w = reinterpret_cast<const uint32_t *>(slot);   // little-endian: high words at 1, 3
    if (o >= w[1]) {
        const unsigned long long k = ((unsigned long long)o << 32) | (unsigned long long)(0xFFFFFFFFu - pos);
        if (k > slot[0]) atomicMax(&slot[0], k);
    }
    if (~o >= w[3]) {
        const unsigned long long k = ((unsigned long long)(~o) << 32) | (unsigned long long)(0xFFFFFFFFu - pos);
        if (k > slot[1]) atomicMax(&slot[1], k);
    }
}

template <typename T, int KM, int DM>
__device__ __forceinline__ void pass_a_node(const uint64_t *tp, const double *td, int tile, int tn, int j0, int step,
                                            const uint32_t *tids, int64_t base, const T *__restrict__ lo,
                                            const T *__restrict__ hi, int b, int K, int D, double alpha,
                                            const Margins &mg, typename Key<T>::K *__restrict__ lbkey,
                                            typename Key<T>::K *__restrict__ amax, typename Key<T>::K *__restrict__ amin,
                                            unsigned *__restrict__ flags, const WarpKeys &dk)
{
    using KT = Key<T>;
    using KY = typename KT::K;
    constexpr bool F32 = sizeof(T) == 4;
    const int lane = threadIdx.x & 31;
    if constexpr (F32) {
        for (int i = lane; i < warp_key_words(K, D, dk.ndir); i += 32) dk.sk[i] = 0ull;
        __syncwarp();
    }
    // node boxes into registers
    uint64_t bx[KM][DM];
    double blo[KM][DM], bhi[KM][DM];
#pragma unroll
    for (int k = 0; k < KM; ++k)
#pragma unroll
        for (int a = 0; a < DM; ++a) {
            const bool in = k < K && a < D;
            const size_t o = ((size_t)b * K + k) * D + a;
            if constexpr (F32) {
                bx[k][a] = in ? pk((float)lo[o], -(float)hi[o]) : pk(0.f, -0.f);
            } else {
                blo[k][a] = in ? (double)lo[o] : 0.0;
                bhi[k][a] = in ? (double)hi[o] : 0.0;
            }
        }
    KY acc_lb = KT::none();
    KY acc_max[F32 ? 1 : KM][DM], acc_min[F32 ? 1 : KM][DM];   // double data only
    if constexpr (!F32) {
#pragma unroll
        for (int k = 0; k < KM; ++k)
#pragma unroll
            for (int a = 0; a < DM; ++a) { acc_max[k][a] = KT::none(); acc_min[k][a] = KT::none(); }
    }
    bool infeasible = false;
    for (int j = j0; j < tn; j += step) {
        const uint32_t pos = tids ? tids[j] : (uint32_t)(base + j);
        T x[DM];
        uint64_t px[DM];
#pragma unroll
        for (int a = 0; a < DM; ++a) {
            if constexpr (F32) {
                px[a] = a < D ? tp[(size_t)a * tile + j] : pk(0.f, -0.f);
                x[a] = upk(px[a]).x;
            } else {
                x[a] = a < D ? td[(size_t)a * tile + j] : 0.0;
            }
        }
        T bmin = T(0);
        int left = 0, k1 = -1;
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            if (k < K) {
                T v;
                bool excl;
                if constexpr (F32) {
                    v = box_dist_pad<DM>(px, bx[k]);
                    excl = v > mg.t_alpha;
                } else {
                    v = box_dist_f64<DM>(reinterpret_cast<const double *>(x), blo[k], bhi[k], D);
                    excl = v > alpha;
                }
                bmin = (k == 0 || v < bmin) ? v : bmin;
                if (!excl) { ++left; k1 = k; }
            }
        }
        acc_lb = kmax<T>(acc_lb, KT::max_of(bmin, pos));
        if (left == 0) infeasible = true;
        if (left == 1) {
            if constexpr (!F32) {
#pragma unroll
                for (int k = 0; k < KM; ++k)
                    if (k == k1) {
#pragma unroll
                        for (int a = 0; a < DM; ++a)
                            if (a < D) {
                                acc_max[k][a] = kmax<T>(acc_max[k][a], KT::max_of(x[a], pos));
                                acc_min[k][a] = kmax<T>(acc_min[k][a], KT::min_of(x[a], pos));
                            }
                    }
            } else {
                unsigned long long *sa = dk.sk + (size_t)k1 * D * 2;
#pragma unroll
                for (int a = 0; a < DM; ++a)
                    if (a < D) raise_keys(sa + 2 * a, x[a], pos);
                if (dk.ndir > 0) {
                    unsigned long long *s = dk.sk + (size_t)2 * K * D + (size_t)k1 * dk.ndir * 2;
                    int q = 0;
#pragma unroll
                    for (int a = 0; a < DM; ++a)
#pragma unroll
                        for (int c = a + 1; c < DM; ++c)
                            if (c < D && q < dk.ndir) {
                                raise_keys(s + 2 * q, __fadd_rn(x[a], x[c]), pos);
                                raise_keys(s + 2 * q + 2, __fsub_rn(x[a], x[c]), pos);
                                q += 2;
                            }
                }
            }
        }
    }
    // warp reduction, then one atomic per accumulator and warp
    acc_lb = warp_kmax<T>(acc_lb);
    if (lane == 0 && !KT::is_none(acc_lb)) KT::atomic_max(&lbkey[b], acc_lb, &flags[b]);
    if constexpr (!F32) {
#pragma unroll
        for (int k = 0; k < KM; ++k)
#pragma unroll
            for (int a = 0; a < DM; ++a)
                if (k < K && a < D) {
                    const KY m1 = warp_kmax<T>(acc_max[k][a]);
                    const KY m2 = warp_kmax<T>(acc_min[k][a]);
                    const size_t o = ((size_t)b * K + k) * D + a;
                    if (lane == 0 && !KT::is_none(m1)) KT::atomic_max(&amax[o], m1, &flags[b]);
                    if (lane == 0 && !KT::is_none(m2)) KT::atomic_max(&amin[o], m2, &flags[b]);
                }
    }
    if (__any_sync(0xffffffffu, infeasible) && lane == 0) atomicOr(&flags[b], 1u);
    if constexpr (F32) {
        __syncwarp();
        for (int i = lane; i < K * D; i += 32) {
            const size_t o = (size_t)b * K * D + i;
            if (dk.sk[2 * i]) atomicMax(&amax[o], dk.sk[2 * i]);
            if (dk.sk[2 * i + 1]) atomicMax(&amin[o], dk.sk[2 * i + 1]);
        }
        const unsigned long long *sd = dk.sk + (size_t)2 * K * D;
        for (int i = lane; i < K * dk.ndir; i += 32) {
            const size_t o = (size_t)b * K * dk.ndir + i;
            if (sd[2 * i]) atomicMax(&dk.dmax[o], sd[2 * i]);
            if (sd[2 * i + 1]) atomicMax(&dk.dmin[o], sd[2 * i + 1]);
        }
        __syncwarp();   // the slot is rewritten by the warp's next node
    }
}

// Stages samples of a tile in shared memory: float data as (x, -x) pairs,
// double data as values.  ids: gather by sample id (list mode), else rows
// base .. base + tn of the view.
template <typename T>
__device__ __forceinline__ void stage_tile_a(const T *__restrict__ X, int64_t ld, int D, int tile, int tn, int64_t base,
                                             const uint32_t *ids, uint64_t *tp, double *td)
{
    for (int i = threadIdx.x; i < D * tile; i += kThreads) {
        const int a = i / tile, j = i - a * tile;
        T v = T(0);
        if (j < tn) v = ids ? X[(size_t)a * ld + ids[j]] : X[(size_t)a * ld + base + j];
        if constexpr (sizeof(T) == 4) tp[i] = pk(v, -v);
        else td[i] = v;
    }
}

template <typename T, int KM, int DM>
__global__ void __launch_bounds__(kThreads)
visit_a_kernel(const T *__restrict__ X, int64_t ld, int64_t n, int tile, const T *__restrict__ lo,
               const T *__restrict__ hi, int B, int K, int D, double alpha, Margins mg,
               typename Key<T>::K *__restrict__ lbkey, typename Key<T>::K *__restrict__ amax,
               typename Key<T>::K *__restrict__ amin, unsigned *__restrict__ flags, int ndir,
               unsigned long long *__restrict__ dmax, unsigned long long *__restrict__ dmin)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *tp = reinterpret_cast<uint64_t *>(smem);
    double *td = reinterpret_cast<double *>(smem);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // per-warp key slots after the tile
    const WarpKeys dk{ndir,
                      reinterpret_cast<unsigned long long *>(smem + (size_t)D * tile * 8) +
                          (size_t)warp * warp_key_words(K, D, ndir),
                      dmax, dmin};
    for (int64_t base = (int64_t)blockIdx.x * tile; base < n; base += (int64_t)gridDim.x * tile) {
        const int tn = (int)((n - base) < (int64_t)tile ? (n - base) : (int64_t)tile);
        __syncthreads();
        stage_tile_a<T>(X, ld, D, tile, tn, base, nullptr, tp, td);
        __syncthreads();
        for (int b = warp; b < B; b += NWV)
            pass_a_node<T, KM, DM>(tp, td, tile, tn, lane, 32, nullptr, base, lo, hi, b, K, D, alpha, mg, lbkey, amax,
                                   amin, flags, dk);
    }
}

// List mode: work item w = one tile of a group's sample-id list (see
// ListBatch); the CTA evaluates every node of the group on the staged tile.
template <typename T, int KM, int DM>
__global__ void __launch_bounds__(kThreads, 3)
visit_a_list_kernel(const T *__restrict__ X, int64_t ld, ListBatch L, int tile,
                    const T *__restrict__ lo, const T *__restrict__ hi, int K, int D, double alpha, Margins mg,
                    typename Key<T>::K *__restrict__ lbkey, typename Key<T>::K *__restrict__ amax,
                    typename Key<T>::K *__restrict__ amin, unsigned *__restrict__ flags, int ndir,
                    unsigned long long *__restrict__ dmax, unsigned long long *__restrict__ dmin)
{
    extern __shared__ __align__(16) unsigned char smem[];
    uint64_t *tp = reinterpret_cast<uint64_t *>(smem);
    double *td = reinterpret_cast<double *>(smem);
    uint32_t *tids = reinterpret_cast<uint32_t *>(smem + (size_t)D * tile * 8);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // per-warp key slots after the ids (tile is a multiple of 32)
    const WarpKeys dk{ndir, reinterpret_cast<unsigned long long *>(tids + tile) + (size_t)warp * warp_key_words(K, D, ndir),
                      dmax, dmin};
    for (int64_t w = blockIdx.x; w < L.W; w += gridDim.x) {
        int b;
        int64_t st;
        list_item(L.tile_prefix, L.B, w, tile, &b, &st);
        const int64_t nb = L.seg_n[b];
        const int tn = (int)((nb - st) < (int64_t)tile ? (nb - st) : (int64_t)tile);
        __syncthreads();
        for (int j = threadIdx.x; j < tn; j += kThreads) tids[j] = L.pool[L.seg_off[b] + st + j];
        __syncthreads();
        stage_tile_a<T>(X, ld, D, tile, tn, 0, tids, tp, td);
        __syncthreads();
        // the group's nodes share the tile: min(G, warps) teams of warps, team
        // t takes nodes n0 + t, n0 + t + teams, ... over the whole tile
        const int n0 = L.node_start ? L.node_start[b] : b, n1 = L.node_start ? L.node_start[b + 1] : b + 1;
        const int teams = (n1 - n0) < NWV ? (n1 - n0) : NWV, wpt = NWV / teams, team = warp / wpt;
        if (team < teams)
            for (int nd = n0 + team; nd < n1; nd += teams)
                pass_a_node<T, KM, DM>(tp, td, tile, tn, (warp % wpt) * 32 + lane, wpt * 32, tids, 0, lo, hi, nd, K, D,
                                       alpha, mg, lbkey, amax, amin, flags, dk);
    }
}

// ------------------------------------------------------- finalize pass A

template <typename T>
__device__ __forceinline__ T round_dn(double v)
{
    if constexpr (sizeof(T) == 4) return __double2float_rd(v);
    else return v;
}
template <typename T>
__device__ __forceinline__ T round_up(double v)
{
    if constexpr (sizeof(T) == 4) return __double2float_ru(v);
    else return v;
}

struct FinA {
    const int64_t *seeds;       // [K] original ids or null
    const uint32_t *ids;        // view position -> id, or null
    double r_up;                // sqrt(alpha) rounded up
    double alpha;
    double defl, slack;         // certified lower-bound deflation
    double seed_defl;           // float data: deflation of the seed test (1 for double)
    int cap, RM;
    // float data, wide path: arg-extreme keys along the attribute-pair
    // directions [B][K][ndir] (direction q: pair q / 2 of the pairs a < b in
    // lexicographic order, x_a + x_b for even q, x_a - x_b for odd q)
    int ndir;
    const unsigned long long *dmax, *dmin;
};

template <typename T>
__global__ void finalize_a_kernel(int B, int K, int D, const T *__restrict__ lo, const T *__restrict__ hi,
                                  const typename Key<T>::K *__restrict__ lbkey,
                                  const typename Key<T>::K *__restrict__ amax,
                                  const typename Key<T>::K *__restrict__ amin, unsigned *__restrict__ flags,
                                  const T *__restrict__ Xf, int64_t ldf, FinA f, T *__restrict__ blo,
                                  T *__restrict__ bhi, int64_t *__restrict__ reps, int *__restrict__ nreps,
                                  T *__restrict__ repx, int *__restrict__ allhave, double *__restrict__ lb,
                                  double *__restrict__ lb_raw, int64_t *__restrict__ lbarg)
{
    using KT = Key<T>;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    bool inf = (flags[b] & 1u) != 0;
    // lower bound of the input box
    {
        const auto k = lbkey[b];
        const bool none = KT::is_none(k);
        const double raw = none ? 0.0 : (double)KT::vmax(k);
        if (lb_raw) lb_raw[b] = raw;
        if (lb) lb[b] = fmax(0.0, __dsub_rd(__dmul_rd(raw, f.defl), f.slack));
        if (lbarg) {
            const int64_t p = none ? -1 : (int64_t)KT::pos(k);
            lbarg[b] = (p < 0 || !f.ids) ? p : (int64_t)f.ids[p];
        }
    }
    int have = 1;
    for (int k = 0; k < K; ++k) {
        const size_t o0 = ((size_t)b * K + k) * D;
        int64_t seed = f.seeds ? f.seeds[k] : -1;
        if (seed >= 0) {
            // seed consistency: box k farther than alpha from seed k
            double acc = 0.0;
            for (int a = 0; a < D; ++a) {
                const double x = (double)Xf[(size_t)a * ldf + seed];
                const double mu = mid3d((double)lo[o0 + a], x, (double)hi[o0 + a]);
                const double d = __dsub_rn(x, mu);
                acc = __dadd_rn(acc, __dmul_rn(d, d));
            }
            if (__dmul_rd(acc, f.seed_defl) > f.alpha) inf = true;
        }
        bool nonempty = seed >= 0;
        int64_t amin_id[kMaxD], amax_id[kMaxD];
        for (int a = 0; a < D; ++a) {
            const size_t o = o0 + a;
            double vmx = 0, vmn = 0;
            int64_t imx = -1, imn = -1;
            if (!KT::is_none(amax[o])) {
                vmx = (double)KT::vmax(amax[o]);
                const int64_t p = KT::pos(amax[o]);
                imx = f.ids ? (int64_t)f.ids[p] : p;
                vmn = (double)KT::vmin(amin[o]);
                const int64_t q = KT::pos(amin[o]);
                imn = f.ids ? (int64_t)f.ids[q] : q;
                nonempty = true;
            }
            if (seed >= 0) {
                const double sx = (double)Xf[(size_t)a * ldf + seed];
                if (imx < 0 || sx > vmx || (sx == vmx && seed < imx)) { vmx = sx; imx = seed; }
                if (imn < 0 || sx < vmn || (sx == vmn && seed < imn)) { vmn = sx; imn = seed; }
            }
            amin_id[a] = imn;
            amax_id[a] = imx;
            T l = lo[o], h = hi[o];
            if (imx >= 0) {
                const T l2 = round_dn<T>(nextafter(__dsub_rn(vmx, f.r_up), -__builtin_huge_val()));
                const T h2 = round_up<T>(nextafter(__dadd_rn(vmn, f.r_up), __builtin_huge_val()));
                if (l2 > l) l = l2;
                if (h2 < h) h = h2;
            }
            if (l > h) inf = true;
            blo[o] = l;
            bhi[o] = h;
        }
        // representatives: seed, then arg-min / arg-max of each attribute
        int nr = 0;
        int64_t *rp = reps + ((size_t)b * K + k) * f.RM;
        auto add = [&](int64_t v) {
            if (v < 0 || nr >= f.cap) return;
            for (int q = 0; q < nr; ++q)
                if (rp[q] == v) return;
            rp[nr++] = v;
        };
        add(seed);
        if (nonempty)
            for (int a = 0; a < D; ++a) {
                add(amin_id[a]);
                add(amax_id[a]);
            }
        if constexpr (sizeof(T) == 4) {
            // then the arg-min and arg-max along each pair direction, the seed
            // taking part as an assigned sample of cluster k
            int pa = 0, pb = 1;
            for (int q = 0; q < f.ndir && nonempty && nr < f.cap; ++q) {
                if (q > 0 && !(q & 1)) {
                    if (++pb == D) { ++pa; pb = pa + 1; }
                }
                const size_t o = ((size_t)b * K + k) * f.ndir + q;
                float vmx = 0.f, vmn = 0.f;
                int64_t imx = -1, imn = -1;
                if (!KT::is_none(f.dmax[o])) {
                    vmx = KT::vmax(f.dmax[o]);
                    const int64_t p = KT::pos(f.dmax[o]);
                    imx = f.ids ? (int64_t)f.ids[p] : p;
                    vmn = KT::vmin(f.dmin[o]);
                    const int64_t p2 = KT::pos(f.dmin[o]);
                    imn = f.ids ? (int64_t)f.ids[p2] : p2;
                }
                if (seed >= 0) {
                    const float xa = Xf[(size_t)pa * ldf + seed], xb = Xf[(size_t)pb * ldf + seed];
                    const float sv = (q & 1) ? __fsub_rn(xa, xb) : __fadd_rn(xa, xb);
                    if (imx < 0 || sv > vmx || (sv == vmx && seed < imx)) { vmx = sv; imx = seed; }
                    if (imn < 0 || sv < vmn || (sv == vmn && seed < imn)) { vmn = sv; imn = seed; }
                }
                add(imn);
                add(imx);
            }
        }
        for (int q = nr; q < f.RM; ++q) rp[q] = -1;
        nreps[(size_t)b * K + k] = nr;
        T *rx = repx + ((size_t)b * K + k) * f.RM * D;
        for (int q = 0; q < nr; ++q)
            for (int a = 0; a < D; ++a) rx[(size_t)q * D + a] = Xf[(size_t)a * ldf + rp[q]];
        if (nr == 0) have = 0;
    }
    allhave[b] = have;
    if (inf) atomicOr(&flags[b], 1u);
}

// ------------------------------------------------------------ pass B
//
// Only two kinds of samples need representative distances: samples that the
// center-based rule left unassigned (the sample-based rule tests them against
// every representative) and samples inside some box M'^k (the ball test of
// cluster k).  Each warp first flags its slice of the tile and compacts the
// flagged samples into a list in shared memory, then processes the list with
// every lane busy.

constexpr int kSub = 256;   // samples flagged per warp before processing

// Per-warp shared-memory state of pass B for one node: the node's boxes
// (read by every lane, so kept once per warp instead of once per thread) and
// the warp's running bounding boxes, merged into global memory at the end.
template <typename T, int KM, int DM>
struct PBSlot {
    uint64_t bx[KM][DM];                 // float data: packed (lo, -hi) of the input boxes
    T ilo[KM][DM], ihi[KM][DM];          // double data: input boxes
    T l[KM][DM], h[KM][DM], mid[KM][DM]; // box-BT boxes and their midpoints
    OrdT<T> smax[KM][DM], smin[KM][DM];  // bbox of S_+ (ordered integers)
    OrdT<T> jmax[KM][DM], jmin[KM][DM];  // bbox of the sample-based assigned samples
};

__device__ __forceinline__ unsigned to_ord(float v) { return ord_f32(v); }
__device__ __forceinline__ unsigned long long to_ord(double v) { return ord_f64(v); }

// Words of one staged representative: float data packs coordinate pairs
// (DM + 1) / 2 u64, double data keeps DM values.
template <typename T, int DM>
constexpr int rep_words() { return sizeof(T) == 4 ? (DM + 1) / 2 : DM; }

template <typename T, int KM, int DM>
__device__ __forceinline__ void pass_b_node(const T *tx, int tile, int tn, int jstart, int wstep, const uint32_t *tids,
                                            const uint32_t *__restrict__ ids, int64_t base, uint32_t *list,
                                            PBSlot<T, KM, DM> *ws, uint64_t *wrep, int b, int K, int D, int RM,
                                            const T *__restrict__ lo_in, const T *__restrict__ hi_in,
                                            const T *__restrict__ blo, const T *__restrict__ bhi,
                                            const T *__restrict__ repx, const int *__restrict__ nreps,
                                            const int *__restrict__ allhave, double alpha, const Margins &mg,
                                            const int64_t *seed_id, unsigned long long *__restrict__ cnt,
                                            OrdT<T> *__restrict__ smax, OrdT<T> *__restrict__ smin,
                                            OrdT<T> *__restrict__ jmax, OrdT<T> *__restrict__ jmin,
                                            typename Key<T>::K *__restrict__ cand, unsigned *__restrict__ flags)
{
    using KT = Key<T>;
    using KY = typename KT::K;
    using OT = OrdT<T>;
    constexpr bool F32 = sizeof(T) == 4;
    constexpr int DH = (DM + 1) / 2;
    const int lane = threadIdx.x & 31;
    const double four_alpha = 4.0 * alpha;
    // node b: input boxes (center-based status), box-BT boxes, midpoints
    for (int i = lane; i < KM * DM; i += 32) {
        const int k = i / DM, a = i % DM;
        const bool in = k < K && a < D;
        const size_t o = ((size_t)b * K + k) * D + a;
        if constexpr (F32) ws->bx[k][a] = in ? pk((float)lo_in[o], -(float)hi_in[o]) : pk(0.f, -0.f);
        else { ws->ilo[k][a] = in ? lo_in[o] : T(0); ws->ihi[k][a] = in ? hi_in[o] : T(0); }
        const T lv = in ? blo[o] : T(0), hv = in ? bhi[o] : T(0);
        ws->l[k][a] = lv;
        ws->h[k][a] = hv;
        if constexpr (F32) ws->mid[k][a] = (float)(0.5 * ((double)lv + (double)hv));
        else ws->mid[k][a] = 0.5 * (lv + hv);
        ws->smax[k][a] = (OT)0;
        ws->smin[k][a] = ~(OT)0;
        ws->jmax[k][a] = (OT)0;
        ws->jmin[k][a] = ~(OT)0;
    }
    int nr[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) nr[k] = k < K ? nreps[(size_t)b * K + k] : 0;
    const bool have = allhave[b] != 0;
    // the node's representatives into the warp's slot wrep [K][RM][words]
    constexpr int RW = rep_words<T, DM>();
    {
        const T *rxb = repx + (size_t)b * K * RM * D;
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            if (k >= K) continue;
            const T *src = rxb + (size_t)k * RM * D;
            for (int i = lane; i < nr[k] * RW; i += 32) {
                const int r = i / RW, p = i - r * RW;
                if constexpr (F32) {
                    const float v0 = 2 * p < D ? (float)src[(size_t)r * D + 2 * p] : 0.f;
                    const float v1 = 2 * p + 1 < D ? (float)src[(size_t)r * D + 2 * p + 1] : 0.f;
                    wrep[((size_t)k * RM + r) * RW + p] = pk(v0, v1);
                } else {
                    const double v = p < D ? (double)src[(size_t)r * D + p] : 0.0;
                    wrep[((size_t)k * RM + r) * RW + p] = (uint64_t)__double_as_longlong(v);
                }
            }
        }
    }
    unsigned long long c_cnt[KM];
    KY c_cand[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        c_cnt[k] = 0;
        c_cand[k] = KT::none();
    }
    __syncwarp();
    bool infeasible = false;
    for (int r0 = jstart; r0 < tn; r0 += 8 * wstep) {
        // phase 1: flag the samples that need representative distances
        int count = 0;
        for (int g = 0; g < 8; ++g) {
            const int jb = r0 + g * wstep;
            if (jb >= tn) break;   // uniform across the warp
            const int j = jb + lane;
            uint32_t fl = 0u;
            if (j < tn) {
                T x[DM];
#pragma unroll
                for (int a = 0; a < DM; ++a) x[a] = a < D ? tx[(size_t)a * tile + j] : T(0);
                // clusters the center-based rule leaves open (only needed when the
                // sample-based rule can run: every cluster has representatives)
                int left = 0;
#pragma unroll
                for (int k = 0; k < KM; ++k)
                    if (have && k < K) {
                        bool excl;
                        if constexpr (F32) {
                            uint64_t px[DM];
#pragma unroll
                            for (int a = 0; a < DM; ++a) px[a] = pk(x[a], -x[a]);
                            excl = box_dist_f32<DM>(px, ws->bx[k]) > mg.t_alpha;
                        } else {
                            excl = box_dist_f64<DM>(reinterpret_cast<const double *>(x),
                                                    reinterpret_cast<const double *>(ws->ilo[k]),
                                                    reinterpret_cast<const double *>(ws->ihi[k]), D) > alpha;
                        }
                        if (!excl) ++left;
                    }
                if (have && left >= 2) {
                    // the seeds count as assigned in every node
                    const int64_t id = tids ? (int64_t)tids[j] : (ids ? (int64_t)ids[base + j] : base + j);
                    bool is_seed = false;
#pragma unroll
                    for (int k = 0; k < KM; ++k)
                        if (seed_id[k] == id) is_seed = true;
                    if (!is_seed) fl |= 1u;
                }
#pragma unroll
                for (int k = 0; k < KM; ++k)
                    if (k < K) {
                        bool inb = true;
#pragma unroll
                        for (int a = 0; a < DM; ++a)
                            if (a < D && (x[a] < ws->l[k][a] || x[a] > ws->h[k][a])) inb = false;
                        if (inb) fl |= 2u << k;
                    }
            }
            const unsigned bal = __ballot_sync(0xffffffffu, fl != 0u);
            if (fl) list[count + __popc(bal & ((1u << lane) - 1u))] = (uint32_t)j | (fl << 16);
            count += __popc(bal);
        }
        __syncwarp();
        // phase 2: representative distances of the flagged samples
        for (int e = lane; e < count; e += 32) {
            const uint32_t ent = list[e];
            const int j = (int)(ent & 0xFFFFu);
            const uint32_t fl = ent >> 16;
            const uint32_t pos = tids ? tids[j] : (uint32_t)(base + j);
            T x[DM];
#pragma unroll
            for (int a = 0; a < DM; ++a) x[a] = a < D ? tx[(size_t)a * tile + j] : T(0);
            uint64_t px[DH];
            if constexpr (F32) {
#pragma unroll
                for (int p = 0; p < DH; ++p) px[p] = pk(x[2 * p], 2 * p + 1 < DM ? x[2 * p + 1] : 0.f);
            }
            // distances to the representatives of the clusters that need them:
            // far4[k] = some representative of k proved farther than 4 alpha
            // (Lemma 2), far1[k] = some proved farther than alpha (ball test).
            // Chunks of 4 representatives are decided by their largest
            // distance (a short last chunk repeats the last representative);
            // far4 implies far1, so a cluster's scan stops at its first far4,
            // or at its first far1 when only the ball test needs it
            const T th1 = F32 ? (T)mg.t_alpha : (T)alpha, th4 = F32 ? (T)mg.t_four : (T)four_alpha;
            bool far4[KM], far1[KM];
#pragma unroll
            for (int k = 0; k < KM; ++k) {
                far4[k] = far1[k] = false;
                const bool need = k < K && ((fl & 1u) || (fl & (2u << k)));
                if (!need) continue;
                const bool want4 = (fl & 1u) != 0u;
                const uint64_t *rk = wrep + (size_t)k * RM * RW;
                const int nk = nr[k];
                for (int r0 = 0; r0 < nk; r0 += 4) {
                    T d[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int r = r0 + u < nk ? r0 + u : nk - 1;
                        if constexpr (F32) d[u] = pt_dist_f32<2 * DH>(px, rk + (size_t)r * RW);
                        else
                            d[u] = pt_dist_f64<DM>(reinterpret_cast<const double *>(x),
                                                   reinterpret_cast<const double *>(rk + (size_t)r * RW), D);
                    }
                    T m;
                    if constexpr (F32) m = fmaxf(fmaxf(d[0], d[1]), fmaxf(d[2], d[3]));
                    else m = fmax(fmax(d[0], d[1]), fmax(d[2], d[3]));
                    if (m > th1) {
                        far1[k] = true;
                        if (m > th4) { far4[k] = true; break; }
                        if (!want4) break;
                    }
                }
            }
            // sample-based assignment of an unassigned sample (Algorithm 3, Lemma 2)
            if (fl & 1u) {
                int left = 0, k1 = -1;
#pragma unroll
                for (int k = 0; k < KM; ++k)
                    if (k < K && !far4[k]) { ++left; k1 = k; }
                if (left == 0) infeasible = true;
                if (left == 1)
                    for (int a = 0; a < D; ++a) {
                        // a plain read skips the atomics that cannot change the value
                        const OT v = to_ord(x[a]);
                        if (v > ws->jmax[k1][a]) atomicMax(&ws->jmax[k1][a], v);
                        if (v < ws->jmin[k1][a]) atomicMin(&ws->jmin[k1][a], v);
                    }
            }
            // ball-based tightening and centers on samples (Algorithm 4)
#pragma unroll
            for (int k = 0; k < KM; ++k)
                if (k < K && (fl & (2u << k))) {
                    if (far1[k]) continue;
                    ++c_cnt[k];
                    for (int a = 0; a < D; ++a) {
                        const OT v = to_ord(x[a]);
                        if (v > ws->smax[k][a]) atomicMax(&ws->smax[k][a], v);
                        if (v < ws->smin[k][a]) atomicMin(&ws->smin[k][a], v);
                    }
                    T dm;
                    if constexpr (F32) {
                        uint64_t pm[DH];
#pragma unroll
                        for (int p = 0; p < DH; ++p)
                            pm[p] = pk(ws->mid[k][2 * p], 2 * p + 1 < DM ? ws->mid[k][2 * p + 1] : 0.f);
                        dm = pt_dist_f32<2 * DH>(px, pm);
                    } else {
                        dm = pt_dist_f64<DM>(reinterpret_cast<const double *>(x),
                                             reinterpret_cast<const double *>(ws->mid[k]), D);
                    }
                    c_cand[k] = kmax<T>(c_cand[k], KT::min_of(dm, pos));
                }
        }
        __syncwarp();
    }
    // reduce and merge
#pragma unroll
    for (int k = 0; k < KM; ++k)
        if (k < K) {
            unsigned long long cn = c_cnt[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) cn += __shfl_xor_sync(0xffffffffu, cn, o);
            const KY cd = warp_kmax<T>(c_cand[k]);
            const size_t ok_ = (size_t)b * K + k;
            if (lane == 0 && cn) atomicAdd(&cnt[ok_], cn);
            if (lane == 0 && !KT::is_none(cd)) KT::atomic_max(&cand[ok_], cd, &flags[b]);
        }
    __syncwarp();
    for (int i = lane; i < K * D; i += 32) {
        const int k = i / D, a = i % D;
        const size_t o = ((size_t)b * K + k) * D + a;
        if (ws->smax[k][a] != (OT)0) atomicMax(&smax[o], ws->smax[k][a]);
        if (ws->smin[k][a] != ~(OT)0) atomicMin(&smin[o], ws->smin[k][a]);
        if (ws->jmax[k][a] != (OT)0) atomicMax(&jmax[o], ws->jmax[k][a]);
        if (ws->jmin[k][a] != ~(OT)0) atomicMin(&jmin[o], ws->jmin[k][a]);
    }
    __syncwarp();   // the slot is rewritten by the warp's next node
    if (__any_sync(0xffffffffu, infeasible) && lane == 0) atomicOr(&flags[b], 1u);
}

template <typename T, int KM, int DM>
__global__ void __launch_bounds__(kThreads, 3)
visit_b_kernel(const T *__restrict__ X, int64_t ld, int64_t n, int tile, int B, int K, int D, int RM,
               const T *__restrict__ lo_in, const T *__restrict__ hi_in, const T *__restrict__ blo,
               const T *__restrict__ bhi, const T *__restrict__ repx, const int *__restrict__ nreps,
               const int *__restrict__ allhave, double alpha, Margins mg, const int64_t *__restrict__ seeds,
               const uint32_t *__restrict__ ids, unsigned long long *__restrict__ cnt,
               OrdT<T> *__restrict__ smax, OrdT<T> *__restrict__ smin, OrdT<T> *__restrict__ jmax,
               OrdT<T> *__restrict__ jmin, typename Key<T>::K *__restrict__ cand, unsigned *__restrict__ flags)
{
    int64_t seed_id[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) seed_id[k] = (seeds && k < K) ? seeds[k] : -1;
    extern __shared__ __align__(16) unsigned char smem[];
    T *tx = reinterpret_cast<T *>(smem);                                        // [D][tile]
    uint32_t *lists = reinterpret_cast<uint32_t *>(tx + (size_t)D * tile);      // [warps][kSub]
    auto *slots = reinterpret_cast<PBSlot<T, KM, DM> *>(lists + NWV * kSub);   // [warps]
    const int warp = threadIdx.x >> 5;
    uint32_t *list = lists + warp * kSub;
    uint64_t *wrep = reinterpret_cast<uint64_t *>(slots + NWV) + (size_t)warp * KM * RM * rep_words<T, DM>();
    for (int64_t base = (int64_t)blockIdx.x * tile; base < n; base += (int64_t)gridDim.x * tile) {
        const int tn = (int)((n - base) < (int64_t)tile ? (n - base) : (int64_t)tile);
        __syncthreads();
        for (int i = threadIdx.x; i < D * tile; i += kThreads) {
            const int a = i / tile, j = i - a * tile;
            tx[i] = j < tn ? X[(size_t)a * ld + base + j] : T(0);
        }
        __syncthreads();
        for (int b = warp; b < B; b += NWV)
            pass_b_node<T, KM, DM>(tx, tile, tn, 0, 32, nullptr, ids, base, list, slots + warp, wrep, b, K, D, RM,
                                        lo_in, hi_in, blo, bhi, repx, nreps, allhave, alpha, mg, seed_id, cnt, smax,
                                        smin, jmax, jmin, cand, flags);
    }
}

// List mode of pass B (see visit_a_list_kernel).
template <typename T, int KM, int DM>
__global__ void __launch_bounds__(kThreads, 3)
visit_b_list_kernel(const T *__restrict__ X, int64_t ld, ListBatch L, int tile, int K,
                    int D, int RM, const T *__restrict__ lo_in, const T *__restrict__ hi_in, const T *__restrict__ blo,
                    const T *__restrict__ bhi, const T *__restrict__ repx, const int *__restrict__ nreps,
                    const int *__restrict__ allhave, double alpha, Margins mg, const int64_t *__restrict__ seeds,
                    unsigned long long *__restrict__ cnt, OrdT<T> *__restrict__ smax, OrdT<T> *__restrict__ smin,
                    OrdT<T> *__restrict__ jmax, OrdT<T> *__restrict__ jmin, typename Key<T>::K *__restrict__ cand,
                    unsigned *__restrict__ flags)
{
    int64_t seed_id[KM];
#pragma unroll
    for (int k = 0; k < KM; ++k) seed_id[k] = (seeds && k < K) ? seeds[k] : -1;
    extern __shared__ __align__(16) unsigned char smem[];
    T *tx = reinterpret_cast<T *>(smem);                                        // [D][tile]
    uint32_t *lists = reinterpret_cast<uint32_t *>(tx + (size_t)D * tile);      // [warps][kSub]
    auto *slots = reinterpret_cast<PBSlot<T, KM, DM> *>(lists + NWV * kSub);   // [warps]
    uint32_t *tids = reinterpret_cast<uint32_t *>(slots + NWV);                 // [tile]
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t *list = lists + warp * kSub;
    // [warps][KM][RM][words] after the ids (tile is a multiple of 32)
    uint64_t *wrep = reinterpret_cast<uint64_t *>(tids + tile) + (size_t)warp * KM * RM * rep_words<T, DM>();
    for (int64_t w = blockIdx.x; w < L.W; w += gridDim.x) {
        int b;
        int64_t st;
        list_item(L.tile_prefix, L.B, w, tile, &b, &st);
        const int64_t nb = L.seg_n[b];
        const int tn = (int)((nb - st) < (int64_t)tile ? (nb - st) : (int64_t)tile);
        __syncthreads();
        for (int j = threadIdx.x; j < tn; j += kThreads) tids[j] = L.pool[L.seg_off[b] + st + j];
        __syncthreads();
        for (int i = threadIdx.x; i < D * tile; i += kThreads) {
            const int a = i / tile, j = i - a * tile;
            tx[i] = j < tn ? X[(size_t)a * ld + tids[j]] : T(0);
        }
        __syncthreads();
        const int n0 = L.node_start ? L.node_start[b] : b, n1 = L.node_start ? L.node_start[b + 1] : b + 1;
        const int teams = (n1 - n0) < NWV ? (n1 - n0) : NWV, wpt = NWV / teams, team = warp / wpt;
        if (team < teams)
            for (int nd = n0 + team; nd < n1; nd += teams)
                pass_b_node<T, KM, DM>(tx, tile, tn, (warp % wpt) * 32, wpt * 32, tids, nullptr, 0, list,
                                       slots + warp, wrep, nd, K, D, RM, lo_in, hi_in, blo, bhi, repx, nreps, allhave,
                                       alpha, mg, seed_id, cnt, smax, smin, jmax, jmin, cand, flags);
        (void)lane;
    }
}

template <typename T>
__global__ void finalize_b_kernel(int B, int K, int D, const unsigned long long *__restrict__ cnt,
                                  const OrdT<T> *__restrict__ smax, const OrdT<T> *__restrict__ smin,
                                  const OrdT<T> *__restrict__ jmax, const OrdT<T> *__restrict__ jmin,
                                  const typename Key<T>::K *__restrict__ cand, const unsigned *__restrict__ flags,
                                  const uint32_t *__restrict__ ids, double r_up, T *__restrict__ lo_out,
                                  T *__restrict__ hi_out, int64_t *__restrict__ counts, int64_t *__restrict__ cand_out,
                                  int8_t *__restrict__ status)
{
    using KT = Key<T>;
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= B) return;
    bool inf = (flags[b] & 1u) != 0;
    bool leaf = true;
    const OrdT<T> NONE_MAX = 0, NONE_MIN = (OrdT<T>)~(OrdT<T>)0;
    for (int k = 0; k < K; ++k) {
        const size_t ok = (size_t)b * K + k;
        if (counts) counts[ok] = (int64_t)cnt[ok];
        if (cnt[ok] == 0) inf = true;
        if (cand_out) {
            const auto c = cand[ok];
            const int64_t p = KT::is_none(c) ? -1 : (int64_t)KT::pos(c);
            cand_out[ok] = (p < 0 || !ids) ? p : (int64_t)ids[p];
        }
        for (int a = 0; a < D; ++a) {
            const size_t o = ok * D + a;
            T l, h;
            if (cnt[ok] == 0) {
                l = T(1);
                h = T(0);
            } else {
                l = from_ord(smin[o]);
                h = from_ord(smax[o]);
            }
            if (jmax[o] != NONE_MAX && jmin[o] != NONE_MIN) {
                const double vmx = (double)from_ord(jmax[o]), vmn = (double)from_ord(jmin[o]);
                const T l2 = round_dn<T>(nextafter(__dsub_rn(vmx, r_up), -__builtin_huge_val()));
                const T h2 = round_up<T>(nextafter(__dadd_rn(vmn, r_up), __builtin_huge_val()));
                if (l2 > l) l = l2;
                if (h2 < h) h = h2;
            }
            if (!(l <= h)) inf = true;
            if (h > l) leaf = false;
            lo_out[o] = l;
            hi_out[o] = h;
        }
    }
    status[b] = inf ? 1 : (leaf ? 2 : 0);
}

// ------------------------------------------------------ sample reduction

template <typename T, int KM, int DM>
__global__ void __launch_bounds__(kThreads)
sr_kernel(const T *__restrict__ X, int64_t ld, int64_t n, int M, int K, int D, const T *__restrict__ lo,
          const T *__restrict__ hi, const T *__restrict__ repx, const int *__restrict__ nreps, int R,
          double beta_glob, double alpha, Margins mg, uint8_t *__restrict__ mask,
          unsigned long long *__restrict__ n_active)
{
    constexpr bool F32 = sizeof(T) == 4;
    unsigned long long kept = 0;
    for (int64_t s = (int64_t)blockIdx.x * kThreads + threadIdx.x; s < n; s += (int64_t)gridDim.x * kThreads) {
        if (!mask[s]) continue;
        T x[DM];
        uint64_t px[DM];
#pragma unroll
        for (int a = 0; a < DM; ++a) {
            x[a] = a < D ? X[(size_t)a * ld + s] : T(0);
            if constexpr (F32) px[a] = pk(x[a], -x[a]);
        }
        bool redundant = true;
        for (int m = 0; m < M && redundant; ++m) {
            // redundant for the lower bound: alpha_s(M) < beta_glob (Eq. 13)
            T as = T(0);
            for (int k = 0; k < K; ++k) {
                const size_t o = ((size_t)m * K + k) * D;
                T v;
                if constexpr (F32) {
                    uint64_t bx[DM];
#pragma unroll
                    for (int a = 0; a < DM; ++a) bx[a] = a < D ? pk(lo[o + a], -hi[o + a]) : pk(0.f, -0.f);
                    v = corner_dist_f32<DM>(px, bx);
                } else {
                    double l[DM], h[DM];
#pragma unroll
                    for (int a = 0; a < DM; ++a) { l[a] = a < D ? lo[o + a] : 0.0; h[a] = a < D ? hi[o + a] : 0.0; }
                    v = corner_dist_f64<DM>(reinterpret_cast<const double *>(x), l, h, D);
                }
                as = (k == 0 || v < as) ? v : as;
            }
            bool lb_red;
            if constexpr (F32) lb_red = proved_lt(as, mg.infl, mg.slack, mg.beta_dn);
            else lb_red = as < beta_glob;
            if (!lb_red) { redundant = false; break; }
            // redundant for the upper bound: x outside M^k, or some representative farther than alpha
            for (int k = 0; k < K && redundant; ++k) {
                const size_t o = ((size_t)m * K + k) * D;
                bool inb = true;
#pragma unroll
                for (int a = 0; a < DM; ++a)
                    if (a < D && (x[a] < lo[o + a] || x[a] > hi[o + a])) inb = false;
                if (!inb) continue;
                bool excl = false;
                const int nr = nreps ? nreps[(size_t)m * K + k] : 0;
                for (int r = 0; r < nr && !excl; ++r) {
                    const T *c = repx + (((size_t)m * K + k) * R + r) * D;
                    if constexpr (F32) {
                        uint64_t pxx[(DM + 1) / 2], pc[(DM + 1) / 2];
#pragma unroll
                        for (int p = 0; p < (DM + 1) / 2; ++p) {
                            pxx[p] = pk(x[2 * p], 2 * p + 1 < DM ? x[2 * p + 1] : 0.f);
                            pc[p] = pk(2 * p < D ? c[2 * p] : 0.f, 2 * p + 1 < D ? c[2 * p + 1] : 0.f);
                        }
                        const float d = pt_dist_f32<2 * ((DM + 1) / 2)>(pxx, pc);
                        excl = proved_gt(d, mg.defl, mg.slack, mg.alpha_up);
                    } else {
                        double cc[DM];
#pragma unroll
                        for (int a = 0; a < DM; ++a) cc[a] = a < D ? c[a] : 0.0;
                        excl = pt_dist_f64<DM>(reinterpret_cast<const double *>(x), cc, D) > alpha;
                    }
                }
                if (!excl) redundant = false;
            }
        }
        if (redundant) mask[s] = 0;
        else ++kept;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) kept += __shfl_xor_sync(0xffffffffu, kept, o);
    if ((threadIdx.x & 31) == 0 && kept) atomicAdd(n_active, kept);
}

__global__ void gather_reps_kernel(int M, int K, int D, int R, const int64_t *__restrict__ reps,
                                   const void *__restrict__ Xf, int64_t ldf, int f32, void *__restrict__ repx,
                                   int *__restrict__ nreps)
{
    const int mk = blockIdx.x * blockDim.x + threadIdx.x;
    if (mk >= M * K) return;
    int nr = 0;
    for (int r = 0; r < R; ++r) {
        const int64_t id = reps[(size_t)mk * R + r];
        if (id < 0) continue;
        for (int a = 0; a < D; ++a) {
            const size_t dst = ((size_t)mk * R + nr) * D + a;
            if (f32) static_cast<float *>(repx)[dst] = static_cast<const float *>(Xf)[(size_t)a * ldf + id];
            else static_cast<double *>(repx)[dst] = static_cast<const double *>(Xf)[(size_t)a * ldf + id];
        }
        ++nr;
    }
    nreps[mk] = nr;
}

// ------------------------------------------------------------ host side

template <typename F>
kc_status grid_of(kc_ctx *c, F fn, size_t smem, int64_t work, int *grid)
{
    if (smem > 48 * 1024)
        KC_CUDA(c, cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int per_sm = 0;
    KC_CUDA(c, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kThreads, smem));
    if (per_sm < 1) return set_err(c, KC_EINTERNAL, "tightening kernel does not fit (smem %zu)", smem);
    int64_t g = (int64_t)per_sm * c->num_sms;
    if (g > work) g = work;
    *grid = (int)(g < 1 ? 1 : g);
    return KC_OK;
}

Margins make_margins(kc_ctx *c, double alpha, double beta_glob)
{
    Margins m{};
    const double g = gamma_n(f32_roundings(c->D), kU32);
    m.defl = (float)(1.0 - g);
    if ((double)m.defl > 1.0 - g) m.defl = nextafterf(m.defl, 0.f);
    m.infl = (float)(1.0 / (1.0 - g));
    if ((double)m.infl < 1.0 / (1.0 - g)) m.infl = nextafterf(m.infl, 2.f);
    m.slack = (float)((c->D + 2) * 1.401298464324817e-45);
    auto up = [](double v) {
        float f = (float)v;
        if ((double)f < v) f = nextafterf(f, __builtin_huge_valf());
        return f;
    };
    auto dn = [](double v) {
        float f = (float)v;
        if ((double)f > v) f = nextafterf(f, -__builtin_huge_valf());
        return f;
    };
    m.alpha_up = up(alpha);
    m.four_up = up(4.0 * alpha);
    m.beta_dn = dn(beta_glob);
    m.t_alpha = up(((double)m.alpha_up + (double)m.slack) / (double)m.defl * (1.0 + 1e-6));
    m.t_four = up(((double)m.four_up + (double)m.slack) / (double)m.defl * (1.0 + 1e-6));
    return m;
}

int reps_cap(int D, int cap) { return std::min(cap, std::min(kMaxReps, 2 * D + 1)); }

// Attribute-pair directions of the representatives: 2 min(D(D-1)/2, 16).
int pair_dirs(int D) { return 2 * std::min(D * (D - 1) / 2, kMaxPairs); }

// Representatives per cluster: min(cap, 2D + 1, 50) along the attributes,
// or, with pair directions (ndir > 0), up to min(cap, 50, 2D + 1 + 2 ndir).
int reps_slots(int D, int cap, int ndir)
{
    return std::max(1, ndir > 0 ? std::min(std::min(cap, kMaxReps), 1 + 2 * D + 2 * ndir) : reps_cap(D, cap));
}

template <typename T, int KM, int DM>
kc_status tighten_impl(kc_ctx *c, const View &v, const void *lo_, const void *hi_, int B, double alpha,
                       const int64_t *seeds, int cap, bool dirs, void *lo_out_, void *hi_out_, int64_t *counts,
                       int64_t *cand_out, double *lb, double *lb_raw, int64_t *lbarg, int8_t *status, VisitScratch *vs,
                       const ListBatch *L = nullptr)
{
    using KY = typename Key<T>::K;
    const int K_ = c->K, D = c->D;
    const int ndir = (dirs && sizeof(T) == 4) ? pair_dirs(D) : 0;
    const int RM = reps_slots(D, cap, ndir);
    const T *lo = static_cast<const T *>(lo_);
    const T *hi = static_cast<const T *>(hi_);
    const size_t KD = (size_t)B * K_ * D, BK = (size_t)B * K_;
    // workspace
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_lbkey = take(B * sizeof(KY)), o_amax = take(KD * sizeof(KY)), o_amin = take(KD * sizeof(KY));
    const size_t o_flags = take(B * 4), o_blo = take(KD * sizeof(T)), o_bhi = take(KD * sizeof(T));
    const size_t o_reps = take(BK * RM * 8), o_nreps = take(BK * 4), o_repx = take(BK * RM * D * sizeof(T));
    const size_t o_have = take(B * 4), o_cnt = take(BK * 8), o_smax = take(KD * sizeof(OrdT<T>));
    const size_t o_smin = take(KD * sizeof(OrdT<T>)), o_jmax = take(KD * sizeof(OrdT<T>));
    const size_t o_jmin = take(KD * sizeof(OrdT<T>)), o_cand = take(BK * sizeof(KY));
    const size_t o_dmax = take(BK * ndir * 8), o_dmin = take(BK * ndir * 8);
    KC_TRY(ensure(c, vs->buf, off));
    char *w = static_cast<char *>(vs->buf.p);
    KY *lbkey = reinterpret_cast<KY *>(w + o_lbkey), *amax = reinterpret_cast<KY *>(w + o_amax);
    KY *amin = reinterpret_cast<KY *>(w + o_amin), *cand = reinterpret_cast<KY *>(w + o_cand);
    unsigned long long *dmax = reinterpret_cast<unsigned long long *>(w + o_dmax);
    unsigned long long *dmin = reinterpret_cast<unsigned long long *>(w + o_dmin);
    unsigned *flags = reinterpret_cast<unsigned *>(w + o_flags);
    T *blo = reinterpret_cast<T *>(w + o_blo), *bhi = reinterpret_cast<T *>(w + o_bhi);
    int64_t *reps = reinterpret_cast<int64_t *>(w + o_reps);
    int *nreps = reinterpret_cast<int *>(w + o_nreps), *have = reinterpret_cast<int *>(w + o_have);
    T *repx = reinterpret_cast<T *>(w + o_repx);
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(w + o_cnt);
    OrdT<T> *smax = reinterpret_cast<OrdT<T> *>(w + o_smax), *smin = reinterpret_cast<OrdT<T> *>(w + o_smin);
    OrdT<T> *jmax = reinterpret_cast<OrdT<T> *>(w + o_jmax), *jmin = reinterpret_cast<OrdT<T> *>(w + o_jmin);
    // zero everything up to the min accumulators, which start at all-ones
    KC_CUDA(c, cudaMemsetAsync(w, 0, o_smin, c->stream));
    KC_CUDA(c, cudaMemsetAsync(w + o_smin, 0xFF, o_jmax - o_smin, c->stream));
    KC_CUDA(c, cudaMemsetAsync(w + o_jmax, 0, o_jmin - o_jmax, c->stream));
    KC_CUDA(c, cudaMemsetAsync(w + o_jmin, 0xFF, o_cand - o_jmin, c->stream));
    KC_CUDA(c, cudaMemsetAsync(w + o_cand, 0, off - o_cand, c->stream));

    const Margins mg = make_margins(c, alpha, 0.0);
    const double r_up = nextafter(std::sqrt(alpha), __builtin_huge_val());
    // pass A
    const int tileA = (int)std::max<int64_t>(256, std::min<int64_t>(2048, (64 * 1024) / (D * 8)) / 32 * 32);
    const size_t dkA = sizeof(T) == 4 ? (size_t)NWV * warp_key_words(K_, D, ndir) * 8 : 0;   // per-warp key slots
    const size_t smemA = (size_t)D * tileA * 8 + dkA;
    int gA = 1;
    const int64_t tilesA = (v.n + tileA - 1) / tileA;
    auto kA = visit_a_kernel<T, KM, DM>;
    if (L) {
        // list mode (float data): one node per work item, tile = list_tile() gathered ids
        if constexpr (sizeof(T) == 4) {
            const int lt = list_tile();
            const size_t smem = (size_t)D * lt * 8 + (size_t)lt * 4 + dkA;
            auto kAL = visit_a_list_kernel<T, KM, DM>;
            int g = 1;
            KC_TRY(grid_of(c, kAL, smem, std::max<int64_t>(1, L->W), &g));
            if (L->W > 0) {
                kAL<<<g, kThreads, smem, c->stream>>>(static_cast<const T *>(c->X), c->ldx, *L, lt, lo, hi, K_, D,
                                                      alpha, mg, lbkey, amax, amin, flags, ndir, dmax, dmin);
                KC_TRY(after_launch(c, "tighten pass A (lists)"));
            }
        } else {
            return set_err(c, KC_EINTERNAL, "list-mode tightening is for float data");
        }
    } else {
        KC_TRY(grid_of(c, kA, smemA, tilesA, &gA));
        if (sizeof(T) == 8) gA = 1;   // single-writer key merge (see Key<double>)
        if (v.n > 0) {
            kA<<<gA, kThreads, smemA, c->stream>>>(static_cast<const T *>(v.X), v.ld, v.n, tileA, lo, hi, B, K_, D,
                                                  alpha, mg, lbkey, amax, amin, flags, ndir, dmax, dmin);
            KC_TRY(after_launch(c, "tighten pass A"));
        }
    }
    FinA fa;
    fa.seeds = seeds;
    fa.ids = L ? nullptr : v.ids;   // list-mode keys already hold sample ids
    fa.r_up = r_up;
    fa.alpha = alpha;
    fa.defl = deflate_factor(c->dt, D);
    fa.slack = underflow_slack(c->dt, D);
    fa.seed_defl = sizeof(T) == 4 ? 1.0 - gamma_n(f64_roundings(D), kU64) : 1.0;
    fa.cap = RM;
    fa.RM = RM;
    fa.ndir = ndir;
    fa.dmax = dmax;
    fa.dmin = dmin;
    finalize_a_kernel<T><<<(B + 127) / 128, 128, 0, c->stream>>>(
        B, K_, D, lo, hi, lbkey, amax, amin, flags, static_cast<const T *>(c->X), c->ldx, fa, blo, bhi, reps, nreps,
        repx, have, lb, lb_raw, lbarg);
    KC_TRY(after_launch(c, "tighten finalize A"));
    // pass B
    const int tileB = (int)std::max<int64_t>(256, std::min<int64_t>(2048, (32 * 1024) / (D * (int64_t)sizeof(T))) / 32 * 32);
    static_assert(kThreads / 32 * kSub * 4 <= 16 * 1024, "pass B lists");
    const size_t slotB = (size_t)NWV * sizeof(PBSlot<T, KM, DM>);
    const size_t repB = (size_t)NWV * KM * RM * rep_words<T, DM>() * 8;   // per-warp representatives
    const size_t smemB = (size_t)D * tileB * sizeof(T) + (size_t)NWV * kSub * 4 + slotB + repB;
    int gB = 1;
    auto kB = visit_b_kernel<T, KM, DM>;
    if (L) {
        if constexpr (sizeof(T) == 4) {
            const int lt = list_tile();
            const size_t smem = (size_t)D * lt * sizeof(T) + (size_t)NWV * kSub * 4 + slotB + (size_t)lt * 4 + repB;
            auto kBL = visit_b_list_kernel<T, KM, DM>;
            int g = 1;
            KC_TRY(grid_of(c, kBL, smem, std::max<int64_t>(1, L->W), &g));
            if (L->W > 0) {
                kBL<<<g, kThreads, smem, c->stream>>>(static_cast<const T *>(c->X), c->ldx, *L, lt, K_, D, RM, lo, hi,
                                                      blo, bhi, repx, nreps, have, alpha, mg, seeds, cnt, smax, smin,
                                                      jmax, jmin, cand, flags);
                KC_TRY(after_launch(c, "tighten pass B (lists)"));
            }
        }
    } else {
    KC_TRY(grid_of(c, kB, smemB, (v.n + tileB - 1) / tileB, &gB));
    if (sizeof(T) == 8) gB = 1;   // single-writer key merge (see Key<double>)
    if (v.n > 0) {
        kB<<<gB, kThreads, smemB, c->stream>>>(static_cast<const T *>(v.X), v.ld, v.n, tileB, B, K_, D, RM, lo, hi, blo,
                                              bhi, repx, nreps, have, alpha, mg, seeds, v.ids, cnt, smax, smin, jmax, jmin,
                                              cand, flags);
        KC_TRY(after_launch(c, "tighten pass B"));
    }
    }
    finalize_b_kernel<T><<<(B + 127) / 128, 128, 0, c->stream>>>(B, K_, D, cnt, smax, smin, jmax, jmin, cand, flags,
                                                                L ? nullptr : v.ids, r_up, static_cast<T *>(lo_out_),
                                                                static_cast<T *>(hi_out_), counts, cand_out, status);
    KC_TRY(after_launch(c, "tighten finalize B"));
    vs->reps = reps;
    vs->nreps = nreps;
    vs->repx = repx;
    vs->RM = RM;
    return KC_OK;
}

// The wide path (float data, K <= 16, D <= 128): the workspace, finalize
// kernels and outputs of tighten_impl, passes A and B from kc_wide.cu.
// Representatives per cluster: min(cap, 2D + 1, 50) along the attributes, or,
// with `dirs`, up to min(cap, 50) with the attribute-pair directions after
// the attributes.
kc_status tighten_wide(kc_ctx *c, const View &v, const void *lo_, const void *hi_, int B, double alpha,
                       const int64_t *seeds, int cap, bool dirs, void *lo_out_, void *hi_out_, int64_t *counts,
                       int64_t *cand_out, double *lb, double *lb_raw, int64_t *lbarg, int8_t *status, VisitScratch *vs,
                       const ListBatch *L = nullptr, bool all_balls = false)
{
    using T = float;
    using KY = unsigned long long;
    const int K_ = c->K, D = c->D;
    const int ndir = dirs ? pair_dirs(D) : 0;
    const int RM = reps_slots(D, cap, ndir);
    const T *lo = static_cast<const T *>(lo_);
    const T *hi = static_cast<const T *>(hi_);
    const size_t KD = (size_t)B * K_ * D, BK = (size_t)B * K_;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~(size_t)255;
        return o;
    };
    const size_t o_lbkey = take(B * sizeof(KY)), o_amax = take(KD * sizeof(KY)), o_amin = take(KD * sizeof(KY));
    const size_t o_flags = take(B * 4), o_blo = take(KD * sizeof(T)), o_bhi = take(KD * sizeof(T));
    const size_t o_reps = take(BK * RM * 8), o_nreps = take(BK * 4), o_repx = take(BK * RM * D * sizeof(T));
    const size_t o_have = take(B * 4), o_cnt = take(BK * 8), o_smax = take(KD * 4);
    const size_t o_smin = take(KD * 4), o_jmax = take(KD * 4);
    const size_t o_jmin = take(KD * 4), o_cand = take(BK * sizeof(KY));
    const size_t o_dmax = take(BK * ndir * sizeof(KY)), o_dmin = take(BK * ndir * sizeof(KY));
    KC_TRY(ensure(c, vs->buf, off));
    char *w = static_cast<char *>(vs->buf.p);
    KY *lbkey = reinterpret_cast<KY *>(w + o_lbkey), *amax = reinterpret_cast<KY *>(w + o_amax);
    KY *amin = reinterpret_cast<KY *>(w + o_amin), *cand = reinterpret_cast<KY *>(w + o_cand);
    KY *dmax = reinterpret_cast<KY *>(w + o_dmax), *dmin = reinterpret_cast<KY *>(w + o_dmin);
    unsigned *flags = reinterpret_cast<unsigned *>(w + o_flags);
    T *blo = reinterpret_cast<T *>(w + o_blo), *bhi = reinterpret_cast<T *>(w + o_bhi);
    int64_t *reps = reinterpret_cast<int64_t *>(w + o_reps);
    int *nreps = reinterpret_cast<int *>(w + o_nreps), *have = reinterpret_cast<int *>(w + o_have);
    T *repx = reinterpret_cast<T *>(w + o_repx);
    unsigned long long *cnt = reinterpret_cast<unsigned long long *>(w + o_cnt);
    unsigned *smax = reinterpret_cast<unsigned *>(w + o_smax), *smin = reinterpret_cast<unsigned *>(w + o_smin);
    unsigned *jmax = reinterpret_cast<unsigned *>(w + o_jmax), *jmin = reinterpret_cast<unsigned *>(w + o_jmin);
    KC_CUDA(c, cudaMemsetAsync(w, 0, o_smin, c->stream));
    KC_CUDA(c, cudaMemsetAsync(w + o_smin, 0xFF, o_jmax - o_smin, c->stream));
    KC_CUDA(c, cudaMemsetAsync(w + o_jmax, 0, o_jmin - o_jmax, c->stream));
    KC_CUDA(c, cudaMemsetAsync(w + o_jmin, 0xFF, o_cand - o_jmin, c->stream));
    KC_CUDA(c, cudaMemsetAsync(w + o_cand, 0, off - o_cand, c->stream));

    const Margins mg = make_margins(c, alpha, 0.0);
    const double r_up = nextafter(std::sqrt(alpha), __builtin_huge_val());
    KC_TRY(launch_wide_a(c, v, L, lo, hi, B, mg, lbkey, amax, amin, flags, ndir, dmax, dmin));
    FinA fa;
    fa.seeds = seeds;
    fa.ids = L ? nullptr : v.ids;
    fa.r_up = r_up;
    fa.alpha = alpha;
    fa.defl = deflate_factor(c->dt, D);
    fa.slack = underflow_slack(c->dt, D);
    fa.seed_defl = 1.0 - gamma_n(f64_roundings(D), kU64);
    fa.cap = RM;
    fa.RM = RM;
    fa.ndir = ndir;
    fa.dmax = dmax;
    fa.dmin = dmin;
    finalize_a_kernel<T><<<(B + 127) / 128, 128, 0, c->stream>>>(
        B, K_, D, lo, hi, lbkey, amax, amin, flags, static_cast<const T *>(c->X), c->ldx, fa, blo, bhi, reps, nreps,
        repx, have, lb, lb_raw, lbarg);
    KC_TRY(after_launch(c, "tighten finalize A"));
    if (all_balls)
        KC_TRY(launch_wide_ball_all(c, v, lo, hi, B, mg, blo, bhi, have, seeds, cnt, cand, smax, smin, jmax, jmin, flags,
                                    vs));
    else
        KC_TRY(launch_wide_b(c, v, L, lo, hi, B, mg, blo, bhi, repx, nreps, have, seeds, RM, cnt, cand, smax, smin,
                             jmax, jmin, flags));
    finalize_b_kernel<T><<<(B + 127) / 128, 128, 0, c->stream>>>(B, K_, D, cnt, smax, smin, jmax, jmin, cand, flags,
                                                                L ? nullptr : v.ids, r_up, static_cast<T *>(lo_out_),
                                                                static_cast<T *>(hi_out_), counts, cand_out, status);
    KC_TRY(after_launch(c, "tighten finalize B"));
    vs->reps = reps;
    vs->nreps = nreps;
    vs->repx = repx;
    vs->RM = RM;
    return KC_OK;
}

// Shape dispatch of the tightening: the register kernels for the shapes
// listed here, the shared-memory kernels (kc_wide.cu) for the other float
// shapes.  Representatives: at most ball_cap (<= 0: 50); float data keep the
// pair-direction keys whenever the cap can reach them (the attribute
// extremes may number fewer than 2D + 1 distinct samples), double data stop
// after the attribute extremes.
kc_status launch_tighten_any(kc_ctx *c, const View &v, const ListBatch *L, const void *lo, const void *hi, int B,
                             double alpha, const int64_t *seeds_dev, int ball_cap, void *lo_out, void *hi_out,
                             int64_t *counts, int64_t *cand, double *lb, double *lb_raw, int64_t *lbarg, int8_t *status,
                             VisitScratch *vs)
{
    if (B <= 0) return KC_OK;
    const int cap = ball_cap > 0 ? ball_cap : 50;
    const int K = c->K, D = c->D;
    const bool dirs = c->dt == KC_F32 && cap >= 2 && D >= 2;
    if (ball_cap == KC_BALLS_ALL) {
        // every sample of J_A^k a representative: the tiled pass of kc_wide.cu
        if (c->dt != KC_F32 || L || D > 16)
            return set_err(c, KC_EINVAL,
                           "ball_cap = KC_BALLS_ALL: float data, D <= 16, a shared sample set (D=%d)", D);
        return tighten_wide(c, v, lo, hi, B, alpha, seeds_dev, cap, dirs, lo_out, hi_out, counts, cand, lb, lb_raw,
                            lbarg, status, vs, nullptr, true);
    }
#define KC_TIGHTEN(T_, KM_, DM_)                                                                                      \
    return tighten_impl<T_, KM_, DM_>(c, v, lo, hi, B, alpha, seeds_dev, cap, dirs, lo_out, hi_out, counts, cand, lb, \
                                      lb_raw, lbarg, status, vs, L)
    if (c->dt == KC_F32) {
        if (K == 3 && D == 3) KC_TIGHTEN(float, 3, 3);
        if (K == 3 && D == 4) KC_TIGHTEN(float, 3, 4);
        if (K <= 4 && D <= 2) KC_TIGHTEN(float, 4, 2);
        if (K <= 4 && D <= 4) KC_TIGHTEN(float, 4, 4);
        if (K <= 2 && D <= 8) KC_TIGHTEN(float, 2, 8);
        return tighten_wide(c, v, lo, hi, B, alpha, seeds_dev, cap, dirs, lo_out, hi_out, counts, cand, lb, lb_raw,
                            lbarg, status, vs, L);
    }
    if (L) return set_err(c, KC_EINTERNAL, "list-mode tightening is for float data");
    if (K <= 4 && D <= 2) KC_TIGHTEN(double, 4, 2);
    if (K <= 4 && D <= 4) KC_TIGHTEN(double, 4, 4);
#undef KC_TIGHTEN
    return set_err(c, KC_EINVAL, "kc_tighten: double data supported for K <= 4, D <= 4 (K=%d, D=%d)", K, D);
}

}  // namespace

kc_status launch_tighten_view(kc_ctx *c, const View &v, const void *lo, const void *hi, int B, double alpha,
                              const int64_t *seeds_dev, int ball_cap, void *lo_out, void *hi_out, int64_t *counts,
                              int64_t *cand, double *lb, double *lb_raw, int64_t *lbarg, int8_t *status,
                              VisitScratch *vs)
{
    return launch_tighten_any(c, v, nullptr, lo, hi, B, alpha, seeds_dev, ball_cap, lo_out, hi_out, counts, cand, lb,
                              lb_raw, lbarg, status, vs);
}

kc_status launch_tighten_list(kc_ctx *c, const ListBatch &L, const void *lo, const void *hi, int B, double alpha,
                              const int64_t *seeds_dev, int ball_cap, void *lo_out, void *hi_out, int64_t *counts,
                              int64_t *cand, double *lb, double *lb_raw, int64_t *lbarg, int8_t *status,
                              VisitScratch *vs)
{
    if (c->dt != KC_F32) return set_err(c, KC_EINTERNAL, "list-mode tightening is for float data");
    return launch_tighten_any(c, full_view(c), &L, lo, hi, B, alpha, seeds_dev, ball_cap, lo_out, hi_out, counts,
                              cand, lb, lb_raw, lbarg, status, vs);
}

kc_status launch_sample_reduction_view(kc_ctx *c, const View &v, const void *lo, const void *hi, int M,
                                       const void *repx, const int *nreps, int R, double beta_glob, double alpha,
                                       uint8_t *mask, unsigned long long *n_active)
{
    if (c->D > 8) return set_err(c, KC_EINVAL, "sample reduction: supported for D <= 8");
    KC_CUDA(c, cudaMemsetAsync(n_active, 0, 8, c->stream));
    if (v.n == 0 || M <= 0) return KC_OK;
    const Margins mg = make_margins(c, alpha, beta_glob);
    const int64_t blocks = (v.n + kThreads - 1) / kThreads;
    const int grid = (int)std::min<int64_t>(blocks, (int64_t)c->num_sms * 8);
    if (c->dt == KC_F32) {
        if (c->D <= 4)
            sr_kernel<float, 16, 4><<<grid, kThreads, 0, c->stream>>>(
                static_cast<const float *>(v.X), v.ld, v.n, M, c->K, c->D, static_cast<const float *>(lo),
                static_cast<const float *>(hi), static_cast<const float *>(repx), nreps, R, beta_glob, alpha, mg, mask,
                n_active);
        else
            sr_kernel<float, 16, 8><<<grid, kThreads, 0, c->stream>>>(
                static_cast<const float *>(v.X), v.ld, v.n, M, c->K, c->D, static_cast<const float *>(lo),
                static_cast<const float *>(hi), static_cast<const float *>(repx), nreps, R, beta_glob, alpha, mg, mask,
                n_active);
    } else {
        if (c->D <= 4)
            sr_kernel<double, 16, 4><<<grid, kThreads, 0, c->stream>>>(
                static_cast<const double *>(v.X), v.ld, v.n, M, c->K, c->D, static_cast<const double *>(lo),
                static_cast<const double *>(hi), static_cast<const double *>(repx), nreps, R, beta_glob, alpha, mg,
                mask, n_active);
        else
            sr_kernel<double, 16, 8><<<grid, kThreads, 0, c->stream>>>(
                static_cast<const double *>(v.X), v.ld, v.n, M, c->K, c->D, static_cast<const double *>(lo),
                static_cast<const double *>(hi), static_cast<const double *>(repx), nreps, R, beta_glob, alpha, mg,
                mask, n_active);
    }
    return after_launch(c, "sample reduction");
}

kc_status launch_gather_reps(kc_ctx *c, int M, int R, const int64_t *reps, void *repx, int *nreps)
{
    if (M <= 0) return KC_OK;
    const int MK = M * c->K;
    gather_reps_kernel<<<(MK + 127) / 128, 128, 0, c->stream>>>(M, c->K, c->D, R, reps, c->X, c->ldx,
                                                                 c->dt == KC_F32, repx, nreps);
    return after_launch(c, "gather representatives");
}

}  // namespace kc
