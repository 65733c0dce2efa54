// kc_solve.cu -- the branch and bound of Algorithm 1 on the GPU, and the
// public entry points of the tightening (Algorithms 3-4) and sample
// reduction (Algorithm 5) kernels.
//
// Schedule of one batch (host control, all sample-level work in kernels):
//   1. pop up to B open nodes with the smallest (lower bound, id);
//   2. tighten them over the current sample set: certified lower bound of the
//      node, cluster assignment, box/ball bounds tightening, "centers on
//      samples" boxes, counts and an upper-bound candidate per cluster;
//   3. evaluate the candidates' objective (float screen, exact double value);
//   4. prune (bound >= incumbent), drop infeasible nodes, close leaves, and
//      branch the rest at the midpoint of the chosen variable (max range, or
//      the learned scorer's pick between two rules);
//   5. sample reduction (Section 4.2): with per-node lists (float data), the
//      branched node's list is filtered to the samples that are not
//      redundant for both bounds, and the same pass bounds both children over
//      it; with one shared sample set, every i_sr batches the set is reduced
//      against the hulls of the open nodes and compacted;
//   6. bound the children as they are created (those not bounded by the
//      filter get a bound launch over their list); only children below the
//      incumbent enter the open set, keyed by max(parent bound, own bound).
// A visited node's bound is evaluated again by the tightening pass, over the
// samples it holds then, and its key is the larger of the two.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <set>
#include <vector>

#include "kc_internal.cuh"

namespace kc {

namespace {

double now_s()
{
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

template <typename T>
T next_up(T v)
{
    return std::nextafter(v, std::numeric_limits<T>::infinity());
}

// Branching value (Section 3.3): the midpoint of [lo, hi] in the data's
// precision; children [lo, m] and [succ(m), hi] so each sample value falls in
// exactly one child and both children are strictly smaller.  Requires lo < hi.
template <typename T>
void split_point(T lo, T hi, T *m_out, T *succ_out)
{
    T m = (T)(0.5 * ((double)lo + (double)hi));
    if (m >= hi) m = lo;
    if (m < lo) m = lo;
    *m_out = m;
    *succ_out = next_up(m);
}

template <typename T>
struct Node {
    std::vector<T> lo, hi;   // [K][D]
    double key;              // certified lower bound known for the node
    int64_t id;
    int64_t parent;
    int depth;
    double pkey = 0.0;       // the parent's bound
    int64_t group = 0;       // its ancestor at depth 8 (itself above that depth)
    float prio = 0.f;        // learned priority (ties of equal keys: smaller first)
    int list = -1;           // handle of its surviving-sample list (per-node list mode)
    int64_t wit = -1;        // a sample whose distance to the node's boxes attains `key` (-1: none known)
    int8_t fwait = 0;        // generations still to skip list filtering (after filters that dropped little)
    int8_t fstreak = 0;      // consecutive such filters along the path
};

template <typename T>
struct NodeCmp {
    bool operator()(const Node<T> &a, const Node<T> &b) const
    {
        if (a.key != b.key) return a.key > b.key;
        if (a.prio != b.prio) return a.prio > b.prio;
        return a.id > b.id;
    }
};

// Squared distance in attribute order (double), for the seed test on host.
double sqdist_host(const std::vector<double> &x, const std::vector<double> &y)
{
    double acc = 0.0;
    for (size_t a = 0; a < x.size(); ++a) {
        volatile double d = x[a] - y[a];
        volatile double p = d * d;
        acc = acc + p;
    }
    return acc;
}

// Device arena of per-node sample-id lists (Section 4.2: a sample redundant
// for both bounds in a node stays redundant in every descendant, so a node's
// children only need the samples that survive in it).  Lists are immutable
// and shared by reference: both children of a node hold its filtered list,
// and a child whose parent could not be filtered (or gained little) holds the
// parent's list.  Space is managed on the host: best fit over free ranges,
// coalesced on release.
struct ListArena {
    struct Rec {
        int64_t off = 0, n = 0;
        int refs = 0;
    };
    DevBuf pool;                                   // uint32 sample ids
    int64_t cap = 0, used = 0, peak = 0;
    std::map<int64_t, int64_t> by_off;             // free ranges: offset -> length
    std::set<std::pair<int64_t, int64_t>> by_len;  // (length, offset)
    std::vector<Rec> recs;
    std::vector<int> spare;

    uint32_t *ids() const { return static_cast<uint32_t *>(pool.p); }
    void reset(int64_t capacity)
    {
        cap = capacity;
        used = peak = 0;
        by_off.clear();
        by_len.clear();
        recs.clear();
        spare.clear();
        if (cap > 0) put(0, cap);
    }
    void put(int64_t off, int64_t len)
    {
        by_off[off] = len;
        by_len.insert({len, off});
    }
    void drop(std::map<int64_t, int64_t>::iterator it)
    {
        by_len.erase({it->second, it->first});
        by_off.erase(it);
    }
    // offset of n free entries, or -1
    int64_t alloc(int64_t n)
    {
        if (n <= 0) return 0;
        auto it = by_len.lower_bound({n, INT64_MIN});
        if (it == by_len.end()) return -1;
        const int64_t len = it->first, off = it->second;
        drop(by_off.find(off));
        if (len > n) put(off + n, len - n);
        used += n;
        peak = std::max(peak, used);
        return off;
    }
    void release(int64_t off, int64_t n)
    {
        if (n <= 0) return;
        used -= n;
        int64_t o = off, l = n;
        auto nx = by_off.lower_bound(off);
        if (nx != by_off.begin()) {
            auto pv = std::prev(nx);
            if (pv->first + pv->second == o) {
                o = pv->first;
                l += pv->second;
                drop(pv);
            }
        }
        nx = by_off.lower_bound(o + l);
        if (nx != by_off.end() && nx->first == o + l) {
            l += nx->second;
            drop(nx);
        }
        put(o, l);
    }
    int make(int64_t off, int64_t n)
    {
        int h;
        if (!spare.empty()) {
            h = spare.back();
            spare.pop_back();
        } else {
            h = (int)recs.size();
            recs.push_back(Rec{});
        }
        recs[h] = Rec{off, n, 0};
        return h;
    }
    void ref(int h) { recs[h].refs += 1; }
    void unref(int h)
    {
        if (h < 0) return;
        if (--recs[h].refs == 0) {
            release(recs[h].off, recs[h].n);
            spare.push_back(h);
        }
    }
};

struct SolveBufs {
    DevBuf boxes, outs, sets, mask, counts, xbuf[2], idbuf[2], extra, lists;
    void *lpin = nullptr;   // pinned mirror of the list-batch descriptors
};

// Coordinates of B samples (by id) -> out [B][D] in the data type.
template <typename T>
__global__ void gather_points_kernel(const T *__restrict__ X, int64_t ld, int D, const int64_t *__restrict__ ids, int B,
                                     T *__restrict__ out)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < B * D; i += gridDim.x * blockDim.x) {
        const int b = i / D, a = i % D;
        const int64_t id = ids[b];
        out[i] = id >= 0 ? X[(size_t)a * ld + id] : T(0);
    }
}

// Branching rule 0 (Section 3.3): the max-range variable (smallest k*D+a on ties).
template <typename T>
int rule_max_range(const T *lo, const T *hi, int KD)
{
    int bi = -1;
    double br = 0.0;
    for (int i = 0; i < KD; ++i) {
        const double r = (double)hi[i] - (double)lo[i];
        if (r > br) { br = r; bi = i; }
    }
    return bi;
}

// Branching rule 1: the box nearest to the sample x attaining the node's lower
// bound, on the attribute (with positive range) where x lies farthest outside
// it.  -1 when x is inside every nearest box or no such attribute exists.
template <typename T>
int rule_argmax_gap(const T *lo, const T *hi, const T *x, int K, int D)
{
    int kb = -1;
    double best = 0.0;
    for (int k = 0; k < K; ++k) {
        double acc = 0.0;
        for (int a = 0; a < D; ++a) {
            const double xv = (double)x[a], l = (double)lo[k * D + a], h = (double)hi[k * D + a];
            const double d = xv < l ? l - xv : (xv > h ? xv - h : 0.0);
            acc += d * d;
        }
        if (kb < 0 || acc < best) { best = acc; kb = k; }
    }
    if (kb < 0 || !(best > 0.0)) return -1;
    int ab = -1;
    double g = 0.0;
    for (int a = 0; a < D; ++a) {
        const double xv = (double)x[a], l = (double)lo[kb * D + a], h = (double)hi[kb * D + a];
        if (!(h > l)) continue;
        const double d = xv < l ? l - xv : (xv > h ? xv - h : 0.0);
        if (d > g) { g = d; ab = a; }
    }
    return ab < 0 ? -1 : kb * D + ab;
}

template <typename T>
kc_status solve_impl(kc_ctx *c, const kc_solve_opts &o, kc_result *res)
{
    const double t0 = now_s();
    const int K = c->K, D = c->D, KD = K * D;
    const double tol = o.tol;
    SolveBufs sb;
    ListArena arena;
    auto cleanup = [&]() {
        for (DevBuf *b : {&sb.boxes, &sb.outs, &sb.sets, &sb.mask, &sb.counts, &sb.xbuf[0], &sb.xbuf[1], &sb.idbuf[0],
                          &sb.idbuf[1], &sb.extra, &sb.lists, &arena.pool})
            if (b->p) cudaFree(b->p);
        if (sb.lpin) cudaFreeHost(sb.lpin);
    };
    struct Guard {
        std::function<void()> f;
        ~Guard() { f(); }
    } guard{[&]() {
        cudaStreamSynchronize(c->stream);
        cleanup();
    }};

    // ---- root: M0, FFT upper bound (Algorithm 2), seeds (Section 4.1.1)
    std::vector<T> root_lo(D), root_hi(D);
    KC_TRY(ensure(c, sb.outs, 4096));
    {
        char *d = static_cast<char *>(sb.outs.p);
        int *flag = reinterpret_cast<int *>(d + 2048);
        KC_TRY(launch_root_box(c, d, d + 1024, flag));
        KC_CUDA(c, cudaMemcpyAsync(root_lo.data(), d, D * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaMemcpyAsync(root_hi.data(), d + 1024, D * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
    }
    KC_TRY(ensure(c, sb.sets, 4096));
    int64_t *T_dev = static_cast<int64_t *>(sb.sets.p);
    double *v_dev = reinterpret_cast<double *>(static_cast<char *>(sb.sets.p) + 1024);
    std::vector<int64_t> inc(K), trial(K);
    double alpha = __builtin_huge_val();
    // FFT from fft_starts start samples (seed mod N, then steps of a large odd
    // multiplier); the best objective is the first incumbent
    for (int i = 0; i < std::max(1, o.fft_starts); ++i) {
        const int64_t start = (int64_t)((o.seed + (uint64_t)i * 2654435761ull) % (uint64_t)c->N);
        KC_CUDA(c, cudaMemcpyAsync(T_dev, &start, 8, cudaMemcpyHostToDevice, c->stream));
        for (int t = 1; t < K; ++t)
            KC_TRY(launch_objective(c, full_view(c), T_dev, 1, t, __builtin_huge_val(), v_dev, T_dev + t));
        KC_TRY(launch_objective(c, full_view(c), T_dev, 1, K, __builtin_huge_val(), v_dev, nullptr));
        double a = 0.0;
        KC_CUDA(c, cudaMemcpyAsync(trial.data(), T_dev, K * 8, cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaMemcpyAsync(&a, v_dev, 8, cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaStreamSynchronize(c->stream));
        if (a < alpha) {
            alpha = a;
            inc = trial;
        }
    }
    KC_CUDA(c, cudaMemcpyAsync(T_dev, inc.data(), K * 8, cudaMemcpyHostToDevice, c->stream));
    res->fft_objective = alpha;

    bool seeds_found = false;
    if (o.use_bt) {
        std::vector<std::vector<double>> sx(K, std::vector<double>(D));
        std::vector<T> tmp(D);
        for (int k = 0; k < K; ++k) {
            for (int a = 0; a < D; ++a)
                KC_CUDA(c, cudaMemcpyAsync(&tmp[a], static_cast<const T *>(c->X) + (size_t)a * c->ldx + inc[k],
                                           sizeof(T), cudaMemcpyDeviceToHost, c->stream));
            KC_CUDA(c, cudaStreamSynchronize(c->stream));
            for (int a = 0; a < D; ++a) sx[k][a] = (double)tmp[a];
        }
        seeds_found = true;
        for (int i = 0; i < K && seeds_found; ++i)
            for (int j = i + 1; j < K; ++j)
                if (!(sqdist_host(sx[i], sx[j]) > 4.0 * alpha)) { seeds_found = false; break; }
    }
    const bool use_sb = o.use_bt && !seeds_found;
    int64_t *seeds_dev = nullptr;
    if (seeds_found) {
        seeds_dev = T_dev + 64;
        KC_CUDA(c, cudaMemcpyAsync(seeds_dev, inc.data(), K * 8, cudaMemcpyHostToDevice, c->stream));
    }
    res->seeds_found = seeds_found;
    const std::vector<int64_t> inc_seeds = inc;

    // ---- open nodes: a binary heap on (key, id)
    std::vector<Node<T>> heap;
    NodeCmp<T> cmp;
    {
        Node<T> r;
        r.lo.resize(KD);
        r.hi.resize(KD);
        for (int k = 0; k < K; ++k)
            for (int a = 0; a < D; ++a) { r.lo[k * D + a] = root_lo[a]; r.hi[k * D + a] = root_hi[a]; }
        r.key = 0.0;
        r.pkey = 0.0;
        r.id = 0;
        r.parent = -1;
        r.depth = 0;
        heap.push_back(std::move(r));
    }
    int64_t next_id = 1;
    std::vector<double> range0(D);
    for (int a = 0; a < D; ++a) range0[a] = std::max((double)root_hi[a] - (double)root_lo[a], 1e-300);
    kc_mlp *scorer = (o.order == 1) ? c->scorer : nullptr;
    const double rule_width = o.rule_width > 0 ? (double)o.rule_width : 4.0;

    const int Bmax = o.batch > 0 ? o.batch : 256;
    // device batch buffers
    const size_t box_bytes = (size_t)Bmax * KD * sizeof(T);
    KC_TRY(ensure(c, sb.boxes, 4 * box_bytes + 1024));
    T *d_lo = static_cast<T *>(sb.boxes.p);
    T *d_hi = reinterpret_cast<T *>(static_cast<char *>(sb.boxes.p) + box_bytes);
    T *d_lo2 = reinterpret_cast<T *>(static_cast<char *>(sb.boxes.p) + 2 * box_bytes);
    T *d_hi2 = reinterpret_cast<T *>(static_cast<char *>(sb.boxes.p) + 3 * box_bytes);
    const size_t o_cand = 0, o_lb = o_cand + (size_t)Bmax * K * 8, o_st = o_lb + (size_t)Bmax * 8;
    const size_t o_sets = o_st + ((Bmax + 255) & ~255), o_val = o_sets + (size_t)Bmax * K * 8;
    const size_t outs_bytes = o_val + (size_t)Bmax * 8 + 256;
    KC_TRY(ensure(c, sb.outs, outs_bytes));
    char *ob = static_cast<char *>(sb.outs.p);
    int64_t *d_cand = reinterpret_cast<int64_t *>(ob + o_cand);
    double *d_lb = reinterpret_cast<double *>(ob + o_lb);
    int8_t *d_st = reinterpret_cast<int8_t *>(ob + o_st);
    int64_t *d_sets = reinterpret_cast<int64_t *>(ob + o_sets);
    double *d_val = reinterpret_cast<double *>(ob + o_val);
    // pinned host mirror: boxes in (2), boxes out (2), cand, lb, status, sets, val
    const size_t pin_bytes = 4 * box_bytes + outs_bytes;
    KC_TRY(ensure_pinned(c, pin_bytes));
    char *pb = static_cast<char *>(c->pinned);
    T *h_lo = reinterpret_cast<T *>(pb), *h_hi = reinterpret_cast<T *>(pb + box_bytes);
    T *h_lo2 = reinterpret_cast<T *>(pb + 2 * box_bytes), *h_hi2 = reinterpret_cast<T *>(pb + 3 * box_bytes);
    char *po = pb + 4 * box_bytes;
    int64_t *h_cand = reinterpret_cast<int64_t *>(po + o_cand);
    double *h_lb = reinterpret_cast<double *>(po + o_lb);
    int8_t *h_st = reinterpret_cast<int8_t *>(po + o_st);
    int64_t *h_sets = reinterpret_cast<int64_t *>(po + o_sets);
    double *h_val = reinterpret_cast<double *>(po + o_val);

    // per-batch extras: argmax ids, counts, argmax coordinates, scorer I/O, label boxes
    const size_t e_arg = 0, e_cnt = e_arg + (size_t)Bmax * 8, e_pts = e_cnt + (size_t)Bmax * K * 8;
    const size_t e_feat = e_pts + (((size_t)Bmax * D * sizeof(T) + 255) & ~(size_t)255);
    const size_t e_out = e_feat + (size_t)Bmax * 12 * 4, e_lbox = e_out + (size_t)Bmax * 2 * 4 + 256;
    const size_t e_llb = e_lbox + 2 * (size_t)4 * Bmax * KD * sizeof(T), e_raw = e_llb + (size_t)4 * Bmax * 8;
    const size_t e_ref = e_raw + (size_t)Bmax * 8, e_kar = e_ref + (size_t)Bmax * 8, e_rfw = e_kar + (size_t)Bmax * 8;
    const size_t extra_bytes = e_rfw + (size_t)Bmax * 8 + 256;
    KC_TRY(ensure(c, sb.extra, extra_bytes));
    char *xb = static_cast<char *>(sb.extra.p);
    int64_t *d_arg = reinterpret_cast<int64_t *>(xb + e_arg);
    int64_t *d_cnt = reinterpret_cast<int64_t *>(xb + e_cnt);
    T *d_pts = reinterpret_cast<T *>(xb + e_pts);
    float *d_feat = reinterpret_cast<float *>(xb + e_feat);
    float *d_out = reinterpret_cast<float *>(xb + e_out);
    T *d_llo = reinterpret_cast<T *>(xb + e_lbox);
    T *d_lhi = d_llo + (size_t)4 * Bmax * KD;
    double *d_llb = reinterpret_cast<double *>(xb + e_llb);
    double *d_raw = reinterpret_cast<double *>(xb + e_raw);
    double *d_ref = reinterpret_cast<double *>(xb + e_ref);
    int64_t *d_kar = reinterpret_cast<int64_t *>(xb + e_kar);   // children's bound witnesses
    int64_t *d_rfw = reinterpret_cast<int64_t *>(xb + e_rfw);   // refined bounds' witnesses
    std::vector<int64_t> h_arg(Bmax), h_cnt((size_t)Bmax * K);
    std::vector<T> h_pts((size_t)Bmax * D);
    std::vector<float> h_feat((size_t)Bmax * 12), h_out((size_t)Bmax * 2);
    std::vector<T> h_llo((size_t)4 * Bmax * KD), h_lhi((size_t)4 * Bmax * KD);
    std::vector<double> h_ub(Bmax);

    std::vector<double> h_raw(Bmax), h_ref(Bmax);
    std::vector<int64_t> h_refw(Bmax), h_kar(Bmax);
    // Float data: a bound whose float value cannot decide the prune (its
    // certified value is below the threshold, the float value plus its error
    // bound is not) is re-evaluated in double over the same samples (the
    // ambiguous band of the rounding margin).
    const double g32 = gamma_n(f32_roundings(D), kU32);
    std::vector<int> amb;
    std::vector<double> amb_raw;
    auto ambiguous = [&](double key, double raw) {
        const double thr = alpha - tol * alpha;
        return c->dt == KC_F32 && key < thr && raw * (1.0 + g32) * (1.0 + 1e-9) >= thr;
    };
    int64_t refined = 0, filtered = 0, dropped = 0;

    // ---- per-node surviving-sample lists (float data)
    // per-node lists: float data with D <= 8 (the list kernels' register
    // tiles); wider data scan one shared sample set
    const bool lists = o.lists != 0 && c->dt == KC_F32 && c->D <= 8;
    const int LT = list_tile();
    const size_t slot_bytes = ((size_t)3 * (Bmax + 1) * 8 + (size_t)(2 * Bmax + 1) * 4 + 255) & ~(size_t)255;
    const int kSlots = 6;   // batch, its refinement, upper bounds, filter, children, their refinement
    const size_t l_keys = (size_t)kSlots * slot_bytes, l_vmax = l_keys + (size_t)Bmax * 8;
    const size_t l_thr = l_vmax + (size_t)Bmax * 8, l_beta = l_thr + (size_t)Bmax * 4;
    const size_t l_off = l_beta + (size_t)Bmax * 4, l_cap = l_off + (size_t)Bmax * 8, l_n = l_cap + (size_t)Bmax * 8;
    const size_t l_cvar = l_n + (size_t)Bmax * 8, l_csplit = l_cvar + (size_t)Bmax * 4;
    const size_t l_ckeys = l_csplit + (size_t)2 * Bmax * 4, l_clb = l_ckeys + (size_t)2 * Bmax * 8;
    const size_t l_craw = l_clb + (size_t)2 * Bmax * 8, l_carg = l_craw + (size_t)2 * Bmax * 8;
    const size_t l_wid = l_carg + (size_t)2 * Bmax * 8;
    const size_t l_end = l_wid + (size_t)Bmax * 4 + 256;
    unsigned long long *d_keys = nullptr, *d_vmax = nullptr, *d_outn = nullptr, *d_ckeys = nullptr;
    float *d_thr = nullptr, *d_beta = nullptr, *d_csplit = nullptr;
    int64_t *d_outoff = nullptr, *d_outcap = nullptr;
    int *d_cvar = nullptr;
    double *d_clb = nullptr, *d_craw = nullptr;
    int64_t *d_carg = nullptr;
    unsigned *d_wid = nullptr;
    int root_list = -1;
    if (lists) {
        KC_TRY(ensure(c, sb.lists, l_end));
        char *lb = static_cast<char *>(sb.lists.p);
        d_keys = reinterpret_cast<unsigned long long *>(lb + l_keys);
        d_vmax = reinterpret_cast<unsigned long long *>(lb + l_vmax);
        d_thr = reinterpret_cast<float *>(lb + l_thr);
        d_beta = reinterpret_cast<float *>(lb + l_beta);
        d_outoff = reinterpret_cast<int64_t *>(lb + l_off);
        d_outcap = reinterpret_cast<int64_t *>(lb + l_cap);
        d_outn = reinterpret_cast<unsigned long long *>(lb + l_n);
        d_cvar = reinterpret_cast<int *>(lb + l_cvar);
        d_csplit = reinterpret_cast<float *>(lb + l_csplit);
        d_ckeys = reinterpret_cast<unsigned long long *>(lb + l_ckeys);
        d_clb = reinterpret_cast<double *>(lb + l_clb);
        d_craw = reinterpret_cast<double *>(lb + l_craw);
        d_carg = reinterpret_cast<int64_t *>(lb + l_carg);
        d_wid = reinterpret_cast<unsigned *>(lb + l_wid);
        if (cudaMallocHost(&sb.lpin, (size_t)kSlots * slot_bytes) != cudaSuccess) {
            sb.lpin = nullptr;
            cudaGetLastError();
            return set_err(c, KC_ENOMEM, "kc_solve: pinned list descriptors");
        }
        size_t fr = 0, tot = 0;
        KC_CUDA(c, cudaMemGetInfo(&fr, &tot));
        int64_t cap = o.arena_mb > 0 ? (int64_t)o.arena_mb * (1 << 20) / 4
                                     : std::min<int64_t>((int64_t)(fr / 2 / 4), 4096 * c->N);
        cap = std::max<int64_t>(cap, c->N);
        KC_TRY(ensure(c, arena.pool, (size_t)cap * 4));
        arena.reset(cap);
        const int64_t off = arena.alloc(c->N);
        KC_TRY(launch_iota(c, arena.ids() + off, c->N));
        root_list = arena.make(off, c->N);
        arena.ref(root_list);
        heap.front().list = root_list;
    }
    // descriptors of n nodes' lists in slot `slot`: handle_of(i) names node i's
    // list; rows (or NULL) gives each node's row in per-batch arrays; with
    // `group`, consecutive nodes holding the same list form one group that
    // shares each staged tile
    auto make_lb = [&](int slot, int n, const std::function<int(int)> &handle_of, const int *rows, ListBatch *L,
                       const int **rows_dev, bool group = false) -> kc_status {
        char *hp = static_cast<char *>(sb.lpin) + (size_t)slot * slot_bytes;
        char *dp = static_cast<char *>(sb.lists.p) + (size_t)slot * slot_bytes;
        int64_t *so = reinterpret_cast<int64_t *>(hp), *sn = so + (Bmax + 1), *tp = sn + (Bmax + 1);
        int *rm = reinterpret_cast<int *>(tp + (Bmax + 1)), *ns = rm + Bmax;
        tp[0] = 0;
        int G = 0, prev = -1;
        for (int i = 0; i < n; ++i) {
            const int h = handle_of(i);
            if (rows) rm[i] = rows[i];
            if (group && G > 0 && h == prev) continue;
            const ListArena::Rec &r = arena.recs[h];
            so[G] = r.off;
            sn[G] = r.n;
            tp[G + 1] = tp[G] + (r.n + LT - 1) / LT;
            ns[G] = i;
            ++G;
            prev = h;
        }
        ns[G] = n;
        KC_CUDA(c, cudaMemcpyAsync(dp, hp, slot_bytes, cudaMemcpyHostToDevice, c->stream));
        const int64_t *sod = reinterpret_cast<const int64_t *>(dp);
        L->pool = arena.ids();
        L->seg_off = sod;
        L->seg_n = sod + (Bmax + 1);
        L->tile_prefix = sod + 2 * (Bmax + 1);
        const int *rmd = reinterpret_cast<const int *>(sod + 3 * (Bmax + 1));
        L->node_start = group ? rmd + Bmax : nullptr;
        L->B = G;
        L->W = tp[G];
        if (rows_dev) *rows_dev = rmd;
        return KC_OK;
    };
    auto list_n = [&](int h) { return h >= 0 ? arena.recs[h].n : (int64_t)0; };
    // refined certified bounds of the boxes src[which[i]] -> h_ref[i]
    // (list mode: over each node's own list, list_of(j) naming box j's list)
    auto refine_nodes = [&](const View &vw, const T *src_lo, const T *src_hi, const double *raw,
                            const std::function<int(int)> *list_of, int slot) -> kc_status {
        const int n = (int)amb.size();
        amb_raw.resize(n);
        for (int i = 0; i < n; ++i) {
            std::memcpy(&h_llo[(size_t)i * KD], src_lo + (size_t)amb[i] * KD, KD * sizeof(T));
            std::memcpy(&h_lhi[(size_t)i * KD], src_hi + (size_t)amb[i] * KD, KD * sizeof(T));
            amb_raw[i] = raw[amb[i]];
        }
        KC_CUDA(c, cudaMemcpyAsync(d_llo, h_llo.data(), (size_t)n * KD * sizeof(T), cudaMemcpyHostToDevice, c->stream));
        KC_CUDA(c, cudaMemcpyAsync(d_lhi, h_lhi.data(), (size_t)n * KD * sizeof(T), cudaMemcpyHostToDevice, c->stream));
        if (list_of) {
            ListBatch L;
            KC_TRY(make_lb(slot, n, [&](int i) { return (*list_of)(amb[i]); }, nullptr, &L, nullptr));
            KC_TRY(launch_seg_refine(c, L, d_llo, d_lhi, n, amb_raw.data(), d_thr, d_vmax, d_ref, d_wid, d_rfw));
        } else {
            KC_TRY(launch_lower_bounds_refine(c, vw, d_llo, d_lhi, n, amb_raw.data(), d_ref, nullptr, d_rfw));
        }
        KC_CUDA(c, cudaMemcpyAsync(h_ref.data(), d_ref, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaMemcpyAsync(h_refw.data(), d_rfw, (size_t)n * 8, cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaStreamSynchronize(c->stream));
        return KC_OK;
    };

    View cur = full_view(c);
    int ping = 0;
    int64_t visits = 0, batches = 0, created = 1;
    kc_status status = KC_OK;
    std::vector<Node<T>> batch;
    std::vector<int> live;
    // node log: closed on every return path
    std::unique_ptr<FILE, int (*)(FILE *)> log_file(o.log_path ? fopen(o.log_path, "w") : nullptr, &fclose);
    if (o.log_path && !log_file) return set_err(c, KC_EINVAL, "kc_solve: cannot open log_path '%s'", o.log_path);
    FILE *log = log_file.get();
    double prof[5] = {0, 0, 0, 0, 0};
    double tA = 0, last_trace = t0;

    auto prune_threshold = [&]() { return alpha - tol * alpha; };
    auto drop_list = [&](Node<T> &nd) {
        if (lists) arena.unref(nd.list);
        nd.list = -1;
    };

    for (;;) {
        // stop test: the smallest key over the open nodes against alpha
        if (!heap.empty() && heap.front().key >= prune_threshold()) {
            // the heap is ordered: every node is prunable
            for (Node<T> &nd : heap) drop_list(nd);
            heap.clear();
        }
        if (heap.empty()) break;
        if (alpha - heap.front().key <= tol * alpha) break;
        if (o.node_limit > 0 && visits >= o.node_limit) { status = KC_ELIMIT; break; }
        if (o.time_limit_s > 0 && now_s() - t0 > o.time_limit_s) { status = KC_ETIMEOUT; break; }

        // 1. select
        batch.clear();
        while (!heap.empty() && (int)batch.size() < Bmax) {
            std::pop_heap(heap.begin(), heap.end(), cmp);
            Node<T> nd = std::move(heap.back());
            heap.pop_back();
            if (nd.key >= prune_threshold()) {
                drop_list(nd);
                continue;
            }
            batch.push_back(std::move(nd));
        }
        if (batch.empty()) continue;
        // nodes holding the same list are bounded together (one staged tile each)
        if (lists)
            std::stable_sort(batch.begin(), batch.end(), [](const Node<T> &a, const Node<T> &b) { return a.list < b.list; });
        const int B = (int)batch.size();
        for (int b = 0; b < B; ++b) {
            std::memcpy(h_lo + (size_t)b * KD, batch[b].lo.data(), KD * sizeof(T));
            std::memcpy(h_hi + (size_t)b * KD, batch[b].hi.data(), KD * sizeof(T));
        }
        KC_CUDA(c, cudaMemcpyAsync(d_lo, h_lo, (size_t)B * KD * sizeof(T), cudaMemcpyHostToDevice, c->stream));
        KC_CUDA(c, cudaMemcpyAsync(d_hi, h_hi, (size_t)B * KD * sizeof(T), cudaMemcpyHostToDevice, c->stream));

        const int Bp = B;
        if (o.verbose) { KC_CUDA(c, cudaStreamSynchronize(c->stream)); tA = now_s(); }

        // 2b. tighten the survivors
        ListBatch Lb;
        const std::function<int(int)> batch_list = [&](int b) { return batch[b].list; };
        if (lists) KC_TRY(make_lb(0, Bp, batch_list, nullptr, &Lb, nullptr, true));
        if (lists) {
            const bool bt = o.use_bt != 0;
            KC_TRY(launch_tighten_list(c, Lb, d_lo, d_hi, Bp, bt ? alpha : __builtin_huge_val(), bt ? seeds_dev : nullptr,
                                       bt ? o.ball_cap : 1, d_lo2, d_hi2, d_cnt, d_cand, d_lb, d_raw, d_arg, d_st,
                                       &c->vs));
        } else if (o.use_bt) {
            KC_TRY(launch_tighten_view(c, cur, d_lo, d_hi, Bp, alpha, seeds_dev, o.ball_cap, d_lo2, d_hi2, d_cnt,
                                       d_cand, d_lb, d_raw, d_arg, d_st, &c->vs));
        } else {
            KC_TRY(launch_tighten_view(c, cur, d_lo, d_hi, Bp, __builtin_huge_val(), nullptr, 1, d_lo2, d_hi2, d_cnt,
                                       d_cand, d_lb, d_raw, d_arg, d_st, &c->vs));
        }
        KC_CUDA(c, cudaMemcpyAsync(h_raw.data(), d_raw, (size_t)Bp * 8, cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaMemcpyAsync(h_arg.data(), d_arg, (size_t)Bp * 8, cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaMemcpyAsync(h_cnt.data(), d_cnt, (size_t)Bp * K * 8, cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaMemcpyAsync(h_lo2, d_lo2, (size_t)Bp * KD * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaMemcpyAsync(h_hi2, d_hi2, (size_t)Bp * KD * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaMemcpyAsync(h_cand, d_cand, (size_t)Bp * K * 8, cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaMemcpyAsync(h_lb, d_lb, (size_t)Bp * 8, cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaMemcpyAsync(h_st, d_st, (size_t)Bp, cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaStreamSynchronize(c->stream));
        if (o.verbose) { prof[1] += now_s() - tA; tA = now_s(); }
        visits += Bp;
        ++batches;

        // 3. upper bounds of the live nodes' candidates
        live.clear();
        amb.clear();
        for (int b = 0; b < Bp; ++b) {
            h_ub[b] = __builtin_huge_val();
            if (h_lb[b] > batch[b].key) {
                batch[b].key = h_lb[b];
                batch[b].wit = h_arg[b];
            }
            if (h_st[b] != 1 && ambiguous(batch[b].key, h_raw[b])) amb.push_back(b);
        }
        if (!amb.empty()) {
            KC_TRY(refine_nodes(cur, h_lo, h_hi, h_raw.data(), lists ? &batch_list : nullptr, 1));
            for (size_t i = 0; i < amb.size(); ++i)
                if (h_ref[i] > batch[amb[i]].key) {
                    batch[amb[i]].key = h_ref[i];
                    batch[amb[i]].wit = h_refw[i];
                }
            refined += (int64_t)amb.size();
        }
        for (int b = 0; b < Bp; ++b) {
            if (h_st[b] == 1 || batch[b].key >= prune_threshold()) continue;
            live.push_back(b);
        }
        if (!live.empty()) {
            const int S = (int)live.size();
            // evaluation order: nodes whose lists hold at least a quarter of
            // the samples first -- their sets are evaluated over all samples
            // in one pass that every set shares -- then the others, each over
            // its own list (its candidate lies in the node's boxes, where every
            // dropped sample is nearer to it than the node's bound, so the
            // list's maximum is the full-data objective)
            std::vector<int> ev(live);
            int S_long = 0;
            if (lists) {
                std::stable_partition(ev.begin(), ev.end(),
                                      [&](int b) { return list_n(batch[b].list) * 4 >= c->N; });
                for (int b : ev) S_long += list_n(batch[b].list) * 4 >= c->N ? 1 : 0;
            }
            for (int i = 0; i < S; ++i)
                for (int k = 0; k < K; ++k) h_sets[(size_t)i * K + k] = h_cand[(size_t)ev[i] * K + k];
            KC_CUDA(c, cudaMemcpyAsync(d_sets, h_sets, (size_t)S * K * 8, cudaMemcpyHostToDevice, c->stream));
            if (lists) {
                if (S_long > 0) KC_TRY(launch_objective(c, full_view(c), d_sets, S_long, K, alpha, d_val, nullptr));
                if (S > S_long) {
                    ListBatch Lu;
                    KC_TRY(make_lb(2, S - S_long, [&](int i) { return batch[ev[S_long + i]].list; }, nullptr, &Lu,
                                   nullptr));
                    KC_TRY(launch_seg_objective(c, Lu, d_sets + (size_t)S_long * K, S - S_long, alpha, d_keys, d_vmax,
                                                d_thr, d_val + S_long));
                }
            } else {
                KC_TRY(launch_objective(c, cur, d_sets, S, K, alpha, d_val, nullptr));
            }
            KC_CUDA(c, cudaMemcpyAsync(h_val, d_val, (size_t)S * 8, cudaMemcpyDeviceToHost, c->stream));
            KC_CUDA(c, cudaStreamSynchronize(c->stream));
            for (int i = 0; i < S; ++i) h_ub[ev[i]] = h_val[i];
            for (int i = 0; i < S; ++i)
                if (h_val[i] < alpha) {
                    alpha = h_val[i];
                    for (int k = 0; k < K; ++k) inc[k] = h_sets[(size_t)i * K + k];
                }
        }
        if (o.verbose) { prof[2] += now_s() - tA; tA = now_s(); }

        // 4. prune, close leaves, choose the branching variable, branch
        std::vector<int> br;          // batch indices of the nodes to branch
        std::vector<Node<T>> kids;
        std::vector<int> kid_fused;   // index into flb/fraw, or -1
        std::vector<int> rule0;       // their max-range variable
        for (int b : live) {
            Node<T> &nd = batch[b];
            if (nd.key >= prune_threshold()) continue;
            T *lo = h_lo2 + (size_t)b * KD, *hi = h_hi2 + (size_t)b * KD;
            const bool leaf = h_st[b] == 2;
            if (use_sb && !leaf) {
                // symmetry breaking mu^1_1 <= ... <= mu^K_1 (Section 4.1.3)
                for (int k = 1; k < K; ++k)
                    if (lo[(k - 1) * D] > lo[k * D]) lo[k * D] = lo[(k - 1) * D];
                for (int k = K - 2; k >= 0; --k)
                    if (hi[(k + 1) * D] < hi[k * D]) hi[k * D] = hi[(k + 1) * D];
                bool empty = false;
                for (int k = 0; k < K; ++k)
                    if (lo[k * D] > hi[k * D]) empty = true;
                if (empty) continue;
            }
            if (leaf) continue;
            const int bi = rule_max_range<T>(lo, hi, KD);
            if (bi < 0) {
                // every box became a point after symmetry breaking: visit again
                Node<T> again;
                again.lo.assign(lo, lo + KD);
                again.hi.assign(hi, hi + KD);
                again.key = nd.key;
                again.pkey = nd.key;
                again.id = next_id++;
                again.parent = nd.id;
                again.depth = nd.depth + 1;
                again.group = nd.group;
                again.list = nd.list;
                if (lists) arena.ref(again.list);
                heap.push_back(std::move(again));
                std::push_heap(heap.begin(), heap.end(), cmp);
                continue;
            }
            br.push_back(b);
            rule0.push_back(bi);
        }
        const int NB = (int)br.size();
        std::vector<int> rule1(NB, -1), choice(rule0);
        std::vector<float> prio(NB, 0.f);
        const bool want_feat = scorer != nullptr || log != nullptr;
        if (NB > 0 && want_feat) {
            // coordinates of each node's lower-bound sample, for rule 1
            std::vector<int64_t> ids(NB);
            for (int i = 0; i < NB; ++i) ids[i] = h_arg[br[i]];
            KC_CUDA(c, cudaMemcpyAsync(d_sets, ids.data(), (size_t)NB * 8, cudaMemcpyHostToDevice, c->stream));
            gather_points_kernel<T><<<(NB * D + 255) / 256, 256, 0, c->stream>>>(
                static_cast<const T *>(c->X), c->ldx, D, d_sets, NB, d_pts);
            KC_TRY(after_launch(c, "gather points"));
            KC_CUDA(c, cudaMemcpyAsync(h_pts.data(), d_pts, (size_t)NB * D * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
            KC_CUDA(c, cudaStreamSynchronize(c->stream));
            for (int i = 0; i < NB; ++i) {
                const int b = br[i];
                rule1[i] = rule_argmax_gap<T>(h_lo2 + (size_t)b * KD, h_hi2 + (size_t)b * KD, &h_pts[(size_t)i * D], K, D);
                // node features (the scorer's 12 inputs)
                const Node<T> &nd = batch[b];
                const T *lo = h_lo2 + (size_t)b * KD, *hi = h_hi2 + (size_t)b * KD;
                float *f = &h_feat[(size_t)i * 12];
                double cnt = 0.0, lmean = 0.0, lmax = -1e300, lmin = 1e300, zero = 0.0;
                for (int k = 0; k < K; ++k) cnt += (double)h_cnt[(size_t)b * K + k];
                for (int k = 0; k < K; ++k)
                    for (int a2 = 0; a2 < D; ++a2) {
                        const double r = (double)hi[k * D + a2] - (double)lo[k * D + a2];
                        const double lr = std::log2(r / range0[a2] + 9.094947017729282e-13) / 40.0;
                        lmean += lr;
                        lmax = std::max(lmax, lr);
                        lmin = std::min(lmin, lr);
                        if (!(r > 0)) zero += 1.0;
                    }
                lmean /= KD;
                const double al = alpha > 0 ? alpha : 1.0;
                f[0] = (float)std::min(2.0, nd.key / al);
                f[1] = (float)std::max(-1.0, std::min(1.0, (alpha - nd.key) / al));
                f[2] = (float)(std::log2(1.0 + nd.depth) / 8.0);
                f[3] = (float)(std::log10(1.0 + cnt) / std::log10(1.0 + (double)K * c->N));
                const double nact = lists ? (double)list_n(nd.list) : (double)cur.n;
                f[4] = (float)(std::log10(1.0 + nact) / std::log10(1.0 + (double)c->N));
                f[5] = (float)lmean;
                f[6] = (float)lmax;
                f[7] = (float)lmin;
                f[8] = (float)(zero / KD);
                // range of rule 1's variable against the largest range (0 when rule 1 has none)
                {
                    const int v0 = rule0[i], v1 = rule1[i];
                    const double r0 = (double)hi[v0] - (double)lo[v0];
                    const double r1 = v1 >= 0 ? (double)hi[v1] - (double)lo[v1] : 0.0;
                    f[9] = v1 >= 0 && r0 > 0 ? (float)(std::log2(r1 / r0 + 9.094947017729282e-13) / -40.0) : 1.f;
                }
                f[10] = std::isfinite(h_ub[b]) ? (float)std::max(-1.0, std::min(1.0, (h_ub[b] - alpha) / al)) : 1.f;
                f[11] = (float)std::max(0.0, std::min(1.0, (nd.key - nd.pkey) / al));
            }
            if (scorer) {
                KC_CUDA(c, cudaMemcpyAsync(d_feat, h_feat.data(), (size_t)NB * 12 * 4, cudaMemcpyHostToDevice, c->stream));
                KC_TRY(mlp_forward_device(scorer, d_feat, NB, d_out, c->stream));
                c->launches += 1;
                KC_CUDA(c, cudaMemcpyAsync(h_out.data(), d_out, (size_t)NB * 2 * 4, cudaMemcpyDeviceToHost, c->stream));
                KC_CUDA(c, cudaStreamSynchronize(c->stream));
                // output r: predicted cost of branching with rule r; take the cheaper,
                // but rule 1 only on a variable whose range is at least 1/rule_width
                // (default 1/4) of the largest: splitting one short side over and
                // over leaves the other boxes large, and tightening and list
                // filtering then stall
                for (int i = 0; i < NB; ++i) {
                    const float c0 = h_out[(size_t)i * 2], c1 = h_out[(size_t)i * 2 + 1];
                    const T *lb2 = h_lo2 + (size_t)br[i] * KD, *hb2 = h_hi2 + (size_t)br[i] * KD;
                    const bool wide = rule1[i] >= 0 &&
                                      rule_width * ((double)hb2[rule1[i]] - (double)lb2[rule1[i]]) >=
                                          (double)hb2[rule0[i]] - (double)lb2[rule0[i]];
                    const bool take1 = wide && (double)c1 < (double)c0 - o.rule_margin;
                    if (take1) choice[i] = rule1[i];
                    prio[i] = take1 ? c1 : c0;
                }
            }
            if (o.explore > 0) {
                // training data: on explore % of the nodes where the two rules
                // differ, a uniformly random rule, drawn from the seed and the node
                // id (splitmix64 finalizer)
                for (int i = 0; i < NB; ++i) {
                    if (rule1[i] < 0 || rule1[i] == rule0[i]) continue;
                    uint64_t z = o.seed + 0x9E3779B97F4A7C15ull * (uint64_t)(batch[br[i]].id + 1);
                    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
                    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
                    z ^= z >> 31;
                    if ((z & 0xFFFFFFFFull) % 100 < (uint64_t)o.explore) choice[i] = (z >> 63) ? rule1[i] : rule0[i];
                }
            }
        }
        // the children's sample list: the samples of the node's list that are
        // not redundant for both bounds in its tightened boxes (Section 4.2);
        // the parent's list when there is no room or little is dropped
        // The filter also bounds the children over the surviving samples
        // (flb/fraw[2 * row + side]); fused_row[i]: node i's row, or -1.
        // by default a child shares its parent's list (also when no filter runs)
        std::vector<int> kid_list(NB, -1), fused_row(NB, -1);
        std::vector<int8_t> kid_fwait(NB, 0), kid_fstreak(NB, 0);
        for (int i = 0; i < NB; ++i) {
            const Node<T> &nd = batch[br[i]];
            kid_list[i] = nd.list;
            kid_fwait[i] = nd.fwait > 0 ? (int8_t)(nd.fwait - 1) : (int8_t)0;
            kid_fstreak[i] = nd.fstreak;
        }
        std::vector<double> flb, fraw;
        std::vector<int64_t> farg;
        if (lists && NB > 0 && o.i_sr > 0 && batches % o.i_sr == 0) {
            std::vector<int> fi, rows, cand;
            std::vector<int64_t> offs, caps;
            std::vector<float> bdn;
            const int64_t room = arena.cap - arena.used;
            for (int i = 0; i < NB; ++i) {
                const Node<T> &nd = batch[br[i]];
                const int64_t n = list_n(nd.list);
                if (n < 2 * LT || nd.fwait > 0) continue;
                if (n > 4 * room) {
                    // no room for what a filter of this list would keep: skip it
                    // (and the next generation's) instead of scanning in vain
                    kid_fwait[i] = 1;
                    continue;
                }
                cand.push_back(i);
            }
            // a filter writes its survivors straight into a region as long as
            // its list while those regions fit in half the free arena; beyond
            // that the longest lists are counted first (no output) and written
            // in a second pass once their survivors' number is known
            std::vector<char> counted(NB, 0);
            {
                int64_t total = 0;
                for (int i : cand) total += list_n(batch[br[i]].list);
                std::vector<int> byn(cand);
                std::stable_sort(byn.begin(), byn.end(), [&](int x, int y) {
                    return list_n(batch[br[x]].list) > list_n(batch[br[y]].list);
                });
                const int64_t budget = (arena.cap - arena.used) / 2;
                for (int i : byn) {
                    if (total <= budget) break;
                    counted[i] = 1;
                    total -= list_n(batch[br[i]].list);
                }
            }
            for (int i : cand) {
                const int b = br[i];
                const int64_t n = list_n(batch[b].list);
                int64_t off = -1;
                if (!counted[i]) {
                    off = arena.alloc(n);
                    if (off < 0) counted[i] = 1;
                }
                fi.push_back(i);
                rows.push_back(b);
                offs.push_back(off);
                caps.push_back(off >= 0 ? n : 0);
                float f = (float)batch[b].key;
                if ((double)f > batch[b].key) f = nextafterf(f, -1.f);
                bdn.push_back(f);
            }
            const int nf = (int)fi.size();
            if (nf > 0) {
                for (int q = 0; q < nf; ++q) {
                    std::memcpy(&h_llo[(size_t)q * KD], h_lo2 + (size_t)rows[q] * KD, KD * sizeof(T));
                    std::memcpy(&h_lhi[(size_t)q * KD], h_hi2 + (size_t)rows[q] * KD, KD * sizeof(T));
                }
                KC_CUDA(c, cudaMemcpyAsync(d_llo, h_llo.data(), (size_t)nf * KD * sizeof(T), cudaMemcpyHostToDevice, c->stream));
                KC_CUDA(c, cudaMemcpyAsync(d_lhi, h_lhi.data(), (size_t)nf * KD * sizeof(T), cudaMemcpyHostToDevice, c->stream));
                KC_CUDA(c, cudaMemcpyAsync(d_beta, bdn.data(), (size_t)nf * 4, cudaMemcpyHostToDevice, c->stream));
                KC_CUDA(c, cudaMemcpyAsync(d_outoff, offs.data(), (size_t)nf * 8, cudaMemcpyHostToDevice, c->stream));
                KC_CUDA(c, cudaMemcpyAsync(d_outcap, caps.data(), (size_t)nf * 8, cudaMemcpyHostToDevice, c->stream));
                // the children's split (branching variable and value, as below)
                std::vector<int> cvar(nf);
                std::vector<float> csplit((size_t)2 * nf);
                for (int q = 0; q < nf; ++q) {
                    const int v = choice[fi[q]];
                    const T *lq = h_lo2 + (size_t)rows[q] * KD, *hq = h_hi2 + (size_t)rows[q] * KD;
                    T m, succ;
                    split_point<T>(lq[v], hq[v], &m, &succ);
                    cvar[q] = v;
                    csplit[2 * q] = (float)m;
                    csplit[2 * q + 1] = (float)succ;
                }
                KC_CUDA(c, cudaMemcpyAsync(d_cvar, cvar.data(), (size_t)nf * 4, cudaMemcpyHostToDevice, c->stream));
                KC_CUDA(c, cudaMemcpyAsync(d_csplit, csplit.data(), (size_t)2 * nf * 4, cudaMemcpyHostToDevice, c->stream));
                ListBatch Lf;
                const int *rows_dev = nullptr;
                KC_TRY(make_lb(3, nf, [&](int q) { return batch[rows[q]].list; }, rows.data(), &Lf, &rows_dev));
                const bool bt = o.use_bt != 0;
                KC_TRY(launch_seg_filter(c, Lf, d_llo, d_lhi, nf, d_beta, alpha, bt ? c->vs.repx : nullptr,
                                         bt ? c->vs.nreps : nullptr, c->vs.RM, rows_dev, arena.ids(), d_outoff,
                                         d_outcap, d_outn, d_cvar, d_csplit, d_ckeys, d_clb, d_craw, d_carg));
                std::vector<unsigned long long> kept(nf);
                flb.resize((size_t)2 * nf);
                fraw.resize((size_t)2 * nf);
                farg.resize((size_t)2 * nf);
                KC_CUDA(c, cudaMemcpyAsync(kept.data(), d_outn, (size_t)nf * 8, cudaMemcpyDeviceToHost, c->stream));
                KC_CUDA(c, cudaMemcpyAsync(flb.data(), d_clb, (size_t)2 * nf * 8, cudaMemcpyDeviceToHost, c->stream));
                KC_CUDA(c, cudaMemcpyAsync(fraw.data(), d_craw, (size_t)2 * nf * 8, cudaMemcpyDeviceToHost, c->stream));
                KC_CUDA(c, cudaMemcpyAsync(farg.data(), d_carg, (size_t)2 * nf * 8, cudaMemcpyDeviceToHost, c->stream));
                KC_CUDA(c, cudaStreamSynchronize(c->stream));
                for (int q = 0; q < nf; ++q) fused_row[fi[q]] = q;
                std::vector<int> second;   // counted filters worth writing: rows q
                for (int q = 0; q < nf; ++q) {
                    const int i = fi[q];
                    const int64_t n = list_n(batch[rows[q]].list), m = (int64_t)kept[q];
                    // a counted (long) list is written only when the survivors are
                    // at most N/16: longer lists stay shared with the parent, so the
                    // nodes holding them keep sharing each staged tile
                    const bool worth = offs[q] >= 0 ? (double)m <= 0.95 * (double)n
                                                    : (double)m <= 0.95 * (double)n && m * 16 <= c->N;
                    if (!worth) {
                        if (offs[q] >= 0) arena.release(offs[q], n);
                        else {
                            // a long list that does not shrink enough: its descendants
                            // skip 1, 3, 7, 15 generations of filtering after 1, 2, 3, 4+
                            // such filters in a row
                            const int st = std::min(4, kid_fstreak[i] + 1);
                            kid_fstreak[i] = (int8_t)st;
                            kid_fwait[i] = (int8_t)((1 << st) - 1);
                        }
                        continue;
                    }
                    kid_fstreak[i] = 0;
                    if (offs[q] >= 0) {
                        arena.release(offs[q] + m, n - m);
                        kid_list[i] = arena.make(offs[q], m);
                        filtered += 1;
                        dropped += n - m;
                    } else {
                        second.push_back(q);
                    }
                }
                if (!second.empty()) {
                    // write the counted filters' survivors (same decisions as the
                    // counting pass; each region holds exactly its count)
                    std::vector<int> rows2, q2;
                    std::vector<int64_t> offs2, caps2;
                    std::vector<float> bdn2;
                    for (int q : second) {
                        const int64_t m = (int64_t)kept[q];
                        const int64_t off = arena.alloc(m);
                        if (off < 0) continue;   // no room: the children keep the parent's list
                        q2.push_back(q);
                        rows2.push_back(rows[q]);
                        offs2.push_back(off);
                        caps2.push_back(m);
                        bdn2.push_back(bdn[q]);
                    }
                    const int n2 = (int)q2.size();
                    if (n2 > 0) {
                        for (int t = 0; t < n2; ++t) {
                            std::memcpy(&h_llo[(size_t)t * KD], h_lo2 + (size_t)rows2[t] * KD, KD * sizeof(T));
                            std::memcpy(&h_lhi[(size_t)t * KD], h_hi2 + (size_t)rows2[t] * KD, KD * sizeof(T));
                        }
                        KC_CUDA(c, cudaMemcpyAsync(d_llo, h_llo.data(), (size_t)n2 * KD * sizeof(T), cudaMemcpyHostToDevice, c->stream));
                        KC_CUDA(c, cudaMemcpyAsync(d_lhi, h_lhi.data(), (size_t)n2 * KD * sizeof(T), cudaMemcpyHostToDevice, c->stream));
                        KC_CUDA(c, cudaMemcpyAsync(d_beta, bdn2.data(), (size_t)n2 * 4, cudaMemcpyHostToDevice, c->stream));
                        KC_CUDA(c, cudaMemcpyAsync(d_outoff, offs2.data(), (size_t)n2 * 8, cudaMemcpyHostToDevice, c->stream));
                        KC_CUDA(c, cudaMemcpyAsync(d_outcap, caps2.data(), (size_t)n2 * 8, cudaMemcpyHostToDevice, c->stream));
                        ListBatch L2;
                        const int *rows2_dev = nullptr;
                        KC_TRY(make_lb(3, n2, [&](int t) { return batch[rows2[t]].list; }, rows2.data(), &L2, &rows2_dev));
                        KC_TRY(launch_seg_filter(c, L2, d_llo, d_lhi, n2, d_beta, alpha, bt ? c->vs.repx : nullptr,
                                                 bt ? c->vs.nreps : nullptr, c->vs.RM, rows2_dev, arena.ids(), d_outoff,
                                                 d_outcap, d_outn, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr));
                        std::vector<unsigned long long> kept2(n2);
                        KC_CUDA(c, cudaMemcpyAsync(kept2.data(), d_outn, (size_t)n2 * 8, cudaMemcpyDeviceToHost, c->stream));
                        KC_CUDA(c, cudaStreamSynchronize(c->stream));
                        for (int t = 0; t < n2; ++t) {
                            const int q = q2[t];
                            const int64_t n = list_n(batch[rows[q]].list), m = (int64_t)kept[q];
                            if ((int64_t)kept2[t] != m) {
                                // cannot happen (identical decisions); keep the parent's list
                                arena.release(offs2[t], m);
                                continue;
                            }
                            kid_list[fi[q]] = arena.make(offs2[t], m);
                            filtered += 1;
                            dropped += n - m;
                        }
                    }
                }
            }
        }
        for (int i = 0; i < NB; ++i) {
            const int b = br[i];
            Node<T> &nd = batch[b];
            const T *lo = h_lo2 + (size_t)b * KD, *hi = h_hi2 + (size_t)b * KD;
            if (log) {
                fprintf(log, "{\"id\":%lld,\"parent\":%lld,\"depth\":%d,\"lb\":%.17g,\"alpha\":%.17g,\"rule\":%d,"
                             "\"rule0\":%d,\"rule1\":%d,\"n\":%lld,\"feat\":[",
                        (long long)nd.id, (long long)nd.parent, nd.depth, nd.key, alpha, choice[i] == rule0[i] ? 0 : 1,
                        rule0[i], rule1[i], (long long)(lists ? list_n(nd.list) : cur.n));
                for (int q = 0; q < 12; ++q) fprintf(log, q ? ",%.8g" : "%.8g", (double)h_feat[(size_t)i * 12 + q]);
                fprintf(log, "]}\n");
            }
            const int bi = choice[i];
            T m, succ;
            split_point<T>(lo[bi], hi[bi], &m, &succ);
            for (int side = 0; side < 2; ++side) {
                Node<T> ch;
                ch.lo.assign(lo, lo + KD);
                ch.hi.assign(hi, hi + KD);
                if (side == 0) ch.hi[bi] = m;
                else ch.lo[bi] = succ;
                ch.key = nd.key;
                ch.pkey = nd.key;
                ch.wit = nd.wit;   // the parent's witness is at least as far from the child's smaller boxes
                ch.prio = prio[i];
                ch.id = next_id++;
                ch.parent = nd.id;
                ch.depth = nd.depth + 1;
                ch.group = ch.depth <= 8 ? ch.id : nd.group;
                ch.list = kid_list[i];
                ch.fwait = kid_fwait[i];
                ch.fstreak = kid_fstreak[i];
                if (lists) {
                    // every node of a list-mode solve holds a list (an empty one is
                    // a valid list of length 0; a missing one is a logic error)
                    if (ch.list < 0 || ch.list >= (int)arena.recs.size())
                        return set_err(c, KC_EINTERNAL, "kc_solve: child %lld without a sample list",
                                       (long long)ch.id);
                    arena.ref(ch.list);
                }
                kids.push_back(std::move(ch));
                kid_fused.push_back(fused_row[i] >= 0 ? 2 * fused_row[i] + side : -1);
            }
        }
        // bound the children as they are created (Algorithm 1, Bounding); only
        // those below the incumbent enter the open set
        std::vector<double> klb((size_t)Bmax), kraw((size_t)Bmax);
        std::vector<int64_t> kwit((size_t)Bmax);
        for (size_t k0 = 0; k0 < kids.size(); k0 += (size_t)Bmax) {
            const int nk = (int)std::min(kids.size() - k0, (size_t)Bmax);
            for (int q = 0; q < nk; ++q) {
                std::memcpy(h_lo + (size_t)q * KD, kids[k0 + q].lo.data(), KD * sizeof(T));
                std::memcpy(h_hi + (size_t)q * KD, kids[k0 + q].hi.data(), KD * sizeof(T));
            }
            const std::function<int(int)> kid_of = [&](int q) { return kids[k0 + q].list; };
            // children bounded by the filter take its values; the rest are
            // bounded here over their lists (or the shared set)
            std::vector<int> sub;
            for (int q = 0; q < nk; ++q) {
                const int f = kid_fused[k0 + q];
                if (f >= 0) {
                    klb[q] = flb[f];
                    kraw[q] = fraw[f];
                    kwit[q] = farg[f];
                } else {
                    sub.push_back(q);
                }
            }
            if (!sub.empty()) {
                const int ns = (int)sub.size();
                for (int t = 0; t < ns; ++t) {
                    std::memcpy(&h_llo[(size_t)t * KD], h_lo + (size_t)sub[t] * KD, KD * sizeof(T));
                    std::memcpy(&h_lhi[(size_t)t * KD], h_hi + (size_t)sub[t] * KD, KD * sizeof(T));
                }
                KC_CUDA(c, cudaMemcpyAsync(d_lo, h_llo.data(), (size_t)ns * KD * sizeof(T), cudaMemcpyHostToDevice, c->stream));
                KC_CUDA(c, cudaMemcpyAsync(d_hi, h_lhi.data(), (size_t)ns * KD * sizeof(T), cudaMemcpyHostToDevice, c->stream));
                if (lists) {
                    ListBatch Lk;
                    KC_TRY(make_lb(4, ns, [&](int t) { return kids[k0 + sub[t]].list; }, nullptr, &Lk, nullptr, true));
                    KC_TRY(launch_seg_lb(c, Lk, d_lo, d_hi, ns, d_keys, d_lb, d_raw, d_kar));
                } else {
                    KC_TRY(launch_lower_bounds_view(c, cur, d_lo, d_hi, ns, d_lb, d_raw, d_kar, 0));
                }
                KC_CUDA(c, cudaMemcpyAsync(h_lb, d_lb, (size_t)ns * 8, cudaMemcpyDeviceToHost, c->stream));
                KC_CUDA(c, cudaMemcpyAsync(h_raw.data(), d_raw, (size_t)ns * 8, cudaMemcpyDeviceToHost, c->stream));
                KC_CUDA(c, cudaMemcpyAsync(h_kar.data(), d_kar, (size_t)ns * 8, cudaMemcpyDeviceToHost, c->stream));
                KC_CUDA(c, cudaStreamSynchronize(c->stream));
                for (int t = 0; t < ns; ++t) {
                    klb[sub[t]] = h_lb[t];
                    kraw[sub[t]] = h_raw[t];
                    kwit[sub[t]] = h_kar[t];
                }
            }
            amb.clear();
            for (int q = 0; q < nk; ++q) {
                if (klb[q] > kids[k0 + q].key) {
                    kids[k0 + q].key = klb[q];
                    kids[k0 + q].wit = kwit[q];
                }
                if (ambiguous(kids[k0 + q].key, kraw[q])) amb.push_back(q);
            }
            if (!amb.empty()) {
                KC_TRY(refine_nodes(cur, h_lo, h_hi, kraw.data(), lists ? &kid_of : nullptr, 5));
                for (size_t i = 0; i < amb.size(); ++i)
                    if (h_ref[i] > kids[k0 + amb[i]].key) {
                        kids[k0 + amb[i]].key = h_ref[i];
                        kids[k0 + amb[i]].wit = h_refw[i];
                    }
                refined += (int64_t)amb.size();
            }
            for (int q = 0; q < nk; ++q) {
                Node<T> &ch = kids[k0 + q];
                ++created;
                if (log) {
                    // every bounded child: its boxes and certified bound, for
                    // checking bounds and prunes against a double evaluation
                    fprintf(log, "{\"child\":%lld,\"parent\":%lld,\"key\":%.17g,\"pruned\":%d,\"w\":%lld,\"lo\":[",
                            (long long)ch.id, (long long)ch.parent, ch.key, ch.key >= prune_threshold() ? 1 : 0,
                            (long long)ch.wit);
                    // 9 significant digits round-trip a float, 17 a double
                    const char *f0 = sizeof(T) == 4 ? "%.9g" : "%.17g", *f1 = sizeof(T) == 4 ? ",%.9g" : ",%.17g";
                    for (int i = 0; i < KD; ++i) fprintf(log, i ? f1 : f0, (double)ch.lo[i]);
                    fprintf(log, "],\"hi\":[");
                    for (int i = 0; i < KD; ++i) fprintf(log, i ? f1 : f0, (double)ch.hi[i]);
                    fprintf(log, "]}\n");
                }
                if (ch.key >= prune_threshold()) {
                    drop_list(ch);
                    continue;
                }
                heap.push_back(std::move(ch));
                std::push_heap(heap.begin(), heap.end(), cmp);
            }
        }
        kids.clear();
        kid_fused.clear();
        for (Node<T> &nd : batch) drop_list(nd);

        if (o.verbose) { prof[3] += now_s() - tA; tA = now_s(); }
        // 5. sample reduction against the hull of the open nodes (Algorithm 5)
        if (!lists && o.i_sr > 0 && c->D <= 8 && batches % o.i_sr == 0 && !heap.empty() &&
            heap.front().key < prune_threshold()) {
            // one hull box per group of open nodes (a group = the descendants of
            // one node at depth 8): every node's box lies inside its group's
            // hull, so redundancy against the hulls implies it against the nodes
            std::vector<int64_t> gid;
            std::vector<T> hlo, hhi;
            {
                std::vector<std::pair<int64_t, int>> order;
                order.reserve(heap.size());
                for (int i = 0; i < (int)heap.size(); ++i) order.push_back({heap[i].group, i});
                std::sort(order.begin(), order.end());
                for (size_t q = 0; q < order.size(); ++q) {
                    const Node<T> &nd = heap[order[q].second];
                    if (q == 0 || order[q].first != order[q - 1].first) {
                        gid.push_back(order[q].first);
                        hlo.insert(hlo.end(), nd.lo.begin(), nd.lo.end());
                        hhi.insert(hhi.end(), nd.hi.begin(), nd.hi.end());
                    } else {
                        T *gl = &hlo[hlo.size() - KD], *gh = &hhi[hhi.size() - KD];
                        for (int i = 0; i < KD; ++i) {
                            gl[i] = std::min(gl[i], nd.lo[i]);
                            gh[i] = std::max(gh[i], nd.hi[i]);
                        }
                    }
                }
            }
            int G = (int)gid.size();
            if (G > Bmax) {
                // too many groups for the batch buffers: merge neighbours pairwise
                const int f = (G + Bmax - 1) / Bmax;
                int w = 0;
                for (int g = 0; g < G; g += f, ++w) {
                    for (int i = 0; i < KD; ++i) { hlo[(size_t)w * KD + i] = hlo[(size_t)g * KD + i]; hhi[(size_t)w * KD + i] = hhi[(size_t)g * KD + i]; }
                    for (int g2 = g + 1; g2 < std::min(G, g + f); ++g2)
                        for (int i = 0; i < KD; ++i) {
                            hlo[(size_t)w * KD + i] = std::min(hlo[(size_t)w * KD + i], hlo[(size_t)g2 * KD + i]);
                            hhi[(size_t)w * KD + i] = std::max(hhi[(size_t)w * KD + i], hhi[(size_t)g2 * KD + i]);
                        }
                }
                G = w;
            }
            const double beta_glob = heap.front().key;
            std::memcpy(h_lo, hlo.data(), (size_t)G * KD * sizeof(T));
            std::memcpy(h_hi, hhi.data(), (size_t)G * KD * sizeof(T));
            KC_CUDA(c, cudaMemcpyAsync(d_lo, h_lo, (size_t)G * KD * sizeof(T), cudaMemcpyHostToDevice, c->stream));
            KC_CUDA(c, cudaMemcpyAsync(d_hi, h_hi, (size_t)G * KD * sizeof(T), cudaMemcpyHostToDevice, c->stream));
            const int64_t ncur = cur.n;
            KC_TRY(ensure(c, sb.mask, (size_t)ncur + 256));
            KC_TRY(ensure(c, sb.counts, (size_t)compact_blocks(ncur) * 4 + 4096));
            uint8_t *mask = static_cast<uint8_t *>(sb.mask.p);
            unsigned long long *n_keep_dev =
                reinterpret_cast<unsigned long long *>(static_cast<char *>(sb.counts.p) + compact_blocks(ncur) * 4);
            n_keep_dev = reinterpret_cast<unsigned long long *>(((uintptr_t)n_keep_dev + 15) & ~(uintptr_t)15);
            KC_CUDA(c, cudaMemsetAsync(mask, 1, (size_t)ncur, c->stream));
            const void *repx = nullptr;
            const int *nreps = nullptr;
            if (seeds_found) {
                // the seeds are the assigned samples known in every node: one
                // representative per cluster, the same for every group
                std::vector<int64_t> rp((size_t)G * K);
                for (int g = 0; g < G; ++g)
                    for (int k = 0; k < K; ++k) rp[(size_t)g * K + k] = inc_seeds[k];
                KC_CUDA(c, cudaMemcpyAsync(d_sets, rp.data(), rp.size() * 8, cudaMemcpyHostToDevice, c->stream));
                KC_TRY(launch_gather_reps(c, G, 1, d_sets, d_lo2, reinterpret_cast<int *>(d_llb)));
                repx = d_lo2;
                nreps = reinterpret_cast<const int *>(d_llb);
            }
            KC_TRY(launch_sample_reduction_view(c, cur, d_lo, d_hi, G, repx, nreps, 1, beta_glob, alpha, mask,
                                                n_keep_dev));
            unsigned long long n_keep = 0;
            KC_CUDA(c, cudaMemcpyAsync(&n_keep, n_keep_dev, 8, cudaMemcpyDeviceToHost, c->stream));
            KC_CUDA(c, cudaStreamSynchronize(c->stream));
            if ((int64_t)n_keep < ncur && n_keep > 0 && (double)n_keep < 0.95 * (double)ncur) {
                const int nxt = ping ^ 1;
                const int64_t ld = ((int64_t)n_keep + 63) / 64 * 64;
                KC_TRY(ensure(c, sb.xbuf[nxt], (size_t)D * ld * sizeof(T)));
                KC_TRY(ensure(c, sb.idbuf[nxt], (size_t)ld * 4));
                unsigned long long *tot = n_keep_dev;
                KC_TRY(launch_compact(c, cur, mask, sb.xbuf[nxt].p, ld, static_cast<uint32_t *>(sb.idbuf[nxt].p),
                                      static_cast<unsigned *>(sb.counts.p), tot));
                View nv;
                nv.X = sb.xbuf[nxt].p;
                nv.ld = ld;
                nv.n = (int64_t)n_keep;
                nv.ids = static_cast<const uint32_t *>(sb.idbuf[nxt].p);
                cur = nv;
                ping = nxt;
            }
        }
        if (o.verbose) {
            KC_CUDA(c, cudaStreamSynchronize(c->stream));
            prof[4] += now_s() - tA;
            tA = now_s();
            if (batches % 100 == 0 || tA - last_trace >= 10.0) {
                last_trace = tA;
                const double beta = heap.empty() ? alpha : std::min(heap.front().key, alpha);
                fprintf(stderr, "[kc_solve] t %.1f s batch %lld visits %lld open %zu alpha %.17g beta %.17g gap %.3e "
                                "active %lld\n",
                        tA - t0, (long long)batches, (long long)visits, heap.size(), alpha, beta,
                        alpha > 0 ? (alpha - beta) / alpha : 0.0, (long long)(lists ? arena.used : cur.n));
            }
        }
    }
    log_file.reset();
    log = nullptr;
    if (o.verbose)
        fprintf(stderr, "[kc_solve] seconds: tighten %.3f, upper bounds %.3f, branch+child bounds %.3f, "
                        "sample reduction %.3f; batches %lld, visits %lld, created %lld, refined %lld\n",
                prof[1], prof[2], prof[3], prof[4], (long long)batches, (long long)visits, (long long)created,
                (long long)refined);
    if (o.verbose && lists)
        fprintf(stderr, "[kc_solve] lists: %lld filtered, %lld entries dropped, arena peak %lld of %lld entries\n",
                (long long)filtered, (long long)dropped, (long long)arena.peak, (long long)arena.cap);

    // ---- certificate: the incumbent's objective over all N samples in double
    KC_CUDA(c, cudaMemcpyAsync(T_dev, inc.data(), K * 8, cudaMemcpyHostToDevice, c->stream));
    KC_TRY(launch_objective(c, full_view(c), T_dev, 1, K, __builtin_huge_val(), v_dev, nullptr));
    double obj = 0.0;
    KC_CUDA(c, cudaMemcpyAsync(&obj, v_dev, 8, cudaMemcpyDeviceToHost, c->stream));
    KC_CUDA(c, cudaStreamSynchronize(c->stream));
    double lbound;
    if (heap.empty()) lbound = tol > 0 ? std::min(obj, alpha * (1.0 - tol)) : obj;
    else lbound = std::min(heap.front().key, tol > 0 ? alpha * (1.0 - tol) : alpha);
    res->objective = obj;
    res->lower_bound = std::min(lbound, obj);
    res->gap = obj > 0 ? (obj - res->lower_bound) / obj : 0.0;
    for (int k = 0; k < 16; ++k) res->centers[k] = k < K ? inc[k] : -1;
    res->nodes = visits;
    res->batches = batches;
    if (lists) {
        int64_t longest = 0;
        for (const Node<T> &nd : heap) longest = std::max(longest, list_n(nd.list));
        res->active_final = longest;
    } else {
        res->active_final = cur.n;
    }
    res->seconds = now_s() - t0;
    res->status = status;
    res->lists_filtered = filtered;
    res->samples_dropped = dropped;
    return status;
}

}  // namespace

}  // namespace kc

using namespace kc;

extern "C" {

kc_status kc_tighten(kc_ctx *c, const void *lo, const void *hi, int32_t B, double alpha, const int64_t *seeds,
                     int32_t ball_cap, void *lo_out, void *hi_out, int64_t *counts, int64_t *cand, double *lb_out,
                     int8_t *status)
{
    if (!c) return KC_EINVAL;
    if (B < 0) return set_err(c, KC_EINVAL, "kc_tighten: B=%d < 0", B);
    if (B == 0) return KC_OK;
    if (!lo || !hi || !lo_out || !hi_out || !status) return set_err(c, KC_EINVAL, "kc_tighten: NULL argument");
    if (!(alpha >= 0.0) || std::isinf(alpha)) return set_err(c, KC_EINVAL, "kc_tighten: alpha must be finite, >= 0");
    if (seeds) {
        std::vector<int64_t> h(c->K);
        if (is_device_ptr(seeds)) {
            KC_CUDA(c, cudaMemcpyAsync(h.data(), seeds, c->K * 8, cudaMemcpyDeviceToHost, c->stream));
            KC_CUDA(c, cudaStreamSynchronize(c->stream));
        } else {
            std::memcpy(h.data(), seeds, c->K * 8);
        }
        for (int k = 0; k < c->K; ++k)
            if (h[k] < 0 || h[k] >= c->N) return set_err(c, KC_EINVAL, "kc_tighten: seed index out of range");
    }
    const size_t box = (size_t)B * c->K * c->D * c->esize;
    Stager sg(c);
    const int ilo = sg.add(lo, box, true), ihi = sg.add(hi, box, true);
    const int isd = sg.add(seeds, (size_t)c->K * 8, true);
    const int ilo2 = sg.add(lo_out, box, false), ihi2 = sg.add(hi_out, box, false);
    const int icn = sg.add(counts, (size_t)B * c->K * 8, false), icd = sg.add(cand, (size_t)B * c->K * 8, false);
    const int ilb = sg.add(lb_out, (size_t)B * 8, false), ist = sg.add(status, (size_t)B, false);
    KC_TRY(sg.begin());
    KC_TRY(launch_tighten_view(c, full_view(c), sg.dev(ilo), sg.dev(ihi), B, alpha,
                               static_cast<const int64_t *>(sg.dev(isd)), ball_cap, sg.dev(ilo2), sg.dev(ihi2),
                               static_cast<int64_t *>(sg.dev(icn)), static_cast<int64_t *>(sg.dev(icd)),
                               static_cast<double *>(sg.dev(ilb)), nullptr, nullptr,
                               static_cast<int8_t *>(sg.dev(ist)), &c->vs));
    return sg.finish();
}

kc_status kc_sample_reduction(kc_ctx *c, const void *lo, const void *hi, int32_t M, const int64_t *reps, int32_t R,
                              double beta_glob, double alpha, uint8_t *active_inout, int64_t *n_active_out)
{
    if (!c) return KC_EINVAL;
    if (M < 0 || R < 0) return set_err(c, KC_EINVAL, "kc_sample_reduction: negative size");
    if (!lo || !hi || !active_inout) return set_err(c, KC_EINVAL, "kc_sample_reduction: NULL argument");
    if (reps && R > kMaxReps) return set_err(c, KC_EINVAL, "kc_sample_reduction: R > %d", kMaxReps);
    const size_t box = (size_t)M * c->K * c->D * c->esize;
    Stager sg(c);
    const int ilo = sg.add(lo, box, true), ihi = sg.add(hi, box, true);
    const int irp = sg.add(reps, (size_t)M * c->K * R * 8, true);
    // the mask is read and written: stage it as an input, copy it back after
    const bool mask_host = !is_device_ptr(active_inout);
    const int imk = sg.add(active_inout, (size_t)c->N, true);
    KC_TRY(sg.begin());
    const size_t rx_bytes = (size_t)M * c->K * std::max(R, 1) * c->D * c->esize;
    KC_TRY(ensure(c, c->work, rx_bytes + (size_t)M * c->K * 4 + 512));
    char *w = static_cast<char *>(c->work.p);
    void *repx = w;
    int *nreps = reinterpret_cast<int *>(w + ((rx_bytes + 255) & ~(size_t)255));
    unsigned long long *nact = reinterpret_cast<unsigned long long *>(
        w + ((rx_bytes + 255) & ~(size_t)255) + (((size_t)M * c->K * 4 + 255) & ~(size_t)255));
    if (reps) {
        {
            // validate indices on the host
            std::vector<int64_t> h((size_t)M * c->K * R);
            KC_CUDA(c, cudaMemcpyAsync(h.data(), sg.dev(irp), h.size() * 8, cudaMemcpyDeviceToHost, c->stream));
            KC_CUDA(c, cudaStreamSynchronize(c->stream));
            for (int64_t v : h)
                if (v >= c->N) return set_err(c, KC_EINVAL, "kc_sample_reduction: representative out of range");
        }
        KC_TRY(launch_gather_reps(c, M, R, static_cast<const int64_t *>(sg.dev(irp)), repx, nreps));
    }
    uint8_t *mask = static_cast<uint8_t *>(sg.dev(imk));
    KC_TRY(launch_sample_reduction_view(c, full_view(c), sg.dev(ilo), sg.dev(ihi), M, reps ? repx : nullptr,
                                        reps ? nreps : nullptr, std::max(R, 1), beta_glob, alpha, mask, nact));
    if (mask_host)
        KC_CUDA(c, cudaMemcpyAsync(active_inout, mask, (size_t)c->N, cudaMemcpyDeviceToHost, c->stream));
    if (n_active_out) {
        unsigned long long n = 0;
        KC_CUDA(c, cudaMemcpyAsync(&n, nact, 8, cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaStreamSynchronize(c->stream));
        int64_t v = (int64_t)n;
        if (is_device_ptr(n_active_out))
            KC_CUDA(c, cudaMemcpy(n_active_out, &v, 8, cudaMemcpyHostToDevice));
        else
            *n_active_out = v;
    }
    KC_CUDA(c, cudaStreamSynchronize(c->stream));
    return KC_OK;
}

kc_status kc_set_scorer(kc_ctx *c, kc_mlp *m)
{
    if (!c) return KC_EINVAL;
    c->scorer = m;
    return KC_OK;
}

void kc_solve_defaults(kc_solve_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-12;
    o->ball_cap = 50;
    o->i_sr = 1;
    o->use_bt = 1;
    o->lists = 1;
    o->rule_width = 4;
}

kc_status kc_solve(kc_ctx *c, double tol, const kc_solve_opts *opt, kc_result *out)
{
    if (!c) return KC_EINVAL;
    if (!out) return set_err(c, KC_EINVAL, "kc_solve: out is NULL");
    kc_solve_opts o;
    if (opt) o = *opt;
    else kc_solve_defaults(&o);
    if (tol >= 0) o.tol = tol;
    if (!(o.tol >= 0.0) || o.tol >= 1.0) return set_err(c, KC_EINVAL, "kc_solve: tol must be in [0, 1)");
    if (o.batch < 0 || o.batch > 4096) return set_err(c, KC_EINVAL, "kc_solve: batch must be in [0, 4096]");
    if (o.order != 0 && o.order != 1) return set_err(c, KC_EINVAL, "kc_solve: order must be 0 or 1");
    if (o.order == 1 && !c->scorer) return set_err(c, KC_EINVAL, "kc_solve: order = 1 needs kc_set_scorer");
    if (o.lists != 0 && o.lists != 1) return set_err(c, KC_EINVAL, "kc_solve: lists must be 0 or 1");
    if (o.arena_mb < 0) return set_err(c, KC_EINVAL, "kc_solve: arena_mb must be >= 0");
    if (o.ball_cap == KC_BALLS_ALL && (c->dt != KC_F32 || c->D > 16 || (o.lists && c->D <= 8)))
        return set_err(c, KC_EINVAL, "kc_solve: ball_cap = KC_BALLS_ALL needs float data, D <= 16 and lists = 0");
    if (o.explore < 0 || o.explore > 100) return set_err(c, KC_EINVAL, "kc_solve: explore must be in [0, 100]");
    if (!(o.rule_margin >= 0.0)) return set_err(c, KC_EINVAL, "kc_solve: rule_margin must be >= 0");
    if (o.fft_starts < 0 || o.fft_starts > 4096) return set_err(c, KC_EINVAL, "kc_solve: fft_starts must be in [0, 4096]");
    if (o.rule_width < 0) return set_err(c, KC_EINVAL, "kc_solve: rule_width must be >= 0");
    std::memset(out, 0, sizeof(*out));
    if (c->dt == KC_F32) return solve_impl<float>(c, o, out);
    return solve_impl<double>(c, o, out);
}

}  // extern "C"
