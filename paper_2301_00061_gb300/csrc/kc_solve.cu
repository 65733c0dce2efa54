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
//      branch the rest on the max-range variable at its midpoint; children
//      inherit the parent's certified bound as their key;
//   5. every i_sr batches, sample reduction against the hull of the open
//      nodes, then compaction of the surviving samples.
// Bounds are computed when a node is visited rather than when it is created
// (the children of one batch are bounded in the next), so one pass per node
// evaluates its bound, tightens it and yields its candidate.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
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
};

template <typename T>
struct NodeCmp {
    bool operator()(const Node<T> &a, const Node<T> &b) const
    {
        return a.key > b.key || (a.key == b.key && a.id > b.id);
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

struct SolveBufs {
    DevBuf boxes, outs, sets, mask, counts, xbuf[2], idbuf[2];
};

template <typename T>
kc_status solve_impl(kc_ctx *c, const kc_solve_opts &o, kc_result *res)
{
    const double t0 = now_s();
    const int K = c->K, D = c->D, KD = K * D;
    const double tol = o.tol;
    SolveBufs sb;
    auto cleanup = [&]() {
        for (DevBuf *b : {&sb.boxes, &sb.outs, &sb.sets, &sb.mask, &sb.counts, &sb.xbuf[0], &sb.xbuf[1], &sb.idbuf[0],
                          &sb.idbuf[1]})
            if (b->p) cudaFree(b->p);
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
    const int64_t start = (int64_t)(o.seed % (uint64_t)c->N);
    KC_TRY(ensure(c, sb.sets, 4096));
    int64_t *T_dev = static_cast<int64_t *>(sb.sets.p);
    double *v_dev = reinterpret_cast<double *>(static_cast<char *>(sb.sets.p) + 1024);
    KC_CUDA(c, cudaMemcpyAsync(T_dev, &start, 8, cudaMemcpyHostToDevice, c->stream));
    for (int t = 1; t < K; ++t)
        KC_TRY(launch_objective(c, full_view(c), T_dev, 1, t, __builtin_huge_val(), v_dev, T_dev + t));
    KC_TRY(launch_objective(c, full_view(c), T_dev, 1, K, __builtin_huge_val(), v_dev, nullptr));
    std::vector<int64_t> inc(K);
    double alpha = 0.0;
    KC_CUDA(c, cudaMemcpyAsync(inc.data(), T_dev, K * 8, cudaMemcpyDeviceToHost, c->stream));
    KC_CUDA(c, cudaMemcpyAsync(&alpha, v_dev, 8, cudaMemcpyDeviceToHost, c->stream));
    KC_CUDA(c, cudaStreamSynchronize(c->stream));
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
        r.id = 0;
        r.parent = -1;
        r.depth = 0;
        heap.push_back(std::move(r));
    }
    int64_t next_id = 1;

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

    View cur = full_view(c);
    int ping = 0;
    int64_t visits = 0, batches = 0;
    kc_status status = KC_OK;
    std::vector<Node<T>> batch;
    std::vector<int> live;
    FILE *log = o.log_path ? fopen(o.log_path, "w") : nullptr;

    auto prune_threshold = [&]() { return alpha - tol * alpha; };

    for (;;) {
        // stop test: the smallest key over the open nodes against alpha
        while (!heap.empty() && heap.front().key >= prune_threshold()) {
            // the heap is ordered: every node is prunable
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
            if (nd.key >= prune_threshold()) continue;
            batch.push_back(std::move(nd));
        }
        if (batch.empty()) continue;
        const int B = (int)batch.size();
        for (int b = 0; b < B; ++b) {
            std::memcpy(h_lo + (size_t)b * KD, batch[b].lo.data(), KD * sizeof(T));
            std::memcpy(h_hi + (size_t)b * KD, batch[b].hi.data(), KD * sizeof(T));
        }
        KC_CUDA(c, cudaMemcpyAsync(d_lo, h_lo, (size_t)B * KD * sizeof(T), cudaMemcpyHostToDevice, c->stream));
        KC_CUDA(c, cudaMemcpyAsync(d_hi, h_hi, (size_t)B * KD * sizeof(T), cudaMemcpyHostToDevice, c->stream));

        // 2. bound + tighten
        if (o.use_bt) {
            KC_TRY(launch_tighten_view(c, cur, d_lo, d_hi, B, alpha, seeds_dev, o.ball_cap, d_lo2, d_hi2, nullptr,
                                       d_cand, d_lb, nullptr, nullptr, d_st, &c->vs));
        } else {
            KC_TRY(launch_tighten_view(c, cur, d_lo, d_hi, B, __builtin_huge_val(), nullptr, 1, d_lo2, d_hi2, nullptr,
                                       d_cand, d_lb, nullptr, nullptr, d_st, &c->vs));
        }
        KC_CUDA(c, cudaMemcpyAsync(h_lo2, d_lo2, (size_t)B * KD * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaMemcpyAsync(h_hi2, d_hi2, (size_t)B * KD * sizeof(T), cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaMemcpyAsync(h_cand, d_cand, (size_t)B * K * 8, cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaMemcpyAsync(h_lb, d_lb, (size_t)B * 8, cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaMemcpyAsync(h_st, d_st, (size_t)B, cudaMemcpyDeviceToHost, c->stream));
        KC_CUDA(c, cudaStreamSynchronize(c->stream));
        visits += B;
        ++batches;

        // 3. upper bounds of the live nodes' candidates
        live.clear();
        for (int b = 0; b < B; ++b) {
            const double lb = std::max(h_lb[b], batch[b].key);
            batch[b].key = lb;
            if (h_st[b] == 1 || lb >= prune_threshold()) continue;
            live.push_back(b);
        }
        if (!live.empty()) {
            const int S = (int)live.size();
            for (int i = 0; i < S; ++i)
                for (int k = 0; k < K; ++k) h_sets[(size_t)i * K + k] = h_cand[(size_t)live[i] * K + k];
            KC_CUDA(c, cudaMemcpyAsync(d_sets, h_sets, (size_t)S * K * 8, cudaMemcpyHostToDevice, c->stream));
            KC_TRY(launch_objective(c, cur, d_sets, S, K, alpha, d_val, nullptr));
            KC_CUDA(c, cudaMemcpyAsync(h_val, d_val, (size_t)S * 8, cudaMemcpyDeviceToHost, c->stream));
            KC_CUDA(c, cudaStreamSynchronize(c->stream));
            for (int i = 0; i < S; ++i)
                if (h_val[i] < alpha) {
                    alpha = h_val[i];
                    for (int k = 0; k < K; ++k) inc[k] = h_sets[(size_t)i * K + k];
                }
        }

        // 4. prune, close leaves, branch
        for (int b : live) {
            Node<T> &nd = batch[b];
            if (nd.key >= prune_threshold()) continue;
            T *lo = h_lo2 + (size_t)b * KD, *hi = h_hi2 + (size_t)b * KD;
            bool leaf = h_st[b] == 2;
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
            if (log)
                fprintf(log, "{\"id\":%lld,\"parent\":%lld,\"depth\":%d,\"lb\":%.17g,\"alpha\":%.17g,\"status\":%d}\n",
                        (long long)nd.id, (long long)nd.parent, nd.depth, nd.key, alpha, (int)h_st[b]);
            if (leaf) continue;
            int bi = -1;
            double br = 0.0;
            for (int i = 0; i < KD; ++i) {
                const double r = (double)hi[i] - (double)lo[i];
                if (r > br) { br = r; bi = i; }
            }
            if (bi < 0) {
                // every box became a point after symmetry breaking: visit again
                Node<T> again;
                again.lo.assign(lo, lo + KD);
                again.hi.assign(hi, hi + KD);
                again.key = nd.key;
                again.id = next_id++;
                again.parent = nd.id;
                again.depth = nd.depth + 1;
                heap.push_back(std::move(again));
                std::push_heap(heap.begin(), heap.end(), cmp);
                continue;
            }
            T m, succ;
            split_point<T>(lo[bi], hi[bi], &m, &succ);
            for (int side = 0; side < 2; ++side) {
                Node<T> ch;
                ch.lo.assign(lo, lo + KD);
                ch.hi.assign(hi, hi + KD);
                if (side == 0) ch.hi[bi] = m;
                else ch.lo[bi] = succ;
                ch.key = nd.key;
                ch.id = next_id++;
                ch.parent = nd.id;
                ch.depth = nd.depth + 1;
                heap.push_back(std::move(ch));
                std::push_heap(heap.begin(), heap.end(), cmp);
            }
        }

        // 5. sample reduction against the hull of the open nodes (Algorithm 5)
        if (o.i_sr > 0 && batches % o.i_sr == 0 && !heap.empty() && heap.front().key < prune_threshold()) {
            std::vector<T> hlo(KD), hhi(KD);
            for (int i = 0; i < KD; ++i) { hlo[i] = heap[0].lo[i]; hhi[i] = heap[0].hi[i]; }
            for (const auto &nd : heap)
                for (int i = 0; i < KD; ++i) {
                    hlo[i] = std::min(hlo[i], nd.lo[i]);
                    hhi[i] = std::max(hhi[i], nd.hi[i]);
                }
            const double beta_glob = heap.front().key;
            // hull boxes and the seed representatives go after the batch boxes
            std::memcpy(h_lo, hlo.data(), KD * sizeof(T));
            std::memcpy(h_hi, hhi.data(), KD * sizeof(T));
            KC_CUDA(c, cudaMemcpyAsync(d_lo, h_lo, KD * sizeof(T), cudaMemcpyHostToDevice, c->stream));
            KC_CUDA(c, cudaMemcpyAsync(d_hi, h_hi, KD * sizeof(T), cudaMemcpyHostToDevice, c->stream));
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
                KC_TRY(launch_gather_reps(c, 1, 1, seeds_dev, d_lo2, reinterpret_cast<int *>(d_sets)));
                repx = d_lo2;
                nreps = reinterpret_cast<const int *>(d_sets);
            }
            KC_TRY(launch_sample_reduction_view(c, cur, d_lo, d_hi, 1, repx, nreps, 1, beta_glob, alpha, mask,
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
    }
    if (log) fclose(log);

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
    res->active_final = cur.n;
    res->seconds = now_s() - t0;
    res->status = status;
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

void kc_solve_defaults(kc_solve_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->tol = 1e-12;
    o->ball_cap = 50;
    o->i_sr = 1;
    o->use_bt = 1;
    o->use_graph = 1;
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
    if (o.order != 0) return set_err(c, KC_EINVAL, "kc_solve: learned ordering needs scorer weights");
    std::memset(out, 0, sizeof(*out));
    if (c->dt == KC_F32) return solve_impl<float>(c, o, out);
    return solve_impl<double>(c, o, out);
}

}  // extern "C"
