// kc_internal.cuh -- private declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <type_traits>
#include <cmath>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/kc.h"

namespace kc {

constexpr int kMaxK = 16;
constexpr int kMaxD = 128;
constexpr int kMaxReps = 50;
constexpr int kMaxPairs = 16;   // attribute pairs a < b along which representatives are taken
constexpr int kThreads = 256;

// Growable device buffer owned by a context.
struct DevBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

// Workspace and outputs of one tightening call that later steps reuse.
struct VisitScratch {
    DevBuf buf;
    DevBuf jbuf;                     // every-sample representatives: the sets J_A^k as lists
    const int64_t *reps = nullptr;   // [B][K][RM] representative sample ids (-1 unused)
    const int *nreps = nullptr;      // [B][K]
    const void *repx = nullptr;      // [B][K][RM][D] their coordinates
    int RM = 0;
};

}  // namespace kc

struct kc_mlp;

struct kc_ctx {
    int dev = 0;
    int num_sms = 0;
    size_t smem_optin = 0;       // max dynamic shared memory per block
    cudaStream_t stream = nullptr;
    int64_t N = 0;
    int D = 0, K = 0;
    kc_dtype dt = KC_F32;
    size_t esize = 4;
    int64_t ldx = 0;             // padded row length of the attribute-major copy
    void *X = nullptr;           // [D][ldx] owned device copy
    // scratch
    kc::DevBuf part;             // per-CTA partial results
    kc::DevBuf stage_in;         // staged host inputs
    kc::DevBuf stage_out;        // device-side outputs destined for host
    kc::DevBuf work;             // per-call work arrays
    kc::VisitScratch vs;         // tightening workspace
    kc_mlp *scorer = nullptr;    // learned node scorer used by kc_solve with order = 1
    void *pinned = nullptr;      // pinned host staging
    size_t pinned_bytes = 0;
    int64_t launches = 0;
    std::string err;
    // launch shape of the float lower-bound kernel, set by kc_autotune (kc_lb.cu)
    int lb_st = 0;               // samples per thread of the float lower-bound kernel
    int lb_chunk = 0;            // node chunk of the float lower-bound kernel (0: largest that fits)
};

namespace kc {

// ------------------------------------------------------------------ errors

kc_status set_err(kc_ctx *c, kc_status st, const char *fmt, ...);

#define KC_CUDA(ctx, call)                                                              \
    do {                                                                                \
        cudaError_t e_ = (call);                                                        \
        if (e_ != cudaSuccess)                                                          \
            return ::kc::set_err((ctx), KC_ECUDA, "%s: %s (%s:%d)", #call,              \
                                 cudaGetErrorString(e_), __FILE__, __LINE__);           \
    } while (0)

#define KC_TRY(expr)                                                                    \
    do {                                                                                \
        kc_status s_ = (expr);                                                          \
        if (s_ != KC_OK) return s_;                                                     \
    } while (0)

// Checks the launch that was just issued and counts it.
kc_status after_launch(kc_ctx *c, const char *what);

// ------------------------------------------------------------ buffers

kc_status ensure(kc_ctx *c, DevBuf &b, size_t bytes);
kc_status ensure_pinned(kc_ctx *c, size_t bytes);
bool is_device_ptr(const void *p);

// A host or device array argument resolved to a device pointer.  Inputs in
// host memory are copied into `buf` (cudaMemcpyAsync on the context stream);
// outputs in host memory get device scratch and are copied back by
// finish_outputs().
struct OutArg {
    void *user = nullptr;   // caller pointer
    void *dev = nullptr;    // where kernels write
    size_t bytes = 0;
    bool host = false;
};

// --------------------------------------------------------- rounding margins

// gamma_n = n u / (1 - n u): relative error bound of n roundings (Higham 3.1).
inline double gamma_n(int n, double u) { return (n * u) / (1.0 - n * u); }

// Float evaluation of a clamp or point distance in this library: the
// difference (one rounding, squared), ceil(D/2) fused multiply-adds in each
// of two interleaved chains, one final add.
inline int f32_roundings(int D) { return 2 + (D + 1) / 2 + 1; }
// Double evaluation in attribute order with separate multiply and add.
inline int f64_roundings(int D) { return D + 3; }

constexpr double kU32 = 5.9604644775390625e-08;   // 2^-24
constexpr double kU64 = 1.1102230246251565e-16;   // 2^-53

// Multiplier that maps an evaluated distance to a certified lower bound
// (applied with round-down); and the absolute slack for underflow.
inline double deflate_factor(kc_dtype dt, int D)
{
    double g = dt == KC_F32 ? gamma_n(f32_roundings(D), kU32) : gamma_n(f64_roundings(D) + 1, kU64);
    return (1.0 - g) * (1.0 - 4 * kU64);
}
inline double underflow_slack(kc_dtype dt, int D)
{
    return dt == KC_F32 ? (D + 2) * 1.401298464324817e-45 : (D + 2) * 4.9406564584124654e-324;
}

// A set of samples the kernels stream: attribute-major rows X[a*ld + pos],
// pos < n; ids[pos] is the sample's index in the full dataset (NULL: pos).
struct View {
    const void *X = nullptr;
    int64_t ld = 0;
    int64_t n = 0;
    const uint32_t *ids = nullptr;
};
inline View full_view(const kc_ctx *c)
{
    View v;
    v.X = c->X;
    v.ld = c->ldx;
    v.n = c->N;
    return v;
}

// Thresholds of the float proofs in the tightening kernels: a distance d
// evaluated as d' satisfies d' (1 - g) <= d <= d' / (1 - g).
struct Margins {
    float defl, infl, slack;     // float evaluation of a D-term distance
    float alpha_up, four_up;     // alpha and 4 alpha rounded up to float
    float beta_dn;               // beta_glob rounded down to float
    // single-compare proofs: a float distance d' > t_alpha proves d > alpha,
    // d' > t_four proves d > 4 alpha (t = RU((RU(target) + slack) / defl * (1 + 1e-6)))
    float t_alpha, t_four;
};

// Per-node sample-id lists of a batch of nodes (device arrays).  Nodes that
// share one list form a group: group g's list is pool[seg_off[g] ..
// seg_off[g] + seg_n[g]) and its nodes are node_start[g] .. node_start[g + 1]
// - 1 (node_start NULL: group g is node g alone).  Work item w covers entries
// [t * list_tile(), (t + 1) * list_tile()) of group g's list, where g is the
// group with tile_prefix[g] <= w < tile_prefix[g + 1] and t = w - tile_prefix[g];
// a staged tile serves every node of its group.
struct ListBatch {
    const uint32_t *pool = nullptr;
    const int64_t *seg_off = nullptr;
    const int64_t *seg_n = nullptr;
    const int64_t *tile_prefix = nullptr;   // [B + 1]
    const int *node_start = nullptr;        // [B + 1] or NULL
    int B = 0;                              // groups
    int64_t W = 0;                          // tile_prefix[B]
};

// ----------------------------------------------------------- kernel launchers
// (implemented in the .cu files; all run on c->stream)

// Lower bounds of B nodes (device lo/hi [B][K][D]) -> device lb, lb_raw, argmax.
kc_status launch_lower_bounds(kc_ctx *c, const void *lo, const void *hi, int B, double *lb,
                              double *lb_raw, int64_t *argmax);
kc_status launch_lower_bounds_view(kc_ctx *c, const View &v, const void *lo, const void *hi, int B,
                                   double *lb, double *lb_raw, int64_t *arg, int st_override);
kc_status launch_lower_bounds_cfg(kc_ctx *c, const View &v, const void *lo, const void *hi, int B, double *lb,
                                  double *lb_raw, int64_t *arg, int st_override, int chunk_override);
kc_status launch_lower_bounds_refine(kc_ctx *c, const View &v, const void *lo, const void *hi, int B,
                                     const double *raw_host, double *lb_out, double *lb_exact_out, int64_t *arg);
kc_status autotune_lower_bounds(kc_ctx *c, const void *lo, const void *hi, int B, double *lb_scratch, int *st_out,
                                int *chunk_out, float *ms_out);

// Objective (Eq. 1) of S center sets given by device indices [S][K] ->
// device values [S] (double, exact serial-double value) and argmax [S].
// alpha_cut: sets whose float screen proves a value >= alpha_cut are not
// evaluated exactly (their val is set to +inf); pass +inf to evaluate all.
// pts (nullable, device [S][Kc][D] of the data type): the centers as points
// instead of sample indices (centers is then ignored).
kc_status launch_objective(kc_ctx *c, const View &v, const int64_t *centers, int S, int Kc,
                           double alpha_cut, double *val, int64_t *arg, const void *pts = nullptr);

// Per-attribute min/max of the data; *nonfinite set if any NaN/Inf.
kc_status launch_root_box(kc_ctx *c, void *lo, void *hi, int *nonfinite_dev);

// Attribute-major padded copy from the user's layout.
kc_status launch_ingest(kc_ctx *c, const void *src, kc_layout layout, int64_t N, int D);
// Rows s0 .. s0 + n of a row-major dataset staged on the device as [n][D]
// into the context's attribute-major copy (padding not touched).
kc_status launch_ingest_rows(kc_ctx *c, const void *chunk_dev, int64_t s0, int64_t n);

// Cluster assignment + bounds tightening of B nodes over a sample view (see kc.h).
kc_status launch_tighten_view(kc_ctx *c, const View &v, const void *lo, const void *hi, int B, double alpha,
                              const int64_t *seeds_dev, int ball_cap, void *lo_out, void *hi_out, int64_t *counts,
                              int64_t *cand, double *lb, double *lb_raw, int64_t *lbarg, int8_t *status,
                              VisitScratch *vs);

// Sample reduction (Algorithm 5) of the samples of a view against M nodes
// with representative coordinates repx [M][K][R][D] (nreps [M][K]).
kc_status launch_sample_reduction_view(kc_ctx *c, const View &v, const void *lo, const void *hi, int M,
                                       const void *repx, const int *nreps, int R, double beta_glob, double alpha,
                                       uint8_t *mask, unsigned long long *n_active);

// Passes A and B of the float tightening for any K <= 16, D <= 128 (kc_wide.cu;
// the workspace and finalize kernels are kc_visit.cu's).
// Step B with every sample of J_A^k as a representative of k (no budget):
// builds the sets J_A^k of the B nodes as lists of view positions in
// vs->jbuf, then runs the tiled sample x J_A^k pass; same accumulators as
// launch_wide_b.
kc_status launch_wide_ball_all(kc_ctx *c, const View &v, const float *lo, const float *hi, int B, const Margins &mg,
                               const float *blo, const float *bhi, const int *allhave, const int64_t *seeds,
                               unsigned long long *cnt, unsigned long long *cand, unsigned *smax, unsigned *smin,
                               unsigned *jmax, unsigned *jmin, unsigned *flags, VisitScratch *vs);

// ndir > 0 (at most 32): also the arg-extreme keys of the assigned samples
// along the attribute-pair directions, dmax / dmin [B][K][ndir].
kc_status launch_wide_a(kc_ctx *c, const View &v, const ListBatch *L, const float *lo, const float *hi, int B,
                        const Margins &mg, unsigned long long *lbkey, unsigned long long *amax,
                        unsigned long long *amin, unsigned *flags, int ndir, unsigned long long *dmax,
                        unsigned long long *dmin);
kc_status launch_wide_b(kc_ctx *c, const View &v, const ListBatch *L, const float *lo, const float *hi, int B,
                        const Margins &mg, const float *blo, const float *bhi, const float *repx, const int *nreps,
                        const int *allhave, const int64_t *seeds, int RM, unsigned long long *cnt,
                        unsigned long long *cand, unsigned *smax, unsigned *smin, unsigned *jmax, unsigned *jmin,
                        unsigned *flags);

// Coordinates of representative ids [M][K][R] (-1 = unused) -> repx, nreps.
kc_status launch_gather_reps(kc_ctx *c, int M, int R, const int64_t *reps, void *repx, int *nreps);

// Stable compaction of the view's samples with mask[pos] != 0 into Xo [D][ldo]
// and ids ido; the kept count lands in *total_dev.  scratch_counts needs
// compact_blocks(v.n) entries.
kc_status launch_compact(kc_ctx *c, const View &v, const uint8_t *mask, void *Xo, int64_t ldo, uint32_t *ido,
                         unsigned *scratch_counts, unsigned long long *total_dev);
int64_t compact_blocks(int64_t n);

// Staging of one call's array arguments.  Inputs in host memory are copied to
// device scratch; outputs in host memory are written to device scratch and
// copied back by finish().
struct Stager {
    kc_ctx *c;
    struct Item {
        const void *user;
        size_t bytes;
        size_t off;
        bool in;
        bool host;
    };
    std::vector<Item> items;
    size_t total = 0;
    explicit Stager(kc_ctx *cc) : c(cc) {}

    // Registers an argument; returns its index.
    int add(const void *user, size_t bytes, bool in)
    {
        Item it{user, bytes, 0, in, user != nullptr && !is_device_ptr(user)};
        if (it.host) {
            it.off = total;
            total += (bytes + 255) & ~(size_t)255;
        }
        items.push_back(it);
        return (int)items.size() - 1;
    }
    // Allocates scratch and copies host inputs; then dev(i) is valid.
    kc_status begin()
    {
        if (total == 0) return KC_OK;
        KC_TRY(ensure(c, c->stage_in, total));
        for (auto &it : items)
            if (it.host && it.in && it.bytes)
                KC_CUDA(c, cudaMemcpyAsync(static_cast<char *>(c->stage_in.p) + it.off, it.user, it.bytes,
                                           cudaMemcpyHostToDevice, c->stream));
        return KC_OK;
    }
    void *dev(int i) const
    {
        const Item &it = items[i];
        if (!it.user) return nullptr;
        return it.host ? static_cast<char *>(c->stage_in.p) + it.off : const_cast<void *>(it.user);
    }
    bool any_host_out() const
    {
        for (auto &it : items)
            if (it.host && !it.in) return true;
        return false;
    }
    // Copies host outputs back and waits when any output is in host memory.
    kc_status finish()
    {
        bool wait = false;
        for (auto &it : items)
            if (it.host && !it.in && it.bytes) {
                KC_CUDA(c, cudaMemcpyAsync(const_cast<void *>(it.user), static_cast<char *>(c->stage_in.p) + it.off,
                                           it.bytes, cudaMemcpyDeviceToHost, c->stream));
                wait = true;
            }
        if (wait) KC_CUDA(c, cudaStreamSynchronize(c->stream));
        return KC_OK;
    }
};


// Scores B nodes: device features [B][12] -> device outputs [B][2].
kc_status mlp_forward_device(kc_mlp *m, const float *feats, int B, float *out, cudaStream_t stream);

// ---- per-node sample lists (kc_lists.cu)
int list_tile();
kc_status launch_iota(kc_ctx *c, uint32_t *p, int64_t n);
kc_status launch_seg_lb(kc_ctx *c, const ListBatch &L, const void *lo, const void *hi, int B, unsigned long long *keys,
                        double *lb, double *raw, int64_t *arg);
// wit (nullable, device [B]): the sample attaining each refined value (wid:
// device scratch [B]), found by a second pass over the lists.
kc_status launch_seg_refine(kc_ctx *c, const ListBatch &L, const void *lo, const void *hi, int B, const double *raw_host,
                            float *thr_dev, unsigned long long *vmax, double *out, unsigned *wid, int64_t *wit);
kc_status launch_seg_objective(kc_ctx *c, const ListBatch &L, const int64_t *centers, int B, double alpha_cut,
                               unsigned long long *keys, unsigned long long *vmax, float *thr, double *val);
kc_status launch_seg_filter(kc_ctx *c, const ListBatch &L, const void *lo, const void *hi, int B,
                            const float *beta_dn_dev, double alpha, const void *repx, const int *nreps, int RM,
                            const int *rmap, uint32_t *out_pool, const int64_t *out_off, const int64_t *out_cap,
                            unsigned long long *out_n, const int *cvar, const float *csplit,
                            unsigned long long *ckeys, double *child_lb, double *child_raw, int64_t *child_arg);
// Tightening of B nodes, each over its own list (float data).
kc_status launch_tighten_list(kc_ctx *c, const ListBatch &L, const void *lo, const void *hi, int B, double alpha,
                              const int64_t *seeds_dev, int ball_cap, void *lo_out, void *hi_out, int64_t *counts,
                              int64_t *cand, double *lb, double *lb_raw, int64_t *lbarg, int8_t *status,
                              VisitScratch *vs);

}  // namespace kc
