/*
 * kc.h -- C ABI of the GB300 K-center branch-and-bound library (libkc.so).
 *
 * The library evaluates the data-parallel steps of the reduced-space branch
 * and bound for K-center clustering of Ren, You, Hua, Ji and Cao ("A Global
 * Optimization Algorithm for K-Center Clustering of One Billion Samples"):
 * node lower bounds (Section 3.1), upper bounds (Section 3.2), farthest first
 * traversal (Algorithm 2), cluster assignment and bounds tightening
 * (Section 4.1, Algorithms 3-4), sample reduction (Section 4.2, Algorithm 5)
 * and the branch-and-bound loop itself (Algorithm 1), on one CUDA GPU.
 *
 * Notation: N samples (the paper's S), D attributes (the paper's A), K
 * clusters, B nodes.  A node is K axis-aligned boxes, one per cluster:
 * lo[k*D + a] <= mu^k_a <= hi[k*D + a]; a batch of B nodes is the arrays
 * lo[B][K][D] and hi[B][K][D] in the data's element type.  All distances are
 * squared Euclidean (Eq. 1).  Ties in every argmax/argmin go to the smallest
 * sample index.
 *
 * Pointers.  Every array argument may be host memory (pageable or pinned) or
 * device memory of the context's GPU; the library checks which with
 * cudaPointerGetAttributes and stages host arrays through its own buffers.
 * Calls are ordered on the context's stream.  A call whose outputs are all in
 * device memory returns without waiting for the GPU; a call with any output in
 * host memory returns after the results are written.
 *
 * Errors.  Every call returns a kc_status; nothing is thrown across the ABI.
 * On failure the outputs are unspecified and kc_last_error() describes the
 * cause.  After KC_ECUDA the context should be destroyed; after any other
 * error it stays usable.  Limits: 1 <= K <= 16, 1 <= D <= 128,
 * K <= N <= 4,294,967,294.
 */
#ifndef KC_H_
#define KC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kc_ctx kc_ctx;

typedef enum {
    KC_OK = 0,
    KC_EINVAL = 1,     /* bad argument or non-finite data */
    KC_ENOMEM = 2,     /* device or host allocation failed */
    KC_ECUDA = 3,      /* a CUDA call failed; destroy the context */
    KC_ETIMEOUT = 4,   /* kc_solve stopped at its time limit */
    KC_ELIMIT = 5,     /* kc_solve stopped at its node limit */
    KC_EINTERNAL = 6
} kc_status;

typedef enum { KC_F32 = 0, KC_F64 = 1 } kc_dtype;
typedef enum { KC_ROW_MAJOR = 0, KC_COL_MAJOR = 1 } kc_layout;

/*
 * kc_create -- upload a dataset and make a context.
 *   X       N*D values of type dt; KC_ROW_MAJOR: X[s*D + a]; KC_COL_MAJOR:
 *           X[a*N + s].  Host or device.  The library keeps its own
 *           device copy (attribute-major, padded rows), so X may be freed
 *           after the call returns.
 *   stream  a cudaStream_t (e.g. torch.cuda.current_stream().cuda_stream),
 *           or NULL for the legacy default stream.  The context must only be
 *           used from one host thread at a time.
 *   out     receives the context; NULL on failure.
 * Rejects NaN or infinite data with KC_EINVAL.  The dataset X of Eq. 1.
 */
kc_status kc_create(const void *X, int64_t N, int32_t D, int32_t K, kc_dtype dt, kc_layout layout,
                    void *stream, kc_ctx **out);

/* Frees the context and everything it owns.  NULL is accepted. */
void kc_destroy(kc_ctx *ctx);

/* Message of the last failed call on this context (never NULL). */
const char *kc_last_error(const kc_ctx *ctx);

/* Message of the last failed kc_create in this process (never NULL). */
const char *kc_create_error(void);

/* Changes the stream later calls are ordered on. */
kc_status kc_set_stream(kc_ctx *ctx, void *stream);

/* Number of this library's own kernels launched on the context so far. */
int64_t kc_launch_count(const kc_ctx *ctx);

/*
 * kc_root_box -- the region of centers M0 (Section 2.1): lo[a] = min_s x_{s,a},
 * hi[a] = max_s x_{s,a} (the same box for every cluster).  lo, hi: D values of
 * the data type.  Exact (no rounding).
 */
kc_status kc_root_box(kc_ctx *ctx, void *lo, void *hi);

/*
 * kc_lower_bounds -- the closed-form node lower bound of Section 3.1:
 *   beta(M) = max_s min_k beta_s^k(M^k),  beta_s^k = sum_a (x_{s,a} - mid{lo, x_{s,a}, hi})^2
 * (Eqs. 9-11), for B nodes, over all N samples.
 *   lo, hi     [B][K][D] of the data type, lo <= hi.
 *   lb_out     [B] double: a certified bound, never above the exact real value
 *              of beta(M); for float data it is the float evaluation deflated
 *              by its proved rounding-error bound (relative gap at most
 *              2 gamma_n, n = ceil(D/2) + 3, gamma_n = n u / (1 - n u),
 *              u = 2^-24: below 1e-6 for D <= 10, 1.3e-6 at D = 16; in
 *              practice far smaller), for double data the double evaluation deflated by a
 *              few units in the last place.
 *   lb_raw_out [B] double or NULL: the value as evaluated (float data: the
 *              float result; double data: bit-identical to a serial
 *              double-precision evaluation in attribute order).
 *   argmax_out [B] int64 or NULL: a sample attaining the evaluated maximum
 *              (smallest index on ties).
 * Node batches larger than the shared-memory budget are processed in chunks.
 */
kc_status kc_lower_bounds(kc_ctx *ctx, const void *lo, const void *hi, int32_t B, double *lb_out,
                          double *lb_raw_out, int64_t *argmax_out);

/*
 * kc_lower_bounds_noalloc -- the float lower bound of kc_lower_bounds without a
 * context and without allocating any memory.  The paper has no counterpart:
 * this entry point exists for callers that cannot allocate GPU memory at the
 * point where they need bounds -- a process whose device memory is already
 * reserved by another allocator (a framework's caching pool holding nearly
 * all of it), or a latency-critical loop where the device-wide
 * synchronization that cudaMalloc / cudaFree can imply is not acceptable.
 *   X          device, float, attribute-major: X[a*ld + s]; when X is 16-byte
 *              aligned and ld is a multiple of 4 the vectorized kernel is used.
 *   N, ld, D, K  samples, row length (ld >= N), attributes, clusters.
 *   lo, hi     device [B][K][D] float boxes.
 *   lb_out, lb_raw_out, argmax_out  device, as in kc_lower_bounds (the last
 *              two may be NULL).
 *   stream     cudaStream_t the work is ordered on.
 * Every non-NULL array must be device (or managed) memory of the current
 * GPU; anything else -- a host array in particular -- returns KC_EINVAL
 * before any launch (checked with cudaPointerGetAttributes, which allocates
 * nothing).  If a CUDA error is already pending in the calling thread the
 * call returns KC_ECUDA at once, launches nothing and leaves that error in
 * place for its owner.
 * Scratch is one fixed array in the library (512 partial results for each of
 * 256 nodes, 1 MiB, kept by every GPU that loads the library until the
 * process exits); nodes are processed 256 at a time and B may be at most
 * 4096 (larger B returns KC_EINVAL).  The first call on a device looks up the
 * array's device address with that device current and keeps it for the
 * process; make that first call before any stream capture, and do not call
 * the entry point on a device after cudaDeviceReset (the kept address would
 * be stale).  Every call reuses the same array, so calls that can overlap on
 * the GPU (different streams, no ordering between them) race and must not be
 * issued.  Returns KC_EINVAL for bad sizes or pointers, KC_ECUDA if a CUDA
 * call fails.  Nothing is written to an error string.
 */
kc_status kc_lower_bounds_noalloc(const float *X, int64_t N, int64_t ld, int32_t D, int32_t K,
                                  const float *lo, const float *hi, int32_t B, double *lb_out,
                                  double *lb_raw_out, int64_t *argmax_out, void *stream);

/*
 * kc_autotune -- picks the launch shape of the float lower-bound kernel
 * (samples per thread, nodes per launch: occupancy against extra passes over
 * the samples) by timing each candidate with CUDA events on the given batch
 * of B nodes (lo, hi as in kc_lower_bounds), and keeps the fastest for later
 * kc_lower_bounds calls on this context.  Outputs (host, each may be NULL):
 * the chosen samples per thread, nodes per launch, and its time per batch in
 * ms.  Double data: nothing to tune (outputs 0).  A scheduling choice; the
 * paper has no counterpart (the bound itself is Section 3.1's).
 */
kc_status kc_autotune(kc_ctx *ctx, const void *lo, const void *hi, int32_t B, int32_t *samples_per_thread_out,
                      int32_t *nodes_per_launch_out, float *ms_out);

/*
 * kc_upper_bound -- the objective of Eq. 1 at S center sets on samples
 * (the upper bound alpha(M) of Eq. 12):
 *   alpha = max_s min_k ||x_s - x_{c_k}||^2.
 *   centers    [S][K] int64 sample indices in [0, N).
 *   ub_out     [S] double: the value in double precision, bit-identical to a
 *              serial double evaluation (attribute order, no fused multiply-add),
 *              over all N samples.
 *   worst_out  [S] int64 or NULL: the sample attaining it (smallest index on ties).
 * Float data are screened in float with a proved error bound and only the
 * samples that can attain the maximum are re-evaluated in double.
 */
kc_status kc_upper_bound(kc_ctx *ctx, const int64_t *centers, int32_t S, double *ub_out,
                         int64_t *worst_out);

/*
 * kc_upper_bound_points -- the objective of Eq. 1 at S sets of Kc centers given
 * as points (not necessarily samples): max_s min_k ||x_s - mu_k||^2 over all N
 * samples, evaluated as kc_upper_bound does (float data: float screen, double
 * re-evaluation of the samples that can attain the maximum).  Used where a
 * center's coordinates are known but the sample is not in this context (the
 * samples split across several contexts, Section 4.3), and for centers off the
 * samples.
 *   pts        [S][Kc][D] of the data type, finite (KC_EINVAL otherwise).
 *   Kc         centers per set, 1 <= Kc <= 16 (any, not only K); S <= 65536.
 *   ub_out     [S] double; worst_out [S] int64 or NULL (smallest index on ties).
 */
kc_status kc_upper_bound_points(kc_ctx *ctx, const void *pts, int32_t S, int32_t Kc, double *ub_out,
                                int64_t *worst_out);

/*
 * kc_fft -- Farthest First Traversal, Algorithm 2: start at sample `start`,
 * then repeatedly add the sample farthest (in double precision) from the
 * chosen set until K are chosen.  centers_out: K int64; obj_out: the
 * objective (Eq. 1) of the chosen set, or NULL.
 */
kc_status kc_fft(kc_ctx *ctx, int64_t start, int64_t *centers_out, double *obj_out);

/*
 * kc_fft_multi -- Algorithm 2 from S start samples at once (the paper's
 * heuristic baseline runs FFT from many random starts and keeps the best,
 * Section 6): set s starts at starts[s] and repeatedly adds the sample
 * farthest (in double precision, smallest index on ties) from its chosen
 * points until K are chosen.  Each of the K - 1 passes over the samples
 * serves all S sets.  Every set equals what kc_fft returns for its start.
 *   starts       [S] int64 sample indices in [0, N); 0 <= S <= 65536.
 *   centers_out  [S][K] int64.
 *   obj_out      [S] double objective (Eq. 1) of each set, or NULL.
 */
kc_status kc_fft_multi(kc_ctx *ctx, const int64_t *starts, int32_t S, int64_t *centers_out, double *obj_out);

/*
 * kc_lower_bounds_subset -- the closed-form lower bound of kc_lower_bounds
 * (Section 3.1, Eqs. 9-11) of B nodes over a subset of the samples given by
 * their indices (the reduced data set that sample reduction leaves,
 * Section 4.2): beta(M) = max over s in ids of min_k beta_s^k.  Each
 * sample's coordinates are gathered by index; all B nodes share each
 * gathered tile.
 *   ids        [n] uint32 sample indices (any order, repeats allowed); every
 *              index must be < N (checked with one pass over the ids:
 *              KC_EINVAL otherwise).  n = 0 gives bound 0 and argmax -1.
 *   lo, hi     [B][K][D] float boxes, 0 <= B <= 4096.
 *   lb_out, lb_raw_out, argmax_out  as in kc_lower_bounds (the argmax is a
 *              sample index, smallest on ties).
 *   kernel_ms_out  host float or NULL: the device time of the bound launch
 *              (key reset, the gather-and-bound kernel and its finalize),
 *              measured with CUDA events on the context's stream; the call
 *              then waits for it.
 * Float data with D <= 8 only (KC_EINVAL otherwise).
 */
kc_status kc_lower_bounds_subset(kc_ctx *ctx, const uint32_t *ids, int64_t n, const void *lo, const void *hi,
                                 int32_t B, double *lb_out, double *lb_raw_out, int64_t *argmax_out,
                                 float *kernel_ms_out);

/*
 * kc_fp32_probe -- measures the FP32 arithmetic throughput of the current GPU
 * that bounds the float lower-bound kernel (a measurement aid; the paper has
 * no counterpart).  Every thread of a full-GPU launch runs independent chains
 * of one instruction mix with no memory traffic; the fastest of five timed
 * launches (CUDA events on `stream`) is reported as FP32 lane operations per
 * second, counting a packed f32x2 subtraction or fused multiply-add as two
 * lane operations and a 3-input max.f32 as one.
 *   mode  0: packed fused multiply-adds (fma.rn.f32x2) only;
 *         1: 3-input maxima (max.f32) only;
 *         2: the bound kernel's clamp-distance term: per two attributes two
 *            packed subtractions, two 3-input maxima and one packed fused
 *            multiply-add (4 lane operations per attribute).
 *   lane_ops_per_s  receives the rate; ms_out (or NULL) the launch time.
 * Allocates and frees a small device buffer.
 */
kc_status kc_fp32_probe(int32_t mode, void *stream, double *lane_ops_per_s, float *ms_out);

/*
 * kc_tighten -- cluster assignment and bounds tightening of B nodes given an
 * upper bound alpha (Section 4.1, Algorithms 3 and 4):
 *   step A  center-based assignment: sample s leaves cluster k when
 *           beta_s^k > alpha (Lemma 1); one cluster left assigns s to it;
 *   box-BT  M'^k = M^k cap [max_j x_j - sqrt(alpha), min_j x_j + sqrt(alpha)]
 *           over the samples j assigned to k (and the seed of k);
 *   step B  sample-based assignment against the representatives of each
 *           cluster (the seed, then the assigned samples with the smallest
 *           and largest value of each attribute, then -- see ball_cap --
 *           of x_a + x_b and of x_a - x_b for attribute pairs a < b):
 *           ||x_s - x_j||^2 > 4 alpha excludes k (Lemma 2);
 *   ball-BT S_+^k = samples in M'^k within sqrt(alpha) of every
 *           representative of k; M^k_hat = bbox(S_+^k) cap box-BT of the
 *           step-B assignments ("centers on samples", Algorithm 4).
 * For float data every exclusion is taken only where the float evaluation
 * proves it, so the tightened boxes contain the exact ones; for double data
 * the decisions equal a serial double evaluation.
 *   lo, hi          [B][K][D] input boxes.
 *   alpha           the upper bound (double).
 *   seeds           [K] int64 sample indices pre-assigned to clusters
 *                   (Section 4.1.1), or NULL.
 *   lo_out, hi_out  [B][K][D] tightened boxes (may alias lo, hi).
 *   counts          [B][K] int64 |S_+^k|, or NULL.
 *   cand            [B][K] int64: the sample of S_+^k closest to the midpoint
 *                   of M'^k (an upper-bound candidate), -1 if none, or NULL.
 *   lb_out          [B] double certified lower bound of the input boxes, or NULL.
 *   status          [B] int8: 0 feasible, 1 proved to hold no solution of
 *                   value <= alpha, 2 leaf (every tightened box is a point).
 * ball_cap: the representatives' budget ("at most 50 balls" of Section
 * 4.1.2), at most min(ball_cap, 50) per cluster; <= 0 selects the default
 * of 50, except KC_BALLS_ALL: every sample of J_A^k (the samples step A
 * assigns to k, and the seed of k) is a representative of k -- the ball-BT
 * without a budget, S x |J_A^k| distances per node, run as a tiled pass
 * (float data, D <= 16; otherwise KC_EINVAL).  In order: the seed, the arg-min and arg-max of each attribute,
 * then, for float data, the arg-min and arg-max of x_a + x_b and of
 * x_a - x_b (added in float) for the first min(D(D-1)/2, 16) pairs a < b in
 * lexicographic order; ties go to the smaller sample index, duplicates are
 * skipped.  Double data stop after the attribute extremes (2D + 1).
 * Shapes: float data any K <= 16 and D <= 128 (K <= 4 with D <= 4 and K <= 2
 * with D <= 8 run kernels with the node's state in registers, compiled per
 * shape; the others kernels whose node state lives in shared memory sized at
 * launch); double data K <= 4 with D <= 4.  Other shapes return KC_EINVAL.
 */
#define KC_BALLS_ALL (-1)
kc_status kc_tighten(kc_ctx *ctx, const void *lo, const void *hi, int32_t B, double alpha,
                     const int64_t *seeds, int32_t ball_cap, void *lo_out, void *hi_out,
                     int64_t *counts, int64_t *cand, double *lb_out, int8_t *status);

/*
 * kc_sample_reduction -- Algorithm 5 against a list of M nodes: sample s is
 * deleted when in every node it is redundant for the lower bound
 * (alpha_s(M) = min_k max over mu in M^k of ||x_s - mu||^2 < beta_glob,
 * Eq. 13) and for the upper bound (for every k: x_s outside M^k, or some
 * representative j of k has ||x_s - x_j||^2 > alpha, Section 4.2.2).
 *   lo, hi        [M][K][D] node boxes.
 *   reps          [M][K][R] int64 representatives (-1 = unused slot), or NULL.
 *   R             slots per cluster in reps.
 *   beta_glob     the best lower bound; alpha the upper bound.
 *   active_inout  [N] uint8 mask: 1 = sample still present; cleared where
 *                 the sample is deleted.  Float data delete only where the
 *                 float evaluation proves redundancy.
 *   n_active_out  remaining samples, or NULL.
 * Shapes: D <= 8 (KC_EINVAL otherwise).
 */
kc_status kc_sample_reduction(kc_ctx *ctx, const void *lo, const void *hi, int32_t M,
                              const int64_t *reps, int32_t R, double beta_glob, double alpha,
                              uint8_t *active_inout, int64_t *n_active_out);

/*
 * The learned node scorer: a 12 -> 64 -> 64 -> 2 perceptron with ReLU
 * activations, bfloat16 weight matrices and float32 biases, activations and
 * accumulation.  Output r predicts the cost (log2 of the list entries scanned
 * by the branched nodes of the subtree, / 40) of branching a node with rule r:
 * rule 0 is the max-range rule of Section 3.3, rule 1 splits the box nearest to
 * the sample attaining the node's lower bound, on the attribute where that
 * sample lies farthest outside it (taken only where that attribute's range is
 * at least 1/4 of the largest, kc_solve_opts.rule_width).  The solver takes the cheaper rule and orders
 * equal lower bounds by the smaller predicted cost.  The paper has no
 * learned component: the exact lower bound still decides every prune, so the
 * certified optimum cannot change.  Parameters are one float vector of 5122
 * values [W1 64x12, b1 64, W2 64x64, b2 64, W3 2x64, b3 2] (row major);
 * training minimizes the mean of m0 (y0 - t0)^2 / 2 + m1 (y1 - t1)^2 / 2 with
 * Adam.  Arrays may be host or device memory.
 */
typedef struct kc_mlp kc_mlp;
kc_status kc_mlp_create(const float *params, void *stream, kc_mlp **out);
void kc_mlp_destroy(kc_mlp *m);
const char *kc_mlp_last_error(const kc_mlp *m);
kc_status kc_mlp_get_params(kc_mlp *m, float *params);
/* feats [B][12] -> out [B][2]. */
kc_status kc_mlp_forward(kc_mlp *m, const float *feats, int32_t B, float *out);
/* Mean loss and its gradient (5122 floats) over n samples; targets, masks [n][2]. */
kc_status kc_mlp_grad(kc_mlp *m, const float *feats, const float *targets, const float *masks, int32_t n,
                      float *loss_out, float *grad_out);
/* epochs x ceil(n / batch) Adam steps (lr, beta1 0.9, beta2 0.999, eps 1e-8) over
 * a permutation of the samples drawn from `seed` every epoch; loss_out (host or
 * NULL) receives the mean loss over all n samples afterwards. */
kc_status kc_mlp_train(kc_mlp *m, const float *feats, const float *targets, const float *masks, int32_t n,
                       int32_t epochs, int32_t batch, float lr, uint64_t seed, float *loss_out);
/* Attaches a scorer to a context (NULL detaches); kc_solve with order = 1 uses it.
 * The scorer must outlive its use by the context. */
kc_status kc_set_scorer(kc_ctx *ctx, kc_mlp *m);

/* Options of kc_solve; kc_solve_defaults() fills the defaults shown. */
typedef struct {
    double tol;            /* 1e-12: stop when (UB - LB) / UB <= tol (Section 6.1 gap) */
    double time_limit_s;   /* 0: none */
    int64_t node_limit;    /* 0: none */
    int32_t batch;         /* 0: automatic; nodes bounded per launch */
    int32_t ball_cap;      /* 50: representatives per cluster, as kc_tighten's ball_cap
                              (KC_BALLS_ALL: float data, D <= 16, lists = 0) */
    int32_t i_sr;          /* 1: sample reduction every i_sr batches, 0: off */
    int32_t use_bt;        /* 1: assignment + bounds tightening (BB+CF+BT); 0: BB+CF */
    int32_t order;         /* 0: best bound, max-range branching; 1: learned scorer (kc_set_scorer) */
    int32_t lists;         /* 1: every node keeps its own list of surviving samples (float data, Section
                              4.2); 0: all nodes of a batch scan one shared sample set */
    int32_t verbose;       /* 0; 1: per-phase timings on stderr */
    int32_t explore;       /* 0; p in (0, 100]: on p % of the nodes where the two branching rules
                              differ, take a random one (seeded by seed and node id): training
                              data for the scorer, with log_path */
    int32_t arena_mb;      /* 0: automatic; device memory (MiB) that holds the per-node lists */
    uint64_t seed;         /* 0: FFT start = seed mod N */
    const char *log_path;  /* NULL, or a file receiving one JSON line per branched node (scorer
                              features) and one per bounded child (boxes, certified bound, pruned) */
    double rule_margin;    /* 0: with order = 1, rule 1 is taken only when its predicted cost is
                              lower than max-range's by more than this (cost units: log2 / 40) */
    int32_t fft_starts;    /* 1 (0 = 1): FFT runs from this many start samples (seed mod N, then
                              steps of 2654435761 mod N); the best is the first incumbent and
                              kc_result.fft_objective */
    int32_t rule_width;    /* 4 (0 = 4): with order = 1, rule 1 only on a variable whose range is
                              at least 1/rule_width of the largest range */
} kc_solve_opts;

typedef struct {
    double objective;      /* incumbent objective recomputed in double over all N samples */
    double lower_bound;    /* certified lower bound on the optimum */
    double gap;            /* (objective - lower_bound) / objective */
    int64_t centers[16];   /* K sample indices */
    int64_t nodes;         /* nodes visited */
    int64_t batches;       /* bounding launches */
    int64_t active_final;  /* samples left after sample reduction (per-node lists: the longest list of
                              an open node, 0 when none is open) */
    double fft_objective;  /* objective of the root FFT solution */
    double seconds;        /* wall time of the solve */
    int32_t seeds_found;   /* the FFT points were K initial seeds (Section 4.1.1) */
    int32_t status;        /* KC_OK, KC_ETIMEOUT or KC_ELIMIT */
    int64_t lists_filtered;   /* per-node lists: nodes whose children got a shorter list */
    int64_t samples_dropped;  /* per-node lists: list entries dropped over the solve */
} kc_result;

void kc_solve_defaults(kc_solve_opts *opt);

/*
 * kc_solve -- the branch and bound of Algorithm 1 to a certified optimum:
 * root box, FFT upper bound and seeds (Algorithm 2, Section 4.1.1), then
 * batches of open nodes with the smallest bounds are tightened, given an
 * upper-bound candidate and branched on the GPU (max-range variable or the
 * scorer's rule, midpoint value); children are bounded when created and every
 * node whose certified lower bound reaches UB (1 - tol) is pruned.  Sample
 * reduction (Section 4.2) runs per node: with opt->lists (float data) each
 * node's children scan only the samples that survive in it; otherwise one
 * shared sample set is reduced between batches.  Float bounds that cannot
 * decide a prune are re-evaluated in double.  The returned objective is
 * recomputed in double over all samples.  opt may be NULL (defaults); tol
 * overrides opt->tol when >= 0.  Returns KC_OK at optimality within tol,
 * KC_ETIMEOUT / KC_ELIMIT (with *out filled) at a limit, KC_EINVAL for
 * options out of range, KC_ENOMEM when the list arena or buffers do not fit.
 * Shapes: those of kc_tighten (float K <= 16, D <= 128; double K <= 4 with
 * D <= 4); other shapes return KC_EINVAL.  Float data with D > 8 scan one
 * shared sample set (no per-node lists) without sample reduction.
 */
kc_status kc_solve(kc_ctx *ctx, double tol, const kc_solve_opts *opt, kc_result *out);

#ifdef __cplusplus
}
#endif

#endif /* KC_H_ */
