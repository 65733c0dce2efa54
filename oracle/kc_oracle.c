/*
 * kc_oracle.c -- plain, slow CPU oracle for the reduced-space branch and bound
 * for K-center clustering (Ren, You, Hua, Ji, Cao, "A Global Optimization
 * Algorithm for K-Center Clustering of One Billion Samples").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may link, load or
 * call this file: only the tests, the smoke check and the CPU baseline leg of
 * the benchmark do.  It shares no code with the CUDA library.
 *
 * Conventions
 *   - X is row major, X[s*D + a] = x_{s,a}, in double.  Data stored in float
 *     is promoted exactly to double before it reaches this file.
 *   - A node is K boxes, lo[k*D + a] <= mu^k_a <= hi[k*D + a].
 *   - All distances are squared Euclidean (Eq. 1).  Every distance is summed
 *     over a = 0..D-1 in order, as acc = acc + d*d with two roundings (the
 *     file is compiled with -ffp-contract=off).
 *   - Ties in every argmax / argmin go to the smallest sample index.
 *   - `active` (nullable) is the sample-reduction mask: only samples with
 *     active[s] != 0 take part (Algorithm 5 deletes the others).
 *
 * Where the paper is silent or garbled, the reading taken here is stated in
 * the comment of the function that applies it.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define KCO_MAXK 16
#define KCO_MAXD 128
#define KCO_MAXREPS 50
/* ball_cap value: every sample assigned to cluster k in step A is a
 * representative of k (no budget; the paper's unrestricted ball-BT) */
#define KCO_BALLS_ALL (-1)

/* ---------------------------------------------------------------------- */
/* Elementary pieces                                                       */
/* ---------------------------------------------------------------------- */

/* mid{l, x, h}: the median of three numbers (l <= h), the minimiser of
 * (x - mu)^2 over mu in [l, h] (Section 3.1, analytic solution of Eq. 11). */
static double mid3(double l, double x, double h)
{
    if (x < l) return l;
    if (x > h) return h;
    return x;
}

/* ||x - y||^2 summed in attribute order (Eq. 1). */
static double sqdist(const double *x, const double *y, int D)
{
    double acc = 0.0;
    for (int a = 0; a < D; ++a) {
        double d = x[a] - y[a];
        acc = acc + d * d;
    }
    return acc;
}

/* beta_s^k(M^k) = min over mu in M^k of ||x_s - mu||^2, Eq. 11, evaluated at
 * its closed-form minimiser mu_a = mid{lo_a, x_a, hi_a}. */
double kco_beta_sk(const double *x, const double *lo, const double *hi, int D)
{
    double acc = 0.0;
    for (int a = 0; a < D; ++a) {
        double mu = mid3(lo[a], x[a], hi[a]);
        double d = x[a] - mu;
        acc = acc + d * d;
    }
    return acc;
}

/* alpha_s(M^k) for one cluster: max over mu in M^k of ||x_s - mu||^2 (Eq. 13),
 * attained at the corner mu_a = lo_a if |lo_a - x_a| > |hi_a - x_a| else hi_a. */
static double farthest_corner_sk(const double *x, const double *lo, const double *hi, int D)
{
    double acc = 0.0;
    for (int a = 0; a < D; ++a) {
        double mu = (fabs(lo[a] - x[a]) > fabs(hi[a] - x[a])) ? lo[a] : hi[a];
        double d = x[a] - mu;
        acc = acc + d * d;
    }
    return acc;
}

static int is_active(const uint8_t *active, int64_t s) { return active == NULL || active[s] != 0; }

static int in_box(const double *x, const double *lo, const double *hi, int D)
{
    for (int a = 0; a < D; ++a)
        if (x[a] < lo[a] || x[a] > hi[a]) return 0;
    return 1;
}

/* ---------------------------------------------------------------------- */
/* Root region M0 (Section 2.1)                                             */
/* ---------------------------------------------------------------------- */

/* M0: lo_a = min_s x_{s,a}, hi_a = max_s x_{s,a} (the same box for every k). */
int kco_root_box(const double *X, int64_t N, int D, double *lo, double *hi)
{
    if (N <= 0 || D <= 0) return 1;
    for (int a = 0; a < D; ++a) { lo[a] = X[a]; hi[a] = X[a]; }
    for (int64_t s = 1; s < N; ++s)
        for (int a = 0; a < D; ++a) {
            double v = X[s * D + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Lower bound (Section 3.1)                                               */
/* ---------------------------------------------------------------------- */

/* beta(M) = max_s min_k beta_s^k(M^k)  (Eq. 9 with Eqs. 10-11).
 * Writes the bound and the sample attaining it (-1 if no active sample). */
int kco_lower_bound(const double *X, int64_t N, int D, int K, const double *lo, const double *hi,
                    const uint8_t *active, double *beta, int64_t *argmax)
{
    double best = -1.0;
    int64_t arg = -1;
    for (int64_t s = 0; s < N; ++s) {
        if (!is_active(active, s)) continue;
        const double *x = X + s * D;
        double bs = INFINITY;
        for (int k = 0; k < K; ++k) {
            double v = kco_beta_sk(x, lo + k * D, hi + k * D, D);
            if (v < bs) bs = v;
        }
        if (bs > best) { best = bs; arg = s; }
    }
    *beta = arg < 0 ? 0.0 : best;
    if (argmax) *argmax = arg;
    return 0;
}

/* The lower bound of B nodes; node b's boxes start at lo + b*K*D. */
int kco_lower_bounds(const double *X, int64_t N, int D, int K, const double *lo, const double *hi,
                     int B, const uint8_t *active, double *beta, int64_t *argmax)
{
    for (int b = 0; b < B; ++b)
        kco_lower_bound(X, N, D, K, lo + (int64_t)b * K * D, hi + (int64_t)b * K * D, active,
                        beta + b, argmax ? argmax + b : NULL);
    return 0;
}

/* kco_lower_bounds spread over the host cores (the timed CPU baseline): the
 * samples are cut into contiguous blocks, OpenMP threads evaluate
 * kco_lower_bound on (block, node) pairs, and the block results of a node
 * are merged in block order, a later block winning only with a strictly
 * larger value.  Value and argmax therefore equal the serial loop's.
 * Returns the number of threads used. */
int kco_lower_bounds_par(const double *X, int64_t N, int D, int K, const double *lo, const double *hi,
                         int B, double *beta, int64_t *argmax)
{
    int nt = 1;
#ifdef _OPENMP
    nt = omp_get_max_threads();
#endif
    int64_t nblk = (int64_t)nt * 4;
    if (nblk > N) nblk = N > 0 ? N : 1;
    double *bv = (double *)malloc(sizeof(double) * (size_t)nblk * (size_t)(B > 0 ? B : 1));
    int64_t *ba = (int64_t *)malloc(sizeof(int64_t) * (size_t)nblk * (size_t)(B > 0 ? B : 1));
    if (!bv || !ba) { free(bv); free(ba); return -1; }
    const int64_t pairs = nblk * (int64_t)B;
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1)
#endif
    for (int64_t q = 0; q < pairs; ++q) {
        const int64_t j = q / B;
        const int b = (int)(q % B);
        const int64_t s0 = N * j / nblk, s1 = N * (j + 1) / nblk;
        kco_lower_bound(X + s0 * D, s1 - s0, D, K, lo + (int64_t)b * K * D, hi + (int64_t)b * K * D, NULL,
                        &bv[q], &ba[q]);
        if (ba[q] >= 0) ba[q] += s0;
    }
    for (int b = 0; b < B; ++b) {
        double best = 0.0;
        int64_t arg = -1;
        for (int64_t j = 0; j < nblk; ++j) {
            const int64_t q = j * B + b;
            if (ba[q] >= 0 && (arg < 0 || bv[q] > best)) { best = bv[q]; arg = ba[q]; }
        }
        beta[b] = best;
        if (argmax) argmax[b] = arg;
    }
    free(bv);
    free(ba);
    return nt;
}

/* Certificate replay (O5), pruned nodes: for node m with boxes lo/hi + m*K*D
 * and witness sample wit[m], out[m] = min_k beta_{wit}^k(M^k), the closed
 * form of Section 3.1 at that one sample.  beta(M) is a maximum over samples,
 * so beta(M) >= out[m]: out[m] >= threshold proves that the node holds no
 * solution below the threshold without evaluating the other samples.
 * out[m] = -1 when wit[m] < 0 (no witness). */
int kco_witness_values(const double *X, int64_t N, int D, int K, const double *lo, const double *hi, int64_t M,
                       const int64_t *wit, double *out)
{
    for (int64_t m = 0; m < M; ++m) {
        if (wit[m] < 0 || wit[m] >= N) { out[m] = -1.0; continue; }
        const double *x = X + wit[m] * D;
        double v = INFINITY;
        for (int k = 0; k < K; ++k) {
            double b = kco_beta_sk(x, lo + (m * K + k) * D, hi + (m * K + k) * D, D);
            if (b < v) v = b;
        }
        out[m] = v;
    }
    return 0;
}

/* The matrix beta_s^k (N x K, row major): test helper for the closed form. */
int kco_beta_matrix(const double *X, int64_t N, int D, int K, const double *lo, const double *hi,
                    double *out)
{
    for (int64_t s = 0; s < N; ++s)
        for (int k = 0; k < K; ++k)
            out[s * K + k] = kco_beta_sk(X + s * D, lo + k * D, hi + k * D, D);
    return 0;
}

/* alpha_s(M) = min_k max over mu^k in M^k of ||x_s - mu^k||^2 (Eq. 13), N values. */
int kco_alpha_s(const double *X, int64_t N, int D, int K, const double *lo, const double *hi,
                double *out)
{
    for (int64_t s = 0; s < N; ++s) {
        double best = INFINITY;
        for (int k = 0; k < K; ++k) {
            double v = farthest_corner_sk(X + s * D, lo + k * D, hi + k * D, D);
            if (v < best) best = v;
        }
        out[s] = best;
    }
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Upper bound (Section 3.2)                                               */
/* ---------------------------------------------------------------------- */

/* alpha = max_s min_k ||x_s - x_{c_k}||^2 for centers on samples c (Eq. 12 and
 * the objective of Eq. 1).  Writes the value and the sample attaining it. */
int kco_objective(const double *X, int64_t N, int D, int K, const int64_t *centers,
                  const uint8_t *active, double *value, int64_t *argmax)
{
    double best = -1.0;
    int64_t arg = -1;
    for (int64_t s = 0; s < N; ++s) {
        if (!is_active(active, s)) continue;
        double q = INFINITY;
        for (int k = 0; k < K; ++k) {
            double v = sqdist(X + s * D, X + centers[k] * D, D);
            if (v < q) q = v;
        }
        if (q > best) { best = q; arg = s; }
    }
    *value = arg < 0 ? 0.0 : best;
    if (argmax) *argmax = arg;
    return 0;
}

/* Eq. 1 at K centres given as points mu (K x D, row major), which need not be
 * samples: max_s min_k ||x_s - mu_k||^2 and the sample attaining it. */
int kco_objective_points(const double *X, int64_t N, int D, int K, const double *mu, double *value,
                         int64_t *argmax)
{
    double best = -1.0;
    int64_t arg = -1;
    for (int64_t s = 0; s < N; ++s) {
        double q = INFINITY;
        for (int k = 0; k < K; ++k) {
            double v = sqdist(X + s * D, mu + k * D, D);
            if (v < q) q = v;
        }
        if (q > best) {   /* strictly larger: ties keep the smaller index */
            best = q;
            arg = s;
        }
    }
    *value = arg < 0 ? 0.0 : best;
    if (argmax) *argmax = arg;
    return 0;
}

/* Candidate centre of one box (Section 3.2, children): the active sample
 * inside [lo, hi] closest to the box midpoint (lo + hi) / 2.  -1 if the box
 * holds no active sample.  (Reading: candidates are drawn from X cap M^k.) */
int64_t kco_mid_candidate(const double *X, int64_t N, int D, const double *lo, const double *hi,
                          const uint8_t *active, double *dist_out)
{
    double mid[KCO_MAXD];
    for (int a = 0; a < D; ++a) mid[a] = 0.5 * (lo[a] + hi[a]);
    double best = INFINITY;
    int64_t arg = -1;
    for (int64_t s = 0; s < N; ++s) {
        if (!is_active(active, s)) continue;
        const double *x = X + s * D;
        if (!in_box(x, lo, hi, D)) continue;
        double v = sqdist(x, mid, D);
        if (v < best) { best = v; arg = s; }
    }
    if (dist_out) *dist_out = best;
    return arg;
}

/* Farthest First Traversal, Algorithm 2: start at sample `start`, then add the
 * sample farthest from the chosen set (d(x_s, T) = min over T) until |T| = K.
 * Writes the K indices and the objective (Eq. 1) of the chosen set. */
int kco_fft(const double *X, int64_t N, int D, int K, int64_t start, int64_t *centers, double *obj)
{
    double *dmin = (double *)malloc(sizeof(double) * (size_t)N);
    if (!dmin) return 2;
    centers[0] = start;
    for (int64_t s = 0; s < N; ++s) dmin[s] = sqdist(X + s * D, X + start * D, D);
    for (int t = 1; t < K; ++t) {
        double best = -1.0;
        int64_t arg = 0;
        for (int64_t s = 0; s < N; ++s)
            if (dmin[s] > best) { best = dmin[s]; arg = s; }
        centers[t] = arg;
        for (int64_t s = 0; s < N; ++s) {
            double v = sqdist(X + s * D, X + arg * D, D);
            if (v < dmin[s]) dmin[s] = v;
        }
    }
    double best = -1.0;
    for (int64_t s = 0; s < N; ++s)
        if (dmin[s] > best) best = dmin[s];
    *obj = best;
    free(dmin);
    return 0;
}

/* Exact optimum of Eq. 1 by enumerating every K-subset of samples in
 * lexicographic order (the first subset reaching the minimum is kept).
 * Feasible only for tiny N. */
int kco_bruteforce(const double *X, int64_t N, int D, int K, double *obj, int64_t *centers)
{
    if (K < 1 || K > KCO_MAXK || N < K) return 1;
    int64_t c[KCO_MAXK];
    for (int k = 0; k < K; ++k) c[k] = k;
    double best = INFINITY;
    for (;;) {
        double v;
        kco_objective(X, N, D, K, c, NULL, &v, NULL);
        if (v < best) {
            best = v;
            for (int k = 0; k < K; ++k) centers[k] = c[k];
        }
        int i = K - 1;
        while (i >= 0 && c[i] == N - K + i) --i;
        if (i < 0) break;
        ++c[i];
        for (int j = i + 1; j < K; ++j) c[j] = c[j - 1] + 1;
    }
    *obj = best;
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Outward rounding to the data's precision                                */
/* ---------------------------------------------------------------------- */

/* Box bounds produced by bounds tightening are rounded outward to a value the
 * data type can hold (float data: is_f32 = 1), so the tightened box always
 * contains the exact real-number box (reading of Algorithm 4 under rounding). */
static double round_down_dt(double v, int is_f32)
{
    if (!is_f32) return v;
    float f = (float)v;
    if ((double)f > v) f = nextafterf(f, -INFINITY);
    return (double)f;
}

static double round_up_dt(double v, int is_f32)
{
    if (!is_f32) return v;
    float f = (float)v;
    if ((double)f < v) f = nextafterf(f, INFINITY);
    return (double)f;
}

/* Branching value (Section 3.3): the midpoint of [lo, hi] in the data's
 * precision; children are [lo, m] and [succ(m), hi] where succ is the next
 * value of the data type, so every sample value lies in exactly one child and
 * both children are strictly smaller than the parent (reading of the
 * midpoint rule for finite precision).  Requires lo < hi. */
static void split_point(double lo, double hi, int is_f32, double *m_out, double *succ_out)
{
    if (is_f32) {
        float m = (float)(0.5 * (lo + hi));
        if ((double)m >= hi) m = (float)lo;
        if ((double)m < lo) m = (float)lo;
        *m_out = (double)m;
        *succ_out = (double)nextafterf(m, INFINITY);
    } else {
        double m = 0.5 * (lo + hi);
        if (m >= hi) m = lo;
        if (m < lo) m = lo;
        *m_out = m;
        *succ_out = nextafter(m, INFINITY);
    }
}

/* The branching value of [lo, hi] and its successor, for the tests. */
void kco_split_point(double lo, double hi, int is_f32, double *m_out, double *succ_out)
{
    split_point(lo, hi, is_f32, m_out, succ_out);
}

/* ---------------------------------------------------------------------- */
/* Cluster assignment and bounds tightening (Section 4.1, Algorithms 3, 4) */
/* ---------------------------------------------------------------------- */

typedef struct {
    int32_t status;                 /* 0 feasible, 1 infeasible (proved empty), 2 leaf */
    double beta;                    /* node lower bound beta(M) over active samples */
    int64_t beta_arg;
    double lo[KCO_MAXK * KCO_MAXD]; /* tightened box */
    double hi[KCO_MAXK * KCO_MAXD];
    int64_t count[KCO_MAXK];        /* |S_+^k|: samples allowed as centre k */
    int64_t cand[KCO_MAXK];         /* UB candidate per cluster (closest to box-BT midpoint) */
    int64_t n_assigned[KCO_MAXK];   /* |J^k| after both assignment rules */
    int32_t n_reps[KCO_MAXK];
    int64_t reps[KCO_MAXK * KCO_MAXREPS];
    double blo[KCO_MAXK * KCO_MAXD];  /* the box-BT box M' of step A */
    double bhi[KCO_MAXK * KCO_MAXD];
} kco_tighten_out;

/* Representatives ("balls") of cluster k, from its assigned set (reading of
 * the "at most 50 balls" of Section 4.1.2): the seed of cluster k (if seeds
 * exist), then the assigned samples attaining the minimum and the maximum of
 * x along a fixed list of directions -- first the D attributes (x_a), then,
 * for float data, the first P = min(D(D-1)/2, 16) attribute pairs a < b in
 * lexicographic order, each as x_a + x_b and then x_a - x_b -- smallest index
 * on ties, duplicates skipped, at most `cap` of them (for double data the
 * list stops after the attributes).  Arrays hold those
 * arg-extremes (-1 if none): amin_idx/amax_idx [D], dmin_idx/dmax_idx [2P]
 * (sum of pair p at 2p, difference at 2p + 1). */
#define KCO_MAXPAIRS 16
static int build_reps(int64_t seed_k, const int64_t *amin_idx, const int64_t *amax_idx, int D,
                      const int64_t *dmin_idx, const int64_t *dmax_idx, int ndir, int cap, int64_t *reps)
{
    int n = 0;
#define KCO_ADD_REP(idx)                                            \
    do {                                                            \
        int64_t v_ = (idx);                                         \
        if (v_ >= 0 && n < cap) {                                   \
            int dup_ = 0;                                           \
            for (int q_ = 0; q_ < n; ++q_) if (reps[q_] == v_) dup_ = 1; \
            if (!dup_) reps[n++] = v_;                              \
        }                                                           \
    } while (0)
    KCO_ADD_REP(seed_k);
    for (int a = 0; a < D; ++a) {
        KCO_ADD_REP(amin_idx[a]);
        KCO_ADD_REP(amax_idx[a]);
    }
    for (int q = 0; q < ndir; ++q) {
        KCO_ADD_REP(dmin_idx[q]);
        KCO_ADD_REP(dmax_idx[q]);
    }
#undef KCO_ADD_REP
    return n;
}

/* The value of sample x along direction q of the pair list (see build_reps),
 * in the data's precision: float data add or subtract in float. */
static double dir_value(const double *x, int D, int q, int is_f32)
{
    const int p = q / 2;
    int a = 0, b = 1, t = p;
    for (a = 0; a < D - 1; ++a) {
        if (t < D - 1 - a) { b = a + 1 + t; break; }
        t -= D - 1 - a;
    }
    if (is_f32) {
        const float fa = (float)x[a], fb = (float)x[b];
        const float v = (q & 1) ? fa - fb : fa + fb;
        return (double)v;
    }
    return (q & 1) ? x[a] - x[b] : x[a] + x[b];
}

/* One node's cluster assignment and bounds tightening.
 *
 * Step A (Algorithm 3, center-based): for every active sample compute
 *   beta_s^k; exclude k when beta_s^k > alpha (Lemma 1).  A sample with
 *   exactly one cluster k' left is assigned to k'; with none left the node
 *   cannot hold a solution of value <= alpha (infeasible).  J_A^k = seed of k
 *   plus the samples assigned to k.
 * Box-based BT (Section 4.1.2): M'^k = M^k cap [max_j x_j - r, min_j x_j + r]
 *   over j in J_A^k, r = sqrt(alpha) rounded up, bounds rounded outward.
 *   With seeds, a node whose box k is farther than alpha from seed k holds
 *   no such solution either (infeasible).
 * Step B (Algorithm 3, sample-based, when every J_A^k is non-empty): a
 *   sample not assigned in step A (assigned samples help pre-assign the other
 *   samples, Section 4.1.1) is excluded from k when some representative j of
 *   k has ||x_s - x_j||^2 > 4 alpha (Lemma 2); exactly one cluster left
 *   assigns it (J_B), none left makes the node infeasible.
 * Ball-based BT and "centers on samples" (Algorithm 4): S_+^k = active
 *   samples in M'^k within sqrt(alpha) of every representative of k;
 *   M^k_hat = bbox(S_+^k) cap box-BT over J_B^k.
 * Also returns beta(M) (from step A's values), |S_+^k|, and the candidate
 * centre per cluster: the sample of S_+^k closest to the midpoint of M'^k.
 * A node whose tightened boxes all have zero range is a leaf (status 2).
 */
int kco_tighten(const double *X, int64_t N, int D, int K, const double *lo, const double *hi,
                double alpha, const int64_t *seeds, const uint8_t *active, int is_f32,
                int ball_cap, kco_tighten_out *out)
{
    if (K > KCO_MAXK || D > KCO_MAXD) return 1;
    /* at most ball_cap representatives (<= 0: the default of 50, which is
     * also the largest); pair directions for float data only.  KCO_BALLS_ALL:
     * step B tests against every sample of J_A^k instead (the reported
     * representatives are then the default ones, for information) */
    const int diag = is_f32 != 0;
    const int all_balls = ball_cap == KCO_BALLS_ALL;
    if (ball_cap <= 0 || ball_cap > KCO_MAXREPS) ball_cap = KCO_MAXREPS;
    const int npairs = D * (D - 1) / 2 < KCO_MAXPAIRS ? D * (D - 1) / 2 : KCO_MAXPAIRS;
    const int ndir = diag ? 2 * npairs : 0;
    const int KD = K * D;
    int8_t *asg = (int8_t *)malloc((size_t)N);
    if (!asg) return 2;
    memset(out, 0, sizeof(*out));
    out->status = 0;

    /* step A */
    double jmin[KCO_MAXK * KCO_MAXD], jmax[KCO_MAXK * KCO_MAXD];
    int64_t jmin_i[KCO_MAXK * KCO_MAXD], jmax_i[KCO_MAXK * KCO_MAXD];
    int64_t na[KCO_MAXK];
    for (int i = 0; i < KD; ++i) { jmin[i] = INFINITY; jmax[i] = -INFINITY; jmin_i[i] = -1; jmax_i[i] = -1; }
    for (int k = 0; k < K; ++k) na[k] = 0;
    double beta = -1.0;
    int64_t beta_arg = -1;
    int infeasible = 0;
    for (int64_t s = 0; s < N; ++s) {
        asg[s] = -1;
        if (!is_active(active, s)) continue;
        const double *x = X + s * D;
        double bmin = INFINITY;
        int left = 0, kk = -1;
        for (int k = 0; k < K; ++k) {
            double v = kco_beta_sk(x, lo + k * D, hi + k * D, D);
            if (v < bmin) bmin = v;
            if (!(v > alpha)) { ++left; kk = k; }
        }
        if (bmin > beta) { beta = bmin; beta_arg = s; }
        if (left == 0) infeasible = 1;
        if (left == 1) asg[s] = (int8_t)kk;
    }
    if (seeds)
        for (int k = 0; k < K; ++k) {
            /* seeds are assigned in every node; a node whose box k is farther
             * than alpha from seed k cannot hold a solution of value <= alpha */
            if (kco_beta_sk(X + seeds[k] * D, lo + k * D, hi + k * D, D) > alpha) infeasible = 1;
            asg[seeds[k]] = (int8_t)k;
        }
    double dmin[KCO_MAXK * 2 * KCO_MAXPAIRS], dmax[KCO_MAXK * 2 * KCO_MAXPAIRS];
    int64_t dmin_i[KCO_MAXK * 2 * KCO_MAXPAIRS], dmax_i[KCO_MAXK * 2 * KCO_MAXPAIRS];
    for (int i = 0; i < KCO_MAXK * 2 * KCO_MAXPAIRS; ++i) {
        dmin[i] = INFINITY; dmax[i] = -INFINITY; dmin_i[i] = -1; dmax_i[i] = -1;
    }
    for (int64_t s = 0; s < N; ++s) {
        int k = asg[s];
        if (k < 0) continue;
        ++na[k];
        const double *x = X + s * D;
        for (int a = 0; a < D; ++a) {
            int i = k * D + a;
            if (x[a] < jmin[i]) { jmin[i] = x[a]; jmin_i[i] = s; }
            if (x[a] > jmax[i]) { jmax[i] = x[a]; jmax_i[i] = s; }
        }
        for (int q = 0; q < ndir; ++q) {
            const double v = dir_value(x, D, q, is_f32);
            const int i = k * 2 * KCO_MAXPAIRS + q;
            if (v < dmin[i]) { dmin[i] = v; dmin_i[i] = s; }
            if (v > dmax[i]) { dmax[i] = v; dmax_i[i] = s; }
        }
    }
    out->beta = beta_arg < 0 ? 0.0 : beta;
    out->beta_arg = beta_arg;

    /* box-based BT over J_A */
    double r = nextafter(sqrt(alpha), INFINITY);
    double blo[KCO_MAXK * KCO_MAXD], bhi[KCO_MAXK * KCO_MAXD];
    for (int k = 0; k < K; ++k)
        for (int a = 0; a < D; ++a) {
            int i = k * D + a;
            blo[i] = lo[i];
            bhi[i] = hi[i];
            if (na[k] > 0) {
                double l = round_down_dt(nextafter(jmax[i] - r, -INFINITY), is_f32);
                double h = round_up_dt(nextafter(jmin[i] + r, INFINITY), is_f32);
                if (l > blo[i]) blo[i] = l;
                if (h < bhi[i]) bhi[i] = h;
            }
            if (blo[i] > bhi[i]) infeasible = 1;
        }

    memcpy(out->blo, blo, sizeof(double) * KD);
    memcpy(out->bhi, bhi, sizeof(double) * KD);

    /* representatives from J_A */
    int all_have = 1;
    for (int k = 0; k < K; ++k) {
        out->n_reps[k] = build_reps(seeds ? seeds[k] : -1, jmin_i + k * D, jmax_i + k * D, D,
                                    dmin_i + k * 2 * KCO_MAXPAIRS, dmax_i + k * 2 * KCO_MAXPAIRS, ndir,
                                    ball_cap, out->reps + k * KCO_MAXREPS);
        if (out->n_reps[k] == 0) all_have = 0;
    }

    /* J_A^k as index lists (for KCO_BALLS_ALL): samples with asg == k, in order */
    int64_t *jl = NULL, joff[KCO_MAXK + 1];
    if (all_balls) {
        jl = (int64_t *)malloc(sizeof(int64_t) * (size_t)(N > 0 ? N : 1));
        if (!jl) { free(asg); return 2; }
        for (int k = 0; k <= K; ++k) joff[k] = 0;
        for (int64_t s = 0; s < N; ++s)
            if (asg[s] >= 0) ++joff[asg[s] + 1];
        for (int k = 0; k < K; ++k) joff[k + 1] += joff[k];
        int64_t fill[KCO_MAXK];
        for (int k = 0; k < K; ++k) fill[k] = joff[k];
        for (int64_t s = 0; s < N; ++s)
            if (asg[s] >= 0) jl[fill[asg[s]]++] = s;
    }

    /* step B */
    double slo[KCO_MAXK * KCO_MAXD], shi[KCO_MAXK * KCO_MAXD];
    double bmin2[KCO_MAXK * KCO_MAXD], bmax2[KCO_MAXK * KCO_MAXD];
    int64_t nb[KCO_MAXK];
    double cdist[KCO_MAXK], mid[KCO_MAXK * KCO_MAXD];
    for (int i = 0; i < KD; ++i) {
        slo[i] = INFINITY; shi[i] = -INFINITY; bmin2[i] = INFINITY; bmax2[i] = -INFINITY;
        mid[i] = 0.5 * (blo[i] + bhi[i]);
    }
    for (int k = 0; k < K; ++k) { out->count[k] = 0; out->cand[k] = -1; cdist[k] = INFINITY; nb[k] = 0; }
    const double four_alpha = 4.0 * alpha;
    for (int64_t s = 0; s < N; ++s) {
        if (!is_active(active, s)) continue;
        const double *x = X + s * D;
        if (all_have && asg[s] < 0) {
            int left = 0, kk = -1;
            for (int k = 0; k < K; ++k) {
                int excl = 0;
                if (all_balls) {
                    for (int64_t q = joff[k]; q < joff[k + 1] && !excl; ++q)
                        if (sqdist(x, X + jl[q] * D, D) > four_alpha) excl = 1;
                } else {
                    for (int q = 0; q < out->n_reps[k] && !excl; ++q)
                        if (sqdist(x, X + out->reps[k * KCO_MAXREPS + q] * D, D) > four_alpha) excl = 1;
                }
                if (!excl) { ++left; kk = k; }
            }
            if (left == 0) infeasible = 1;
            if (left == 1) {
                ++nb[kk];
                for (int a = 0; a < D; ++a) {
                    int i = kk * D + a;
                    if (x[a] < bmin2[i]) bmin2[i] = x[a];
                    if (x[a] > bmax2[i]) bmax2[i] = x[a];
                }
            }
        }
        for (int k = 0; k < K; ++k) {
            if (!in_box(x, blo + k * D, bhi + k * D, D)) continue;
            int ok = 1;
            if (all_balls) {
                for (int64_t q = joff[k]; q < joff[k + 1] && ok; ++q)
                    if (sqdist(x, X + jl[q] * D, D) > alpha) ok = 0;
            } else {
                for (int q = 0; q < out->n_reps[k] && ok; ++q)
                    if (sqdist(x, X + out->reps[k * KCO_MAXREPS + q] * D, D) > alpha) ok = 0;
            }
            if (!ok) continue;
            ++out->count[k];
            for (int a = 0; a < D; ++a) {
                int i = k * D + a;
                if (x[a] < slo[i]) slo[i] = x[a];
                if (x[a] > shi[i]) shi[i] = x[a];
            }
            double dm = sqdist(x, mid + k * D, D);
            if (dm < cdist[k]) { cdist[k] = dm; out->cand[k] = s; }
        }
    }
    for (int k = 0; k < K; ++k) {
        out->n_assigned[k] = na[k] + nb[k];
        if (out->count[k] == 0) infeasible = 1;
        for (int a = 0; a < D; ++a) {
            int i = k * D + a;
            double l = slo[i], h = shi[i];
            if (nb[k] > 0) {
                double l2 = round_down_dt(nextafter(bmax2[i] - r, -INFINITY), is_f32);
                double h2 = round_up_dt(nextafter(bmin2[i] + r, INFINITY), is_f32);
                if (l2 > l) l = l2;
                if (h2 < h) h = h2;
            }
            out->lo[i] = l;
            out->hi[i] = h;
            if (!(l <= h)) infeasible = 1;
        }
    }
    free(asg);
    free(jl);
    if (infeasible) { out->status = 1; return 0; }
    int leaf = 1;
    for (int i = 0; i < KD; ++i)
        if (out->hi[i] > out->lo[i]) leaf = 0;
    out->status = leaf ? 2 : 0;
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Symmetry breaking (Section 4.1.3)                                       */
/* ---------------------------------------------------------------------- */

/* mu^1_1 <= mu^2_1 <= ... <= mu^K_1 on the first attribute, propagated to the
 * boxes: lo^k_0 >= lo^{k-1}_0 forward and hi^k_0 <= hi^{k+1}_0 backward.
 * Returns 1 when some box becomes empty. */
static int symmetry_break(double *lo, double *hi, int K, int D)
{
    for (int k = 1; k < K; ++k)
        if (lo[(k - 1) * D] > lo[k * D]) lo[k * D] = lo[(k - 1) * D];
    for (int k = K - 2; k >= 0; --k)
        if (hi[(k + 1) * D] < hi[k * D]) hi[k * D] = hi[(k + 1) * D];
    for (int k = 0; k < K; ++k)
        if (lo[k * D] > hi[k * D]) return 1;
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Sample reduction (Section 4.2, Algorithm 5)                             */
/* ---------------------------------------------------------------------- */

/* A sample is deleted when, in every node of the list, it is redundant for the
 * lower bound (alpha_s(M) < beta_glob, Section 4.2.1) and for the upper bound
 * (for every k: x_s outside M^k or some representative j of k has
 * ||x_s - x_j||^2 > alpha, Section 4.2.2).  `reps`/`n_reps` give each node's
 * representatives (KCO_MAXREPS slots per cluster); a node with n_reps NULL uses
 * none.  Returns the number of samples deleted. */
int64_t kco_sample_reduction(const double *X, int64_t N, int D, int K, int n_nodes,
                             const double *lo, const double *hi, const int64_t *reps,
                             const int32_t *n_reps, double beta_glob, double alpha,
                             uint8_t *active)
{
    const int KD = K * D;
    int64_t deleted = 0;
    for (int64_t s = 0; s < N; ++s) {
        if (!active[s]) continue;
        const double *x = X + s * D;
        int redundant = 1;
        for (int m = 0; m < n_nodes && redundant; ++m) {
            const double *l = lo + (int64_t)m * KD, *h = hi + (int64_t)m * KD;
            double as = INFINITY;
            for (int k = 0; k < K; ++k) {
                double v = farthest_corner_sk(x, l + k * D, h + k * D, D);
                if (v < as) as = v;
            }
            if (!(as < beta_glob)) { redundant = 0; break; }
            for (int k = 0; k < K && redundant; ++k) {
                if (!in_box(x, l + k * D, h + k * D, D)) continue;
                int excl = 0;
                if (n_reps) {
                    int nr = n_reps[m * K + k];
                    const int64_t *rp = reps + ((int64_t)m * K + k) * KCO_MAXREPS;
                    for (int q = 0; q < nr && !excl; ++q)
                        if (sqdist(x, X + rp[q] * D, D) > alpha) excl = 1;
                }
                if (!excl) redundant = 0;
            }
        }
        if (redundant) { active[s] = 0; ++deleted; }
    }
    return deleted;
}

/* ---------------------------------------------------------------------- */
/* Branch and bound (Algorithm 1)                                          */
/* ---------------------------------------------------------------------- */

typedef struct {
    double tol;          /* stop when (alpha - beta)/alpha <= tol; prune beta >= alpha(1 - tol) */
    int32_t use_bt;      /* 1: BB+CF+BT (assignment, tightening); 0: BB+CF */
    int32_t use_sr;      /* sample reduction (Algorithm 5) */
    int32_t i_sr;        /* run sample reduction every i_sr iterations */
    int32_t ball_cap;    /* representatives per cluster, at most 50 (<= 0: 50) */
    int32_t is_f32;      /* data are float values promoted to double */
    int64_t seed;        /* FFT start = seed mod N */
    int64_t node_limit;  /* 0: none */
    double time_limit;   /* seconds, 0: none */
} kco_opts;

typedef struct {
    double objective;
    double lower_bound;
    int64_t centers[KCO_MAXK];
    int64_t nodes;        /* nodes selected and processed (iterations) */
    int64_t created;      /* nodes pushed to the open set */
    int32_t seeds_found;
    int32_t status;       /* 0 optimal within tol, 4 time limit, 5 node limit */
    int64_t active_final; /* samples left after sample reduction */
    double fft_objective;
} kco_result;

typedef struct {
    double lo[KCO_MAXK * KCO_MAXD];
    double hi[KCO_MAXK * KCO_MAXD];
    double beta;
    int64_t id;
} kco_node;

typedef struct {
    kco_node *v;
    int64_t n, cap;
} kco_nodes;

static int nodes_push(kco_nodes *q, const kco_node *nd)
{
    if (q->n == q->cap) {
        int64_t nc = q->cap ? 2 * q->cap : 64;
        kco_node *nv = (kco_node *)realloc(q->v, sizeof(kco_node) * (size_t)nc);
        if (!nv) return 2;
        q->v = nv;
        q->cap = nc;
    }
    q->v[q->n++] = *nd;
    return 0;
}

/* Bound a freshly created child (Algorithm 1, Bounding): returns 0 when some
 * cluster box holds no active sample (the child is not added), else 1 with
 * beta(M_i) and the UB candidates (closest sample to each box midpoint). */
static int bound_child(const double *X, int64_t N, int D, int K, kco_node *c, const uint8_t *active,
                       int64_t *cand)
{
    for (int k = 0; k < K; ++k) {
        cand[k] = kco_mid_candidate(X, N, D, c->lo + k * D, c->hi + k * D, active, NULL);
        if (cand[k] < 0) return 0;
    }
    kco_lower_bound(X, N, D, K, c->lo, c->hi, active, &c->beta, NULL);
    return 1;
}

int kco_solve(const double *X, int64_t N, int D, int K, const kco_opts *opt, kco_result *res)
{
    if (K < 1 || K > KCO_MAXK || D < 1 || D > KCO_MAXD || N < K) return 1;
    const int KD = K * D;
    clock_t t0 = clock();
    memset(res, 0, sizeof(*res));
    uint8_t *active = (uint8_t *)malloc((size_t)N);
    if (!active) return 2;
    memset(active, 1, (size_t)N);

    /* root: M0, FFT upper bound (Algorithm 2), initial seeds (Section 4.1.1) */
    double lo0[KCO_MAXD], hi0[KCO_MAXD];
    kco_root_box(X, N, D, lo0, hi0);
    int64_t start = (int64_t)((uint64_t)opt->seed % (uint64_t)N);
    int64_t inc[KCO_MAXK];
    double alpha;
    kco_fft(X, N, D, K, start, inc, &alpha);
    res->fft_objective = alpha;
    int seeds_found = 0;
    if (opt->use_bt) {
        seeds_found = 1;
        for (int i = 0; i < K && seeds_found; ++i)
            for (int j = i + 1; j < K; ++j)
                if (!(sqdist(X + inc[i] * D, X + inc[j] * D, D) > 4.0 * alpha)) { seeds_found = 0; break; }
    }
    int64_t seeds[KCO_MAXK];
    for (int k = 0; k < K; ++k) seeds[k] = inc[k];
    const int use_sb = opt->use_bt && !seeds_found;

    kco_nodes open = {0};
    kco_node root;
    for (int k = 0; k < K; ++k)
        for (int a = 0; a < D; ++a) { root.lo[k * D + a] = lo0[a]; root.hi[k * D + a] = hi0[a]; }
    kco_lower_bound(X, N, D, K, root.lo, root.hi, NULL, &root.beta, NULL);
    root.id = 0;
    int64_t next_id = 1;
    nodes_push(&open, &root);
    res->created = 1;

    kco_tighten_out *tz = (kco_tighten_out *)malloc(sizeof(kco_tighten_out));
    int64_t *sr_reps = NULL;
    int32_t *sr_nreps = NULL;
    double *sr_lo = NULL, *sr_hi = NULL;
    int64_t iter = 0;
    int status = 0;
    double beta_glob = 0.0;
    for (;;) {
        if (open.n == 0) { beta_glob = alpha; break; }
        /* beta_i = min over open nodes; node selection picks (beta, id) smallest */
        int64_t sel = 0;
        for (int64_t i = 1; i < open.n; ++i)
            if (open.v[i].beta < open.v[sel].beta ||
                (open.v[i].beta == open.v[sel].beta && open.v[i].id < open.v[sel].id))
                sel = i;
        beta_glob = open.v[sel].beta;
        if (alpha - beta_glob <= opt->tol * alpha) break;
        if (opt->node_limit > 0 && iter >= opt->node_limit) { status = 5; break; }
        if (opt->time_limit > 0 && (double)(clock() - t0) / CLOCKS_PER_SEC > opt->time_limit) { status = 4; break; }
        kco_node M = open.v[sel];
        open.v[sel] = open.v[--open.n];
        ++iter;

        /* bounds tightening */
        kco_node Mh = M;
        int leaf = 0;
        int32_t cur_nreps[KCO_MAXK];
        int64_t cur_reps[KCO_MAXK * KCO_MAXREPS];
        for (int k = 0; k < K; ++k) cur_nreps[k] = 0;
        if (opt->use_bt) {
            kco_tighten(X, N, D, K, M.lo, M.hi, alpha, seeds_found ? seeds : NULL, active, opt->is_f32,
                        opt->ball_cap, tz);
            if (tz->status == 1) goto prune_step;
            memcpy(Mh.lo, tz->lo, sizeof(double) * KD);
            memcpy(Mh.hi, tz->hi, sizeof(double) * KD);
            for (int k = 0; k < K; ++k) cur_nreps[k] = tz->n_reps[k];
            memcpy(cur_reps, tz->reps, sizeof(cur_reps));
        } else {
            /* BB+CF keeps only the "centers on samples" tightening */
            for (int k = 0; k < K; ++k) {
                double *l = Mh.lo + k * D, *h = Mh.hi + k * D;
                double bl[KCO_MAXD], bh[KCO_MAXD];
                int64_t cnt = 0;
                for (int a = 0; a < D; ++a) { bl[a] = INFINITY; bh[a] = -INFINITY; }
                for (int64_t s = 0; s < N; ++s) {
                    if (!active[s] || !in_box(X + s * D, l, h, D)) continue;
                    ++cnt;
                    for (int a = 0; a < D; ++a) {
                        double v = X[s * D + a];
                        if (v < bl[a]) bl[a] = v;
                        if (v > bh[a]) bh[a] = v;
                    }
                }
                if (cnt == 0) goto prune_step;
                memcpy(l, bl, sizeof(double) * D);
                memcpy(h, bh, sizeof(double) * D);
            }
        }
        if (use_sb && symmetry_break(Mh.lo, Mh.hi, K, D)) goto prune_step;
        leaf = 1;
        for (int i = 0; i < KD; ++i)
            if (Mh.hi[i] > Mh.lo[i]) leaf = 0;

        /* sample reduction every i_sr iterations, over the open nodes and this one */
        if (opt->use_sr && opt->i_sr > 0 && iter % opt->i_sr == 0) {
            int64_t nn = open.n + 1;
            sr_lo = (double *)realloc(sr_lo, sizeof(double) * (size_t)(nn * KD));
            sr_hi = (double *)realloc(sr_hi, sizeof(double) * (size_t)(nn * KD));
            sr_reps = (int64_t *)realloc(sr_reps, sizeof(int64_t) * (size_t)(nn * K * KCO_MAXREPS));
            sr_nreps = (int32_t *)realloc(sr_nreps, sizeof(int32_t) * (size_t)(nn * K));
            for (int64_t i = 0; i < nn; ++i) {
                const kco_node *src = i < open.n ? &open.v[i] : &Mh;
                memcpy(sr_lo + i * KD, src->lo, sizeof(double) * KD);
                memcpy(sr_hi + i * KD, src->hi, sizeof(double) * KD);
                for (int k = 0; k < K; ++k) {
                    int64_t *rp = sr_reps + (i * K + k) * KCO_MAXREPS;
                    if (i < open.n) {
                        /* open nodes: the seeds are the assignments known there */
                        sr_nreps[i * K + k] = seeds_found ? 1 : 0;
                        rp[0] = seeds[k];
                    } else {
                        sr_nreps[i * K + k] = cur_nreps[k];
                        memcpy(rp, cur_reps + k * KCO_MAXREPS, sizeof(int64_t) * KCO_MAXREPS);
                    }
                }
            }
            kco_sample_reduction(X, N, D, K, (int)nn, sr_lo, sr_hi, sr_reps, sr_nreps, beta_glob, alpha,
                                 active);
        }

        if (!leaf) {
            /* branching: max-range variable (smallest k*D+a on ties), midpoint value */
            int bi = 0;
            double br = -1.0;
            for (int i = 0; i < KD; ++i)
                if (Mh.hi[i] - Mh.lo[i] > br) { br = Mh.hi[i] - Mh.lo[i]; bi = i; }
            double m, succ;
            split_point(Mh.lo[bi], Mh.hi[bi], opt->is_f32, &m, &succ);
            kco_node c[2];
            c[0] = Mh; c[0].hi[bi] = m;
            c[1] = Mh; c[1].lo[bi] = succ;
            for (int i = 0; i < 2; ++i) {
                int64_t cand[KCO_MAXK];
                if (!bound_child(X, N, D, K, &c[i], active, cand)) continue;
                double ub;
                kco_objective(X, N, D, K, cand, active, &ub, NULL);
                if (ub < alpha) { alpha = ub; memcpy(inc, cand, sizeof(int64_t) * K); }
                c[i].id = next_id++;
                ++res->created;
                if (c[i].beta < alpha - opt->tol * alpha) nodes_push(&open, &c[i]);
            }
        } else {
            /* leaf: every box is one point, a sample; its objective is exact */
            int64_t cand[KCO_MAXK];
            int ok = 1;
            for (int k = 0; k < K && ok; ++k) {
                cand[k] = kco_mid_candidate(X, N, D, Mh.lo + k * D, Mh.hi + k * D, active, NULL);
                if (cand[k] < 0) ok = 0;
            }
            if (ok) {
                double ub;
                kco_objective(X, N, D, K, cand, active, &ub, NULL);
                if (ub < alpha) { alpha = ub; memcpy(inc, cand, sizeof(int64_t) * K); }
            }
        }
    prune_step:
        /* remove every node with beta >= alpha (Algorithm 1, Bounding) */
        {
            int64_t w = 0;
            for (int64_t i = 0; i < open.n; ++i)
                if (open.v[i].beta < alpha - opt->tol * alpha) open.v[w++] = open.v[i];
            open.n = w;
        }
    }
    /* the incumbent's objective over all samples, the value reported */
    double obj;
    kco_objective(X, N, D, K, inc, NULL, &obj, NULL);
    res->objective = obj;
    res->lower_bound = beta_glob < obj ? beta_glob : obj;
    memcpy(res->centers, inc, sizeof(int64_t) * K);
    res->nodes = iter;
    res->seeds_found = seeds_found;
    res->status = status;
    int64_t na = 0;
    for (int64_t s = 0; s < N; ++s) na += active[s];
    res->active_final = na;
    free(open.v);
    free(tz);
    free(sr_lo); free(sr_hi); free(sr_reps); free(sr_nreps);
    free(active);
    return 0;
}
