"""Pins for the CPU oracle: each test checks the oracle against something other
than itself -- hand-derived examples (tests/golden), brute force, dense grids,
scipy routines for special cases, and the invariants the paper proves.

The oracle is the parity reference for the CUDA path, so these run on CPU only.
"""
import itertools
import json
import os

import numpy as np
import pytest
from scipy.optimize import minimize
from scipy.spatial.distance import cdist

import oracle
import synth

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "hand_examples.json")))


def _blobs(n, d, seed, k=3):
    return synth.gaussian_mixture(n, d, (1 / k,) * k, (1.0,) * k, (1.0,) * k, 10.0, seed,
                                  dtype=np.float64)


def _objective_np(X, centers):
    """Eq. 1 at fixed centers via scipy's squared-Euclidean cdist."""
    Dm = cdist(X, X[np.asarray(centers)], "sqeuclidean")
    q = Dm.min(axis=1)
    return q.max(), int(np.argmax(q))


def _bruteforce_np(X, k):
    """Independent brute force with itertools and cdist (tiny N only)."""
    Dm = cdist(X, X, "sqeuclidean")
    best = np.inf
    for c in itertools.combinations(range(X.shape[0]), k):
        v = Dm[:, list(c)].min(axis=1).max()
        best = min(best, v)
    return best


# ---------------------------------------------------------------- golden ---

@pytest.mark.parametrize("ex", GOLD["objective"])
def test_golden_objective(ex):
    X = np.array(ex["X"], dtype=np.float64)
    z, c = oracle.bruteforce(X, ex["K"])
    assert z == ex["z"]
    r = oracle.solve(X, ex["K"], tol=0.0)
    assert r["objective"] == ex["z"]
    assert oracle.objective(X, c)[0] == ex["z"]


@pytest.mark.parametrize("ex", GOLD["lower_bound"])
def test_golden_lower_bound(ex):
    X = np.array(ex["X"])
    lo = np.array(ex["lo"]); hi = np.array(ex["hi"])
    bm = oracle.beta_matrix(X, lo, hi)
    assert np.array_equal(bm.min(axis=1), np.array(ex["beta_s"]))
    b, arg = oracle.lower_bound(X, lo, hi)
    assert b == ex["beta"] and arg == ex["argmax"]


@pytest.mark.parametrize("ex", GOLD["farthest_corner"])
def test_golden_farthest_corner(ex):
    x = np.array([ex["x"]])
    out = oracle.alpha_s(x, np.array(ex["lo"]), np.array(ex["hi"]))
    assert out[0] == ex["alpha_s"]


# ----------------------------------------------------- closed forms ---

def test_root_box_is_columnwise_min_max():
    X = _blobs(500, 5, 3)
    lo, hi = oracle.root_box(X)
    assert np.array_equal(lo, X.min(axis=0)) and np.array_equal(hi, X.max(axis=0))


@pytest.mark.parametrize("seed", range(4))
def test_objective_matches_cdist(seed):
    rng = np.random.default_rng(seed)
    X = _blobs(300, 1 + seed * 2, seed)
    c = rng.choice(300, size=4, replace=False)
    v, arg = oracle.objective(X, c)
    v2, arg2 = _objective_np(X, c)
    assert v == pytest.approx(v2, rel=1e-13)
    assert X[arg].tolist() == X[arg2].tolist() or abs(v - v2) < 1e-12 * v2


@pytest.mark.parametrize("d", [1, 2, 3, 5, 8])
def test_beta_sk_is_box_minimum(d):
    """beta_s^k is the minimum of ||x - mu||^2 over the box (Eq. 11):
    compare with a bounded numerical minimiser started from many points."""
    rng = np.random.default_rng(d)
    for _ in range(20):
        lo = rng.uniform(-3, 3, size=d)
        hi = lo + rng.uniform(0, 2, size=d) * (rng.uniform(size=d) < 0.8)
        x = rng.uniform(-6, 6, size=d)
        v = oracle.beta_sk(x, lo, hi)
        best = np.inf
        for _ in range(4):
            x0 = rng.uniform(lo, hi)
            r = minimize(lambda m: np.sum((x - m) ** 2), x0, jac=lambda m: 2 * (m - x),
                         bounds=list(zip(lo, hi)), method="L-BFGS-B", tol=1e-14)
            best = min(best, r.fun)
        assert v <= best * (1 + 1e-9) + 1e-12
        assert v == pytest.approx(best, rel=1e-7, abs=1e-9)


def test_beta_sk_dense_grid_2d():
    """Brute force on a dense grid (with the box's edges) bounds the closed form."""
    rng = np.random.default_rng(11)
    for _ in range(10):
        lo = rng.uniform(0, 2, size=2)
        hi = lo + rng.uniform(0.1, 2, size=2)
        x = rng.uniform(-2, 5, size=2)
        g0 = np.linspace(lo[0], hi[0], 801)
        g1 = np.linspace(lo[1], hi[1], 801)
        G = np.stack(np.meshgrid(g0, g1), -1).reshape(-1, 2)
        grid_min = ((G - x) ** 2).sum(1).min()
        v = oracle.beta_sk(x, lo, hi)
        step = max(hi - lo) / 800
        assert v <= grid_min + 1e-12
        assert grid_min - v <= 2 * step * (np.sqrt(grid_min) + step) + 1e-12


@pytest.mark.parametrize("d", [1, 2, 4, 6])
def test_farthest_corner_is_max_over_corners(d):
    """alpha_s: a convex function's maximum over a box sits at a corner, so
    enumerating all 2^D corners is a brute force for Eq. 13."""
    rng = np.random.default_rng(100 + d)
    k = 3
    X = rng.uniform(-4, 4, size=(40, d))
    lo = rng.uniform(-3, 0, size=(k, d))
    hi = lo + rng.uniform(0, 3, size=(k, d))
    got = oracle.alpha_s(X, lo, hi)
    for s in range(40):
        per_k = []
        for j in range(k):
            corners = np.array(list(itertools.product(*zip(lo[j], hi[j]))))
            per_k.append(((corners - X[s]) ** 2).sum(1).max())
        assert got[s] == pytest.approx(min(per_k), rel=1e-13)


def test_bruteforce_matches_independent_enumeration():
    for seed in range(6):
        X = _blobs(14, 2, seed)
        for k in (1, 2, 3):
            z, c = oracle.bruteforce(X, k)
            assert z == pytest.approx(_bruteforce_np(X, k), rel=1e-13)
            assert oracle.objective(X, c)[0] == z


# -------------------------------------------------------- invariants ---

def test_root_lower_bound_is_zero():
    X = _blobs(400, 3, 5)
    lo, hi = oracle.root_box(X)
    L = np.tile(lo, (3, 1)); H = np.tile(hi, (3, 1))
    assert oracle.lower_bound(X, L, H)[0] == 0.0


def test_lower_bound_at_degenerate_box_is_objective():
    """At M = {mu} with mu on samples the relaxation is exact (Section 5)."""
    X = _blobs(500, 4, 6)
    rng = np.random.default_rng(0)
    for _ in range(10):
        c = rng.choice(500, size=3, replace=False)
        b, _ = oracle.lower_bound(X, X[c], X[c])
        assert b == oracle.objective(X, c)[0]
        assert b == pytest.approx(_objective_np(X, c)[0], rel=1e-13)


def test_lower_bound_below_node_optimum():
    """beta(M) <= z(M) = min over centers in X cap M of the objective."""
    rng = np.random.default_rng(7)
    X = _blobs(24, 2, 8)
    Dm = cdist(X, X, "sqeuclidean")
    for _ in range(30):
        lo, hi = synth.random_boxes(X, 2, 1, int(rng.integers(1 << 30)), 0.2, 0.9)
        lo, hi = lo[0], hi[0]
        inb = [np.where(np.all((X >= lo[j]) & (X <= hi[j]), 1))[0] for j in range(2)]
        if any(len(i) == 0 for i in inb):
            continue
        zM = min(Dm[:, [a, b]].min(1).max() for a in inb[0] for b in inb[1])
        b, _ = oracle.lower_bound(X, lo, hi)
        assert b <= zM + 1e-12


def test_lower_bound_monotone_under_shrink_and_below_alpha_s():
    X = _blobs(2000, 3, 9)
    lo, hi = synth.nested_boxes(X, 3, 12, seed=4, hw_lo=1e-2, hw_hi=8.0)
    betas, _ = oracle.lower_bounds(X, lo, hi)
    assert np.all(np.diff(betas) >= 0)
    for b in (0, 6, 11):
        bs = oracle.beta_matrix(X, lo[b], hi[b]).min(1)
        assert np.all(bs <= oracle.alpha_s(X, lo[b], hi[b]))


def test_fft_is_greedy_and_two_approximation():
    """Algorithm 2: each new point is the farthest from the chosen set, and
    FFT is Gonzalez's 2-approximation, i.e. <= 4 z in squared distances."""
    for seed in range(5):
        X = _blobs(16, 2, 20 + seed)
        for k in (2, 3):
            c, obj = oracle.fft(X, k, start=seed % 16)
            assert c[0] == seed % 16
            for t in range(1, k):
                dmin = cdist(X, X[c[:t]], "sqeuclidean").min(1)
                assert dmin[c[t]] == dmin.max()
                assert c[t] == int(np.argmax(dmin))
            assert obj == pytest.approx(_objective_np(X, c)[0], rel=1e-13)
            z, _ = oracle.bruteforce(X, k)
            assert obj <= 4 * z * (1 + 1e-12)


# ---------------------------------------------------- branch and bound ---

@pytest.mark.parametrize("use_bt,use_sr", [(True, True), (True, False), (False, False)])
@pytest.mark.parametrize("seed", range(5))
def test_solve_matches_bruteforce(seed, use_bt, use_sr):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(8, 30))
    d = int(rng.integers(1, 4))
    X = _blobs(n, d, seed)
    for k in (1, 2, 3):
        r = oracle.solve(X, k, tol=0.0, use_bt=use_bt, use_sr=use_sr, seed=seed)
        z, _ = oracle.bruteforce(X, k)
        assert r["objective"] == pytest.approx(z, rel=1e-12)
        assert r["lower_bound"] <= r["objective"]
        assert oracle.objective(X, r["centers"])[0] == r["objective"]


@pytest.mark.parametrize("ball_cap", [1, 5, oracle.BALLS_ALL])
def test_solve_with_any_representatives_matches_bruteforce(ball_cap):
    """Lemma 2 and the ball test are sound for any set of assigned samples as
    representatives (Section 4.1.2): with one, five or every assigned sample,
    in double and in float data, the branch and bound reaches the brute-force
    optimum."""
    for seed in range(4):
        rng = np.random.default_rng(100 + seed)
        n = int(rng.integers(10, 26))
        for f32 in (False, True):
            X = _blobs(n, 2, 40 + seed)
            if f32:
                X = X.astype(np.float32).astype(np.float64)
            for k in (2, 3):
                r = oracle.solve(X, k, tol=0.0, ball_cap=ball_cap, is_f32=f32, seed=seed)
                z, _ = oracle.bruteforce(X, k)
                assert r["objective"] == pytest.approx(z, rel=1e-12), (seed, f32, k)
                assert r["lower_bound"] <= r["objective"]


def test_solve_float32_data_matches_bruteforce():
    for seed in range(4):
        X = synth.gaussian_mixture(25, 2, (0.5, 0.5), (1.0, 1.0), (1.0, 1.0), 5.0, seed,
                                   dtype=np.float32)
        for k in (2, 3, 4):
            r = oracle.solve(X, k, tol=0.0, is_f32=True)
            z, _ = oracle.bruteforce(X.astype(np.float64), k)
            assert r["objective"] == pytest.approx(z, rel=1e-12)


def test_solve_with_duplicates_and_degenerate_data():
    X = np.array([[1.0, 1.0]] * 5 + [[3.0, 1.0]] * 4 + [[1.0, 7.0]] * 3)
    for k in (1, 2, 3, 4):
        r = oracle.solve(X, k, tol=0.0)
        z, _ = oracle.bruteforce(X, k)
        assert r["objective"] == z
    X1 = np.zeros((7, 2))
    assert oracle.solve(X1, 2)["objective"] == 0.0


def test_small_workload_subsample_bruteforce():
    """Seed-0 subsample (N=60) of the small workload: B&B equals brute force."""
    X, w = synth.make_workload("small")
    Xs = X[synth.subsample_rows(w.n, 60, seed=0)]
    z, _ = oracle.bruteforce(Xs, 3)
    assert z == pytest.approx(_bruteforce_np(Xs, 3), rel=1e-13)
    for bt in (True, False):
        r = oracle.solve(Xs, 3, tol=0.0, use_bt=bt, use_sr=bt)
        assert r["objective"] == pytest.approx(z, rel=1e-12)


def test_small_workload_acceleration_invariance():
    """BB+CF+BT, BB+CF and sample reduction on/off reach the same optimum, and
    acceleration cuts the node count (Section 6.2)."""
    X, w = synth.make_workload("small")
    r_full = oracle.solve(X, 3, tol=1e-12)
    r_nosr = oracle.solve(X, 3, tol=1e-12, use_sr=False)
    r_plain = oracle.solve(X, 3, tol=1e-12, use_bt=False, use_sr=False)
    assert r_full["objective"] == r_nosr["objective"] == pytest.approx(r_plain["objective"], rel=1e-12)
    assert r_full["nodes"] < r_plain["nodes"]
    assert r_full["fft_objective"] <= 4 * r_full["objective"] * (1 + 1e-12)


def test_tighten_keeps_the_optimum():
    """Lemmas 1 and 2: with alpha >= z, any node whose boxes hold the optimal
    centers keeps them after assignment and tightening."""
    rng = np.random.default_rng(3)
    for trial in range(12):
        X = _blobs(40, 2, 50 + trial)
        k = 3
        z, c = oracle.bruteforce(X, k)
        alpha = z * (1.0 + 0.5 * rng.uniform())
        lo0, hi0 = oracle.root_box(X)
        lo = np.empty((k, 2)); hi = np.empty((k, 2))
        for j in range(k):
            w = rng.uniform(0.05, 1.0, size=2) * (hi0 - lo0)
            lo[j] = np.maximum(lo0, X[c[j]] - rng.uniform(0, 1, size=2) * w)
            hi[j] = np.minimum(hi0, lo[j] + w)
            hi[j] = np.maximum(hi[j], X[c[j]])
        t = oracle.tighten(X, lo, hi, alpha)
        assert t["status"] in (0, 2)
        for j in range(k):
            assert np.all(t["lo"][j] <= X[c[j]]) and np.all(X[c[j]] <= t["hi"][j])
            assert t["count"][j] >= 1
        assert t["beta"] <= z


def test_tighten_with_seeds_keeps_the_optimum():
    """Seeds fix cluster labels (Section 4.1.1); relabel the optimum to match."""
    X = np.concatenate([np.random.default_rng(s).normal(m, 0.3, size=(15, 2))
                        for s, m in enumerate(([0, 0], [8, 0], [0, 8]))])
    k = 3
    c, fobj = oracle.fft(X, k, 0)
    Dm = cdist(X[c], X[c], "sqeuclidean")
    assert np.all(Dm[~np.eye(k, dtype=bool)] > 4 * fobj)
    z, copt = oracle.bruteforce(X, k)
    lab = cdist(X[c], X[copt], "sqeuclidean").argmin(1)   # seed j sits with center copt[lab[j]]
    lo0, hi0 = oracle.root_box(X)
    t = oracle.tighten(X, np.tile(lo0, (k, 1)), np.tile(hi0, (k, 1)), fobj, seeds=c)
    assert t["status"] in (0, 2)
    for j in range(k):
        mu = X[copt[lab[j]]]
        assert np.all(t["lo"][j] <= mu) and np.all(mu <= t["hi"][j])
    r = oracle.solve(X, k, tol=0.0)
    assert r["seeds_found"] and r["objective"] == pytest.approx(z, rel=1e-12)


def test_sample_reduction_keeps_bound_samples():
    """A deleted sample can never be the farthest one: after reduction the
    objective at the optimum and the node bounds are unchanged (Section 4.2)."""
    X = _blobs(300, 2, 12)
    k = 3
    r = oracle.solve(X, k, tol=0.0, use_sr=False)
    alpha = r["objective"]
    lo0, hi0 = oracle.root_box(X)
    L = np.tile(lo0, (k, 1))[None]; H = np.tile(hi0, (k, 1))[None]
    # a node well inside: boxes around the optimal centers
    c = r["centers"]
    lo = (X[c] - 0.1)[None]; hi = (X[c] + 0.1)[None]
    beta_glob = oracle.lower_bound(X, lo[0], hi[0])[0]
    act = oracle.sample_reduction(X, lo, hi, beta_glob, alpha, np.ones(300, bool),
                                  reps=[[[int(ci)] for ci in c]])
    assert act.sum() < 300
    assert oracle.lower_bound(X, lo[0], hi[0], active=act)[0] == beta_glob
    assert oracle.objective(X, c, active=act)[0] == alpha
    # the root node keeps everything: alpha_s(M0) is large
    act0 = oracle.sample_reduction(X, L, H, 0.0, alpha, np.ones(300, bool))
    assert act0.all()


def test_tighten_hand_examples():
    """Tightening (Algorithms 3-4) on hand-derived 1-D instances: assignment,
    box-based tightening with the sqrt(alpha) radius, centers on samples,
    candidates, infeasibility and the leaf status."""
    for ex in GOLD["tighten"]:
        X = np.array(ex["X"])
        r = oracle.tighten(X, np.array(ex["lo"]), np.array(ex["hi"]), ex["alpha"])
        assert r["status"] == ex["status"], ex["derivation"]
        assert r["beta"] == ex["beta"]
        if ex["status"] == 0:
            blo, bhi = np.array(ex["box_bt_lo"]), np.array(ex["box_bt_hi"])
            if ex.get("outward"):
                # radius rounded up, bounds rounded outward: at most a few ulps wider
                assert np.all(r["box_bt_lo"] <= blo) and np.all(r["box_bt_lo"] >= blo - 1e-14)
                assert np.all(r["box_bt_hi"] >= bhi) and np.all(r["box_bt_hi"] <= bhi + 1e-14)
            else:
                assert r["box_bt_lo"].tolist() == ex["box_bt_lo"] and r["box_bt_hi"].tolist() == ex["box_bt_hi"]
            assert r["lo"].tolist() == ex["lo_out"] and r["hi"].tolist() == ex["hi_out"]
            assert list(r["count"]) == ex["count"] and list(r["cand"]) == ex["cand"]
            if "n_assigned" in ex:
                assert list(r["n_assigned"]) == ex["n_assigned"]


def test_sample_reduction_hand_examples():
    """Algorithm 5 on hand-derived 1-D instances: both redundancy tests, the
    strict LB-redundancy inequality, deletion only when redundant in every
    node, and the no-representative case."""
    for ex in GOLD["sample_reduction"]:
        lo = np.array([nd["lo"] for nd in ex["nodes"]])
        hi = np.array([nd["hi"] for nd in ex["nodes"]])
        X = np.array(ex["X"])
        act = oracle.sample_reduction(X, lo, hi, ex["beta_glob"], ex["alpha"], np.ones(len(X), bool),
                                      reps=ex["reps"])
        assert act.astype(int).tolist() == ex["active_out"], ex["derivation"]


@pytest.mark.parametrize("ex", GOLD["mid_candidate"], ids=lambda e: e["cite"][:24])
def test_golden_mid_candidate(ex):
    """UB candidate of one box (Section 3.2): the sample inside the box nearest
    to its middle point, smallest index on ties, -1 for an empty box."""
    idx, dist = oracle.mid_candidate(np.array(ex["X"]), np.array(ex["lo"]), np.array(ex["hi"]))
    assert idx == ex["index"], ex["derivation"]
    if idx >= 0:
        assert dist == ex["dist"]


def test_root_box_every_row_position():
    """M0 (Section 2.1) under every order of the rows: each extreme is taken
    whichever position holds it."""
    X = np.array([[0.0, 5.0], [3.0, -1.0], [-2.0, 2.0], [1.0, 7.0]])
    for perm in itertools.permutations(range(4)):
        lo, hi = oracle.root_box(X[list(perm)])
        assert lo.tolist() == [-2.0, -1.0] and hi.tolist() == [3.0, 7.0]


@pytest.mark.parametrize("ex", GOLD["objective_argmax"], ids=lambda e: e["derivation"][:16])
def test_golden_objective_argmax(ex):
    """Objective of a center set and the sample attaining it (Eq. 1)."""
    v, arg = oracle.objective(np.array(ex["X"]), np.array(ex["centers"]))
    assert v == ex["value"] and arg == ex["argmax"], ex["derivation"]


@pytest.mark.parametrize("ex", GOLD["split_point"], ids=lambda e: f'{e["lo"]}-{e["hi"]}')
def test_golden_split_point(ex):
    """Branching value (Section 3.3) and the upper child's lower end."""
    m, succ = oracle.split_point(ex["lo"], ex["hi"], ex["is_f32"])
    assert (m, succ) == (ex["m"], ex["succ"]), ex["derivation"]


def _float32_neighbours(v):
    f = np.float32(v)
    return float(np.nextafter(f, np.float32(-np.inf))), float(np.nextafter(f, np.float32(np.inf)))


def test_box_bt_float_bounds_round_outward():
    """Box-based tightening with float data (Section 4.1.2 under rounding):
    each bound of [max_j x_j - sqrt(alpha), min_j x_j + sqrt(alpha)] is the
    float nearest to the real value on the outside.  Samples 0 and 10, boxes
    [-5, 5] and [8, 12], alpha = 2: the real bounds -sqrt2, sqrt2, 10 - sqrt2,
    10 + sqrt2 are irrational and far (in double terms) from every float, so
    the oracle's bounds must be the largest float below, or the smallest
    float above, the real value -- checked in exact arithmetic."""
    from fractions import Fraction
    X = np.array([[0.0], [10.0]])
    r = oracle.tighten(X, np.array([[-5.0], [8.0]]), np.array([[5.0], [12.0]]), 2.0, is_f32=True)
    for k, c in ((0, 0), (1, 10)):
        lo_v, hi_v = r["box_bt_lo"][k][0], r["box_bt_hi"][k][0]
        assert float(np.float32(lo_v)) == lo_v and float(np.float32(hi_v)) == hi_v
        # lo_v <= c - sqrt2 < next float above lo_v
        t = Fraction(c) - Fraction(lo_v)
        assert t > 0 and t * t >= 2
        t_next = Fraction(c) - Fraction(_float32_neighbours(lo_v)[1])
        assert t_next < 0 or t_next * t_next < 2
        # previous float below hi_v < c + sqrt2 <= hi_v
        u = Fraction(hi_v) - Fraction(c)
        assert u > 0 and u * u >= 2
        u_prev = Fraction(_float32_neighbours(hi_v)[0]) - Fraction(c)
        assert u_prev < 0 or u_prev * u_prev < 2


def test_box_bt_bounds_contain_the_real_interval():
    """Box-based tightening in double never cuts inside the real interval
    [max_j x_j - sqrt(alpha), min_j x_j + sqrt(alpha)] (Section 4.1.2), for
    random radii and sample values, checked in exact arithmetic; and it stays
    within a few units in the last place of it."""
    from fractions import Fraction
    rng = np.random.default_rng(21)
    for _ in range(400):
        alpha = float(rng.uniform(0.01, 100.0))
        xs = np.sort(rng.uniform(-3.0, 3.0, size=2))
        X = np.array([[xs[0]], [xs[1]], [1e6]])
        lo = np.array([[-1e3], [1e5]]); hi = np.array([[1e3], [1e7]])
        r = oracle.tighten(X, lo, hi, alpha)
        assert list(r["n_assigned"]) == [2, 1]
        lv, hv = Fraction(r["box_bt_lo"][0][0]), Fraction(r["box_bt_hi"][0][0])
        M, m = Fraction(float(xs[1])), Fraction(float(xs[0]))
        a = Fraction(alpha)
        assert M - lv > 0 and (M - lv) ** 2 >= a          # lo' <= max x - sqrt(alpha)
        assert hv - m > 0 and (hv - m) ** 2 >= a          # hi' >= min x + sqrt(alpha)
        rt = float(np.sqrt(alpha))
        assert float(M - lv) - rt <= 8 * np.spacing(rt) + 4 * np.spacing(abs(float(M)) + 1.0)
        assert float(hv - m) - rt <= 8 * np.spacing(rt) + 4 * np.spacing(abs(float(m)) + 1.0)


def test_parallel_lower_bounds_equal_serial():
    """The all-cores variant of the bound loop (the timed CPU baseline) gives
    the serial loop's values and argmax bit for bit: random data, ties from
    duplicated rows (the smallest index must win across blocks), fewer
    samples than blocks, and a single sample."""
    rng = np.random.default_rng(4)
    X = rng.normal(size=(5_003, 3))
    X[4000] = X[17]                      # a tie across blocks
    lo = rng.normal(size=(9, 2, 3)) - 0.5
    hi = lo + rng.uniform(0.1, 1.0, size=(9, 2, 3))
    for Xs in (X, X[:5], X[:1]):
        a, b = oracle.lower_bounds(Xs, lo, hi)
        c, d, nt = oracle.lower_bounds_par(Xs, lo, hi)
        assert nt >= 1
        assert np.array_equal(a, c) and np.array_equal(b, d)
    # a box around the duplicated pair's far side: both copies attain the max
    lo2 = np.full((1, 1, 3), -50.0); hi2 = np.full((1, 1, 3), -49.0)
    far = np.argmax(oracle.beta_matrix(X, lo2[0], hi2[0])[:, 0])
    X2 = X.copy(); X2[4999] = X2[far]
    a, b = oracle.lower_bounds(X2, lo2, hi2)
    c, d, _ = oracle.lower_bounds_par(X2, lo2, hi2)
    assert b[0] == d[0] == min(far, 4999) and a[0] == c[0]


def test_objective_at_points():
    """Eq. 1 at centers given as points: at sample points it is the objective
    of those samples; at other points it equals a scipy distance-matrix
    evaluation, and the worst sample is the smallest index of the maximum."""
    from scipy.spatial.distance import cdist
    rng = np.random.default_rng(8)
    X = rng.normal(size=(700, 3))
    c = np.array([3, 250, 699])
    assert oracle.objective_points(X, X[c]) == oracle.objective(X, c)
    mu = rng.uniform(-1, 1, size=(2, 3))
    q = (cdist(X, mu) ** 2).min(1)
    v, a = oracle.objective_points(X, mu)
    assert abs(v - q.max()) <= 1e-12 * q.max() and a == int(np.argmax(q))
    X2 = np.concatenate([X, X[a:a + 1]])          # a duplicate of the worst sample: the first index wins
    assert oracle.objective_points(X2, mu)[1] == a


def test_representatives_along_pair_directions():
    """Reading of the 50-ball budget (Section 4.1.2): the seed, the assigned
    samples at the min and max of each attribute, then the min and max of
    x_a + x_b and of x_a - x_b over the first attribute pairs; duplicates
    skipped, at most ball_cap (default 50); the pair directions for float
    data only.  Hand-derived, one cluster, every sample assigned: s0 (0,0),
    s1 (4,0), s2 (0,4), s3 (3,3), s4 (1,-1), s5 (3.5,-0.875).
      attributes: min x0 s0 (tie with s2: smaller index), max x0 s1,
                  min x1 s4, max x1 s2            -> [0, 1, 4, 2]
      x0 + x1: 0, 4, 4, 6, 0, 2.625: min s0 (dup), max s3 (new)
      x0 - x1: 0, 4, -4, 0, 2, 4.375: min s2 (dup), max s5 (new)  -> [0, 1, 4, 2, 3, 5]
    Every value is exact in float."""
    X = np.array([[0.0, 0.0], [4.0, 0.0], [0.0, 4.0], [3.0, 3.0], [1.0, -1.0], [3.5, -0.875]])
    lo = np.array([[-10.0, -10.0]])
    hi = np.array([[10.0, 10.0]])
    assert oracle.tighten(X, lo, hi, 1e6, ball_cap=50, is_f32=True)["reps"] == [[0, 1, 4, 2, 3, 5]]
    assert oracle.tighten(X, lo, hi, 1e6, is_f32=True)["reps"] == [[0, 1, 4, 2, 3, 5]]   # default 50
    assert oracle.tighten(X, lo, hi, 1e6, ball_cap=5, is_f32=True)["reps"] == [[0, 1, 4, 2, 3]]
    assert oracle.tighten(X, lo, hi, 1e6, ball_cap=4, is_f32=True)["reps"] == [[0, 1, 4, 2]]
    # double data: the attribute extremes only, whatever the cap
    assert oracle.tighten(X, lo, hi, 1e6, ball_cap=50)["reps"] == [[0, 1, 4, 2]]
    assert oracle.tighten(X, lo, hi, 1e6)["reps"] == [[0, 1, 4, 2]]
    # with a seed it comes first and is not repeated
    assert oracle.tighten(X, lo, hi, 1e6, seeds=np.array([3]), is_f32=True)["reps"] == [[3, 0, 1, 4, 2, 5]]
    assert oracle.tighten(X, lo, hi, 1e6, seeds=np.array([3]))["reps"] == [[3, 0, 1, 4, 2]]


def test_pair_direction_values_in_the_data_precision():
    """For float data x_a + x_b is rounded to float before it is compared.
    Samples s0 (2^24, 0), s1 (2^24, 1), s2 (2^24 + 2, -5), s3 (0, 3):
      attributes: min x0 s3, max x0 s2, min x1 s2 (dup), max x1 s3 (dup) -> [3, 2]
      x0 + x1: 2^24, 2^24 + 1, 2^24 - 3, 3 -- in float 2^24 + 1 rounds to 2^24
        (ties to even): the max is s0 (tie with s1, smaller index), where
        the exact sums would pick s1; the min is s3 (dup)
      x0 - x1: 2^24, 2^24 - 1, 2^24 + 7, -3: max s2 (dup), min s3 (dup)."""
    X = np.array([[16777216.0, 0.0], [16777216.0, 1.0], [16777218.0, -5.0], [0.0, 3.0]])
    lo = np.array([[-1e8, -1e8]])
    hi = np.array([[1e8, 1e8]])
    assert oracle.tighten(X, lo, hi, 1e30, ball_cap=50, is_f32=True)["reps"] == [[3, 2, 0]]
    # the same samples shifted off the rounding tie pick s1: the sum decides
    X2 = X.copy()
    X2[1, 1] = 2.0
    assert oracle.tighten(X2, lo, hi, 1e30, ball_cap=50, is_f32=True)["reps"] == [[3, 2, 1]]


def _assign_step_a(X, lo, hi, alpha):
    """Lemma 1 from its definition: beta_s^k = squared distance from x_s to
    box k; k excluded when beta_s^k > alpha; assigned when one cluster is left."""
    d = ((X[:, None, :] - np.clip(X[:, None, :], lo[None], hi[None])) ** 2).sum(2)   # (N, K)
    left = d <= alpha
    return np.where(left.sum(1) == 1, left.argmax(1), -1), left


def test_uncapped_representatives_brute_force():
    """ball_cap = BALLS_ALL (the paper's ball-BT without a budget, Section
    4.1.2 and Algorithm 3): every sample of J_A^k is a representative.  Against
    a direct evaluation of the definitions on small random instances: the
    step-A assignment (Lemma 1), the sample-based assignment of the others
    (Lemma 2: k excluded when some j of J_A^k is farther than 4 alpha), and
    |S_+^k| = samples of the box-BT box within sqrt(alpha) of every j of
    J_A^k; the node's status follows (no cluster left, or an empty S_+)."""
    rng = np.random.default_rng(11)
    checked = 0
    for trial in range(40):
        n, d, k = 60, 2, 2
        cen = np.array([[-4.0, 0.0], [4.0, 0.0]]) + rng.uniform(-1, 1, size=(2, 2))
        X = np.round(np.repeat(cen, n // k, 0) + rng.normal(0, 1.2, size=(n, d)), 2)
        w = rng.uniform(1.0, 3.0, size=(k, d))
        lo, hi = cen - w, cen + w
        alpha = float(rng.uniform(3.0, 25.0))
        r = oracle.tighten(X, lo, hi, alpha, ball_cap=oracle.BALLS_ALL)
        asg, left = _assign_step_a(X, lo, hi, alpha)
        if (left.sum(1) == 0).any():
            assert r["status"] == 1
            continue
        J = [np.flatnonzero(asg == j) for j in range(k)]
        if any(len(j) == 0 for j in J):
            continue   # step B does not run without representatives in every cluster
        dd = ((X[:, None, :] - X[None, :, :]) ** 2).sum(2)
        infeasible = False
        for s_ in np.flatnonzero(asg < 0):
            if not any(not (dd[s_, J[j]] > 4 * alpha).any() for j in range(k)):
                infeasible = True
        count = []
        for j in range(k):
            inb = np.all((X >= r["box_bt_lo"][j]) & (X <= r["box_bt_hi"][j]), axis=1)
            count.append(int(np.sum(inb & (dd[:, J[j]] <= alpha).all(1))))
        if infeasible or min(count) == 0 or np.any(r["box_bt_lo"] > r["box_bt_hi"]):
            assert r["status"] == 1, trial
            continue
        if r["status"] == 1:
            continue   # infeasible through the final boxes (J_B and S_+ boxes disjoint)
        assert list(r["count"]) == count, (trial, r["count"], count)
        checked += 1
    assert checked >= 10


def test_uncapped_representatives_reach_a_hull_vertex_the_budget_misses():
    """Twelve samples on the unit circle at 60, 90, ..., 330, 0, 30 degrees
    (in this index order) and one sample s at 0.1 (cos 240, sin 240), one
    cluster, box [-2, 2]^2, alpha = 1.2 (double data).  Every sample is
    assigned; the default representatives are the attribute extremes: 0, 180,
    90 and 270 degrees (samples 10, 4, 1, 7).  Squared distances from
    s: 1 + 0.01 - 0.2 cos(angle - 240): 1.21 to the point at 60 degrees, 1.1832
    at 30 and 90, at most 1.11 to the four representatives; so s is within
    sqrt(alpha) of every representative (|S_+| = 1: the circle points lie
    outside the box-BT box [1 - sqrt(1.2), sqrt(1.2) - 1]^2; the tightened box
    is the point s, a leaf), but not of the sample at 60 degrees: with every
    assigned sample as a representative S_+ is empty and the node is
    infeasible."""
    ang = np.deg2rad((np.arange(0, 360, 30) + 60) % 360)
    X = np.concatenate([np.stack([np.cos(ang), np.sin(ang)], 1), [[0.1 * np.cos(np.deg2rad(240)),
                                                                   0.1 * np.sin(np.deg2rad(240))]]])
    lo = np.array([[-2.0, -2.0]])
    hi = np.array([[2.0, 2.0]])
    r = oracle.tighten(X, lo, hi, 1.2)
    assert r["status"] == 2 and list(r["count"]) == [1]
    assert sorted(r["reps"][0]) == [1, 4, 7, 10]
    r = oracle.tighten(X, lo, hi, 1.2, ball_cap=oracle.BALLS_ALL)
    assert r["status"] == 1
