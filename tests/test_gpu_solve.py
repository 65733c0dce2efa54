"""Parity of the CUDA tightening, sample-reduction and solver paths with the
CPU oracle (Section 4.1 Algorithms 3-4, Section 4.2 Algorithm 5, Algorithm 1).

Double data: every decision is taken in double on both sides, so statuses,
tightened boxes, counts, candidates and masks are compared exactly.  Float
data: the kernels decide in float with proved margins; inputs are chosen so
that no decision quantity lies within the float error band of its threshold,
and then the outputs must again match exactly (boxes are sample coordinates or
the same double-rounded box-BT bounds).  Solves: the certified objective
equals the oracle's (or brute force's) double value to 1e-12 relative.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2301_00061_gb300 import KCenter  # noqa: E402

DEV = torch.device("cuda:0")


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def _blobs(n, d, k, seed, dtype):
    return synth.gaussian_mixture(n, d, (1 / k,) * k, (1.0,) * k, (1.0,) * k, 10.0, seed, dtype=dtype)


def _nodes_around(X, centers, B, seed, scale=(0.05, 0.6)):
    """B random nodes whose box k is a random sub-box of the root region,
    biased to contain sample centers[k] (a realistic branch-and-bound node)."""
    rng = np.random.default_rng(seed)
    lo0, hi0 = X.min(0).astype(np.float64), X.max(0).astype(np.float64)
    k, d = len(centers), X.shape[1]
    lo = np.empty((B, k, d)); hi = np.empty((B, k, d))
    for b in range(B):
        for j in range(k):
            w = rng.uniform(*scale, size=d) * (hi0 - lo0)
            c = X[centers[j]].astype(np.float64) + rng.normal(0, 0.3, size=d) * w
            lo[b, j] = np.clip(c - rng.uniform(0.2, 0.8, size=d) * w, lo0, hi0)
            hi[b, j] = np.clip(lo[b, j] + w, lo0, hi0)
    return np.ascontiguousarray(lo.astype(X.dtype)), np.ascontiguousarray(hi.astype(X.dtype))


def _compare_tighten(X, lo, hi, alpha, seeds, g, exact_cand=True, ball_cap=0):
    B, k, d = lo.shape
    st = g["status"].cpu().numpy() if hasattr(g["status"], "cpu") else g["status"]
    glo = g["lo"].cpu().numpy() if hasattr(g["lo"], "cpu") else g["lo"]
    ghi = g["hi"].cpu().numpy() if hasattr(g["hi"], "cpu") else g["hi"]
    gcnt = g["count"].cpu().numpy() if hasattr(g["count"], "cpu") else g["count"]
    gcand = g["cand"].cpu().numpy() if hasattr(g["cand"], "cpu") else g["cand"]
    glb = g["lb"].cpu().numpy() if hasattr(g["lb"], "cpu") else g["lb"]
    is_f32 = X.dtype == np.float32
    n_feasible = 0
    for b in range(B):
        r = oracle.tighten(X, lo[b], hi[b], alpha, seeds=seeds, is_f32=is_f32, ball_cap=ball_cap)
        assert glb[b] <= r["beta"] and glb[b] >= r["beta"] * (1 - 1e-6), (b, glb[b], r["beta"])
        assert st[b] == r["status"], (b, st[b], r["status"])
        if r["status"] == 1:
            continue
        n_feasible += 1
        assert np.array_equal(glo[b], r["lo"].astype(X.dtype)), (b, glo[b], r["lo"])
        assert np.array_equal(ghi[b], r["hi"].astype(X.dtype)), (b, ghi[b], r["hi"])
        assert np.array_equal(gcnt[b], r["count"]), (b, gcnt[b], r["count"])
        if exact_cand:
            assert np.array_equal(gcand[b], r["cand"]), (b, gcand[b], r["cand"])
        else:
            # the candidate is an argmin decided in float: its double distance to
            # the midpoint of the box-BT box must equal the exact minimum
            # within the float error, and it must lie in that box
            for j in range(k):
                mid = 0.5 * (r["box_bt_lo"][j] + r["box_bt_hi"][j])
                x = X[gcand[b, j]].astype(np.float64)
                assert np.all(x >= r["box_bt_lo"][j]) and np.all(x <= r["box_bt_hi"][j])
                dg = ((x - mid) ** 2).sum()
                do = ((X[r["cand"][j]].astype(np.float64) - mid) ** 2).sum()
                assert dg <= do * (1 + 1e-5) + 1e-9 * (1 + ((r["box_bt_hi"][j] - r["box_bt_lo"][j]) ** 2).sum()), (b, j, dg, do)
    return n_feasible


def _ambiguous(X, lo, hi, alpha, seeds, band=3e-6, ball_cap=0):
    """True when some decision quantity of the tightening lies within `band`
    (relative) of its threshold, where float and double decisions can differ."""
    Xd = X.astype(np.float64)
    for b in range(lo.shape[0]):
        bm = oracle.beta_matrix(Xd, lo[b], hi[b])
        if np.any(np.abs(bm - alpha) <= band * alpha):
            return True
        r = oracle.tighten(Xd, lo[b], hi[b], alpha, seeds=seeds, is_f32=True, ball_cap=ball_cap)
        for reps in r["reps"]:
            for j in reps:
                dd = ((Xd - Xd[j]) ** 2).sum(1)
                if np.any(np.abs(dd - alpha) <= band * alpha) or np.any(np.abs(dd - 4 * alpha) <= 4 * band * alpha):
                    return True
    return False


@pytest.mark.parametrize("d,k", [(2, 3), (2, 4), (4, 2)])
def test_tighten_f64_exact(d, k):
    X = _blobs(3_001, d, k, seed=d * 7 + k, dtype=np.float64)
    c, fobj = oracle.fft(X, k, 0)
    z = oracle.solve(X, k, tol=1e-12)["objective"]
    kc = KCenter(_t(X), k)
    for alpha in (z * 1.3, fobj):
        lo, hi = _nodes_around(X, c, 24, seed=k)
        for seeds in (None, c):
            g = kc.tighten(_t(lo), _t(hi), alpha, seeds=None if seeds is None else _t(seeds))
            torch.cuda.synchronize()
            nf = _compare_tighten(X, lo, hi, alpha, seeds, g)
            assert nf >= 1


@pytest.mark.parametrize("axes", [False, True])
@pytest.mark.parametrize("d,k", [(2, 3), (4, 3), (2, 4), (3, 3)])
def test_tighten_f32_exact_on_unambiguous_inputs(d, k, axes):
    """axes: ball_cap = 2D + 1 (the attribute extremes, and pair-direction
    extremes only where fewer than 2D + 1 of those are distinct), else the
    default of 50."""
    cap = 2 * d + 1 if axes else 0
    X = _blobs(4_003, d, k, seed=100 + d * 7 + k, dtype=np.float32)
    c, fobj = oracle.fft(X, k, 3)
    kc = KCenter(_t(X), k)
    lo, hi = _nodes_around(X, c, 12, seed=d)
    alpha = fobj * 0.71
    for _ in range(20):
        if not _ambiguous(X, lo, hi, alpha, None, ball_cap=cap):
            break
        alpha *= 1.0000373
    else:
        pytest.skip("could not find an unambiguous alpha")
    g = kc.tighten(_t(lo), _t(hi), alpha, ball_cap=cap)
    torch.cuda.synchronize()
    _compare_tighten(X, lo, hi, alpha, None, g, exact_cand=False, ball_cap=cap)


def _step_a_clear(X64, lo, hi, alpha, band=3e-6):
    """No center-based (Lemma 1) decision lies within `band` of alpha."""
    for b in range(lo.shape[0]):
        bm = oracle.beta_matrix(X64, lo[b], hi[b])
        if np.any(np.abs(bm - alpha) <= band * alpha):
            return False
    return True


def _ambiguous_ball_alpha(X, lo, hi, alpha0, ball_cap=0):
    """An alpha at which the center-based assignment, and so the
    representatives, are decided the same in float and double, but some
    sample s of a box-BT box M'^k lies within sqrt(alpha) of every
    representative of k except one, j, with ||x_s - x_j||^2 just above alpha
    (by 1e-7 relative): the double rule drops s from S_+^k, while the float
    evaluation (error bound ~1e-6 relative) cannot prove it outside.
    Returns (alpha, [(node, k, s)]) or None."""
    X64 = X.astype(np.float64)
    alpha = alpha0
    for _ in range(40):
        if _step_a_clear(X64, lo, hi, alpha):
            best = None
            for b in range(lo.shape[0]):
                r = oracle.tighten(X64, lo[b], hi[b], alpha, is_f32=True, ball_cap=ball_cap)
                if r["status"] == 1:
                    continue
                for k, reps in enumerate(r["reps"]):
                    if not reps:
                        continue
                    inb = np.all((X64 >= r["box_bt_lo"][k]) & (X64 <= r["box_bt_hi"][k]), axis=1)
                    idx = np.flatnonzero(inb)
                    dd = ((X64[idx, None, :] - X64[np.array(reps)][None, :, :]) ** 2).sum(2)   # (n_in, R)
                    over = dd > alpha
                    one = (over.sum(1) == 1)
                    gap = np.where(over, dd / alpha - 1.0, np.inf).min(1)
                    ok = one & (gap < 1e-4) & np.all(np.where(over, True, dd <= alpha * (1 - 3e-6)), axis=1)
                    for i in np.flatnonzero(ok):
                        cand = (gap[i], b, k, int(idx[i]), float(dd[i][over[i]][0]))
                        if best is None or cand[0] < best[0]:
                            best = cand
            if best is not None:
                a2 = best[4] * (1 - 1e-7)
                # moving alpha to a2 must not change the representatives or
                # any other decision of the center-based rule
                if _step_a_clear(X64, lo, hi, a2):
                    same = all(oracle.tighten(X64, lo[b], hi[b], a2, is_f32=True, ball_cap=ball_cap)["reps"] ==
                               oracle.tighten(X64, lo[b], hi[b], alpha, is_f32=True, ball_cap=ball_cap)["reps"]
                               for b in range(lo.shape[0]))
                    if same:
                        return a2, [(best[1], best[2], best[3])]
        alpha *= 1.0000373
    return None


@pytest.mark.parametrize("d,k,cap", [(2, 3, 0), (4, 3, 9)])
def test_tighten_f32_ambiguous_ball_decisions_are_conservative(d, k, cap):
    """Float tightening where float and double decisions differ: alpha is
    placed within the rounding band of a ball-membership test (see
    _ambiguous_ball_alpha).  The kernels take an exclusion only where the
    float evaluation proves it, so against the double oracle: every status 1
    is the oracle's status 1; where the oracle finds the node feasible, the
    tightened boxes contain the oracle's and the counts |S_+^k| are at least
    the oracle's; at the planted pair the count is strictly larger (the
    sample the oracle drops is kept)."""
    X = _blobs(4_003, d, k, seed=300 + d * 7 + k, dtype=np.float32)
    c, fobj = oracle.fft(X, k, 1)
    lo, hi = _nodes_around(X, c, 12, seed=d + 40)
    found = _ambiguous_ball_alpha(X, lo, hi, fobj * 0.71, ball_cap=cap)
    assert found is not None, "no ambiguous ball decision could be placed"
    alpha, planted = found
    kc = KCenter(_t(X), k)
    g = kc.tighten(_t(lo), _t(hi), alpha, ball_cap=cap)
    torch.cuda.synchronize()
    st, glo, ghi = g["status"].cpu().numpy(), g["lo"].cpu().numpy(), g["hi"].cpu().numpy()
    gcnt, glb = g["count"].cpu().numpy(), g["lb"].cpu().numpy()
    for b in range(lo.shape[0]):
        r = oracle.tighten(X, lo[b], hi[b], alpha, is_f32=True, ball_cap=cap)
        assert glb[b] <= r["beta"] and glb[b] >= r["beta"] * (1 - 1e-6)
        if st[b] == 1:
            assert r["status"] == 1, b
        if r["status"] == 1:
            continue
        assert st[b] != 1, b
        assert np.all(glo[b] <= r["lo"].astype(np.float32)) and np.all(ghi[b] >= r["hi"].astype(np.float32)), b
        assert np.all(gcnt[b] >= r["count"]), (b, gcnt[b], r["count"])
    for b, j, s_ in planted:
        r = oracle.tighten(X, lo[b], hi[b], alpha, is_f32=True, ball_cap=cap)
        if r["status"] != 1 and st[b] != 1:
            assert gcnt[b, j] > r["count"][j], (b, j, s_, gcnt[b], r["count"])


def test_tighten_f32_exact_at_one_million_samples():
    """The batched-solve recipe (D=4, K=3, weights .6/.3/.1) at N = 1e6, where
    the shared-set tightening kernels merge the partial keys of thousands of
    CTAs per node.  At this size thousands of decision values lie within
    1e-3 of any alpha, so no alpha keeps them all outside the float error
    band; instead the coordinates are rounded to multiples of 1/4 and the
    node boxes outward to that grid.  Every clamp and sample distance is then
    a multiple of 1/16 computed exactly in float, and alpha is an odd multiple
    of 1/32, so float and double take every decision alike and the outputs
    must equal the double oracle's exactly (statuses, boxes, counts;
    candidates -- nearest to a box-BT midpoint, which is off the grid --
    within the float argmin's error)."""
    X, w = synth.make_workload("batched_solve", n=1_000_000)
    X = (np.round(X.astype(np.float64) * 4) / 4).astype(np.float32)
    c, fobj = oracle.fft(X, w.k, 0)
    lo, hi = _nodes_around(X, c, 8, seed=77, scale=(0.05, 0.5))
    lo = (np.floor(lo.astype(np.float64) * 4) / 4).astype(np.float32)
    hi = (np.ceil(hi.astype(np.float64) * 4) / 4).astype(np.float32)
    kc = KCenter(_t(X), w.k)
    n_feasible = 0
    for cap in (0, 2 * X.shape[1] + 1):   # default (pair directions), attribute extremes
        for f in (0.83, 0.95):
            alpha = (np.round(fobj * f * 16) + 0.5) / 16
            g = kc.tighten(_t(lo), _t(hi), alpha, ball_cap=cap)
            torch.cuda.synchronize()
            n_feasible += _compare_tighten(X, lo, hi, alpha, None, g, exact_cand=False, ball_cap=cap)
    assert n_feasible >= 16


def test_tighten_root_and_ragged_sizes():
    """Root node (all boxes = M0): bound 0, nothing assigned (boxes equal)."""
    X = _blobs(1_037, 2, 3, seed=4, dtype=np.float64)
    kc = KCenter(_t(X), 3)
    lo0, hi0 = oracle.root_box(X)
    L = np.tile(lo0, (1, 3, 1)); H = np.tile(hi0, (1, 3, 1))
    alpha = oracle.fft(X, 3, 0)[1]
    g = kc.tighten(_t(L), _t(H), alpha)
    _compare_tighten(X, L, H, alpha, None, g)
    assert float(g["lb"][0]) == 0.0


@pytest.mark.parametrize("dtype", [np.float64, np.float32])
def test_sample_reduction_matches_oracle(dtype):
    X = _blobs(20_011, 2, 3, seed=5, dtype=dtype)
    r = oracle.solve(X, 3, tol=0.0, use_sr=False)
    c = r["centers"]
    alpha = r["objective"]
    lo = (X[c].astype(np.float64) - 0.3)[None].astype(dtype)
    hi = (X[c].astype(np.float64) + 0.3)[None].astype(dtype)
    beta = oracle.lower_bound(X, lo[0], hi[0])[0] * 0.999
    reps = np.array(c, dtype=np.int64).reshape(1, 3, 1)
    ref = oracle.sample_reduction(X, lo, hi, beta, alpha, np.ones(len(X), bool), reps=[[[int(v)] for v in c]])
    kc = KCenter(_t(X), 3)
    act = np.ones(len(X), np.uint8)
    act, n = kc.sample_reduction(lo, hi, beta, alpha, act, reps=reps)
    assert n == int(ref.sum()) == int(act.sum())
    assert np.array_equal(act.astype(bool), ref)
    assert n < len(X)


def _solve_both(X, k, **kw):
    kc = KCenter(_t(X), k)
    g = kc.solve(tol=1e-12, **kw)
    r = oracle.solve(X, k, tol=1e-12, use_bt=kw.get("use_bt", 1) == 1, use_sr=kw.get("i_sr", 1) > 0)
    return g, r


@pytest.mark.parametrize("n", [60, 300, 1000])
def test_solve_small_workload_f64(n):
    X, w = synth.make_workload("small")
    if n < 1000:
        X = X[synth.subsample_rows(1000, n, seed=0)]
    g, r = _solve_both(X, 3)
    assert g["status"] == 0
    assert abs(g["objective"] - r["objective"]) <= 1e-12 * r["objective"]
    # the stop rule is UB - LB <= 1e-12 UB; the reported LB is UB (1 - 1e-12)
    # rounded to double (error <= 2^-53 UB, 1 - 1e-12 itself off by <= 2^-53)
    # and the reported gap is rounded again: gap <= 1e-12 + 4 * 2^-53.
    assert g["lower_bound"] <= g["objective"] and g["gap"] <= 1e-12 + 4 * 2.0**-53
    assert oracle.objective(X, g["centers"])[0] == g["objective"]
    if n == 60:
        assert abs(g["objective"] - oracle.bruteforce(X, 3)[0]) <= 1e-12 * g["objective"]


# Tree sizes vary by orders of magnitude between instances of one recipe (some
# seeds need 1e5+ nodes at tol 1e-12); these seeds give trees of 1e2-1e3
# nodes that the serial oracle finishes in about a second.
@pytest.mark.parametrize("k,seed", [(2, 2), (3, 7), (4, 4)])
def test_solve_f32_small(k, seed):
    X = _blobs(3_000, 2, k, seed=seed, dtype=np.float32)
    g, r = _solve_both(X, k)
    assert abs(g["objective"] - r["objective"]) <= 1e-12 * r["objective"], (g, r)
    assert oracle.objective(X, g["centers"])[0] == g["objective"]


@pytest.mark.parametrize("lists", [0, 1])
@pytest.mark.parametrize("recipe", ["blobs2", "batched4", "outliers2"])
def test_solve_f32_lists_and_shared_set(recipe, lists):
    """Per-node surviving-sample lists (Section 4.2) and the shared compacted
    set reach the oracle's optimum; list mode really drops samples."""
    if recipe == "blobs2":
        X, k = _blobs(4_000, 2, 3, seed=21, dtype=np.float32), 3
    elif recipe == "batched4":
        X, k = synth.make_workload("batched_solve", n=2_500)[0], 3
    else:
        X, k = synth.make_workload("learned_order", n=3_000)[0], 4
    g, r = _solve_both(X, k, lists=lists)
    assert g["status"] == 0
    assert abs(g["objective"] - r["objective"]) <= 1e-12 * r["objective"], (g, r)
    assert oracle.objective(X, g["centers"])[0] == g["objective"]
    if lists:
        assert g["lists_filtered"] > 0 and g["samples_dropped"] > 0
    else:
        assert g["lists_filtered"] == 0


def test_solve_lists_with_a_full_arena():
    """With the list arena barely larger than the root list most children
    inherit their parent's list; the certificate is unchanged."""
    X = synth.make_workload("batched_solve", n=240_000)[0]
    kc = KCenter(_t(X), 3)
    lim = dict(tol=1e-12, time_limit_s=120.0)
    tight = kc.solve(lists=1, arena_mb=1, **lim)
    roomy = kc.solve(lists=1, **lim)
    shared = kc.solve(lists=0, **lim)
    assert tight["status"] == roomy["status"] == shared["status"] == 0
    z = shared["objective"]
    assert tight["objective"] == roomy["objective"] == z
    assert oracle.objective(X, tight["centers"])[0] == z
    assert tight["samples_dropped"] < roomy["samples_dropped"]


def test_solve_counted_filters_in_a_small_arena():
    """With the list arena holding little more than the root list, the
    longest lists of a batch are filtered in two passes (survivors counted,
    then written into a region of exactly that size), and filters that drop
    little make the descendants skip filtering for a few generations.  The
    certified optimum is the one of a solve with room for every list and of
    the shared-set mode."""
    X = synth.make_workload("batched_solve", n=2_000_000)[0]
    kc = KCenter(_t(X), 3)
    lim = dict(tol=1e-12, time_limit_s=120.0)
    tight = kc.solve(lists=1, arena_mb=10, **lim)
    roomy = kc.solve(lists=1, **lim)
    shared = kc.solve(lists=0, **lim)
    kc.close()
    assert tight["status"] == roomy["status"] == shared["status"] == 0
    assert tight["objective"] == roomy["objective"] == shared["objective"]
    assert oracle.objective(X, tight["centers"])[0] == tight["objective"]
    assert tight["lists_filtered"] > 0 and tight["samples_dropped"] > 0


def test_solve_plain_bb_and_no_sample_reduction():
    X = _blobs(800, 2, 3, seed=11, dtype=np.float64)
    for kw in (dict(use_bt=0, i_sr=0), dict(use_bt=1, i_sr=0), dict(use_bt=1, i_sr=1, batch=8)):
        g, r = _solve_both(X, 3, **kw)
        assert abs(g["objective"] - r["objective"]) <= 1e-12 * r["objective"], (kw, g, r)


def test_solve_bruteforce_tiny_random():
    for seed in range(6):
        rng = np.random.default_rng(seed)
        n = int(rng.integers(10, 40))
        X = _blobs(n, 2, 3, seed=seed, dtype=np.float64)
        for k in (1, 2, 3):
            kc = KCenter(_t(X), k)
            g = kc.solve(tol=0.0)
            z, _ = oracle.bruteforce(X, k)
            assert abs(g["objective"] - z) <= 1e-12 * max(z, 1e-300), (seed, k, g, z)


def test_solve_batched_workload_reduced():
    """The batched-solve workload's recipe (D=4, K=3, weights .6/.3/.1) at
    N=3000, where the serial oracle solves in seconds: the GPU certificate
    equals the oracle's optimum."""
    X, w = synth.make_workload("batched_solve", n=3_000)
    g, r = _solve_both(X, 3)
    assert g["status"] == 0
    assert abs(g["objective"] - r["objective"]) <= 1e-12 * r["objective"], (g, r)


def test_full_size_solves_properties():
    """Full-size recipes, where the serial oracle cannot finish a solve: the
    properties that hold at any size.  The FFT start equals the oracle's FFT;
    the reported objective is the exact double objective of the returned
    centers over all N samples (the oracle recomputes it); the certified lower
    bound never exceeds it; a certified solve meets the 1e-12 stop rule.
    Learned-order recipe at N=1e7 (certifies in seconds) and the batched-solve
    recipe at N=1e7 under a 10 s limit."""
    for name, n, limit in (("learned_order", 10_000_000, 120.0), ("batched_solve", 10_000_000, 10.0)):
        X, w = synth.make_workload(name, n=n)
        kc = KCenter(_t(X), w.k)
        g = kc.solve(tol=1e-12, time_limit_s=limit)
        kc.close()
        assert g["status"] in (0, 4), g
        if name == "learned_order":
            assert g["status"] == 0
            assert g["gap"] <= 1e-12 + 4 * 2.0**-53
        _, fobj = oracle.fft(X, w.k, 0)
        assert g["fft_objective"] == fobj
        assert oracle.objective(X, g["centers"])[0] == g["objective"]
        assert 0.0 <= g["lower_bound"] <= g["objective"] <= g["fft_objective"]


def test_full_size_bounds_and_prunes_replayed(tmp_path):
    """Full-size solves log every child they bound; a seeded sample is
    re-bounded by the oracle in double over all N samples.  Each certified
    bound lies within 1e-6 below the double closed form and never above it,
    and each pruned child's double bound reaches the final incumbent times
    (1 - tol), so the prune was sound.  Learned-order recipe at N=1e7 (solved
    to the certificate) and batched-solve recipe at N=1e7 (first 100,000
    nodes)."""
    import json
    for name, node_limit in (("learned_order", 0), ("batched_solve", 100_000)):
        X, w = synth.make_workload(name, n=10_000_000)
        kc = KCenter(_t(X), w.k)
        log = tmp_path / f"{name}.jsonl"
        g = kc.solve(tol=1e-12, log_path=str(log), node_limit=node_limit)
        kc.close()
        assert g["status"] == (0 if node_limit == 0 else 5)
        kids = [r for r in map(json.loads, open(log)) if "child" in r]
        assert len(kids) > 1000
        rng = np.random.default_rng(0)
        pruned = [r for r in kids if r["pruned"]]
        sample = [kids[i] for i in rng.choice(len(kids), 8, replace=False)]
        sample += [pruned[i] for i in rng.choice(len(pruned), min(8, len(pruned)), replace=False)]
        alpha = g["objective"]
        # the two children of every branched node partition its boxes: equal
        # except at one coordinate, split into [lo, m] and [succ(m), hi] with
        # succ the next float; each child's key is at least its parent's bound
        nodes = {r["id"]: r for r in map(json.loads, open(log)) if "id" in r}
        by_parent = {}
        for r in kids:
            by_parent.setdefault(r["parent"], []).append(r)
        assert all(len(v) == 2 for v in by_parent.values())
        for pid, (c0, c1) in by_parent.items():
            lo0, hi0 = np.array(c0["lo"], np.float32), np.array(c0["hi"], np.float32)
            lo1, hi1 = np.array(c1["lo"], np.float32), np.array(c1["hi"], np.float32)
            if c0["child"] > c1["child"]:
                lo0, hi0, lo1, hi1 = lo1, hi1, lo0, hi0
            split = np.flatnonzero((lo0 != lo1) | (hi0 != hi1))
            assert len(split) == 1, (name, pid)
            i = split[0]
            assert lo0[i] <= hi0[i] < lo1[i] <= hi1[i] and lo1[i] == np.nextafter(hi0[i], np.float32(np.inf))
            assert np.array_equal(np.delete(lo0, i), np.delete(lo1, i)) and np.array_equal(np.delete(hi0, i), np.delete(hi1, i))
            if pid in nodes:
                assert min(c0["key"], c1["key"]) >= nodes[pid]["lb"], (name, pid)
        rep = oracle.replay(X, str(log), g["objective"], g["centers"], 1e-12)
        # prunes are taken against the incumbent of their time, never below
        # the final objective: sound against it in a stopped solve too
        assert rep["ok"] and rep["rebound"] == 0, rep
        for r in sample:
            lo = np.array(r["lo"], np.float32).reshape(w.k, w.d)
            hi = np.array(r["hi"], np.float32).reshape(w.k, w.d)
            beta = oracle.lower_bound(X, lo, hi)[0]
            assert r["key"] <= beta and r["key"] >= beta * (1 - 1e-6), (name, r["child"], r["key"], beta)
            if r["pruned"]:
                assert beta >= alpha * (1 - 1e-12), (name, r["child"], beta, alpha)


def test_certificate_replay_at_one_hundred_million_samples(tmp_path):
    """The learned-order recipe at its full size (N = 1e8, D = 2, K = 4,
    4 blobs + 1 % outliers) solved to the 1e-12 certificate with every bounded
    child logged, then replayed by the oracle (O5): the FP64 objective of the
    returned centers over all 1e8 samples equals the reported one; EVERY
    pruned child is proved prunable (its logged witness sample's closed-form
    value reaches objective * (1 - 1e-12), else a re-bound over all samples);
    every branched node's children partition its boxes."""
    X, w = synth.make_workload("learned_order")
    kc = KCenter(_t(X), w.k)
    log = tmp_path / "c4.jsonl"
    g = kc.solve(tol=1e-12, log_path=str(log))
    kc.close()
    assert g["status"] == 0
    r = oracle.replay(X, str(log), g["objective"], g["centers"], 1e-12)
    print(r)
    assert r["ok"], r
    assert r["pruned"] > 1_000 and r["witness_proved"] >= r["pruned"] - r["rebound"]


def test_solve_degenerate_and_edge_inputs():
    """Edge cases of the method: N = K (every sample its own center, optimum
    0); all samples identical (zero-range root box, optimum 0); one attribute;
    float data smaller than one list tile (per-node lists never filtered);
    options out of range are rejected with a message."""
    from paper_2301_00061_gb300 import KCError
    X = np.array([[0.0, 0.0], [3.0, 1.0], [-2.0, 5.0]], np.float32)
    g = KCenter(_t(X), 3).solve(tol=1e-12)
    assert g["status"] == 0 and g["objective"] == 0.0 and sorted(g["centers"].tolist()) == [0, 1, 2]
    X = np.full((50, 3), 1.25, np.float32)
    g = KCenter(_t(X), 2).solve(tol=1e-12)
    assert g["status"] == 0 and g["objective"] == 0.0
    X = _blobs(500, 1, 3, seed=9, dtype=np.float32)
    g, r = _solve_both(X, 3)
    assert g["status"] == 0 and abs(g["objective"] - r["objective"]) <= 1e-12 * r["objective"]
    for seed in range(3):
        X = _blobs(int(np.random.default_rng(seed).integers(20, 60)), 2, 3, seed=seed, dtype=np.float32)
        g = KCenter(_t(X), 3).solve(tol=0.0, lists=1)
        z, _ = oracle.bruteforce(X, 3)
        assert abs(g["objective"] - z) <= 1e-12 * z, (seed, g, z)
    kc = KCenter(_t(_blobs(200, 2, 3, seed=1, dtype=np.float32)), 3)
    for bad in (dict(explore=101), dict(batch=5000), dict(rule_margin=-1.0), dict(fft_starts=-1), dict(lists=2),
                dict(order=1)):
        with pytest.raises(KCError) as e:
            kc.solve(tol=1e-12, **bad)
        assert "kc_solve" in str(e.value), (bad, str(e.value))
    with pytest.raises(KCError):
        kc.solve(tol=1.5)
    # shapes without a tightening kernel (double data beyond K = 4 or D = 4)
    # are refused, not run
    kc5 = KCenter(_t(_blobs(200, 2, 5, seed=1, dtype=np.float64)), 5)
    with pytest.raises(KCError) as e:
        kc5.solve(tol=1e-12)
    assert e.value.status == 1 and "kc_tighten" in str(e.value)
    kc5.close()


@pytest.mark.parametrize("d,k", [(3, 3), (3, 4), (6, 2), (8, 2), (4, 4), (7, 3), (8, 3), (8, 4), (5, 5)])
def test_solve_f32_lists_other_shapes(d, k):
    """Per-node lists with the remaining compiled tightening shapes (K=3 D=3,
    K<=4 D<=4, K<=2 D<=8) and with the shared-memory kernels in list mode
    (K >= 3 at D = 7, 8, where their sample tile for a shared set is smaller
    than a list batch's work item, and K = 5 at D = 5): the certified optimum
    equals the oracle's.  Seed 1 of each shape gives a tree of 15-4,400
    oracle nodes."""
    X = _blobs(2_500, d, k, seed=1, dtype=np.float32)
    g, r = _solve_both(X, k, lists=1)
    assert g["status"] == 0
    assert abs(g["objective"] - r["objective"]) <= 1e-12 * r["objective"], (g, r)
    assert oracle.objective(X, g["centers"])[0] == g["objective"]


def test_solve_limits_and_repeatability():
    """Stopping rules and determinism.  A time limit or a node limit returns
    KC_ETIMEOUT (4) or KC_ELIMIT (5) with a valid incumbent (its double
    objective over all samples), a certified bound no higher than it and the
    gap between them.  The same solve repeated gives the same optimum,
    centers, bound and node count, and the same bound batch repeated gives
    bitwise-equal outputs: the packed-key reductions do not depend on the
    order in which threads finish."""
    X = _blobs(200_000, 4, 3, seed=3, dtype=np.float32)
    kc = KCenter(_t(X), 3)
    for kw, st in ((dict(time_limit_s=1e-6), 4), (dict(node_limit=1), 5)):
        g = kc.solve(tol=1e-12, **kw)
        assert g["status"] == st, (kw, g)
        assert g["objective"] == oracle.objective(X, g["centers"])[0]
        assert 0.0 <= g["lower_bound"] <= g["objective"]
        assert g["gap"] == pytest.approx((g["objective"] - g["lower_bound"]) / g["objective"], rel=1e-12)
    runs = [kc.solve(tol=1e-12, node_limit=3000) for _ in range(2)]
    for key in ("status", "objective", "lower_bound", "nodes", "batches", "lists_filtered", "samples_dropped"):
        assert runs[0][key] == runs[1][key], (key, runs)
    assert np.array_equal(runs[0]["centers"], runs[1]["centers"])
    lo, hi = _nodes_around(X, runs[0]["centers"], 64, seed=4)
    outs = [[t.cpu().numpy() for t in kc.lower_bounds(_t(lo), _t(hi))] for _ in range(3)]
    for o in outs[1:]:
        for a, b in zip(outs[0], o):
            assert np.array_equal(a.view(np.uint8), b.view(np.uint8))
    kc.close()


@pytest.mark.parametrize("n,seed", [(600, 1), (1_000, 2)])
def test_solve_at_the_microbenchmark_shape(n, seed):
    """The lower-bound microbenchmark's shape (D = 8, K = 5, nested clusters of
    the lb_microbench recipe) solved to the 1e-12 certificate on small N (per-
    node lists, the shared-memory tightening kernels): the oracle's optimum,
    and the objective is the exact double value of the returned centers."""
    X, w = synth.make_workload("lb_microbench", n=n, seed=seed)
    kc = KCenter(_t(X), w.k)
    g = kc.solve(tol=1e-12, time_limit_s=120.0)
    r = oracle.solve(X, w.k, tol=1e-12)
    assert g["status"] == 0 and r["status"] == 0
    assert abs(g["objective"] - r["objective"]) <= 1e-12 * r["objective"], (g, r)
    assert oracle.objective(X, g["centers"])[0] == g["objective"]


@pytest.mark.parametrize("i_sr", [0, 2])
def test_solve_lists_with_filters_off_or_every_other_batch(i_sr):
    """Per-node lists with the children's filter off (i_sr = 0: every child
    keeps its parent's list) or run every other batch: the oracle's optimum."""
    X = _blobs(3_000, 2, 3, seed=5, dtype=np.float32)
    kc = KCenter(_t(X), 3)
    g = kc.solve(tol=1e-12, time_limit_s=60.0, i_sr=i_sr)
    r = oracle.solve(X, 3, tol=1e-12)
    assert g["status"] == 0 and r["status"] == 0
    assert abs(g["objective"] - r["objective"]) <= 1e-12 * r["objective"], (g, r)
