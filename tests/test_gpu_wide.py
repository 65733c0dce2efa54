"""The float tightening kernels for shapes without a compile-time
instantiation (any K <= 16, D <= 128; node state in shared memory) against
the FP64 oracle, and the solver on such shapes (Section 4.1, Algorithms 3-4;
Algorithm 1).

Tightening inputs sit on a grid: coordinates are multiples of 1/4 and node
boxes are rounded outward to that grid, so every clamp and sample distance
is a multiple of 1/16 computed exactly in float (coordinates below 64 in
magnitude, squared distances summing below 2^20), and alpha is an odd
multiple of 1/32: float and double take every decision alike and statuses,
boxes and counts must equal the oracle's (candidates, nearest to an
off-grid midpoint, within the float argmin's error).  The representatives
are the seed and the attribute extremes, then the extremes of x_a + x_b and
x_a - x_b over the first 16 attribute pairs, at most min(ball_cap, 50) per
cluster on both sides: D = 29 .. 128 exercise the cap of 50 within the
attribute extremes, D = 2 .. 16 the pair directions.  Sums and differences
of grid coordinates are exact in float, so they order samples alike on
both sides.
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


def _blobs(n, d, k, seed, dtype=np.float32):
    return synth.gaussian_mixture(n, d, (1 / k,) * k, (1.0,) * k, (1.0,) * k, 10.0, seed, dtype=dtype)


def _grid_case(n, d, k, seed, B, scale):
    X = (np.round(_blobs(n, d, k, seed).astype(np.float64) * 4) / 4).astype(np.float32)
    c, fobj = oracle.fft(X, k, 0)
    rng = np.random.default_rng(seed)
    lo0, hi0 = X.min(0).astype(np.float64), X.max(0).astype(np.float64)
    lo = np.empty((B, k, d))
    hi = np.empty((B, k, d))
    for b in range(B):
        for j in range(k):
            # box j holds the FFT center j, so for alpha >= the FFT objective the
            # node holds a solution and cannot be proved infeasible
            w = rng.uniform(*scale, size=d) * (hi0 - lo0)
            ctr = X[c[j]].astype(np.float64)
            lo[b, j] = np.clip(ctr - rng.uniform(0.2, 0.8, size=d) * w, lo0, hi0)
            hi[b, j] = np.clip(lo[b, j] + w, lo0, hi0)
    lo = (np.floor(lo * 4) / 4).astype(np.float32)
    hi = (np.ceil(hi * 4) / 4).astype(np.float32)
    return X, c, fobj, lo, hi


def _lb_rel_gap(d):
    """Proved relative gap of a certified float bound: 2 gamma_n, n = ceil(D/2) + 3
    roundings, gamma_n = n u / (1 - n u), u = 2^-24 (below 1e-6 up to D = 10)."""
    n = (d + 1) // 2 + 3
    u = 2.0 ** -24
    return 2 * n * u / (1 - n * u)


def _compare(X, lo, hi, alpha, seeds, g, cap):
    rel = _lb_rel_gap(X.shape[1])
    st, glo, ghi = g["status"].cpu().numpy(), g["lo"].cpu().numpy(), g["hi"].cpu().numpy()
    gcnt, gcand, glb = g["count"].cpu().numpy(), g["cand"].cpu().numpy(), g["lb"].cpu().numpy()
    feasible = 0
    for b in range(lo.shape[0]):
        r = oracle.tighten(X, lo[b], hi[b], alpha, seeds=seeds, is_f32=True, ball_cap=cap)
        assert glb[b] <= r["beta"] and glb[b] >= r["beta"] * (1 - rel), (b, glb[b], r["beta"])
        assert st[b] == r["status"], (b, st[b], r["status"])
        if r["status"] == 1:
            continue
        feasible += 1
        assert np.array_equal(glo[b], r["lo"].astype(np.float32)), b
        assert np.array_equal(ghi[b], r["hi"].astype(np.float32)), b
        assert np.array_equal(gcnt[b], r["count"]), (b, gcnt[b], r["count"])
        for j in range(lo.shape[1]):
            mid = 0.5 * (r["box_bt_lo"][j] + r["box_bt_hi"][j])
            x = X[gcand[b, j]].astype(np.float64)
            assert np.all(x >= r["box_bt_lo"][j]) and np.all(x <= r["box_bt_hi"][j])
            dg = ((x - mid) ** 2).sum()
            do = ((X[r["cand"][j]].astype(np.float64) - mid) ** 2).sum()
            assert dg <= do * (1 + 1e-5) + 1e-9 * (1 + ((r["box_bt_hi"][j] - r["box_bt_lo"][j]) ** 2).sum())
    return feasible


@pytest.mark.parametrize("n,d,k,cap,seeded", [
    (6_000, 12, 3, 50, False), (6_000, 16, 5, 50, True), (4_000, 29, 3, 9, False), (4_000, 29, 3, 25, False),
    (4_000, 29, 3, 50, True), (8_000, 2, 5, 50, False), (6_000, 6, 3, 50, False), (3_000, 64, 2, 50, False),
    (3_000, 68, 3, 50, False), (2_000, 128, 2, 50, True)])
def test_wide_tighten_exact_on_grid(n, d, k, cap, seeded):
    X, c, fobj, lo, hi = _grid_case(n, d, k, seed=d + k, B=10, scale=(0.05, 0.5))
    kc = KCenter(_t(X), k)
    seeds = np.array(c, np.int64) if seeded else None
    feasible = 0
    for f in (0.8, 0.95, 1.02, 1.2):
        alpha = (np.round(fobj * f * 16) + 0.5) / 16
        g = kc.tighten(_t(lo), _t(hi), alpha, seeds=None if seeds is None else _t(seeds), ball_cap=cap)
        torch.cuda.synchronize()
        feasible += _compare(X, lo, hi, alpha, seeds, g, cap)
    assert feasible >= 5


@pytest.mark.parametrize("n,d,k,seed", [(1_500, 12, 3, 1), (1_500, 16, 3, 1), (1_000, 29, 3, 1), (2_000, 2, 5, 1),
                                        (1_500, 3, 6, 1), (800, 68, 3, 1)])
def test_wide_solve_matches_oracle(n, d, k, seed):
    """Solves on the wide shapes (D > 8: one shared sample set without sample
    reduction; K = 5, 6 with D <= 8: per-node lists) reach the oracle's
    certified optimum; the objective is the exact double value of the
    returned centers."""
    X = _blobs(n, d, k, seed)
    kc = KCenter(_t(X), k)
    g = kc.solve(tol=1e-12, time_limit_s=120.0)
    r = oracle.solve(X, k, tol=1e-12)
    assert g["status"] == 0 and r["status"] == 0
    assert abs(g["objective"] - r["objective"]) <= 1e-12 * r["objective"], (g, r)
    assert oracle.objective(X, g["centers"])[0] == g["objective"]


@pytest.mark.parametrize("n,d,k,cap,seeded", [
    (8_000, 2, 3, 9, False), (8_000, 2, 4, 50, True), (6_000, 3, 3, 12, True), (6_000, 3, 3, 50, False),
    (6_000, 4, 3, 25, False), (6_000, 4, 4, 50, True), (5_000, 5, 3, 50, False)])
def test_pair_direction_representatives_on_grid(n, d, k, cap, seeded):
    """ball_cap above 2D + 1 on the shapes of the register kernels (K <= 4,
    D <= 4, and D = 5 on the shared-memory kernels): the pair-direction
    representatives change the tightened boxes and counts, and the kernels
    match the oracle exactly."""
    X, c, fobj, lo, hi = _grid_case(n, d, k, seed=3 * d + k, B=10, scale=(0.05, 0.5))
    kc = KCenter(_t(X), k)
    seeds = np.array(c, np.int64) if seeded else None
    feasible = changed = 0
    for f in (0.8, 0.95, 1.02, 1.2):
        alpha = (np.round(fobj * f * 16) + 0.5) / 16
        g = kc.tighten(_t(lo), _t(hi), alpha, seeds=None if seeds is None else _t(seeds), ball_cap=cap)
        torch.cuda.synchronize()
        feasible += _compare(X, lo, hi, alpha, seeds, g, cap)
        for b in range(lo.shape[0]):
            r = oracle.tighten(X, lo[b], hi[b], alpha, seeds=seeds, is_f32=True, ball_cap=cap)
            # the budget of the seed and the attribute extremes alone
            r0 = oracle.tighten(X, lo[b], hi[b], alpha, seeds=seeds, is_f32=True, ball_cap=2 * d + int(seeded))
            if r["status"] != 1 and (not np.array_equal(r["count"], r0["count"])
                                     or not np.array_equal(r["lo"], r0["lo"])
                                     or not np.array_equal(r["hi"], r0["hi"])):
                changed += 1
    assert feasible >= 5
    assert changed >= 1, "the case does not tell the direction representatives from the attribute ones"


@pytest.mark.parametrize("n,d,k,seed", [(2_000, 2, 3, 1), (2_000, 3, 3, 2), (1_500, 4, 4, 1)])
def test_solve_with_pair_direction_representatives(n, d, k, seed):
    """A solve with ball_cap = 50 (per-node lists, wide kernels) reaches the
    oracle's certified optimum under the same budget."""
    X = _blobs(n, d, k, seed)
    kc = KCenter(_t(X), k)
    g = kc.solve(tol=1e-12, time_limit_s=120.0, ball_cap=50)
    r = oracle.solve(X, k, tol=1e-12, ball_cap=50)
    assert g["status"] == 0 and r["status"] == 0
    assert abs(g["objective"] - r["objective"]) <= 1e-12 * r["objective"], (g, r)
    assert oracle.objective(X, g["centers"])[0] == g["objective"]


def test_double_data_keep_the_attribute_extremes():
    """Double data: any ball_cap above 2D + 1 gives the attribute extremes,
    as in the oracle."""
    X = np.round(_blobs(600, 2, 3, 1, dtype=np.float64) * 4) / 4
    c, fobj = oracle.fft(X, 3, 0)
    lo = np.broadcast_to(X.min(0), (1, 3, 2)).copy()
    hi = np.broadcast_to(X.max(0), (1, 3, 2)).copy()
    for i, ctr in enumerate(c):
        lo[0, i] = np.maximum(lo[0, i], X[ctr] - 3)
        hi[0, i] = np.minimum(hi[0, i], X[ctr] + 3)
    kc = KCenter(_t(X), 3)
    alpha = (np.round(fobj * 16) + 0.5) / 16
    outs = []
    for cap in (5, 50, 0):
        g = kc.tighten(_t(lo), _t(hi), alpha, ball_cap=cap)
        torch.cuda.synchronize()
        outs.append({k: v.cpu().numpy() for k, v in g.items()})
        r = oracle.tighten(X, lo[0], hi[0], alpha, ball_cap=cap)
        assert outs[-1]["status"][0] == r["status"]
        if r["status"] != 1:
            assert np.array_equal(outs[-1]["lo"][0], r["lo"]) and np.array_equal(outs[-1]["hi"][0], r["hi"])
            assert np.array_equal(outs[-1]["count"][0], r["count"])
    for o in outs[1:]:
        for k in ("status", "lo", "hi", "count"):
            assert np.array_equal(o[k], outs[0][k])


@pytest.mark.parametrize("n,d,k,seeded,scale", [
    (3_000, 2, 3, False, (0.05, 0.5)), (3_000, 2, 4, True, (0.3, 0.9)), (2_500, 3, 3, False, (0.3, 0.9)),
    (2_500, 4, 3, True, (0.05, 0.5)), (2_000, 8, 2, False, (0.3, 0.9)), (2_000, 12, 3, False, (0.3, 0.9))])
def test_every_sample_representatives_on_grid(n, d, k, seeded, scale):
    """ball_cap = KC_BALLS_ALL: every sample of J_A^k is a representative of
    k (the ball-BT of Section 4.1.2 without a budget; the tiled sample x
    J_A^k pass).  Grid-valued data: the kernels match the oracle exactly.  At
    D <= 4 the default 50 (attribute and pair-direction extremes) almost
    always reach the same result; at D = 8 and 12 (16 of 28 or 66 pairs)
    the cases tell the unbudgeted sets from them."""
    from paper_2301_00061_gb300 import KC_BALLS_ALL
    X, c, fobj, lo, hi = _grid_case(n, d, k, seed=5 * d + k, B=8, scale=scale)
    kc = KCenter(_t(X), k)
    seeds = np.array(c, np.int64) if seeded else None
    feasible = changed = 0
    for f in (0.6, 0.8, 0.95, 1.02, 1.2):
        alpha = (np.round(fobj * f * 16) + 0.5) / 16
        g = kc.tighten(_t(lo), _t(hi), alpha, seeds=None if seeds is None else _t(seeds), ball_cap=KC_BALLS_ALL)
        torch.cuda.synchronize()
        feasible += _compare(X, lo, hi, alpha, seeds, g, oracle.BALLS_ALL)
        for b in range(lo.shape[0]):
            r = oracle.tighten(X, lo[b], hi[b], alpha, seeds=seeds, is_f32=True, ball_cap=oracle.BALLS_ALL)
            r0 = oracle.tighten(X, lo[b], hi[b], alpha, seeds=seeds, is_f32=True)
            if r0["status"] != 1 and (r["status"] != r0["status"] or not np.array_equal(r["count"], r0["count"])):
                changed += 1
    assert feasible >= 4
    if d >= 8:
        assert changed >= 1, "the case does not tell every sample from the default representatives"


def test_every_sample_representatives_tighten_at_least_as_much():
    """At N = 200,000 (the batched-solve recipe, 32 nodes, thousands of CTAs
    and sets J_A^k of tens of thousands of samples): with every assigned
    sample as a representative each node's result is at least as tight as
    with the default 50 -- infeasible wherever the default is, boxes inside
    the default's, counts |S_+^k| no larger -- since each test only gains
    representatives."""
    from paper_2301_00061_gb300 import KC_BALLS_ALL
    X, w = synth.make_workload("batched_solve", n=200_000)
    c, fobj = oracle.fft(X, w.k, 0)
    rng = np.random.default_rng(3)
    lo0, hi0 = X.min(0).astype(np.float64), X.max(0).astype(np.float64)
    B = 32
    lo = np.empty((B, w.k, w.d), np.float32)
    hi = np.empty((B, w.k, w.d), np.float32)
    for b in range(B):
        for j in range(w.k):
            wd = rng.uniform(0.05, 0.4, size=w.d) * (hi0 - lo0)
            ctr = X[c[j]].astype(np.float64)
            lo[b, j] = np.clip(ctr - rng.uniform(0.2, 0.8, size=w.d) * wd, lo0, hi0)
            hi[b, j] = np.clip(lo[b, j] + wd, lo0, hi0)
    kc = KCenter(_t(X), w.k)
    seen = 0
    for f in (0.9, 1.1):
        alpha = fobj * f
        g0 = {q: v.cpu().numpy() for q, v in kc.tighten(_t(lo), _t(hi), alpha).items()}
        ga = {q: v.cpu().numpy() for q, v in kc.tighten(_t(lo), _t(hi), alpha, ball_cap=KC_BALLS_ALL).items()}
        for b in range(B):
            if g0["status"][b] == 1:
                assert ga["status"][b] == 1, b
                continue
            if ga["status"][b] == 1:
                continue
            seen += 1
            assert np.all(ga["lo"][b] >= g0["lo"][b]) and np.all(ga["hi"][b] <= g0["hi"][b]), b
            assert np.all(ga["count"][b] <= g0["count"][b]), (b, ga["count"][b], g0["count"][b])
    assert seen >= 8


def test_solve_with_every_sample_representatives():
    """kc_solve with ball_cap = KC_BALLS_ALL (one shared sample set) reaches
    the oracle's certified optimum; per-node lists refuse it."""
    from paper_2301_00061_gb300 import KC_BALLS_ALL, KCError
    X = _blobs(1_500, 2, 3, 2)
    kc = KCenter(_t(X), 3)
    g = kc.solve(tol=1e-12, time_limit_s=120.0, ball_cap=KC_BALLS_ALL, lists=0)
    r = oracle.solve(X, 3, tol=1e-12)
    assert g["status"] == 0 and r["status"] == 0
    assert abs(g["objective"] - r["objective"]) <= 1e-12 * r["objective"], (g, r)
    with pytest.raises(KCError, match="KC_BALLS_ALL"):
        kc.solve(tol=1e-12, ball_cap=KC_BALLS_ALL)


def test_every_sample_representatives_argument_errors_and_edges():
    """KC_BALLS_ALL is refused for double data and for D > 16 (KC_EINVAL,
    the context stays usable); an empty batch is a no-op; a node whose boxes
    assign nothing (every J_A^k empty) gets no sample-based step, as in the
    oracle."""
    from paper_2301_00061_gb300 import KC_BALLS_ALL, KCError
    Xd = _blobs(400, 2, 3, 1, dtype=np.float64)
    kd = KCenter(_t(Xd), 3)
    lo = np.broadcast_to(Xd.min(0), (1, 3, 2)).copy()
    hi = np.broadcast_to(Xd.max(0), (1, 3, 2)).copy()
    with pytest.raises(KCError, match="KC_BALLS_ALL"):
        kd.tighten(_t(lo), _t(hi), 10.0, ball_cap=KC_BALLS_ALL)
    kd.tighten(_t(lo), _t(hi), 10.0)   # still usable
    X17 = _blobs(300, 17, 2, 1)
    k17 = KCenter(_t(X17), 2)
    lo17 = np.broadcast_to(X17.min(0), (1, 2, 17)).copy()
    hi17 = np.broadcast_to(X17.max(0), (1, 2, 17)).copy()
    with pytest.raises(KCError, match="KC_BALLS_ALL"):
        k17.tighten(_t(lo17), _t(hi17), 10.0, ball_cap=KC_BALLS_ALL)
    X, c, fobj, glo, ghi = _grid_case(1_000, 2, 3, seed=7, B=4, scale=(0.05, 0.5))
    kc = KCenter(_t(X), 3)
    g = kc.tighten(_t(glo[:0]), _t(ghi[:0]), fobj, ball_cap=KC_BALLS_ALL)
    assert g["status"].shape[0] == 0
    # the root: equal boxes, nothing assigned, no sample-based step
    L = np.broadcast_to(X.min(0).astype(np.float32), (1, 3, 2)).copy()
    H = np.broadcast_to(X.max(0).astype(np.float32), (1, 3, 2)).copy()
    alpha = (np.round(fobj * 16) + 0.5) / 16
    g = kc.tighten(_t(L), _t(H), alpha, ball_cap=KC_BALLS_ALL)
    torch.cuda.synchronize()
    _compare(X, L, H, alpha, None, g, oracle.BALLS_ALL)
