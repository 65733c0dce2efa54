"""Planted mistakes in the oracle must fail its pins.

Each mutant below turns one spot of the oracle (``oracle/kc_oracle.c`` or
``oracle/mlp.py``) into a plausible slip: a dropped term, a wrong sign, index
or bound, a transposed operand, a wrong tie-break, a looser test.  The pin
suites (``test_oracle_pins.py`` with ``test_oracle_replay.py``, and
``test_oracle_mlp_pins.py``) are run against
each mutant in a child process and must report a failed assertion.  Mutants
are written to a temporary directory; the committed oracle is never touched.

Left out: a mutant of the symmetry-breaking step that swaps the assignment
direction (the serial branch and bound then stops shrinking boxes and does not
end, which is no assertion), and three that change no result: testing seed k
against box k at 4 alpha instead of alpha (a box farther than alpha from its
seed also fails the ball test, which the seed passes as a representative),
selecting the open node with the largest bound instead of the smallest (the
same optimum by another tree), and giving the open nodes of sample reduction
no representatives (fewer deletions, the same optimum).
"""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
C_SRC = os.path.join(ROOT, "oracle", "kc_oracle.c")
MLP_SRC = os.path.join(ROOT, "oracle", "mlp.py")

# name -> (passage, [(original text, planted text), ...]) in kc_oracle.c
C_MUTANTS = {
    "clamp_upper_side_returns_lo": ("Sec. 3.1, mid{lo, x, hi}",
                                    [("if (x > h) return h;", "if (x > h) return l;")]),
    "distance_sign": ("Eq. 1", [("        double d = x[a] - y[a];\n", "        double d = x[a] + y[a];\n")]),
    "clamp_box_transposed": ("Eq. 11", [("double mu = mid3(lo[a], x[a], hi[a]);",
                                          "double mu = mid3(lo[a], x[a], lo[a]);")]),
    "farthest_corner_is_nearest": ("Eq. 13", [("? lo[a] : hi[a];", "? hi[a] : lo[a];")]),
    "bound_drops_last_cluster": ("Eq. 9", [("double bs = INFINITY;\n        for (int k = 0; k < K; ++k) {",
                                            "double bs = INFINITY;\n        for (int k = 0; k < K - 1; ++k) {")]),
    "bound_argmax_last_on_ties": ("Eq. 9", [("if (bs > best) { best = bs; arg = s; }",
                                             "if (bs >= best) { best = bs; arg = s; }")]),
    "objective_first_center_only": ("Eq. 1", [("double v = sqdist(X + s * D, X + centers[k] * D, D);",
                                               "double v = sqdist(X + s * D, X + centers[0] * D, D);")]),
    "objective_argmax_last_on_ties": ("Eq. 1", [("if (q > best) { best = q; arg = s; }",
                                                 "if (q >= best) { best = q; arg = s; }")]),
    "root_box_skips_row_1": ("Sec. 2.1", [("for (int64_t s = 1; s < N; ++s)\n        for (int a = 0; a < D; ++a) {",
                                           "for (int64_t s = 2; s < N; ++s)\n        for (int a = 0; a < D; ++a) {")]),
    "fft_distance_to_last_center_only": ("Alg. 2", [("if (v < dmin[s]) dmin[s] = v;", "dmin[s] = v;")]),
    "fft_ignores_start": ("Alg. 2", [("dmin[s] = sqdist(X + s * D, X + start * D, D);",
                                      "dmin[s] = sqdist(X + s * D, X + 0 * D, D);")]),
    "bruteforce_skips_subsets": ("Eq. 1", [("while (i >= 0 && c[i] == N - K + i) --i;",
                                            "while (i >= 0 && c[i] >= N - K + i - 1) --i;")]),
    "candidate_half_range": ("Sec. 3.2", [("mid[a] = 0.5 * (lo[a] + hi[a]);", "mid[a] = 0.5 * (hi[a] - lo[a]);")]),
    "split_half_range": ("Sec. 3.3", [("double m = 0.5 * (lo + hi);", "double m = 0.5 * (hi - lo);")]),
    "assign_with_two_clusters_open": ("Alg. 3, Lemma 1", [("if (left == 1) asg[s] = (int8_t)kk;",
                                                           "if (left >= 1) asg[s] = (int8_t)kk;")]),
    "no_cluster_left_not_infeasible": ("Alg. 3, Lemma 1",
                                       [("if (left == 0) infeasible = 1;\n        if (left == 1) asg[s] = (int8_t)kk;",
                                         "if (left == 1) asg[s] = (int8_t)kk;")]),
    "box_bt_wrong_extreme": ("Sec. 4.1.2", [("double l = round_down_dt(nextafter(jmax[i] - r, -INFINITY), is_f32);",
                                             "double l = round_down_dt(nextafter(jmin[i] - r, -INFINITY), is_f32);")]),
    "sample_based_alpha_for_4alpha": ("Alg. 3, Lemma 2", [("KCO_MAXREPS + q] * D, D) > four_alpha",
                                                          "KCO_MAXREPS + q] * D, D) > alpha")]),
    "ball_bt_4alpha_for_alpha": ("Alg. 4", [("KCO_MAXREPS + q] * D, D) > alpha) ok = 0;",
                                            "KCO_MAXREPS + q] * D, D) > four_alpha) ok = 0;")]),
    "centers_on_samples_bbox_dropped": ("Alg. 4", [("double l = slo[i], h = shi[i];",
                                                    "double l = blo[i], h = bhi[i];")]),
    "sr_nonstrict_corner_test": ("Sec. 4.2.1", [("if (!(as < beta_glob))", "if (!(as <= beta_glob))")]),
    "sr_nearest_for_farthest_corner": ("Sec. 4.2.1, Eq. 13",
                                       [("double v = farthest_corner_sk(x, l + k * D, h + k * D, D);",
                                         "double v = kco_beta_sk(x, l + k * D, h + k * D, D);")]),
    "sr_ub_test_4alpha": ("Sec. 4.2.2", [("if (sqdist(x, X + rp[q] * D, D) > alpha) excl = 1;",
                                          "if (sqdist(x, X + rp[q] * D, D) > 4.0 * alpha) excl = 1;")]),
    "sr_first_node_only": ("Alg. 5", [("for (int m = 0; m < n_nodes && redundant; ++m)",
                                       "for (int m = 0; m < 1 && redundant; ++m)")]),
    "seed_in_wrong_cluster": ("Sec. 4.1.1", [("asg[seeds[k]] = (int8_t)k;",
                                              "asg[seeds[k]] = (int8_t)((k + 1) % K);")]),
    "seeds_at_alpha_not_4alpha": ("Sec. 4.1.1", [("> 4.0 * alpha)) { seeds_found = 0; break; }",
                                                  "> alpha)) { seeds_found = 0; break; }")]),
    "float_lower_end_rounded_to_nearest": ("Sec. 4.1.2 under rounding",
                                           [("if ((double)f > v) f = nextafterf(f, -INFINITY);", "")]),
    "float_upper_end_rounded_to_nearest": ("Sec. 4.1.2 under rounding",
                                           [("if ((double)f < v) f = nextafterf(f, INFINITY);", "")]),
    "radius_rounded_to_nearest": ("Sec. 4.1.2 under rounding",
                                  [("double r = nextafter(sqrt(alpha), INFINITY);", "double r = sqrt(alpha);")]),
    "float_split_may_equal_upper_end": ("Sec. 3.3", [("if ((double)m >= hi) m = (float)lo;",
                                                      "if ((double)m > hi) m = (float)lo;")]),
    "step_b_tightening_wrong_extreme": ("Alg. 4", [
        ("double l2 = round_down_dt(nextafter(bmax2[i] - r, -INFINITY), is_f32);",
         "double l2 = round_down_dt(nextafter(bmin2[i] - r, -INFINITY), is_f32);")]),
    "step_b_tightening_skipped": ("Alg. 4", [("if (nb[k] > 0) {", "if (0) {")]),
    "representatives_without_minima": ("Sec. 4.1.2", [("KCO_ADD_REP(amin_idx[a]);", "")]),
    "candidate_tie_to_largest_index": ("Sec. 3.2", [
        ("if (dm < cdist[k]) { cdist[k] = dm; out->cand[k] = s; }",
         "if (dm <= cdist[k]) { cdist[k] = dm; out->cand[k] = s; }")]),
    "witness_value_first_cluster_only": ("Sec. 3.1, replay", [
        ("double b = kco_beta_sk(x, lo + (m * K + k) * D, hi + (m * K + k) * D, D);",
         "double b = kco_beta_sk(x, lo + (m * K + 0) * D, hi + (m * K + 0) * D, D);")]),
    "objective_points_first_center_only": ("Eq. 1", [("double v = sqdist(X + s * D, mu + k * D, D);",
                                                      "double v = sqdist(X + s * D, mu + 0 * D, D);")]),
    "parallel_merge_later_block_on_ties": ("Eq. 9", [("if (ba[q] >= 0 && (arg < 0 || bv[q] > best))",
                                                      "if (ba[q] >= 0 && (arg < 0 || bv[q] >= best))")]),
    "pair_direction_difference_as_sum": ("Sec. 4.1.2, R11", [("const float v = (q & 1) ? fa - fb : fa + fb;",
                                                             "const float v = (q & 1) ? fa + fb : fa + fb;")]),
    "pair_direction_in_double_for_float_data": ("Sec. 4.1.2, R11", [("    if (is_f32) {\n        const float fa",
                                                                    "    if (0) {\n        const float fa")]),
    "pair_directions_dropped": ("Sec. 4.1.2, R11", [("for (int q = 0; q < ndir; ++q) {\n        KCO_ADD_REP",
                                                     "for (int q = 0; q < 0; ++q) {\n        KCO_ADD_REP")]),
    "all_balls_ball_test_skips_first": ("Sec. 4.1.2, Alg. 4", [
        ("for (int64_t q = joff[k]; q < joff[k + 1] && ok; ++q)",
         "for (int64_t q = joff[k] + 1; q < joff[k + 1] && ok; ++q)")]),
    "all_balls_lemma2_at_alpha": ("Lemma 2", [("if (sqdist(x, X + jl[q] * D, D) > four_alpha) excl = 1;",
                                               "if (sqdist(x, X + jl[q] * D, D) > alpha) excl = 1;")]),
}

# name -> (what, [(original, planted), ...]) in mlp.py
MLP_MUTANTS = {
    "relu_dropped_in_forward": ("layer 1", [("h1 = np.maximum(z1, 0.0)", "h1 = z1")]),
    "w2_transposed_both_ways": ("layer 2", [('z2 = h1 @ p["W2"].T + p["b2"]', 'z2 = h1 @ p["W2"] + p["b2"]'),
                                            ('dh1 = dz2 @ p["W2"]', 'dh1 = dz2 @ p["W2"].T')]),
    "mask_dropped_in_gradient": ("loss", [("dy[:, 1] = M[:, 1] * (y[:, 1] - T[:, 1])",
                                           "dy[:, 1] = (y[:, 1] - T[:, 1])")]),
    "bf16_ties_away": ("bf16", [("(u + 0x7FFF + lsb)", "(u + 0x8000)")]),
    "adam_second_moment_uncorrected": ("Adam", [("vh = v / (1 - b2 ** t)", "vh = v / (1 - b2)")]),
    "adam_eps_inside_sqrt": ("Adam", [("np.sqrt(vh) + eps", "np.sqrt(vh + eps)")]),
}

_PIN_ARGS = ["-x", "-q", "-p", "no:cacheprovider", "-m", "not gpu", "--timeout=120", "--timeout-method=thread"]

# runs the MLP pins with oracle.mlp replaced by the module at argv[1]
_MLP_RUNNER = """
import sys, types
import oracle
path = sys.argv[1]
m = types.ModuleType("oracle.mlp")
m.__file__ = path
exec(compile(open(path).read(), path, "exec"), m.__dict__)
sys.modules["oracle.mlp"] = m
oracle.mlp = m
import pytest
sys.exit(pytest.main(["tests/test_oracle_mlp_pins.py"] + sys.argv[2:]))
"""


def _plant(src, edits):
    for old, new in edits:
        assert src.count(old) == 1, f"mutation site not unique: {old!r}"
        src = src.replace(old, new)
    return src


def _run_c(tmp, name, edits):
    src = os.path.join(tmp, name + ".c")
    so = os.path.join(tmp, name + ".so")
    with open(src, "w") as f:
        f.write(_plant(open(C_SRC).read(), edits))
    subprocess.run(["gcc", *oracle.GCC_FLAGS, "-o", so, src, "-lm"], check=True)
    env = dict(os.environ, KCO_ORACLE_LIB=so)
    return subprocess.run([sys.executable, "-m", "pytest", "tests/test_oracle_pins.py", "tests/test_oracle_replay.py",
                           *_PIN_ARGS],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)


def _run_mlp(tmp, name, edits):
    path = os.path.join(tmp, name + "_mlp.py")
    with open(path, "w") as f:
        f.write(_plant(open(MLP_SRC).read(), edits))
    return subprocess.run([sys.executable, "-c", _MLP_RUNNER, path, *_PIN_ARGS],
                          cwd=ROOT, capture_output=True, text=True, timeout=900)


@pytest.fixture(scope="module")
def outcomes(tmp_path_factory):
    pytest.importorskip("pytest_timeout")
    tmp = str(tmp_path_factory.mktemp("mutants"))
    jobs = {("c", "control"): (_run_c, []), ("mlp", "control"): (_run_mlp, [])}
    jobs.update({("c", n): (_run_c, e) for n, (_, e) in C_MUTANTS.items()})
    jobs.update({("mlp", n): (_run_mlp, e) for n, (_, e) in MLP_MUTANTS.items()})
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        futs = {key: ex.submit(fn, tmp, key[1], edits) for key, (fn, edits) in jobs.items()}
        return {key: f.result() for key, f in futs.items()}


@pytest.mark.parametrize("kind", ["c", "mlp"])
def test_unmutated_oracle_passes_its_pins(outcomes, kind):
    r = outcomes[(kind, "control")]
    assert r.returncode == 0, r.stdout[-3000:]


@pytest.mark.parametrize("key", [("c", n) for n in C_MUTANTS] + [("mlp", n) for n in MLP_MUTANTS],
                         ids=lambda k: f"{k[0]}-{k[1]}")
def test_planted_mistake_fails_a_pin(outcomes, key):
    r = outcomes[key]
    out = r.stdout + r.stderr
    assert r.returncode == 1 and "FAILED" in out and "Timeout" not in out, \
        f"mutant {key[1]} not caught by an assertion:\n{out[-3000:]}"
