"""The learned node scorer's CUDA kernels against the FP64 oracle
(oracle/mlp.py) on the same bfloat16-rounded weights, its training, and the
solver with learned ordering (the certified optimum must not change)."""
import numpy as np
import pytest

import oracle
import synth
from oracle import mlp

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2301_00061_gb300 import KCenter, Scorer  # noqa: E402


def _data(n, seed):
    rng = np.random.default_rng(seed)
    X = rng.normal(size=(n, 12)).astype(np.float32)
    T = np.stack([rng.normal(size=n), (rng.uniform(size=n) < 0.4)], 1).astype(np.float32)
    M = (rng.uniform(size=(n, 2)) < 0.8).astype(np.float32)
    return X, T, M


@pytest.mark.parametrize("seed", [0, 1])
def test_forward_matches_oracle(seed):
    theta = mlp.init_params(seed)
    rng = np.random.default_rng(seed)
    theta[mlp.NPARAM - 130:] += rng.normal(size=130).astype(np.float32) * 0.1   # non-zero biases too
    X, _, _ = _data(1000, seed)
    sc = Scorer(theta)
    y = sc.forward(X)
    ref, _ = mlp.forward(theta, X)
    assert np.max(np.abs(y - ref)) <= 1e-4 * max(1.0, np.max(np.abs(ref)))


@pytest.mark.parametrize("n", [1, 31, 32, 33, 777])
def test_gradient_matches_oracle(n):
    theta = mlp.init_params(3)
    X, T, M = _data(n, n)
    sc = Scorer(theta)
    loss, g = sc.grad(X, T, M)
    loss_ref, g_ref = mlp.grad(theta, X, T, M)
    assert abs(loss - loss_ref) <= 1e-5 * max(1.0, abs(loss_ref))
    scale = np.max(np.abs(g_ref))
    assert np.max(np.abs(g - g_ref)) <= 2e-4 * scale + 1e-7, np.max(np.abs(g - g_ref)) / scale


def test_training_fits_a_teacher():
    """Targets from a fixed random teacher network: GPU Adam training must cut
    the loss well below its starting value."""
    teacher = mlp.init_params(11)
    X, _, M = _data(4096, 5)
    y, _ = mlp.forward(teacher, X)
    T = y.astype(np.float32)
    M[:] = 1.0
    student = mlp.init_params(12)
    l0 = mlp.loss(student, X, T, M)
    sc = Scorer(student)
    l1 = sc.train(X, T, M, epochs=40, batch=128, lr=3e-3, seed=1)
    assert l1 < 0.35 * l0, (l0, l1)
    # the trained parameters reproduce the reported loss in the oracle
    assert abs(mlp.loss(sc.params(), X, T, M) - l1) <= 1e-3 * max(1.0, l1)


@pytest.mark.parametrize("steps", [1, 2, 5])
def test_adam_steps_match_oracle(steps):
    """kc_mlp_train with one batch holding every sample (so the batch order
    cannot matter) takes `steps` Adam steps (Kingma & Ba, Algorithm 1: lr
    1e-3, beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected moments).  The
    oracle repeats them: the FP64 gradient on the bf16-rounded weights of
    the float32 master parameters, mlp.adam_step, the parameters stored back
    as float32.  At step 1 every update is +-lr times g / (|g| + eps), so a
    wrong bias correction, a misplaced epsilon or a stale bf16 refresh moves
    a parameter by a large part of lr.  Tolerance: 2 % of lr per step plus
    two float32 ulps where the oracle's gradient is at least 1e-2 of the
    largest one at every step (its sign and the ratios of successive steps
    are then fixed by the FP32 gradient, whose error is far below 1e-4 of the
    largest gradient); elsewhere the Adam step bound, 3 lr per step."""
    theta0 = mlp.init_params(21)
    X, T, M = _data(500, 21)
    sc = Scorer(theta0)
    sc.train(X, T, M, epochs=steps, batch=len(X), lr=1e-3, seed=5)
    got = sc.params().astype(np.float64)

    theta = theta0.astype(np.float32)
    m = np.zeros(mlp.NPARAM)
    v = np.zeros(mlp.NPARAM)
    well = np.ones(mlp.NPARAM, bool)
    for t in range(1, steps + 1):
        _, g = mlp.grad(theta, X, T, M)
        well &= np.abs(g) >= 1e-2 * np.max(np.abs(g))
        new, m, v = mlp.adam_step(theta.astype(np.float64), m, v, g, t, lr=1e-3)
        theta = new.astype(np.float32)
    ref = theta.astype(np.float64)
    moved = np.abs(ref - theta0.astype(np.float64))
    assert np.median(moved[well]) > 0.8e-3 * steps      # the steps did move the parameters
    diff = np.abs(got - ref)
    ulp = np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64)
    tight = diff <= 0.02 * 1e-3 * steps + 2 * ulp
    assert np.all(tight[well]), (np.max(diff[well]), int(np.sum(~tight[well])))
    assert np.all(diff <= 3e-3 * steps), np.max(diff)
    assert well.mean() > 0.3


def test_learned_order_keeps_the_optimum():
    """Any scorer only changes the order of nodes and the branching variable;
    every prune still uses the exact bound.  Here the output layer is zero and
    its biases make rule 1 (seed 0) or max-range (seed 1) the cheaper rule."""
    for seed in (0, 1):
        X = synth.gaussian_mixture(2_500, 2, (0.4, 0.3, 0.3), (1.0,) * 3, (1.0,) * 3, 10.0, seed, dtype=np.float32)
        theta = mlp.init_params(seed)
        theta[-130:] = 0.0
        theta[-1] = -5.0 if seed == 0 else 5.0            # predicted cost of rule 1
        kc = KCenter(torch.from_numpy(X).cuda(), 3)
        sc = Scorer(theta)
        kc.set_scorer(sc)
        g1 = kc.solve(tol=1e-12, order=1)
        g0 = kc.solve(tol=1e-12, order=0)
        r = oracle.solve(X, 3, tol=1e-12)
        assert abs(g1["objective"] - r["objective"]) <= 1e-12 * r["objective"]
        assert abs(g0["objective"] - r["objective"]) <= 1e-12 * r["objective"]


def test_trained_scorer_gains_over_best_bound():
    """The committed scorer (trained on exploring solves of the batched-solve
    family, seeds 100.., and the outlier family, seeds 200..) against plain
    best-bound ordering with max-range branching on held-out instances: eight
    family instances drawn with seed 999, three 3000-sample blob sets whose
    best-bound trees are large, the batched-solve recipe at N = 200,000 and
    three outlier-family instances drawn with seed 998.  Same certified
    optimum on every instance; fewer nodes in total."""
    from paper_2301_00061_gb300 import scorer as S
    w = S.load()
    inst = S.family_instances(8, seed=999)
    for s in (3, 16, 25):
        inst.append((synth.gaussian_mixture(3_000, 2, (1 / 3,) * 3, (1.0,) * 3, (1.0,) * 3, 10.0, s,
                                            dtype=np.float32), 3))
    inst.append((synth.make_workload("batched_solve", n=200_000)[0], 3))
    inst += S.outlier_instances(3, seed=998)
    sc = Scorer(w)
    rows, tot = [], {0: 0, 1: 0}
    for X, k in inst:
        kc = KCenter(torch.from_numpy(X).cuda(), k)
        kc.set_scorer(sc)
        r = {o: kc.solve(tol=1e-12, order=o, time_limit_s=60.0) for o in (0, 1)}
        kc.close()
        assert r[0]["status"] == 0 and r[1]["status"] == 0
        assert r[1]["objective"] == r[0]["objective"]
        rows.append((X.shape, k, r[0]["nodes"], r[1]["nodes"], r[0]["seconds"], r[1]["seconds"]))
        tot[0] += r[0]["nodes"]
        tot[1] += r[1]["nodes"]
    for row in rows:
        print("N=%d D=%d K=%d  best-bound %d nodes %.2f s  learned %d nodes %.2f s" %
              (row[0][0], row[0][1], row[1], row[2], row[4], row[3], row[5]))
    print("total nodes: best-bound %d, learned %d" % (tot[0], tot[1]))
    assert tot[1] < 0.8 * tot[0], tot
