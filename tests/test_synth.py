"""The seeded synthetic inputs: the five workloads' recipes, determinism, and
the structural properties the tests and the benchmark rely on (mixture
weights, outliers inside the inliers' bounding box, nested node boxes)."""
import numpy as np
import pytest

import synth


def test_workload_recipes():
    """The five workloads: shape, element type, cluster count and seed."""
    want = {
        "small": (1_000, 2, 3, "f64", 0),
        "lb_microbench": (10_000_000, 8, 5, "f32", 1),
        "batched_solve": (10_000_000, 4, 3, "f32", 2),
        "learned_order": (100_000_000, 2, 4, "f32", 3),
        "large": (1_000_000_000, 3, 3, "f32", 7),
    }
    assert set(synth.WORKLOADS) == set(want)
    for name, (n, d, k, dt, seed) in want.items():
        w = synth.WORKLOADS[name]
        assert (w.n, w.d, w.k, w.dtype, w.seed) == (n, d, k, dt, seed), name
        assert abs(sum(w.weights) - 1.0) < 1e-12 and len(w.weights) == len(w.sigma_lo) == len(w.sigma_hi)
    assert synth.WORKLOADS["learned_order"].outlier_frac == 0.01
    assert synth.WORKLOADS["batched_solve"].weights == (0.6, 0.3, 0.1)


def test_make_workload_dtype_and_overrides():
    X, w = synth.make_workload("small")
    assert X.shape == (1_000, 2) and X.dtype == np.float64 and w.k == 3
    Y, _ = synth.make_workload("batched_solve", n=5_000)
    assert Y.shape == (5_000, 4) and Y.dtype == np.float32
    Z, _ = synth.make_workload("batched_solve", n=5_000, seed=9)
    assert not np.array_equal(Y, Z)


def test_mixture_is_deterministic_and_independent_of_chunking():
    args = (20_011, 3, (0.5, 0.3, 0.2), (0.5, 1.0, 2.0), (0.5, 1.0, 2.0), 10.0, 4)
    a = synth.gaussian_mixture(*args)
    b = synth.gaussian_mixture(*args)
    c = synth.gaussian_mixture(*args, chunk=1_000)
    assert np.array_equal(a, b) and np.array_equal(a, c)


def test_mixture_weights_and_spread():
    """Labels follow the weights: with well-separated means, the share of
    points nearest to each component mean matches its weight."""
    n = 200_000
    X = synth.gaussian_mixture(n, 2, (0.6, 0.3, 0.1), (0.05,) * 3, (0.05,) * 3, 100.0, 5, dtype=np.float64)
    rng = np.random.default_rng(5)
    means = rng.uniform(0.0, 100.0, size=(3, 2))     # the first draw of the generator
    near = np.argmin(((X[:, None, :] - means[None]) ** 2).sum(-1), axis=1)
    share = np.bincount(near, minlength=3) / n
    assert np.allclose(share, (0.6, 0.3, 0.1), atol=0.005), share
    d = np.sqrt(((X - means[near]) ** 2).sum(-1))
    assert d.max() < 1.0                              # sigma 0.05: every point near its mean


def test_outliers_replace_the_stated_fraction_inside_the_bounding_box():
    n = 100_000
    base = synth.gaussian_mixture(n, 2, (0.25,) * 4, (1.0,) * 4, (1.0,) * 4, 10.0, 3)
    X = synth.gaussian_mixture(n, 2, (0.25,) * 4, (1.0,) * 4, (1.0,) * 4, 10.0, 3, outlier_frac=0.01)
    changed = np.any(X != base, axis=1)
    assert changed.sum() == round(0.01 * n)
    assert np.all(X.min(0) >= base.min(0)) and np.all(X.max(0) <= base.max(0))


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_nested_boxes_are_nested(dtype):
    X = synth.gaussian_mixture(10_000, 8, (0.2,) * 5, (0.5,) * 5, (2.0,) * 5, 20.0, 1, dtype=dtype)
    lo, hi = synth.nested_boxes(X, 5, 256, seed=1)
    assert lo.shape == hi.shape == (256, 5, 8) and lo.dtype == hi.dtype == dtype
    assert np.all(lo <= hi)
    assert np.all(lo[1:] >= lo[:-1]) and np.all(hi[1:] <= hi[:-1])
    assert np.any(lo[1:] > lo[:-1])


def test_random_boxes_inside_the_data_range():
    X = synth.gaussian_mixture(5_000, 3, (0.5, 0.5), (1.0,) * 2, (1.0,) * 2, 10.0, 2)
    lo, hi = synth.random_boxes(X, 2, 50, seed=4, frac_lo=0.1, frac_hi=0.4)
    assert lo.shape == (50, 2, 3) and lo.dtype == X.dtype
    assert np.all(lo <= hi) and np.all(lo >= X.min(0)) and np.all(hi <= X.max(0))


def test_subsample_rows():
    a = synth.subsample_rows(1_000, 60, seed=0)
    assert np.array_equal(a, np.random.default_rng(0).permutation(1_000)[:60])
    assert len(set(a.tolist())) == 60
