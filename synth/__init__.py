"""Seeded synthetic inputs for the K-center branch and bound workloads.

This module only draws random numbers: Gaussian-mixture datasets shaped like the
paper's synthetic sets (Section 6.1: Gaussian clusters, few attributes) and the
random nested center boxes used to exercise the node lower bound.  It holds none
of the method's arithmetic, so both the CPU oracle tests and the CUDA path may
use it.

Draw order for a mixture (fixed so that a seed names one dataset): component
means, component sigmas, component labels (categorical by weight), Gaussian
noise, then (optionally) the uniform outliers and their positions.
"""
from __future__ import annotations

import dataclasses
import numpy as np

__all__ = [
    "Workload",
    "WORKLOADS",
    "gaussian_mixture",
    "make_workload",
    "nested_boxes",
    "random_boxes",
    "subsample_rows",
]


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic workload: dataset shape, mixture recipe and seed."""

    name: str
    n: int
    d: int
    k: int
    dtype: str            # "f32" or "f64": storage (and arithmetic) type of the data
    weights: tuple        # mixture weights (sum to 1)
    sigma_lo: tuple       # per-component sigma (lo == hi means fixed)
    sigma_hi: tuple
    mean_hi: float        # means ~ U[0, mean_hi]^d
    seed: int
    outlier_frac: float = 0.0


# The five workloads, shaped like the paper's (Gaussian clusters; N from 1e3
# to 1e9).  What the paper leaves unstated is chosen here: equal weights
# unless given, sigma 1 unless given, means uniform on [0, mean_hi]^D, and
# a fixed seed per workload.
WORKLOADS = {
    "small": Workload("small", 1_000, 2, 3, "f64", (1 / 3,) * 3, (1.0,) * 3, (1.0,) * 3, 10.0, 0),
    "lb_microbench": Workload("lb_microbench", 10_000_000, 8, 5, "f32", (0.2,) * 5,
                              (0.5,) * 5, (2.0,) * 5, 20.0, 1),
    "batched_solve": Workload("batched_solve", 10_000_000, 4, 3, "f32", (0.6, 0.3, 0.1),
                              (1.0,) * 3, (1.0,) * 3, 10.0, 2),
    "learned_order": Workload("learned_order", 100_000_000, 2, 4, "f32", (0.25,) * 4,
                              (1.0,) * 4, (1.0,) * 4, 10.0, 3, outlier_frac=0.01),
    "large": Workload("large", 1_000_000_000, 3, 3, "f32", (0.5, 0.3, 0.2),
                      (0.5, 1.0, 2.0), (0.5, 1.0, 2.0), 10.0, 7),
}


def gaussian_mixture(n, d, weights, sigma_lo, sigma_hi, mean_hi, seed,
                     outlier_frac=0.0, dtype=np.float32, chunk=1 << 22):
    """Return an (n, d) row-major array drawn from an isotropic Gaussian mixture.

    Means are U[0, mean_hi]^d, each component's sigma is U[sigma_lo, sigma_hi]
    (fixed when equal), labels are categorical by ``weights``.  With
    ``outlier_frac`` > 0 that fraction of rows is replaced by points uniform over
    the inliers' bounding box.  Noise is drawn in chunks so memory stays bounded;
    the values depend only on the arguments.
    """
    rng = np.random.default_rng(seed)
    m = len(weights)
    w = np.asarray(weights, dtype=np.float64)
    w = w / w.sum()
    means = rng.uniform(0.0, mean_hi, size=(m, d))
    lo = np.asarray(sigma_lo, dtype=np.float64)
    hi = np.asarray(sigma_hi, dtype=np.float64)
    sig = rng.uniform(lo, hi) if np.any(hi > lo) else lo.copy()
    labels = rng.choice(m, size=n, p=w)
    out = np.empty((n, d), dtype=dtype)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        lab = labels[s:e]
        z = rng.standard_normal(size=(e - s, d))
        out[s:e] = (means[lab] + sig[lab][:, None] * z).astype(dtype)
    if outlier_frac > 0.0:
        n_out = int(round(outlier_frac * n))
        bmin = out.min(axis=0).astype(np.float64)
        bmax = out.max(axis=0).astype(np.float64)
        pos = rng.choice(n, size=n_out, replace=False)
        out[pos] = rng.uniform(bmin, bmax, size=(n_out, d)).astype(dtype)
    return out


def make_workload(name, n=None, seed=None):
    """Dataset of a named workload; ``n``/``seed`` override its size/seed."""
    w = WORKLOADS[name]
    dt = np.float64 if w.dtype == "f64" else np.float32
    X = gaussian_mixture(n if n is not None else w.n, w.d, w.weights, w.sigma_lo, w.sigma_hi,
                         w.mean_hi, w.seed if seed is None else seed, w.outlier_frac, dt)
    return X, w


def subsample_rows(n, m, seed=0):
    """The first ``m`` entries of a seeded permutation of ``range(n)``."""
    return np.random.default_rng(seed).permutation(n)[:m]


def nested_boxes(X, k, b, seed, hw_lo=1e-3, hw_hi=5.0):
    """``b`` nested node boxes (``lo``, ``hi`` each of shape (b, k, d)).

    For each cluster k a center point is a random sample row; half-widths are
    log-uniform on [hw_lo, hw_hi], sorted in descending order along the node
    axis so that box j+1 lies inside box j.  Bounds are rounded to the data's
    dtype outward-free: lo = c - h, hi = c + h evaluated in that dtype.
    """
    rng = np.random.default_rng(seed)
    n, d = X.shape
    idx = rng.integers(0, n, size=k)
    c = X[idx].astype(X.dtype)                                   # (k, d)
    h = np.exp(rng.uniform(np.log(hw_lo), np.log(hw_hi), size=(b, k, d)))
    h = -np.sort(-h, axis=0)                                     # descending over nodes
    h = h.astype(X.dtype)
    lo = (c[None] - h).astype(X.dtype)
    hi = (c[None] + h).astype(X.dtype)
    # dtype rounding can break strict nesting by one ulp; restore it with a running max/min
    lo = np.maximum.accumulate(lo, axis=0)
    hi = np.minimum.accumulate(hi, axis=0)
    return np.ascontiguousarray(lo), np.ascontiguousarray(hi)


def random_boxes(X, k, b, seed, frac_lo=0.0, frac_hi=0.5):
    """``b`` random node boxes inside the data's bounding box (each (b, k, d)).

    Each side is a random sub-interval of the bounding box whose width is a
    U[frac_lo, frac_hi] fraction of the full range.  Useful for small tests.
    """
    rng = np.random.default_rng(seed)
    n, d = X.shape
    bmin = X.min(axis=0).astype(np.float64)
    bmax = X.max(axis=0).astype(np.float64)
    rngw = bmax - bmin
    w = rng.uniform(frac_lo, frac_hi, size=(b, k, d)) * rngw
    start = bmin + rng.uniform(0.0, 1.0, size=(b, k, d)) * (rngw - w)
    lo = start.astype(X.dtype)
    hi = (start + w).astype(X.dtype)
    hi = np.maximum(hi, lo)
    return np.ascontiguousarray(lo), np.ascontiguousarray(hi)
