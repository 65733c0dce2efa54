"""Samples split across ranks (the sample-level parallel scheme of Section 4.3).

Each rank holds one contiguous block of the N samples, rows offset ..
offset + n_local of the full data set, in its own context; every call below
evaluates the rank's block with the library and combines the ranks' partial
results with collectives on a torch.distributed process group (NCCL between
GPUs; any backend the tensors' device allows).  Only the combining happens
here: index bookkeeping and reductions, no arithmetic of the method.

Exchanges (one or two small collectives per call, sizes independent of N):
  root box        all-reduce min of lo, max of hi (Section 2.1);
  lower bounds    all-reduce max of the evaluated bound, then min of the
                  global index among the ranks that attain it (the smallest
                  sample index on ties, as on one GPU), and max of the
                  certified bound (each rank's is certified for its block, the
                  largest for the union);
  objective       the same max / min-index pair (Eq. 1 is a max over samples);
  center points   a center named by its global index is read on the rank
                  that holds it: all-reduce sum of rows that are zero elsewhere;
  FFT             Algorithm 2 as K - 1 objective exchanges.
Within a block the library's own reductions apply (CTAs, warps), so with one
rank every result equals the single-context call.
"""
from __future__ import annotations

import numpy as np

__all__ = ["ShardedKCenter"]


class ShardedKCenter:
    """K-center calls over samples split across the ranks of ``group``.

    ``local`` evaluates this rank's block: an object with ``root_box()``,
    ``lower_bounds(lo, hi) -> (lb, raw, argmax)`` (argmax local to the block,
    -1 when empty), ``upper_bound_points(pts) -> (value, worst)`` and the
    block's rows ``rows(idx)`` as points; by default a ``KCenter`` on
    ``X_local``.  Arrays in and out are numpy (host); the collectives run on
    CPU tensors for a gloo group and on ``device`` tensors otherwise."""

    def __init__(self, X_local, K, offset, n_total, group=None, local=None, device=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.K = int(K)
        self.offset = int(offset)
        self.n_total = int(n_total)
        self.n_local = int(X_local.shape[0])
        self.X_local = X_local
        self.device = device
        if local is None:
            from . import KCenter
            local = _LibraryBlock(KCenter(X_local, K), X_local)
        self.local = local

    # -------------------------------------------------------------- collectives
    def _tensor(self, a):
        import torch
        # a copy: the all-reduce works in place and must not overwrite the caller's array
        t = torch.from_numpy(np.array(a, copy=True))
        return t.to(self.device) if self.device is not None else t

    def _reduce(self, a, op):
        t = self._tensor(a)
        self.dist.all_reduce(t, op=op, group=self.group)
        return t.cpu().numpy()

    def _max_then_min_index(self, value, local_index):
        """Per entry: the largest value over the ranks, and the smallest
        global index among the ranks that attain it (-1 if none has one)."""
        R = self.dist.ReduceOp
        vmax = self._reduce(np.asarray(value, np.float64), R.MAX)
        big = np.iinfo(np.int64).max
        li = np.asarray(local_index, np.int64)
        cand = np.where((np.asarray(value, np.float64) == vmax) & (li >= 0), li + self.offset, big)
        gidx = self._reduce(cand, R.MIN)
        return vmax, np.where(gidx == big, -1, gidx)

    # ------------------------------------------------------------------ calls
    def root_box(self):
        """Per-attribute min and max over all N samples (Section 2.1)."""
        R = self.dist.ReduceOp
        lo, hi = self.local.root_box()
        lo = np.asarray(lo, np.float64) if self.n_local else np.full(np.shape(lo), np.inf)
        hi = np.asarray(hi, np.float64) if self.n_local else np.full(np.shape(hi), -np.inf)
        return self._reduce(lo, R.MIN), self._reduce(hi, R.MAX)

    def lower_bounds(self, lo, hi):
        """Node lower bounds over all N samples (Section 3.1): (certified
        bound, evaluated bound, global index attaining it), each (B,)."""
        R = self.dist.ReduceOp
        lb, raw, arg = self.local.lower_bounds(lo, hi)
        raw_g, arg_g = self._max_then_min_index(raw, arg)
        lb_g = self._reduce(np.asarray(lb, np.float64), R.MAX)
        return lb_g, raw_g, arg_g

    def points_of(self, idx):
        """Coordinates of samples named by global index (array of any shape),
        read on the rank that holds each: shape idx.shape + (D,)."""
        R = self.dist.ReduceOp
        idx = np.asarray(idx, np.int64)
        d = self.X_local.shape[1]
        out = np.zeros(idx.shape + (d,), np.float64)
        mine = (idx >= self.offset) & (idx < self.offset + self.n_local)
        if np.any(mine):
            out[mine] = np.asarray(self.local.rows(idx[mine] - self.offset), np.float64)
        return self._reduce(out, R.SUM)

    def upper_bound_points(self, pts):
        """Objective of Eq. 1 at sets of center points (S, Kc, D): (value,
        global index of the worst sample), each (S,)."""
        val, worst = self.local.upper_bound_points(pts)
        return self._max_then_min_index(val, worst)

    def upper_bound(self, centers):
        """Objective at center sets given by global sample indices (S, K)."""
        pts = self.points_of(centers).astype(self.X_local.dtype)
        return self.upper_bound_points(pts)

    def fft(self, start):
        """Algorithm 2 from the sample with global index ``start``: K indices
        and the objective of the set."""
        chosen = [int(start)]
        for t in range(1, self.K):
            pts = self.points_of(np.array([chosen])).astype(self.X_local.dtype)
            _, worst = self.upper_bound_points(pts)
            chosen.append(int(worst[0]))
        val, _ = self.upper_bound(np.array([chosen]))
        return np.array(chosen, np.int64), float(val[0])


class _LibraryBlock:
    """This rank's block evaluated by the CUDA library (host arrays in and
    out; the library stages them)."""

    def __init__(self, kc, X_local):
        self.kc = kc
        self.X = X_local

    def root_box(self):
        return self.kc.root_box()

    def lower_bounds(self, lo, hi):
        return self.kc.lower_bounds(np.ascontiguousarray(lo), np.ascontiguousarray(hi))

    def upper_bound_points(self, pts):
        return self.kc.upper_bound_points(np.ascontiguousarray(pts))

    def rows(self, idx):
        X = self.X.cpu().numpy() if hasattr(self.X, "cpu") else np.asarray(self.X)
        return X[np.asarray(idx, np.int64)]
