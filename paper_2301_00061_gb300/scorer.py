"""Training data and training for the learned node scorer.

The solver writes one JSON line per branched node when given a ``log_path``
(features, parent link, the branching rules' variables and, with
``log_labels``, a strong-branching label: 1 when the rule "split the nearest box
where the bound-attaining sample lies farthest outside" gives its two children
a larger mean lower bound than max-range, unmasked only where the two differ).  This module turns such logs into a training set
-- priority target log2(1 + number of branched descendants) / 10, rule target
the label -- and trains the scorer on the GPU with the library's kernels.

    python -m paper_2301_00061_gb300.scorer train --out weights.json
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import tempfile

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "scorer_weights.json")


def read_log(path):
    with open(path) as f:
        return [json.loads(line) for line in f if line.strip()]


def dataset_from_log(records):
    """(features [n,12], targets [n,2], masks [n,2]) from one solve's log."""
    if not records:
        return (np.zeros((0, 12), np.float32), np.zeros((0, 2), np.float32), np.zeros((0, 2), np.float32))
    idx = {r["id"]: i for i, r in enumerate(records)}
    size = np.ones(len(records))
    # children are logged after their parents: accumulate subtree sizes backwards
    for i in range(len(records) - 1, -1, -1):
        p = records[i]["parent"]
        if p in idx:
            size[idx[p]] += size[i]
    X = np.array([r["feat"] for r in records], np.float32)
    T = np.stack([np.log2(1.0 + size) / 10.0, np.array([r["label"] for r in records], np.float64)], 1)
    M = np.stack([np.ones(len(records)), np.array([r["label_mask"] for r in records], np.float64)], 1)
    return X, T.astype(np.float32), M.astype(np.float32)


def family_instances(count, seed=100, n_lo=10_000, n_hi=200_000):
    """Seeded training instances of the batched-solve family: Gaussian mixtures
    with N in [n_lo, n_hi], D in {2, 3, 4}, K in {3, 4}."""
    import synth
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        d = int(rng.choice([2, 3, 4]))
        k = int(rng.choice([3, 4]))
        w = rng.dirichlet(np.ones(k) * 2.0)
        X = synth.gaussian_mixture(n, d, tuple(w), (1.0,) * k, (1.0,) * k, 10.0, seed=int(rng.integers(1 << 30)),
                                   dtype=np.float32)
        out.append((X, k))
    return out


def generate(instances, node_limit=20_000, time_limit=60.0, batch=256):
    """Solve each instance with logging and labels; concatenated dataset."""
    import torch
    from . import KCenter
    feats, targs, masks = [], [], []
    for X, k in instances:
        with tempfile.NamedTemporaryFile(suffix=".jsonl", delete=False) as tf:
            path = tf.name
        try:
            kc = KCenter(torch.from_numpy(X).cuda(), k)
            kc.solve(tol=1e-12, log_path=path, log_labels=1, node_limit=node_limit, time_limit_s=time_limit,
                     batch=batch)
            kc.close()
            Xf, T, M = dataset_from_log(read_log(path))
        finally:
            os.unlink(path)
        feats.append(Xf)
        targs.append(T)
        masks.append(M)
    return np.concatenate(feats), np.concatenate(targs), np.concatenate(masks)


def init_params(seed):
    """He-uniform weights, zero biases (seeded numpy draw)."""
    rng = np.random.default_rng(seed)
    parts = []
    for shape in [(64, 12), (64,), (64, 64), (64,), (2, 64), (2,)]:
        if len(shape) == 2:
            lim = np.sqrt(6.0 / shape[1])
            parts.append(rng.uniform(-lim, lim, size=shape).ravel())
        else:
            parts.append(np.zeros(shape))
    return np.concatenate(parts).astype(np.float32)


def train_scorer(X, T, M, epochs=30, batch=256, lr=2e-3, seed=0):
    """Trains a scorer on the GPU (the library's forward/backward/Adam
    kernels); returns (params, final mean loss)."""
    from . import Scorer
    sc = Scorer(init_params(seed))
    loss = sc.train(X, T, M, epochs=epochs, batch=batch, lr=lr, seed=seed)
    p = sc.params()
    sc.close()
    return p, loss


def save(params, path, meta=None):
    with open(path, "w") as f:
        json.dump({"params": [float(v) for v in params], "meta": meta or {}}, f)


def load(path=DEFAULT_WEIGHTS):
    with open(path) as f:
        return np.array(json.load(f)["params"], np.float32)


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("cmd", choices=["train"])
    ap.add_argument("--out", default=DEFAULT_WEIGHTS)
    ap.add_argument("--instances", type=int, default=12)
    ap.add_argument("--epochs", type=int, default=40)
    ap.add_argument("--node-limit", type=int, default=20_000)
    a = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(HERE))
    inst = family_instances(a.instances)
    X, T, M = generate(inst, node_limit=a.node_limit)
    p, loss = train_scorer(X, T, M, epochs=a.epochs)
    save(p, a.out, {"samples": int(len(X)), "instances": a.instances, "epochs": a.epochs, "loss": loss,
                    "node_limit": a.node_limit,
                    "command": "python -m paper_2301_00061_gb300.scorer train " + " ".join(argv or sys.argv[1:]),
                    "label_rate": float(T[M[:, 1] > 0, 1].mean()) if (M[:, 1] > 0).any() else None})
    print(json.dumps({"samples": int(len(X)), "loss": loss, "out": a.out}))


if __name__ == "__main__":
    main()
