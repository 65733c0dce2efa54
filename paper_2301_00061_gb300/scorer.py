"""Training data and training for the learned node scorer.

The scorer predicts, for a node about to be branched, the cost of branching it
with each rule: output r = log2(1 + the solver's work in the subtree) / 40 when
rule r is applied, the work being the number of list entries the branched nodes
of the subtree scan (the sample count of each node's list, summed) (rule 0: max-range; rule 1: split the box nearest to the
sample attaining the node's bound, on the attribute where that sample lies
farthest outside).  The solver takes the cheaper rule.

Training data come from the solver itself: with ``explore`` set it branches
that percentage of the nodes with a random one of the two rules (where they
differ) and, given a ``log_path``, writes one JSON line per branched node
(features, parent, the rule taken, its list size).  A node's subtree work is
summed from the log and becomes the target of the output of the rule that was taken; where the
two rules coincide it is the target of both.  Stage 1 explores every node under
max-range; stage 2 explores 30 % of the nodes under the stage-1 model, and the
model is retrained on both stages' data.  Training runs on the GPU with the
library's kernels.

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
    """The branched-node records of a solver log (child records are skipped)."""
    with open(path) as f:
        recs = [json.loads(line) for line in f if line.strip()]
    return [r for r in recs if "feat" in r]


def dataset_from_log(records):
    """(features [n,12], targets [n,2], masks [n,2]) from one solve's log."""
    if not records:
        return (np.zeros((0, 12), np.float32), np.zeros((0, 2), np.float32), np.zeros((0, 2), np.float32))
    idx = {r["id"]: i for i, r in enumerate(records)}
    work = np.array([float(r.get("n", 1)) for r in records])
    # children are logged after their parents: accumulate subtree work backwards
    for i in range(len(records) - 1, -1, -1):
        p = records[i]["parent"]
        if p in idx:
            work[idx[p]] += work[i]
    X = np.array([r["feat"] for r in records], np.float32)
    cost = np.log2(1.0 + work) / 40.0
    T = np.stack([cost, cost], 1)
    M = np.zeros((len(records), 2))
    for i, r in enumerate(records):
        if r["rule1"] < 0:
            M[i, 0] = 1.0                      # only max-range applies
        elif r["rule1"] == r["rule0"]:
            M[i, :] = 1.0                      # both rules split the same variable
        else:
            M[i, r["rule"]] = 1.0
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


def outlier_instances(count, seed=200, n_lo=10_000, n_hi=200_000):
    """Seeded training instances shaped like the learned-order workload: four
    equal blobs in 2-D plus 1 % uniform outliers, K = 4."""
    import synth
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi))))
        X = synth.gaussian_mixture(n, 2, (0.25,) * 4, (1.0,) * 4, (1.0,) * 4, 10.0, seed=int(rng.integers(1 << 30)),
                                   outlier_frac=0.01, dtype=np.float32)
        out.append((X, 4))
    return out


def generate(instances, node_limit=20_000, time_limit=60.0, batch=256, seed=1, params=None, explore=100):
    """Solve each instance with exploration and logging; concatenated dataset.
    With ``params``, the scorer they define picks the rule on the nodes that
    are not explored (on-policy data); otherwise max-range does."""
    import torch
    from . import KCenter, Scorer
    sc = Scorer(params) if params is not None else None
    feats, targs, masks = [], [], []
    for i, (X, k) in enumerate(instances):
        with tempfile.NamedTemporaryFile(suffix=".jsonl", delete=False) as tf:
            path = tf.name
        try:
            kc = KCenter(torch.from_numpy(X).cuda(), k)
            if sc is not None:
                kc.set_scorer(sc)
            kc.solve(tol=1e-12, log_path=path, explore=explore, order=1 if sc is not None else 0, seed=seed + i,
                     node_limit=node_limit, time_limit_s=time_limit, batch=batch)
            kc.close()
            Xf, T, M = dataset_from_log(read_log(path))
        finally:
            os.unlink(path)
        feats.append(Xf)
        targs.append(T)
        masks.append(M)
    if sc is not None:
        sc.close()
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
    ap.add_argument("--instances", type=int, default=12, help="batched-solve family instances")
    ap.add_argument("--outlier-instances", type=int, default=6, help="outlier family instances")
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--node-limit", type=int, default=8_000)
    ap.add_argument("--stages", type=int, default=2,
                    help="1: random-rule data only; 2: then on-policy data from the first model, retrain on both")
    ap.add_argument("--explore", type=int, default=30, help="percent of random rules in on-policy stages")
    ap.add_argument("--n-lo", type=int, default=10_000, help="smallest training instance")
    ap.add_argument("--n-hi", type=int, default=200_000, help="largest training instance")
    a = ap.parse_args(argv)
    sys.path.insert(0, os.path.dirname(HERE))
    inst = (family_instances(a.instances, n_lo=a.n_lo, n_hi=a.n_hi) +
            outlier_instances(a.outlier_instances, n_lo=a.n_lo, n_hi=a.n_hi))
    X, T, M = generate(inst, node_limit=a.node_limit)
    p, loss = train_scorer(X, T, M, epochs=a.epochs)
    for r in range(1, a.stages):
        X2, T2, M2 = generate(inst, node_limit=a.node_limit, seed=1000 * r + 1, params=p, explore=a.explore)
        X, T, M = np.concatenate([X, X2]), np.concatenate([T, T2]), np.concatenate([M, M2])
        p, loss = train_scorer(X, T, M, epochs=a.epochs)
    save(p, a.out, {"samples": int(len(X)), "instances": a.instances, "outlier_instances": a.outlier_instances,
                    "epochs": a.epochs, "loss": loss, "node_limit": a.node_limit, "stages": a.stages,
                    "explore": a.explore, "n_lo": a.n_lo, "n_hi": a.n_hi,
                    "command": "python -m paper_2301_00061_gb300.scorer " + " ".join(argv or sys.argv[1:])})
    print(json.dumps({"samples": int(len(X)), "loss": loss, "out": a.out}))


if __name__ == "__main__":
    main()
