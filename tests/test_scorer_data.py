"""Host-side logic of the scorer's training data (no GPU): subtree work is
summed from the solver's node log, the target goes to the output of the rule
that was taken (both outputs where the rules coincide, max-range only where
rule 1 does not apply), and child records are skipped."""
import importlib.util
import json
import os

import numpy as np

# loaded by path: the package itself needs the built CUDA library, this
# module's data functions do not
_spec = importlib.util.spec_from_file_location(
    "kc_scorer_data", os.path.join(os.path.dirname(__file__), "..", "paper_2301_00061_gb300", "scorer.py"))
S = importlib.util.module_from_spec(_spec)
_spec.loader.exec_module(S)


def _rec(i, parent, rule, rule0, rule1, n):
    return {"id": i, "parent": parent, "depth": 0, "lb": 0.0, "alpha": 1.0, "rule": rule, "rule0": rule0,
            "rule1": rule1, "n": n, "feat": [float(i)] * 12}


def test_subtree_work_targets_and_masks(tmp_path):
    # tree: 1 -> (2, 3), 2 -> (4,); node 5's parent was never branched (absent)
    recs = [_rec(1, -1, 1, 0, 3, 100), _rec(2, 1, 0, 2, 2, 40), _rec(3, 1, 0, 1, -1, 30),
            _rec(4, 2, 0, 0, 5, 10), _rec(5, 99, 1, 0, 1, 7)]
    path = tmp_path / "log.jsonl"
    with open(path, "w") as f:
        for r in recs:
            f.write(json.dumps(r) + "\n")
        f.write(json.dumps({"child": 6, "parent": 1, "key": 0.5, "pruned": 1, "lo": [0], "hi": [1]}) + "\n")
    got = S.read_log(path)
    assert [r["id"] for r in got] == [1, 2, 3, 4, 5]
    X, T, M = S.dataset_from_log(got)
    work = np.array([100 + 40 + 30 + 10, 40 + 10, 30, 10, 7], float)
    cost = np.log2(1.0 + work) / 40.0
    assert np.allclose(T[:, 0], cost) and np.allclose(T[:, 1], cost)
    # node 1: rule 1 taken; node 2: rules coincide; node 3: rule 1 absent;
    # node 4: rule 0 taken; node 5: rule 1 taken
    assert M.tolist() == [[0, 1], [1, 1], [1, 0], [1, 0], [0, 1]]
    assert X.shape == (5, 12) and X[2, 0] == 3.0


def test_empty_log():
    X, T, M = S.dataset_from_log([])
    assert X.shape == (0, 12) and T.shape == (0, 2) and M.shape == (0, 2)
