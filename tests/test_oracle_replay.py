"""The certificate replay of the oracle (O5) against hand-built solver logs:
it accepts a consistent log and catches each kind of fault -- a prune whose
witness does not prove it but whose node really is prunable (re-bounded over
all samples and accepted), a prune that is not sound, children that do not
partition their parent, a child key below its parent's bound, and an
objective that does not match the centers."""
import numpy as np
import pytest

import oracle


def _setup():
    rng = np.random.default_rng(3)
    X = rng.uniform(0.0, 10.0, size=(300, 2))
    z, c = oracle.bruteforce(X, 2)
    return X, z, c


def _child(cid, parent, lo, hi, thr, X, key=None, wit=None):
    b, arg = oracle.lower_bound(X, lo, hi)
    key = b if key is None else key
    return {"child": cid, "parent": parent, "key": key, "pruned": int(key >= thr),
            "w": int(arg if wit is None else wit), "lo": lo.ravel().tolist(), "hi": hi.ravel().tolist()}


def _pair(X, thr, pid, lo, hi, k, a, cid0):
    """The two children of box (lo, hi) split at the midpoint of (k, a)."""
    m, succ = oracle.split_point(lo[k, a], hi[k, a])
    lo0, hi0, lo1, hi1 = lo.copy(), hi.copy(), lo.copy(), hi.copy()
    hi0[k, a] = m
    lo1[k, a] = succ
    return [_child(cid0, pid, lo0, hi0, thr, X), _child(cid0 + 1, pid, lo1, hi1, thr, X)]


def _log(X, z, tol):
    thr = z - tol * z
    lo = np.array([[0.0, 0.0], [8.5, 8.5]])
    hi = np.array([[10.0, 10.0], [10.0, 10.0]])
    parent_lb = oracle.lower_bound(X, lo, hi)[0]
    recs = [{"id": 7, "parent": 0, "depth": 1, "lb": parent_lb}]
    recs += _pair(X, thr, 7, lo, hi, 0, 0, 10)
    recs += _pair(X, thr, 8, lo, hi, 0, 1, 12)
    return recs, thr


def test_replay_accepts_a_consistent_log():
    X, z, c = _setup()
    recs, thr = _log(X, z, 0.13)          # a threshold low enough that some children are pruned
    r = oracle.replay(X, recs, z, c, tol=0.13)
    assert r["ok"] and r["objective_ok"] and r["partition_ok"] and r["prunes_ok"]
    assert r["pruned"] >= 1 and r["witness_proved"] == r["pruned"] and r["rebound"] == 0


def test_replay_rebounds_a_prune_whose_witness_does_not_prove_it():
    X, z, c = _setup()
    recs, _ = _log(X, z, 0.13)
    pruned = [r for r in recs if r.get("pruned")]
    assert pruned
    lo = np.array(pruned[0]["lo"]).reshape(2, 2)
    inside = np.flatnonzero(np.all((X >= lo[0]) & (X <= np.array(pruned[0]["hi"]).reshape(2, 2)[0]), axis=1))
    pruned[0]["w"] = int(inside[0])          # a sample inside box 0: value 0, proves nothing
    r = oracle.replay(X, recs, z, c, tol=0.13)
    assert r["rebound"] == 1 and r["prunes_ok"] and r["ok"]


def test_replay_catches_an_unsound_prune():
    X, z, c = _setup()
    recs, _ = _log(X, z, 0.13)
    keep = [r for r in recs if "child" in r and not r["pruned"]]
    assert keep
    keep[0]["pruned"] = 1                    # pruned although its bound is below the threshold
    r = oracle.replay(X, recs, z, c, tol=0.13)
    assert not r["prunes_ok"] and not r["ok"]


def test_replay_catches_broken_partitions_and_keys():
    X, z, c = _setup()
    recs, _ = _log(X, z, 0.13)
    kid = next(r for r in recs if r.get("child") == 11)
    lo = list(kid["lo"])
    lo[0] = float(np.nextafter(lo[0], np.inf))   # a gap between the two children
    kid["lo"] = lo
    assert not oracle.replay(X, recs, z, c, tol=0.13)["partition_ok"]
    recs, _ = _log(X, z, 0.13)
    kid = next(r for r in recs if r.get("child") == 10)
    kid["key"] = recs[0]["lb"] - 1.0              # a child's key below its parent's bound
    assert not oracle.replay(X, recs, z, c, tol=0.13)["partition_ok"]
    recs, _ = _log(X, z, 0.13)
    recs = [r for r in recs if r.get("child") != 13]   # a branched node with one child
    assert not oracle.replay(X, recs, z, c, tol=0.13)["partition_ok"]


def test_replay_checks_the_objective():
    X, z, c = _setup()
    recs, _ = _log(X, z, 0.13)
    r = oracle.replay(X, recs, float(np.nextafter(z, np.inf)), c, tol=0.13)
    assert not r["objective_ok"] and not r["ok"]


def test_witness_values_are_the_closed_form_at_the_witness():
    X, z, c = _setup()
    lo = np.array([[[1.0, 2.0], [6.0, 6.0]]])
    hi = np.array([[[3.0, 4.0], [7.0, 9.0]]])
    d0 = np.array([oracle.beta_sk(x, lo[0, 0], hi[0, 0]) for x in X])
    d1 = np.array([oracle.beta_sk(x, lo[0, 1], hi[0, 1]) for x in X])
    near0, near1 = int(np.argmax(d1 - d0)), int(np.argmax(d0 - d1))   # one sample nearer each box
    assert d0[near0] < d1[near0] and d1[near1] < d0[near1]
    for w in (0, near0, near1, 299):
        v = oracle.witness_values(X, lo, hi, np.array([w]))[0]
        assert v == min(oracle.beta_sk(X[w], lo[0, 0], hi[0, 0]), oracle.beta_sk(X[w], lo[0, 1], hi[0, 1]))
        assert v <= oracle.lower_bound(X, lo[0], hi[0])[0]
    assert oracle.witness_values(X, lo, hi, np.array([-1]))[0] == -1.0


def test_replay_reads_float_boxes_in_float():
    """Boxes of float data are logged with 9 significant digits (enough to
    name a float exactly, not a double): the replay must parse them as floats.
    A prune whose bound equals the threshold only at the float bounds is
    accepted."""
    # sample 0 lies right of box 0, whose upper end 7.395677089691162f prints
    # as 7.39567709: read as a double that end moves right and the distance
    # shrinks below the bound
    X = np.array([[20.0, 3.0], [7.395677089691162, 3.0], [-20.0, -20.0]], np.float32)
    lo = np.array([[[7.395677089691162, 3.0], [-20.0, -20.0]]], np.float32)
    hi = lo.copy()
    beta, arg = oracle.lower_bound(X, lo[0], hi[0])
    assert arg == 0
    fmt = lambda a: [float("%.9g" % v) for v in a.ravel()]   # noqa: E731
    recs = [{"id": 1, "lb": 0.0},
            {"child": 2, "parent": 1, "key": beta, "pruned": 1, "w": 0, "lo": fmt(lo), "hi": fmt(hi)},
            {"child": 3, "parent": 1, "key": 0.0, "pruned": 0, "w": 0,
             "lo": fmt(lo), "hi": fmt(np.nextafter(hi, np.float32(np.inf)))}]
    r = oracle.replay(X, recs, beta, np.array([1, 2]), tol=0.0, is_f32=True, rebound_limit=0)
    assert r["pruned"] == 1 and r["witness_proved"] == 1 and r["prunes_ok"]
