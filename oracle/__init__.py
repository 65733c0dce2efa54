"""CPU oracle for the K-center reduced-space branch and bound.

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of
the benchmark use this package; the product library never does.  The
arithmetic lives in ``kc_oracle.c`` (plain C, FP64, serial); this module builds
it with gcc and marshals numpy arrays.  It shares no code with the CUDA path.

Every function takes X as an (N, D) array; float32 data is promoted exactly to
float64 (pass ``is_f32=True`` where the data's own precision matters: the
branching midpoint and the outward rounding of tightened boxes).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kc_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

MAXK, MAXD, MAXREPS = 16, 128, 50
BALLS_ALL = -1   # ball_cap: every sample assigned to a cluster is one of its representatives


GCC_FLAGS = ["-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math", "-fopenmp"]


def build(force=False):
    """Compile kc_oracle.c into liboracle.so next to it (gcc, no FP contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.run(["gcc", *GCC_FLAGS, "-o", tmp, _SRC, "-lm"], check=True)
    os.replace(tmp, _LIB)
    return _LIB


class TightenOut(C.Structure):
    _fields_ = [
        ("status", C.c_int32),
        ("beta", C.c_double),
        ("beta_arg", C.c_int64),
        ("lo", C.c_double * (MAXK * MAXD)),
        ("hi", C.c_double * (MAXK * MAXD)),
        ("count", C.c_int64 * MAXK),
        ("cand", C.c_int64 * MAXK),
        ("n_assigned", C.c_int64 * MAXK),
        ("n_reps", C.c_int32 * MAXK),
        ("reps", C.c_int64 * (MAXK * MAXREPS)),
        ("blo", C.c_double * (MAXK * MAXD)),
        ("bhi", C.c_double * (MAXK * MAXD)),
    ]


class Opts(C.Structure):
    _fields_ = [
        ("tol", C.c_double),
        ("use_bt", C.c_int32),
        ("use_sr", C.c_int32),
        ("i_sr", C.c_int32),
        ("ball_cap", C.c_int32),
        ("is_f32", C.c_int32),
        ("seed", C.c_int64),
        ("node_limit", C.c_int64),
        ("time_limit", C.c_double),
    ]


class Result(C.Structure):
    _fields_ = [
        ("objective", C.c_double),
        ("lower_bound", C.c_double),
        ("centers", C.c_int64 * MAXK),
        ("nodes", C.c_int64),
        ("created", C.c_int64),
        ("seeds_found", C.c_int32),
        ("status", C.c_int32),
        ("active_final", C.c_int64),
        ("fft_objective", C.c_double),
    ]


_P = C.c_void_p
_I64 = C.c_int64
_I32 = C.c_int
_D = C.c_double


def lib():
    global _lib
    with _lock:
        if _lib is None:
            # KCO_ORACLE_LIB names a prebuilt variant of this file's library
            # (the mutation tests plant a mistake in a copy of kc_oracle.c and
            # check that the pins catch it); otherwise build next to the source
            path = os.environ.get("KCO_ORACLE_LIB")
            if not path:
                path = build()
            L = C.CDLL(path)
            sig = {
                "kco_beta_sk": (_D, [_P, _P, _P, _I32]),
                "kco_root_box": (_I32, [_P, _I64, _I32, _P, _P]),
                "kco_lower_bound": (_I32, [_P, _I64, _I32, _I32, _P, _P, _P, _P, _P]),
                "kco_lower_bounds": (_I32, [_P, _I64, _I32, _I32, _P, _P, _I32, _P, _P, _P]),
                "kco_lower_bounds_par": (_I32, [_P, _I64, _I32, _I32, _P, _P, _I32, _P, _P]),
                "kco_witness_values": (_I32, [_P, _I64, _I32, _I32, _P, _P, _I64, _P, _P]),
                "kco_objective_points": (_I32, [_P, _I64, _I32, _I32, _P, _P, _P]),
                "kco_beta_matrix": (_I32, [_P, _I64, _I32, _I32, _P, _P, _P]),
                "kco_alpha_s": (_I32, [_P, _I64, _I32, _I32, _P, _P, _P]),
                "kco_objective": (_I32, [_P, _I64, _I32, _I32, _P, _P, _P, _P]),
                "kco_mid_candidate": (_I64, [_P, _I64, _I32, _P, _P, _P, _P]),
                "kco_fft": (_I32, [_P, _I64, _I32, _I32, _I64, _P, _P]),
                "kco_bruteforce": (_I32, [_P, _I64, _I32, _I32, _P, _P]),
                "kco_tighten": (_I32, [_P, _I64, _I32, _I32, _P, _P, _D, _P, _P, _I32, _I32, _P]),
                "kco_sample_reduction": (_I64, [_P, _I64, _I32, _I32, _I32, _P, _P, _P, _P, _D, _D, _P]),
                "kco_solve": (_I32, [_P, _I64, _I32, _I32, _P, _P]),
                "kco_split_point": (None, [_D, _D, _I32, _P, _P]),
            }
            for name, (res, args) in sig.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data


def _mask(active):
    return None if active is None else np.ascontiguousarray(active, dtype=np.uint8)


def root_box(X):
    X = _f64(X)
    n, d = X.shape
    lo = np.empty(d); hi = np.empty(d)
    lib().kco_root_box(_ptr(X), n, d, _ptr(lo), _ptr(hi))
    return lo, hi


def beta_sk(x, lo, hi):
    x, lo, hi = _f64(x), _f64(lo), _f64(hi)
    return lib().kco_beta_sk(_ptr(x), _ptr(lo), _ptr(hi), x.shape[0])


def lower_bound(X, lo, hi, active=None):
    """beta(M) and its argmax for one node (lo, hi of shape (K, D))."""
    X, lo, hi = _f64(X), _f64(lo), _f64(hi)
    n, d = X.shape
    k = lo.shape[0]
    b = C.c_double(); arg = C.c_int64()
    m = _mask(active)
    lib().kco_lower_bound(_ptr(X), n, d, k, _ptr(lo), _ptr(hi), _ptr(m), C.addressof(b), C.addressof(arg))
    return b.value, arg.value


def lower_bounds(X, lo, hi, active=None):
    """beta(M) and argmax for B nodes (lo, hi of shape (B, K, D))."""
    X, lo, hi = _f64(X), _f64(lo), _f64(hi)
    n, d = X.shape
    B, k, _ = lo.shape
    beta = np.empty(B); arg = np.empty(B, dtype=np.int64)
    m = _mask(active)
    lib().kco_lower_bounds(_ptr(X), n, d, k, _ptr(lo), _ptr(hi), B, _ptr(m), _ptr(beta), _ptr(arg))
    return beta, arg


def lower_bounds_par(X, lo, hi):
    """lower_bounds (no mask) over all host cores (OpenMP); equal to the
    serial result.  Returns (beta, argmax, threads used)."""
    X, lo, hi = _f64(X), _f64(lo), _f64(hi)
    n, d = X.shape
    B, k, _ = lo.shape
    beta = np.empty(B); arg = np.empty(B, dtype=np.int64)
    nt = lib().kco_lower_bounds_par(_ptr(X), n, d, k, _ptr(lo), _ptr(hi), B, _ptr(beta), _ptr(arg))
    if nt < 0:
        raise MemoryError("lower_bounds_par: allocation failed")
    return beta, arg, nt


def beta_matrix(X, lo, hi):
    X, lo, hi = _f64(X), _f64(lo), _f64(hi)
    n, d = X.shape
    k = lo.shape[0]
    out = np.empty((n, k))
    lib().kco_beta_matrix(_ptr(X), n, d, k, _ptr(lo), _ptr(hi), _ptr(out))
    return out


def alpha_s(X, lo, hi):
    X, lo, hi = _f64(X), _f64(lo), _f64(hi)
    n, d = X.shape
    k = lo.shape[0]
    out = np.empty(n)
    lib().kco_alpha_s(_ptr(X), n, d, k, _ptr(lo), _ptr(hi), _ptr(out))
    return out


def objective(X, centers, active=None):
    """Eq. 1 at centers on samples: (value, argmax sample)."""
    X = _f64(X)
    n, d = X.shape
    c = np.ascontiguousarray(centers, dtype=np.int64)
    v = C.c_double(); arg = C.c_int64()
    m = _mask(active)
    lib().kco_objective(_ptr(X), n, d, c.shape[0], _ptr(c), _ptr(m), C.addressof(v), C.addressof(arg))
    return v.value, arg.value


def objective_points(X, mu):
    """Eq. 1 at centres given as points mu (K, D): (value, argmax sample)."""
    X, mu = _f64(X), _f64(mu)
    n, d = X.shape
    v = C.c_double(); arg = C.c_int64()
    lib().kco_objective_points(_ptr(X), n, d, mu.shape[0], _ptr(mu), C.addressof(v), C.addressof(arg))
    return v.value, arg.value


def mid_candidate(X, lo, hi, active=None):
    X, lo, hi = _f64(X), _f64(lo), _f64(hi)
    n, d = X.shape
    dist = C.c_double()
    m = _mask(active)
    idx = lib().kco_mid_candidate(_ptr(X), n, d, _ptr(lo), _ptr(hi), _ptr(m), C.addressof(dist))
    return idx, dist.value


def split_point(lo, hi, is_f32=False):
    """Branching value m of [lo, hi] (lo < hi) and the lower end succ(m) of the
    upper child: children [lo, m] and [succ(m), hi]."""
    m, succ = C.c_double(), C.c_double()
    lib().kco_split_point(float(lo), float(hi), int(bool(is_f32)), C.addressof(m), C.addressof(succ))
    return m.value, succ.value


def fft(X, k, start):
    X = _f64(X)
    n, d = X.shape
    c = np.empty(k, dtype=np.int64)
    obj = C.c_double()
    lib().kco_fft(_ptr(X), n, d, k, int(start), _ptr(c), C.addressof(obj))
    return c, obj.value


def bruteforce(X, k):
    X = _f64(X)
    n, d = X.shape
    c = np.empty(k, dtype=np.int64)
    obj = C.c_double()
    rc = lib().kco_bruteforce(_ptr(X), n, d, k, C.addressof(obj), _ptr(c))
    if rc:
        raise ValueError("bruteforce: bad arguments")
    return obj.value, c


def tighten(X, lo, hi, alpha, seeds=None, active=None, is_f32=False, ball_cap=0):
    """Cluster assignment + bounds tightening of one node; returns a dict.
    Representatives per cluster: at most min(ball_cap, 50) (ball_cap <= 0:
    50), the seed, then the extremes along the attributes, then, for float
    data, along attribute-pair directions; ball_cap = BALLS_ALL: every sample
    assigned to the cluster in step A (the reported "reps" stay the default
    ones)."""
    X, lo, hi = _f64(X), _f64(lo), _f64(hi)
    n, d = X.shape
    k = lo.shape[0]
    out = TightenOut()
    sd = None if seeds is None else np.ascontiguousarray(seeds, dtype=np.int64)
    m = _mask(active)
    rc = lib().kco_tighten(_ptr(X), n, d, k, _ptr(lo), _ptr(hi), float(alpha), _ptr(sd), _ptr(m),
                           int(bool(is_f32)), int(ball_cap), C.addressof(out))
    if rc:
        raise ValueError("tighten: bad arguments")
    kd = k * d
    return {
        "status": out.status,
        "beta": out.beta,
        "beta_arg": out.beta_arg,
        "lo": np.array(out.lo[:kd]).reshape(k, d),
        "hi": np.array(out.hi[:kd]).reshape(k, d),
        "count": np.array(out.count[:k]),
        "cand": np.array(out.cand[:k]),
        "n_assigned": np.array(out.n_assigned[:k]),
        "reps": [list(out.reps[j * MAXREPS: j * MAXREPS + out.n_reps[j]]) for j in range(k)],
        "box_bt_lo": np.array(out.blo[:kd]).reshape(k, d),
        "box_bt_hi": np.array(out.bhi[:kd]).reshape(k, d),
    }


def sample_reduction(X, lo, hi, beta_glob, alpha, active, reps=None):
    """Algorithm 5 over nodes lo, hi (M, K, D); ``reps`` is a list (per node) of
    lists (per cluster) of sample indices, or None.  Returns the new mask."""
    X, lo, hi = _f64(X), _f64(lo), _f64(hi)
    n, d = X.shape
    M, k, _ = lo.shape
    act = np.ascontiguousarray(active, dtype=np.uint8).copy()
    rp = nr = None
    if reps is not None:
        rp = np.zeros((M, k, MAXREPS), dtype=np.int64)
        nr = np.zeros((M, k), dtype=np.int32)
        for i in range(M):
            for j in range(k):
                r = reps[i][j][:MAXREPS]
                rp[i, j, :len(r)] = r
                nr[i, j] = len(r)
    lib().kco_sample_reduction(_ptr(X), n, d, k, M, _ptr(lo), _ptr(hi), _ptr(rp), _ptr(nr),
                               float(beta_glob), float(alpha), _ptr(act))
    return act.astype(bool)


def solve(X, k, tol=1e-12, use_bt=True, use_sr=True, i_sr=1, ball_cap=0, is_f32=None, seed=0,
          node_limit=0, time_limit=0.0):
    """Serial FP64 branch and bound (Algorithm 1); returns a dict."""
    if is_f32 is None:
        is_f32 = np.asarray(X).dtype == np.float32
    X = _f64(X)
    n, d = X.shape
    o = Opts(tol, int(use_bt), int(use_sr), int(i_sr), int(ball_cap), int(bool(is_f32)), int(seed),
             int(node_limit), float(time_limit))
    r = Result()
    rc = lib().kco_solve(_ptr(X), n, d, k, C.addressof(o), C.addressof(r))
    if rc:
        raise ValueError(f"solve: error {rc}")
    return {
        "objective": r.objective,
        "lower_bound": r.lower_bound,
        "centers": np.array(r.centers[:k]),
        "nodes": r.nodes,
        "created": r.created,
        "seeds_found": bool(r.seeds_found),
        "status": r.status,
        "active_final": r.active_final,
        "fft_objective": r.fft_objective,
    }


def witness_values(X, lo, hi, wit):
    """min_k beta_w^k of M nodes (lo, hi of shape (M, K, D)) at their witness
    samples wit (M,); -1 where wit < 0."""
    X, lo, hi = _f64(X), _f64(lo), _f64(hi)
    n, d = X.shape
    M, k, _ = lo.shape
    w = np.ascontiguousarray(wit, dtype=np.int64)
    out = np.empty(M)
    lib().kco_witness_values(_ptr(X), n, d, k, _ptr(lo), _ptr(hi), M, _ptr(w), _ptr(out))
    return out


def replay(X, records, objective, centers, tol, is_f32=None, rebound_limit=64):
    """Certificate replay (O5) of a logged branch and bound solve.

    ``records``: the solver's log as parsed JSON objects (an iterable of dicts,
    or a path to the JSON-lines file): lines with "child" describe a bounded
    child (parent, key, pruned, witness "w", boxes "lo"/"hi" flattened
    [K][D]); lines with "id" a branched node (its bound "lb").  Checks:
      (i)   the objective of ``centers`` over all N samples (Eq. 1, FP64)
            equals ``objective``;
      (ii)  every pruned child holds no solution below objective * (1 - tol):
            its witness sample's closed-form value (Section 3.1) reaches that
            threshold, which proves beta(M) does; where it does not (or there
            is no witness), beta(M) is re-evaluated over ALL samples on the
            host cores (at most ``rebound_limit`` such nodes);
      (iii) the two children of every branched node partition its boxes:
            equal except at one coordinate, split into [lo, m] and
            [succ(m), hi] with succ the next value of the data type
            (Section 3.3), and each child's key is at least its parent's
            bound.
    Returns a dict of counts; ``ok`` is True when every check passed."""
    import json
    if is_f32 is None:
        is_f32 = np.asarray(X).dtype == np.float32
    if isinstance(records, (str, bytes, os.PathLike)):
        with open(records) as f:
            records = [json.loads(line) for line in f]
    kids = [r for r in records if "child" in r]
    nodes = {r["id"]: r for r in records if "id" in r}
    out = {"children": len(kids), "branched": len(nodes)}
    # (i)
    obj, _ = objective_fn(X, centers)
    out["objective_ok"] = obj == objective
    # (ii)
    thr = objective - tol * objective
    pruned = [r for r in kids if r["pruned"]]
    out["pruned"] = len(pruned)
    ok_prune = True
    n_rebound = 0
    dt = np.float32 if is_f32 else np.float64
    if pruned:
        nd = np.asarray(X).shape[1]
        # the log prints boxes with just enough digits to name their values in
        # the data's type: parse them in that type, then promote exactly
        lo = np.array([r["lo"] for r in pruned], dtype=dt).astype(np.float64)
        hi = np.array([r["hi"] for r in pruned], dtype=dt).astype(np.float64)
        k = lo.shape[1] // nd
        lo = lo.reshape(len(pruned), k, nd)
        hi = hi.reshape(len(pruned), k, nd)
        wit = np.array([r.get("w", -1) for r in pruned], dtype=np.int64)
        v = witness_values(X, lo, hi, wit)
        bad = np.flatnonzero(~(v >= thr))
        out["witness_proved"] = int(len(pruned) - len(bad))
        n_rebound = len(bad)
        if n_rebound > rebound_limit:
            ok_prune = False
        elif n_rebound:
            beta, _, _ = lower_bounds_par(X, lo[bad], hi[bad])
            ok_prune = bool(np.all(beta >= thr))
    out["rebound"] = n_rebound
    out["prunes_ok"] = ok_prune
    # (iii)
    by_parent = {}
    for r in kids:
        by_parent.setdefault(r["parent"], []).append(r)
    part_ok = True
    for pid, pair in by_parent.items():
        if len(pair) != 2:
            part_ok = False
            break
        c0, c1 = sorted(pair, key=lambda r: r["child"])
        lo0, hi0 = np.array(c0["lo"], dt), np.array(c0["hi"], dt)
        lo1, hi1 = np.array(c1["lo"], dt), np.array(c1["hi"], dt)
        split = np.flatnonzero((lo0 != lo1) | (hi0 != hi1))
        if len(split) != 1:
            part_ok = False
            break
        i = split[0]
        if not (lo0[i] <= hi0[i] < lo1[i] <= hi1[i] and lo1[i] == np.nextafter(hi0[i], dt(np.inf))):
            part_ok = False
            break
        if not (np.array_equal(np.delete(lo0, i), np.delete(lo1, i)) and
                np.array_equal(np.delete(hi0, i), np.delete(hi1, i))):
            part_ok = False
            break
        if pid in nodes and min(c0["key"], c1["key"]) < nodes[pid]["lb"]:
            part_ok = False
            break
    out["partition_ok"] = part_ok
    out["ok"] = bool(out["objective_ok"] and ok_prune and part_ok)
    return out


objective_fn = objective
