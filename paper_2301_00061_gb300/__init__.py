"""GB300 K-center branch and bound: Python binding of ``libkc.so``.

The functions below carry the names of the C ABI in ``include/kc.h`` and only
marshal arguments (tensor/array -> pointer, dtype and shape checks); every
step of the computation runs in the library's CUDA kernels.  Arrays may be
torch tensors (CUDA or CPU) or numpy arrays; CUDA tensors are passed as
device pointers, everything else as host pointers.

Importing this package raises ImportError when the library has not been built
(``python -c "import __graft_entry__ as g; g.build()"``): there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = [
    "KCError", "KC_F32", "KC_F64", "KC_ROW_MAJOR", "KC_COL_MAJOR", "SolveOpts", "Result",
    "kc_create", "kc_destroy", "kc_last_error", "kc_set_stream", "kc_launch_count", "kc_root_box",
    "kc_lower_bounds", "kc_lower_bounds_noalloc", "kc_autotune", "kc_upper_bound", "kc_fft", "kc_fft_multi",
    "kc_lower_bounds_subset", "kc_fp32_probe", "kc_upper_bound_points", "kc_tighten", "kc_sample_reduction",
    "kc_solve_defaults", "kc_solve", "KCenter", "library_path", "kc_mlp_create", "kc_mlp_destroy",
    "kc_mlp_get_params", "kc_mlp_forward", "kc_mlp_grad", "kc_mlp_train", "kc_set_scorer", "Scorer",
]

KC_F32, KC_F64 = 0, 1
KC_ROW_MAJOR, KC_COL_MAJOR = 0, 1
KC_BALLS_ALL = -1   # ball_cap: every sample assigned to a cluster is one of its representatives
_STATUS = {0: "KC_OK", 1: "KC_EINVAL", 2: "KC_ENOMEM", 3: "KC_ECUDA", 4: "KC_ETIMEOUT",
           5: "KC_ELIMIT", 6: "KC_EINTERNAL"}


class KCError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class SolveOpts(C.Structure):
    _fields_ = [
        ("tol", C.c_double), ("time_limit_s", C.c_double), ("node_limit", C.c_int64),
        ("batch", C.c_int32), ("ball_cap", C.c_int32), ("i_sr", C.c_int32), ("use_bt", C.c_int32),
        ("order", C.c_int32), ("lists", C.c_int32), ("verbose", C.c_int32), ("explore", C.c_int32),
        ("arena_mb", C.c_int32),
        ("seed", C.c_uint64),
        ("log_path", C.c_char_p),
        ("rule_margin", C.c_double),
        ("fft_starts", C.c_int32),
        ("rule_width", C.c_int32),
    ]


class Result(C.Structure):
    _fields_ = [
        ("objective", C.c_double), ("lower_bound", C.c_double), ("gap", C.c_double),
        ("centers", C.c_int64 * 16), ("nodes", C.c_int64), ("batches", C.c_int64),
        ("active_final", C.c_int64), ("fft_objective", C.c_double), ("seconds", C.c_double),
        ("seeds_found", C.c_int32), ("status", C.c_int32),
        ("lists_filtered", C.c_int64), ("samples_dropped", C.c_int64),
    ]


def library_path():
    return _build.LIB


def _load():
    if not os.path.exists(_build.LIB):
        raise ImportError(f"libkc.so is not built ({_build.LIB}); run __graft_entry__.build()")
    L = C.CDLL(_build.LIB)
    P, I64, I32, D = C.c_void_p, C.c_int64, C.c_int32, C.c_double
    sig = {
        "kc_create": (I32, [P, I64, I32, I32, I32, I32, P, C.POINTER(P)]),
        "kc_destroy": (None, [P]),
        "kc_last_error": (C.c_char_p, [P]),
        "kc_create_error": (C.c_char_p, []),
        "kc_set_stream": (I32, [P, P]),
        "kc_launch_count": (I64, [P]),
        "kc_root_box": (I32, [P, P, P]),
        "kc_lower_bounds": (I32, [P, P, P, I32, P, P, P]),
        "kc_lower_bounds_noalloc": (I32, [P, I64, I64, I32, I32, P, P, I32, P, P, P, P]),
        "kc_autotune": (I32, [P, P, P, I32, P, P, P]),
        "kc_upper_bound": (I32, [P, P, I32, P, P]),
        "kc_fft": (I32, [P, I64, P, P]),
        "kc_fft_multi": (I32, [P, P, I32, P, P]),
        "kc_upper_bound_points": (I32, [P, P, I32, I32, P, P]),
        "kc_lower_bounds_subset": (I32, [P, P, I64, P, P, I32, P, P, P, P]),
        "kc_fp32_probe": (I32, [I32, P, P, P]),
        "kc_tighten": (I32, [P, P, P, I32, D, P, I32, P, P, P, P, P, P]),
        "kc_sample_reduction": (I32, [P, P, P, I32, P, I32, D, D, P, P]),
        "kc_solve_defaults": (None, [C.POINTER(SolveOpts)]),
        "kc_mlp_create": (I32, [P, P, C.POINTER(P)]),
        "kc_mlp_destroy": (None, [P]),
        "kc_mlp_last_error": (C.c_char_p, [P]),
        "kc_mlp_get_params": (I32, [P, P]),
        "kc_mlp_forward": (I32, [P, P, I32, P]),
        "kc_mlp_grad": (I32, [P, P, P, P, I32, P, P]),
        "kc_mlp_train": (I32, [P, P, P, P, I32, I32, I32, C.c_float, C.c_uint64, P]),
        "kc_set_scorer": (I32, [P, P]),
        "kc_solve": (I32, [P, D, C.POINTER(SolveOpts), C.POINTER(Result)]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


_lib = _load()


# ------------------------------------------------------------- marshalling

def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return C.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return C.c_void_p(x.ctypes.data)
    raise TypeError(f"unsupported array type {type(x)}")


def _dtype_code(x):
    name = str(x.dtype)
    if name.endswith("float32"):
        return KC_F32
    if name.endswith("float64"):
        return KC_F64
    raise TypeError(f"data must be float32 or float64, got {x.dtype}")


def _stream_ptr(stream):
    if stream is not None:
        return C.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    except ImportError:
        pass
    return None


def _check(h, st):
    if st != 0:
        msg = _lib.kc_last_error(h).decode() if h else _lib.kc_create_error().decode()
        raise KCError(st, msg)


# ------------------------------------------------------------- C ABI names

def kc_create(X, K, layout=KC_ROW_MAJOR, stream=None):
    """X: (N, D) row-major (or (D, N) with layout=KC_COL_MAJOR) float32/float64."""
    if X.ndim != 2:
        raise ValueError("X must be 2-D")
    n, d = (X.shape[0], X.shape[1]) if layout == KC_ROW_MAJOR else (X.shape[1], X.shape[0])
    h = C.c_void_p()
    st = _lib.kc_create(_ptr(X), n, d, int(K), _dtype_code(X), int(layout), _stream_ptr(stream), C.byref(h))
    _check(None, st)
    return h


def kc_destroy(h):
    _lib.kc_destroy(h)


def kc_last_error(h):
    return _lib.kc_last_error(h).decode()


def kc_set_stream(h, stream):
    _check(h, _lib.kc_set_stream(h, _stream_ptr(stream)))


def kc_launch_count(h):
    return int(_lib.kc_launch_count(h))


def kc_root_box(h, lo, hi):
    _check(h, _lib.kc_root_box(h, _ptr(lo), _ptr(hi)))


def kc_lower_bounds(h, lo, hi, lb, lb_raw=None, argmax=None):
    B = lo.shape[0]
    _check(h, _lib.kc_lower_bounds(h, _ptr(lo), _ptr(hi), B, _ptr(lb), _ptr(lb_raw), _ptr(argmax)))


def kc_autotune(h, lo, hi):
    """Returns (samples per thread, nodes per launch, ms per batch) chosen."""
    st, ch, ms = C.c_int32(), C.c_int32(), C.c_float()
    _check(h, _lib.kc_autotune(h, _ptr(lo), _ptr(hi), lo.shape[0], C.byref(st), C.byref(ch), C.byref(ms)))
    return st.value, ch.value, ms.value


def kc_lower_bounds_noalloc(X, N, ld, D, K, lo, hi, lb, lb_raw=None, argmax=None, stream=None):
    """X: CUDA float32 tensor holding X[a*ld + s] (at least D*ld values);
    lo, hi: CUDA float32 (B, K, D); lb, lb_raw: CUDA float64 with at least B
    values, argmax: CUDA int64 with at least B values (the last two may be
    None).  Every array must be a CUDA tensor: the entry point only takes
    device memory."""
    def cuda_tensor(t, name, dtype_name, min_numel):
        if not (_is_torch(t) and t.is_cuda):
            raise TypeError(f"kc_lower_bounds_noalloc: {name} must be a CUDA tensor")
        if not str(t.dtype).endswith(dtype_name):
            raise TypeError(f"kc_lower_bounds_noalloc: {name} must be {dtype_name}, got {t.dtype}")
        if t.numel() < min_numel:
            raise ValueError(f"kc_lower_bounds_noalloc: {name} holds {t.numel()} values, needs {min_numel}")

    if lo.ndim != 3 or tuple(hi.shape) != tuple(lo.shape) or lo.shape[1] != int(K) or lo.shape[2] != int(D):
        raise ValueError(f"kc_lower_bounds_noalloc: lo, hi must have shape (B, {int(K)}, {int(D)})")
    B = lo.shape[0]
    cuda_tensor(X, "X", "float32", int(D) * int(ld))
    cuda_tensor(lo, "lo", "float32", 0)
    cuda_tensor(hi, "hi", "float32", 0)
    cuda_tensor(lb, "lb", "float64", B)
    if lb_raw is not None:
        cuda_tensor(lb_raw, "lb_raw", "float64", B)
    if argmax is not None:
        cuda_tensor(argmax, "argmax", "int64", B)
    st = _lib.kc_lower_bounds_noalloc(_ptr(X), int(N), int(ld), int(D), int(K), _ptr(lo), _ptr(hi), B, _ptr(lb),
                                      _ptr(lb_raw), _ptr(argmax), _stream_ptr(stream))
    if st != 0:
        raise KCError(st, "kc_lower_bounds_noalloc failed")


def kc_upper_bound(h, centers, ub, worst=None):
    _check(h, _lib.kc_upper_bound(h, _ptr(centers), centers.shape[0], _ptr(ub), _ptr(worst)))


def kc_upper_bound_points(h, pts, ub, worst=None):
    """pts (S, Kc, D) in the data type -> ub (S,) float64, worst (S,) int64."""
    _check(h, _lib.kc_upper_bound_points(h, _ptr(pts), pts.shape[0], pts.shape[1], _ptr(ub), _ptr(worst)))


def kc_fft(h, start, centers, obj=None):
    _check(h, _lib.kc_fft(h, int(start), _ptr(centers), _ptr(obj)))


def kc_fft_multi(h, starts, centers, obj=None):
    """starts (S,) int64 -> centers (S, K) int64, obj (S,) float64 or None."""
    _check(h, _lib.kc_fft_multi(h, _ptr(starts), starts.shape[0], _ptr(centers), _ptr(obj)))


def kc_lower_bounds_subset(h, ids, lo, hi, lb, lb_raw=None, argmax=None, want_kernel_ms=False):
    """ids (n,) uint32 (or int32 holding indices < 2^31); returns the bound
    launch's device time in ms when want_kernel_ms, else None."""
    if not (str(ids.dtype).endswith("uint32") or str(ids.dtype).endswith("int32")):
        raise TypeError(f"ids must be uint32, got {ids.dtype}")
    ms = C.c_float(-1.0)
    _check(h, _lib.kc_lower_bounds_subset(h, _ptr(ids), int(ids.shape[0]), _ptr(lo), _ptr(hi), lo.shape[0],
                                          _ptr(lb), _ptr(lb_raw), _ptr(argmax),
                                          C.byref(ms) if want_kernel_ms else None))
    return ms.value if want_kernel_ms else None


def kc_fp32_probe(mode, stream=None):
    """FP32 lane operations per second of the current GPU for one
    instruction mix (0 packed FMA, 1 three-input max, 2 the bound kernel's
    clamp-distance term); returns (rate, ms)."""
    r, ms = C.c_double(), C.c_float()
    st = _lib.kc_fp32_probe(int(mode), _stream_ptr(stream), C.byref(r), C.byref(ms))
    if st != 0:
        raise KCError(st, "kc_fp32_probe failed")
    return r.value, ms.value


def kc_tighten(h, lo, hi, alpha, seeds=None, ball_cap=0, lo_out=None, hi_out=None, counts=None,
               cand=None, lb=None, status=None):
    B = lo.shape[0]
    _check(h, _lib.kc_tighten(h, _ptr(lo), _ptr(hi), B, float(alpha), _ptr(seeds), int(ball_cap),
                              _ptr(lo_out), _ptr(hi_out), _ptr(counts), _ptr(cand), _ptr(lb),
                              _ptr(status)))


def kc_sample_reduction(h, lo, hi, beta_glob, alpha, active, reps=None, n_active=None):
    M = lo.shape[0]
    R = 0 if reps is None else reps.shape[-1]
    _check(h, _lib.kc_sample_reduction(h, _ptr(lo), _ptr(hi), M, _ptr(reps), R, float(beta_glob),
                                       float(alpha), _ptr(active), _ptr(n_active)))


def kc_solve_defaults():
    o = SolveOpts()
    _lib.kc_solve_defaults(C.byref(o))
    return o


def kc_solve(h, tol=-1.0, opts=None):
    r = Result()
    st = _lib.kc_solve(h, float(tol), C.byref(opts) if opts is not None else None, C.byref(r))
    if st not in (0, 4, 5):
        _check(h, st)
    return r, st


def _mcheck(m, st):
    if st != 0:
        raise KCError(st, _lib.kc_mlp_last_error(m).decode() if m else "kc_mlp_create failed")


def kc_mlp_create(params, stream=None):
    p = np.ascontiguousarray(params, dtype=np.float32) if not _is_torch(params) else params
    m = C.c_void_p()
    _mcheck(None, _lib.kc_mlp_create(_ptr(p), _stream_ptr(stream), C.byref(m)))
    return m


def kc_mlp_destroy(m):
    _lib.kc_mlp_destroy(m)


def kc_mlp_get_params(m, out):
    _mcheck(m, _lib.kc_mlp_get_params(m, _ptr(out)))


def kc_mlp_forward(m, feats, out):
    _mcheck(m, _lib.kc_mlp_forward(m, _ptr(feats), feats.shape[0], _ptr(out)))


def kc_mlp_grad(m, feats, targets, masks, loss_out, grad_out):
    _mcheck(m, _lib.kc_mlp_grad(m, _ptr(feats), _ptr(targets), _ptr(masks), feats.shape[0], _ptr(loss_out),
                                _ptr(grad_out)))


def kc_mlp_train(m, feats, targets, masks, epochs, batch, lr, seed, loss_out=None):
    _mcheck(m, _lib.kc_mlp_train(m, _ptr(feats), _ptr(targets), _ptr(masks), feats.shape[0], int(epochs),
                                 int(batch), float(lr), int(seed), _ptr(loss_out)))


def kc_set_scorer(h, m):
    _check(h, _lib.kc_set_scorer(h, m))


class Scorer:
    """The learned node scorer (12 -> 64 -> 64 -> 2, bf16 weights)."""

    NPARAM = 5122

    def __init__(self, params, stream=None):
        self.m = kc_mlp_create(np.ascontiguousarray(params, dtype=np.float32), stream)

    def close(self):
        if self.m:
            kc_mlp_destroy(self.m)
            self.m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        out = np.empty(self.NPARAM, np.float32)
        kc_mlp_get_params(self.m, out)
        return out

    def forward(self, feats):
        feats = np.ascontiguousarray(feats, dtype=np.float32)
        out = np.empty((feats.shape[0], 2), np.float32)
        kc_mlp_forward(self.m, feats, out)
        return out

    def grad(self, feats, targets, masks):
        loss = np.zeros(1, np.float32)
        g = np.empty(self.NPARAM, np.float32)
        kc_mlp_grad(self.m, np.ascontiguousarray(feats, np.float32), np.ascontiguousarray(targets, np.float32),
                    np.ascontiguousarray(masks, np.float32), loss, g)
        return float(loss[0]), g

    def train(self, feats, targets, masks, epochs=20, batch=256, lr=1e-3, seed=0):
        loss = np.zeros(1, np.float32)
        kc_mlp_train(self.m, np.ascontiguousarray(feats, np.float32), np.ascontiguousarray(targets, np.float32),
                     np.ascontiguousarray(masks, np.float32), epochs, batch, lr, seed, loss)
        return float(loss[0])


# ------------------------------------------------------------- convenience

class KCenter:
    """A dataset resident on the GPU plus the bound / solve calls on it.

    Outputs are allocated where the inputs live: CUDA tensors in -> CUDA
    tensors out, numpy (or CPU tensors) in -> numpy out.
    """

    def __init__(self, X, K, layout=KC_ROW_MAJOR, stream=None):
        self.K = int(K)
        self.dtype = _dtype_code(X)
        self.N = X.shape[0] if layout == KC_ROW_MAJOR else X.shape[1]
        self.D = X.shape[1] if layout == KC_ROW_MAJOR else X.shape[0]
        self.h = kc_create(X, K, layout, stream)

    def close(self):
        if self.h:
            kc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # output allocation next to a reference input
    def _alloc(self, like, shape, kind):
        if like is not None and _is_torch(like) and like.is_cuda:
            import torch
            dt = {"f64": torch.float64, "i64": torch.int64, "i8": torch.int8, "u8": torch.uint8,
                  "data": torch.float32 if self.dtype == KC_F32 else torch.float64}[kind]
            return torch.empty(shape, dtype=dt, device=like.device)
        dt = {"f64": np.float64, "i64": np.int64, "i8": np.int8, "u8": np.uint8,
              "data": np.float32 if self.dtype == KC_F32 else np.float64}[kind]
        return np.empty(shape, dtype=dt)

    def launch_count(self):
        return kc_launch_count(self.h)

    def root_box(self, like=None):
        lo = self._alloc(like, (self.D,), "data")
        hi = self._alloc(like, (self.D,), "data")
        kc_root_box(self.h, lo, hi)
        return lo, hi

    def lower_bounds(self, lo, hi):
        """Certified lower bounds of B nodes (Section 3.1): boxes lo, hi of
        shape (B, K, D) in the data type -> (lb, raw, argmax), each (B,)."""
        B = lo.shape[0]
        lb = self._alloc(lo, (B,), "f64")
        raw = self._alloc(lo, (B,), "f64")
        arg = self._alloc(lo, (B,), "i64")
        kc_lower_bounds(self.h, lo, hi, lb, raw, arg)
        return lb, raw, arg

    def upper_bound(self, centers):
        """Objective (Eq. 1) of S center sets, centers (S, K) int64 sample
        indices -> (value in double, the sample attaining it), each (S,)."""
        S = centers.shape[0]
        ub = self._alloc(centers, (S,), "f64")
        worst = self._alloc(centers, (S,), "i64")
        kc_upper_bound(self.h, centers, ub, worst)
        return ub, worst

    def upper_bound_points(self, pts):
        """Objective (Eq. 1) at S sets of centers given as points, pts of
        shape (S, Kc, D) in the data type -> (value, worst sample), each (S,)."""
        S = pts.shape[0]
        ub = self._alloc(pts, (S,), "f64")
        worst = self._alloc(pts, (S,), "i64")
        kc_upper_bound_points(self.h, pts, ub, worst)
        return ub, worst

    def fft(self, start, like=None):
        """Farthest first traversal (Algorithm 2) from sample `start` ->
        (K center indices, their objective)."""
        c = self._alloc(like, (self.K,), "i64")
        obj = self._alloc(like, (1,), "f64")
        kc_fft(self.h, start, c, obj)
        return c, obj

    def fft_multi(self, starts):
        """Farthest first traversal from every start of `starts` (S,) int64
        at once -> (centers (S, K), objectives (S,))."""
        S = starts.shape[0]
        c = self._alloc(starts, (S, self.K), "i64")
        obj = self._alloc(starts, (S,), "f64")
        kc_fft_multi(self.h, starts, c, obj)
        return c, obj

    def lower_bounds_subset(self, ids, lo, hi):
        """Lower bounds of B nodes over the samples named by `ids` (uint32)
        -> (lb, raw, argmax), each (B,)."""
        B = lo.shape[0]
        lb = self._alloc(lo, (B,), "f64")
        raw = self._alloc(lo, (B,), "f64")
        arg = self._alloc(lo, (B,), "i64")
        kc_lower_bounds_subset(self.h, ids, lo, hi, lb, raw, arg)
        return lb, raw, arg

    def tighten(self, lo, hi, alpha, seeds=None, ball_cap=0):
        """Cluster assignment and bounds tightening of B nodes given the upper
        bound alpha (Algorithms 3-4): tightened boxes, |S_+^k| counts,
        candidates, the input boxes' certified bound and a status per node
        (0 feasible, 1 infeasible, 2 leaf).  ball_cap: representatives per
        cluster, at most min(ball_cap, 50) (<= 0: 50; the seed, attribute
        extremes, then for float data pair-direction extremes), or
        KC_BALLS_ALL: every sample step A assigns to the cluster."""
        B = lo.shape[0]
        lo_o = self._alloc(lo, tuple(lo.shape), "data")
        hi_o = self._alloc(lo, tuple(lo.shape), "data")
        counts = self._alloc(lo, (B, self.K), "i64")
        cand = self._alloc(lo, (B, self.K), "i64")
        lb = self._alloc(lo, (B,), "f64")
        status = self._alloc(lo, (B,), "i8")
        kc_tighten(self.h, lo, hi, alpha, seeds, ball_cap, lo_o, hi_o, counts, cand, lb, status)
        return {"lo": lo_o, "hi": hi_o, "count": counts, "cand": cand, "lb": lb, "status": status}

    def sample_reduction(self, lo, hi, beta_glob, alpha, active, reps=None):
        """Algorithm 5 against M nodes: clears active[s] (uint8, updated in
        place) for samples redundant in every node; returns (active, count)."""
        n_act = self._alloc(lo, (1,), "i64")
        kc_sample_reduction(self.h, lo, hi, beta_glob, alpha, active, reps, n_act)
        return active, int(n_act[0])

    def set_scorer(self, scorer):
        kc_set_scorer(self.h, scorer.m if scorer is not None else None)
        self._scorer = scorer

    def solve(self, tol=1e-12, **kw):
        """Branch and bound to a certified optimum within relative gap `tol`
        (Algorithm 1).  Keyword options are the fields of kc_solve_opts
        (time_limit_s, node_limit, batch, ball_cap, i_sr, use_bt, order,
        lists, verbose, explore, arena_mb, seed, log_path, rule_margin,
        fft_starts, rule_width).  Returns the objective (double, over all
        samples), certified lower bound, gap, centers, counters and the
        status (0 optimal, 4 time limit, 5 node limit)."""
        o = kc_solve_defaults()
        o.tol = tol
        log = kw.pop("log_path", None)
        for k, v in kw.items():
            if not hasattr(o, k):
                raise TypeError(f"unknown solve option {k}")
            setattr(o, k, v)
        if log is not None:
            o.log_path = log.encode()
        r, st = kc_solve(self.h, tol, o)
        return {
            "objective": r.objective, "lower_bound": r.lower_bound, "gap": r.gap,
            "centers": np.array(r.centers[: self.K]), "nodes": r.nodes, "batches": r.batches,
            "active_final": r.active_final, "fft_objective": r.fft_objective, "seconds": r.seconds,
            "seeds_found": bool(r.seeds_found), "status": st,
            "lists_filtered": r.lists_filtered, "samples_dropped": r.samples_dropped,
        }
