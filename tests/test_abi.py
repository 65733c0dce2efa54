"""The C-ABI library builds, loads without a GPU, exports every entry point
that include/kc.h declares, and validates arguments before touching CUDA."""
import ctypes as C
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def kcpkg():
    import __graft_entry__
    __graft_entry__._builder().build()
    import paper_2301_00061_gb300 as pkg
    return pkg


def _declared():
    src = open(os.path.join(ROOT, "include", "kc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(kc_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["kc_create", "kc_destroy", "kc_lower_bounds", "kc_upper_bound", "kc_tighten", "kc_solve",
              "kc_fft", "kc_root_box", "kc_sample_reduction"]:
        assert n in names


def test_library_exports_every_declared_symbol(kcpkg):
    lib = C.CDLL(kcpkg.library_path())
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_argument_validation_without_gpu(kcpkg):
    import numpy as np
    X = np.zeros((10, 2), dtype=np.float32)
    for bad in [dict(K=0), dict(K=17), dict(K=11)]:
        with pytest.raises(kcpkg.KCError) as e:
            kcpkg.kc_create(X, bad["K"])
        assert e.value.status == 1
    with pytest.raises(TypeError):
        kcpkg.kc_create(np.zeros((10, 2), dtype=np.int32), 2)


def test_solve_defaults(kcpkg):
    o = kcpkg.kc_solve_defaults()
    assert o.tol == 1e-12 and o.ball_cap == 50 and o.i_sr == 1 and o.use_bt == 1


def test_null_context_is_rejected(kcpkg):
    lib = C.CDLL(kcpkg.library_path())
    lib.kc_root_box.restype = C.c_int
    assert lib.kc_root_box(None, None, None) == 1
    lib.kc_last_error.restype = C.c_char_p
    assert lib.kc_last_error(None) == b"null context"


def test_import_fails_loudly_without_the_library(tmp_path):
    """A copy of the package without libkc.so refuses to import: no CPU
    fallback exists."""
    import shutil
    import subprocess
    import sys
    pkg = os.path.join(ROOT, "paper_2301_00061_gb300")
    dst = tmp_path / "paper_2301_00061_gb300"
    dst.mkdir()
    for f in os.listdir(pkg):
        if f.endswith(".py") or f.endswith(".json"):
            shutil.copy(os.path.join(pkg, f), dst / f)
    r = subprocess.run([sys.executable, "-c", "import paper_2301_00061_gb300"], cwd=tmp_path,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode != 0 and "ImportError" in r.stderr and "not built" in r.stderr, r.stderr[-2000:]


def test_noalloc_rejects_bad_sizes_before_touching_cuda(kcpkg):
    """kc_lower_bounds_noalloc validates sizes before any CUDA call: more nodes
    than its fixed scratch holds, bad K / D / N / ld and NULL arrays return
    KC_EINVAL (1), an empty batch returns KC_OK, all without a GPU.  (The
    pointers are host buffers that the rejected calls never read.)"""
    import numpy as np
    lib = C.CDLL(kcpkg.library_path())
    f = lib.kc_lower_bounds_noalloc
    P, I64, I32 = C.c_void_p, C.c_int64, C.c_int32
    f.restype = C.c_int
    f.argtypes = [P, I64, I64, I32, I32, P, P, I32, P, P, P, P]
    buf = np.zeros(64, np.float64)
    p = buf.ctypes.data
    ok = dict(X=p, N=10, ld=16, D=2, K=3, lo=p, hi=p, B=1, lb=p)

    def call(**kw):
        a = {**ok, **kw}
        return f(a["X"], a["N"], a["ld"], a["D"], a["K"], a["lo"], a["hi"], a["B"], a["lb"], None, None, None)

    for bad in (dict(B=4097), dict(B=-1), dict(K=0), dict(K=17), dict(D=0), dict(D=129), dict(N=-1),
                dict(ld=9), dict(N=2 ** 32, ld=2 ** 32), dict(X=None), dict(lo=None), dict(hi=None), dict(lb=None)):
        assert call(**bad) == 1, bad
    assert call(B=0) == 0
