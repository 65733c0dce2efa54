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
