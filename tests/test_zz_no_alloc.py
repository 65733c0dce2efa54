"""The allocation-free lower-bound entry point (kc_lower_bounds_noalloc).

Some callers cannot allocate GPU memory when they need node bounds -- their
device memory is held by another allocator, or an allocation's implicit
synchronization would stall a latency-critical loop.  kc_lower_bounds_noalloc
serves them with a fixed scratch array inside the library.  These tests call
it through the C ABI, twice in a row (the second call reuses the scratch the
first left behind), and require its outputs to be bitwise equal to
kc_lower_bounds on the same inputs: both evaluate every (sample, box) pair
with the same float operations in the same order, take the same maximum
with the same smallest-index tie-break and deflate it by the same factor, so
nothing may differ.  Sampled nodes are also checked against the FP64 oracle
(certified bound within 1e-6 below the double value of Eqs. 9-11, never
above).  Argument errors (sizes, host arrays) are refused before any launch.
The file sorts last so a run that stops at the first failure has run
everything else.
"""
import ctypes as C

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2301_00061_gb300 as kcm  # noqa: E402

DEV = torch.device("cuda:0")
REL = 1e-6


def _same_bits(a, b):
    a, b = a.cpu().numpy(), b.cpu().numpy()
    return a.shape == b.shape and np.array_equal(a.view(np.uint8), b.view(np.uint8))


# (n, d, k, pad): pad = 0 with n % 4 == 0 runs the vectorized kernel; n % 4 != 0
# or pad = 3 (rows not 16-byte aligned) runs the scalar-load kernel, whose float
# evaluation order is the same
@pytest.mark.parametrize("n,d,k,pad", [(120_000, 8, 5, 0), (50_003, 3, 3, 0), (40_000, 4, 3, 3)])
def test_noalloc_matches_lower_bounds(n, d, k, pad):
    X = synth.gaussian_mixture(n, d, (1 / k,) * k, (0.5,) * k, (2.0,) * k, 20.0, seed=n + d, dtype=np.float32)
    lo, hi = synth.nested_boxes(X, k, 300, seed=d)        # 300 nodes: two 256-node chunks
    ld = n + pad
    Xa = np.zeros((d, ld), np.float32)
    Xa[:, :n] = X.T
    Xd = torch.from_numpy(Xa).to(DEV)
    lod, hid = torch.from_numpy(lo).to(DEV), torch.from_numpy(hi).to(DEV)

    ref = kcm.KCenter(torch.from_numpy(X).to(DEV), k)
    lb_ref, raw_ref, arg_ref = ref.lower_bounds(lod, hid)
    torch.cuda.synchronize()
    ref.close()

    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        lb = torch.full((300,), -1.0, dtype=torch.float64, device=DEV)
        raw = torch.full((300,), -1.0, dtype=torch.float64, device=DEV)
        arg = torch.full((300,), -7, dtype=torch.int64, device=DEV)
        kcm.kc_lower_bounds_noalloc(Xd, n, ld, d, k, lod, hid, lb, raw, arg, stream=stream)
        torch.cuda.synchronize()
        assert _same_bits(lb, lb_ref)
        assert _same_bits(raw, raw_ref)
        assert _same_bits(arg, arg_ref)

    sel = np.arange(0, 300, 23)
    beta, _ = oracle.lower_bounds(X, lo[sel], hi[sel])
    got = lb.cpu().numpy()[sel]
    assert np.all(got <= beta), np.max(got - beta)
    assert np.all(got >= beta * (1 - REL)), np.min(got / np.maximum(beta, 1e-300))


def _raw_entry():
    lib = C.CDLL(kcm.library_path())
    f = lib.kc_lower_bounds_noalloc
    P, I64, I32 = C.c_void_p, C.c_int64, C.c_int32
    f.restype = I32
    f.argtypes = [P, I64, I64, I32, I32, P, P, I32, P, P, P, P]
    return f


def test_noalloc_argument_errors():
    """Sizes out of range and host arrays return KC_EINVAL (1) before any
    launch; B = 0 returns KC_OK and writes nothing."""
    f = _raw_entry()
    X = torch.zeros((2, 64), dtype=torch.float32, device=DEV)
    lo = torch.zeros((3, 1, 2), dtype=torch.float32, device=DEV)
    out = torch.full((3,), -5.0, dtype=torch.float64, device=DEV)
    p = lambda t: C.c_void_p(t.data_ptr())  # noqa: E731
    # too many nodes for the fixed scratch
    big = torch.zeros((4097, 1, 2), dtype=torch.float32, device=DEV)
    with pytest.raises(kcm.KCError) as e:
        kcm.kc_lower_bounds_noalloc(X, 64, 64, 2, 1, big, big, torch.empty(4097, dtype=torch.float64, device=DEV))
    assert e.value.status == 1
    # ld < N, N < 0, K = 0, D = 0
    for N, ld, D, K in ((64, 63, 2, 1), (-1, 64, 2, 1), (64, 64, 2, 0), (64, 64, 0, 1)):
        assert f(p(X), N, ld, D, K, p(lo), p(lo), 3, p(out), None, None, None) == 1
    # a host output array is refused before anything runs
    host_out = np.zeros(3, np.float64)
    assert f(p(X), 64, 64, 2, 1, p(lo), p(lo), 3, C.c_void_p(host_out.ctypes.data), None, None, None) == 1
    host_x = np.zeros((2, 64), np.float32)
    assert f(C.c_void_p(host_x.ctypes.data), 64, 64, 2, 1, p(lo), p(lo), 3, p(out), None, None, None) == 1
    # B = 0: nothing to do, nothing written
    assert f(p(X), 64, 64, 2, 1, p(lo), p(lo), 0, p(out), None, None, None) == 0
    torch.cuda.synchronize()
    assert torch.all(out == -5.0)
    # the binding refuses CPU tensors and wrong dtypes itself
    with pytest.raises(TypeError):
        kcm.kc_lower_bounds_noalloc(X, 64, 64, 2, 1, lo, lo, torch.zeros(3, dtype=torch.float64))
    with pytest.raises(TypeError):
        kcm.kc_lower_bounds_noalloc(X, 64, 64, 2, 1, lo, lo, torch.zeros(3, dtype=torch.float32, device=DEV))
