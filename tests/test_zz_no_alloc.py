"""The allocation-free lower-bound entry point (kc_lower_bounds_noalloc).

Some callers cannot allocate GPU memory when they need node bounds -- their
device memory is held by another allocator, or an allocation's implicit
synchronization would stall a latency-critical loop.  kc_lower_bounds_noalloc
serves them with a fixed scratch array inside the library.  This test calls it
through the C ABI, twice in a row (the second call reuses scratch the first
left behind), and checks it against kc_lower_bounds on the same inputs with the
tolerance of the other lower-bound tests (certified bounds within 1e-6
relative of each other; both never above the FP64 value).  The file sorts
last so a run that stops at the first failure has run everything else.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2301_00061_gb300 as kcm  # noqa: E402

DEV = torch.device("cuda:0")
REL = 1e-6


@pytest.mark.parametrize("n,d,k,pad", [(120_000, 8, 5, 0), (50_003, 3, 3, 0), (40_000, 4, 3, 3)])
def test_noalloc_matches_lower_bounds(n, d, k, pad):
    X = synth.gaussian_mixture(n, d, (1 / k,) * k, (0.5,) * k, (2.0,) * k, 20.0, seed=n + d, dtype=np.float32)
    lo, hi = synth.nested_boxes(X, k, 300, seed=d)        # 300 nodes: two 256-node chunks
    ld = n + pad                                          # pad = 3 makes rows unaligned: scalar-load kernel
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
        a, b = lb.cpu().numpy(), lb_ref.cpu().numpy()
        assert np.all(np.abs(a - b) <= REL * np.maximum(b, 1e-30))
        assert np.all(np.abs(raw.cpu().numpy() - raw_ref.cpu().numpy()) <= REL * np.maximum(raw_ref.cpu().numpy(), 1e-30))
        same = arg.cpu().numpy() == arg_ref.cpu().numpy()
        assert same.mean() > 0.99


def test_noalloc_rejects_too_many_nodes():
    X = torch.zeros((2, 64), dtype=torch.float32, device=DEV)
    lo = torch.zeros((4097, 1, 2), dtype=torch.float32, device=DEV)
    out = torch.empty(4097, dtype=torch.float64, device=DEV)
    with pytest.raises(kcm.KCError) as e:
        kcm.kc_lower_bounds_noalloc(X, 64, 64, 2, 1, lo, lo, out)
    assert e.value.status == 1
