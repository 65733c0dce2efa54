"""The samples split across ranks (Section 4.3): ``ShardedKCenter`` combines
the ranks' partial results with collectives.  Two gloo ranks on the CPU, each
holding one block of the samples (uneven: 1000 and 1337 rows), with the FP64
oracle evaluating each rank's block in place of the library (no GPU here);
the combined results must equal the oracle's on the whole data set: the root
box; node lower bounds and the sample attaining them, where duplicated rows
put ties across the two blocks (the smallest global index wins, as on one
GPU); the objective of center sets named by global index (the centers' rows
are read on the rank that holds them); and the farthest first traversal."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

N0, N = 1000, 2337
K = 3


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _data():
    rng = np.random.default_rng(4)
    X = np.concatenate([rng.normal(c, 1.0, size=(N // 3 + 1, 3)) for c in ((0, 0, 0), (6, 1, 2), (2, 7, 5))])[:N]
    X[17] = X[1500] = (40.0, 40.0, 40.0)   # the same far point in both blocks: a tie across ranks
    X[2300] = X[999]
    rng2 = np.random.default_rng(5)
    lo = rng2.uniform(-2, 6, size=(12, K, 3))
    hi = lo + rng2.uniform(0.1, 3.0, size=(12, K, 3))
    # boxes inside the data: the duplicated far pair attains the bound
    lo[0] = np.array([0.0, 0.0, 0.0]) - 0.5
    hi[0] = np.array([0.0, 0.0, 0.0]) + 0.5
    centers = rng2.integers(0, N, size=(5, K))
    centers[0] = [5, 1200, 2000]
    return X, lo, hi, centers


class OracleBlock:
    """One rank's block evaluated by the FP64 oracle."""

    def __init__(self, X):
        self.X = X

    def root_box(self):
        import oracle
        return oracle.root_box(self.X)

    def lower_bounds(self, lo, hi):
        import oracle
        beta, arg = oracle.lower_bounds(self.X, lo, hi)
        return beta, beta, arg

    def upper_bound_points(self, pts):
        import oracle
        out = [oracle.objective_points(self.X, p) for p in pts]
        return np.array([v for v, _ in out]), np.array([a for _, a in out], np.int64)

    def rows(self, idx):
        return self.X[idx]


def _worker(rank, ws, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    from paper_2301_00061_gb300.shard import ShardedKCenter
    X, lo, hi, centers = _data()
    a, b = (0, N0) if rank == 0 else (N0, N)
    sk = ShardedKCenter(X[a:b], K, offset=a, n_total=N, local=OracleBlock(X[a:b]))
    out = {"root": sk.root_box(), "lb": sk.lower_bounds(lo, hi), "ub": sk.upper_bound(centers),
           "fft": [sk.fft(s) for s in (0, 1500, N - 1)]}
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


def test_sharded_results_equal_the_whole_data_set():
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=300) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    X, lo, hi, centers = _data()
    rlo, rhi = oracle.root_box(X)
    beta, arg = oracle.lower_bounds(X, lo, hi)
    for rank in (0, 1):
        out = res[rank]
        assert np.array_equal(out["root"][0], rlo) and np.array_equal(out["root"][1], rhi)
        lb, raw, garg = out["lb"]
        assert np.array_equal(raw, beta) and np.array_equal(lb, beta) and np.array_equal(garg, arg)
        for s in range(centers.shape[0]):
            v, w = oracle.objective(X, centers[s])
            assert out["ub"][0][s] == v and out["ub"][1][s] == w
        for (c, obj), start in zip(out["fft"], (0, 1500, N - 1)):
            rc, robj = oracle.fft(X, K, start)
            assert np.array_equal(c, rc) and obj == robj
    assert arg[0] == 17          # the tie across the two blocks went to the smaller index
