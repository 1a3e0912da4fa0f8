"""Host logic of the multi-GPU path on CPU with gloo, world size 2: the data-sharded
class ShardedExactKDE itself (each rank evaluates its block of X, one FP64 all-reduce
of the per-rank partials), and query-row sharding with a gather. No GPU here: the
class is given a local evaluator built on the FP64 oracle, so what is under test is
the sharding, the exchange and the normalisation by the global n."""
import os

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2407_07096_gb300 import dist as D


def test_shard_range_partitions():
    for n in (1, 2, 7, 100, 1001):
        for w in (1, 2, 3, 8):
            if n < w:
                continue
            seen = []
            for r in range(w):
                lo, hi = D.shard_range(n, r, w)
                seen.extend(range(lo, hi))
                assert hi - lo in (n // w, n // w + 1)
            assert seen == list(range(n))
    with pytest.raises(ValueError):
        D.shard_range(10, 2, 2)


class OracleBlock:
    """Local evaluator over one rank's block of X (FP64 oracle on the host)."""

    def __init__(self, X, a, **kw):
        self.X, self.a = np.array(X, dtype=np.float64), a
        self.seen = len(X)

    def query(self, Q):
        import oracle
        return oracle.kde(self.X, Q, self.a, threads=1)

    def close(self):
        pass


def _data():
    rng = np.random.default_rng(0)
    return rng.normal(size=(1001, 5)), rng.normal(size=(37, 5)), 0.4


def _worker(rank, world, port, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        X, Q, a = _data()
        kde = D.ShardedExactKDE(X, a, rank, world, local_factory=OracleBlock)
        tot = kde.query(Q)
        nkde = D.ShardedExactKDE(X, a, rank, world, normalise=True, local_factory=OracleBlock)
        normed = nkde.query(Q)
        qlo, qhi = D.shard_range(len(Q), rank, world)
        rows = torch.from_numpy(oracle.kde(X, Q[qlo:qhi], a, threads=1))
        full = D.gather_rows(rows, len(Q))
        results[rank] = (tot.copy(), normed.copy(), full.numpy().copy(), kde.local.seen, kde.block)
        kde.close()
        nkde.close()
    finally:
        dist.destroy_process_group()


def test_sharded_class_and_query_sharding_world2():
    import oracle
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    results = mgr.dict()
    port = 29500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, results)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    X, Q, a = _data()
    want = oracle.kde(X, Q, a)
    blocks = []
    for r in range(2):
        tot, normed, full, seen, block = results[r]
        assert np.allclose(tot, want, rtol=1e-13, atol=0)
        assert np.allclose(normed, want / len(X), rtol=1e-13, atol=0)
        assert np.allclose(full, want, rtol=1e-13, atol=0)
        assert seen == block[1] - block[0] < len(X)  # each rank held only its block
        blocks.append(block)
    assert blocks == [(0, 500), (500, 1001)]


def test_single_process_needs_no_exchange():
    X, Q, a = _data()
    import oracle
    kde = D.ShardedExactKDE(X, a, 0, 1, local_factory=OracleBlock)
    assert np.allclose(kde.query(Q), oracle.kde(X, Q, a), rtol=1e-13, atol=0)
