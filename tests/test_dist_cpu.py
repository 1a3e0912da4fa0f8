"""Host logic of the multi-GPU path on CPU with gloo, world size 2: data sharding with
an FP64 all-reduce of per-shard partials, and query-row sharding with a gather. The
per-shard partial sums come from the FP64 oracle here (no GPU); the product code under
test is the sharding and the exchange."""
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


def _worker(rank, world, port, results):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import oracle
        rng = np.random.default_rng(0)
        X = rng.normal(size=(1001, 5))
        Q = rng.normal(size=(37, 5))
        a = 0.4
        lo, hi = D.shard_range(len(X), rank, world)
        part = torch.from_numpy(oracle.kde(X[lo:hi], Q, a, threads=1))
        tot = D.allreduce_partials(part)
        qlo, qhi = D.shard_range(len(Q), rank, world)
        rows = torch.from_numpy(oracle.kde(X, Q[qlo:qhi], a, threads=1))
        full = D.gather_rows(rows, len(Q))
        results[rank] = (tot.numpy().copy(), full.numpy().copy())
    finally:
        dist.destroy_process_group()


def test_data_and_query_sharding_world2():
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
    rng = np.random.default_rng(0)
    X = rng.normal(size=(1001, 5))
    Q = rng.normal(size=(37, 5))
    want = oracle.kde(X, Q, 0.4)
    for r in range(2):
        tot, full = results[r]
        assert np.allclose(tot, want, rtol=1e-13, atol=0)
        assert np.allclose(full, want, rtol=1e-13, atol=0)
