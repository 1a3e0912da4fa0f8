"""The data-sharded class on the GPU: two gloo ranks (processes) on the one GPU each
hold half of X in their own library handle, evaluate every query against it, and one
FP64 all-reduce of the partials must give the oracle's densities (1e-4 for the
tensor-core form, the plain form's FP32 tolerance for the plain form). The ranks'
kernels are independent of one another; only the host-side gloo all-reduce joins them.
The sharded result is also compared with an unsharded handle on the same GPU."""
import os

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _data():
    from tests._common import mixture_inputs
    X, Q = mixture_inputs(77, 6001, 700, 16)
    return X, Q, 0.2


def _worker(rank, world, port, results):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from paper_2407_07096_gb300 import dist as D
        X, Q, a = _data()
        out = {}
        for form in ("tc", "simt_f32"):
            kde = D.ShardedExactKDE(X, a, rank, world, form=form)
            host = kde.query(Q)
            dev = kde.query_dev(torch.from_numpy(Q).cuda()).cpu().numpy()
            out[form] = (host.copy(), dev.copy(), kde.local.n)
            kde.close()
        results[rank] = out
    finally:
        dist.destroy_process_group()


def test_sharded_exact_kde_two_ranks_on_one_gpu():
    import torch.multiprocessing as mp
    import oracle
    from paper_2407_07096_gb300 import build
    from paper_2407_07096_gb300.kde import ExactGaussianKDE
    from tests._common import tol_f32
    build.build()
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    results = mgr.dict()
    port = 28500 + (os.getpid() % 1000)
    procs = [ctx.Process(target=_worker, args=(r, 2, port, results)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=300)
        assert p.exitcode == 0
    X, Q, a = _data()
    ref = oracle.kde(X, Q, a)
    _, _, kappa = oracle.kde_log(X, Q, a)
    tol = {"tc": 1e-4, "simt_f32": tol_f32(kappa, X.shape[1])}
    for form in ("tc", "simt_f32"):
        with ExactGaussianKDE(X, a, form=form) as whole:
            unsharded = whole.query(Q)
        for r in range(2):
            host, dev, n_local = results[r][form]
            assert n_local in (3000, 3001)
            assert np.all(oracle.rel_err(host, ref) <= tol[form])
            assert np.array_equal(host, dev)
            assert np.all(oracle.rel_err(host, unsharded) <= 2 * np.asarray(tol[form]))
        assert np.array_equal(results[0][form][0], results[1][form][0])
