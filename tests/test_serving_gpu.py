"""The serving API: continuous batching over resident datasets. Each request's result
must equal a solo query on the same dataset (within the form's tolerance) and the FP64
oracle, whatever it was coalesced with; cancel, timeout, admission and stop behave as
documented."""
import ctypes
import threading

import numpy as np
import pytest

import oracle
from paper_2407_07096_gb300 import datagen as G

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module")
def env():
    from paper_2407_07096_gb300 import build, _lib
    build.build()
    lib = _lib.load()
    from paper_2407_07096_gb300.kde import ExactGaussianKDE
    data = []
    for i, (n, d, a) in enumerate([(20000, 16, 0.1), (5000, 4, 0.5), (8000, 64, 0.02)]):
        mix = G.make_mixture(100 + i, 5, d, -4.0, 4.0, 1.0)
        X = G.sample(mix, i, n, "data")
        data.append((X, mix, a, ExactGaussianKDE(X, a)))
    yield lib, data
    for *_, k in data:
        k.close()


def start(lib, data, slots=4, max_rows=4096, budget=1 << 30):
    from paper_2407_07096_gb300 import _lib as L
    o = L.SrvOpts()
    lib.stag_srv_opts_init(ctypes.byref(o))
    hs = (ctypes.c_void_p * len(data))(*[k._h.value for *_, k in data])
    o.datasets = hs
    o.n_datasets = len(data)
    o.slots = slots
    o.max_rows = max_rows
    o.mem_budget_bytes = budget
    srv = lib.stag_srv_start(ctypes.byref(o))
    assert srv, L.last_error()
    return ctypes.c_void_p(srv), hs


def submit(lib, srv, ds, Q, out):
    t = ctypes.c_uint64()
    rc = lib.stag_srv_submit(srv, ds, Q.ctypes.data, Q.shape[0], out.ctypes.data, ctypes.byref(t))
    assert rc == 0
    return t.value


@pytest.mark.parametrize("slots,budget", [(4, 1 << 30), (1, 1 << 30), (3, 1)])
def test_results_equal_alone_and_in_the_mix(env, slots, budget):
    lib, data = env
    srv, _keep = start(lib, data, slots=slots, budget=budget)
    rng = np.random.default_rng(slots)
    reqs = []
    lock = threading.Lock()

    def producer(seed):
        r = np.random.default_rng(seed)
        for j in range(20):
            ds = int(r.integers(0, len(data)))
            X, mix, a, _ = data[ds]
            m = int(np.exp(r.uniform(0, np.log(600))))
            Q = G.sample(mix, 1000 * seed + j, m, "query")
            out = np.full(m, -1.0)
            t = submit(lib, srv, ds, Q, out)
            with lock:
                reqs.append((t, ds, Q, out))

    threads = [threading.Thread(target=producer, args=(s,)) for s in range(3)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    for t, ds, Q, out in reqs:
        assert lib.stag_srv_wait(srv, t, -1) == 0
    for t, ds, Q, out in reqs:
        X, mix, a, kde = data[ds]
        solo = kde.query(Q)
        ref = oracle.kde(X, Q, a)
        assert oracle.rel_err(out, solo).max() <= TOL
        assert oracle.rel_err(out, ref).max() <= TOL
    done, rows = ctypes.c_int64(), ctypes.c_int64()
    p50, p99 = ctypes.c_double(), ctypes.c_double()
    assert lib.stag_srv_stats(srv, ctypes.byref(done), ctypes.byref(rows), ctypes.byref(p50), ctypes.byref(p99)) == 0
    assert done.value == len(reqs) and rows.value == sum(q.shape[0] for _, _, q, _ in reqs)
    assert 0 < p50.value <= p99.value
    assert lib.stag_srv_stop(srv) == 0
    del rng


def test_cancel_timeout_and_stop(env):
    from paper_2407_07096_gb300 import _lib as L
    lib, data = env
    srv, _keep = start(lib, data, slots=1)
    X, mix, a, kde = data[2]
    Q = G.sample(mix, 7, 4000, "query")
    outs = [np.empty(4000) for _ in range(6)]
    ts = [submit(lib, srv, 2, Q, o) for o in outs]
    # the last request is still queued behind the others on the single slot
    rc = lib.stag_srv_cancel(srv, ts[-1])
    assert rc in (0, L.EINVAL)
    assert lib.stag_srv_wait(srv, ts[-1], -1) == (L.ECANCELED if rc == 0 else 0)
    rc0 = lib.stag_srv_wait(srv, ts[0], 0)
    assert rc0 in (0, L.ETIMEDOUT)
    if rc0 == L.ETIMEDOUT:
        assert lib.stag_srv_wait(srv, ts[0], -1) == 0
    for t in ts[1:-1]:
        assert lib.stag_srv_wait(srv, t, -1) == 0
    ref = oracle.kde(X, Q[:50], a)
    assert oracle.rel_err(outs[0][:50], ref).max() <= TOL
    # bad arguments
    t = ctypes.c_uint64()
    assert lib.stag_srv_submit(srv, 9, Q.ctypes.data, 10, outs[0].ctypes.data, ctypes.byref(t)) == L.EINVAL
    assert lib.stag_srv_submit(srv, 0, Q.ctypes.data, 0, outs[0].ctypes.data, ctypes.byref(t)) == L.EINVAL
    assert lib.stag_srv_wait(srv, 123456789, 0) == L.EINVAL
    assert lib.stag_srv_stop(srv) == 0
