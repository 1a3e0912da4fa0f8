"""Failure detection without faulting the GPU.

* Device side: every mbarrier wait of the tensor-core kernel is bounded. A limit of 1 ms
  (stag_kde_set_wait_limit) and a producer held back for 200 ms by the host-side hook
  STAG_KDE_INJECT_PRODUCER_STALL_NS (the consumers wait on barriers nothing arrives at)
  make the waits expire; the kernel must record the error, stop its other warps, wait
  for its own copies and MMAs, free TMEM and return, the host call must report
  STAG_KDE_ETIMEDOUT with the output untouched, and the same handle must answer the next
  query, at the default limit, like the oracle. (A short limit alone does not expire:
  mbarrier.try_wait suspends until the phase completes, and every phase does.)
* Host side: STAG_KDE_INJECT_ALLOC_FAIL=k fails the k-th device allocation from the
  moment it is set. Each allocation of a create fails in turn and must give NULL with
  STAG_KDE_ENOMEM (nothing leaked: a clean create follows); in the server, a request
  whose admission needs an allocation that fails is refused with ENOMEM while the
  server keeps serving the next requests correctly.
"""
import ctypes
import os

import numpy as np
import pytest

import oracle
from tests._common import mixture_inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_2407_07096_gb300 import build, _lib
    build.build()
    _lib.load()
    return _lib


@pytest.fixture
def inject():
    def arm(k):
        if k is None:
            os.environ.pop("STAG_KDE_INJECT_ALLOC_FAIL", None)
        else:
            os.environ["STAG_KDE_INJECT_ALLOC_FAIL"] = str(k)
    yield arm
    arm(None)


@pytest.mark.parametrize("d", [16, 64])
def test_tc_wait_expiry_is_reported_and_the_handle_recovers(L, d, monkeypatch):
    from paper_2407_07096_gb300.kde import ExactGaussianKDE
    X, Q = mixture_inputs(90 + d, 20000, 1500, d)
    a = 0.5 / d
    ref = oracle.kde(X, Q, a)
    with ExactGaussianKDE(X, a, form="tc") as kde:
        kde.query(Q)  # scratch set up, settings cached
        kde.set_wait_limit(1_000_000)
        monkeypatch.setenv("STAG_KDE_INJECT_PRODUCER_STALL_NS", "200000000")
        out = np.full(len(Q), -7.0)
        lib = L.load()
        rc = lib.stag_kde_query(kde._h, Q.ctypes.data, len(Q), out.ctypes.data)
        monkeypatch.delenv("STAG_KDE_INJECT_PRODUCER_STALL_NS")
        assert rc == L.ETIMEDOUT, (rc, L.last_error())
        assert np.all(out == -7.0)  # untouched on failure
        kde.set_wait_limit(0)
        for _ in range(2):
            got = kde.query(Q)
            assert oracle.rel_err(got, ref).max() <= 1e-4


def test_set_wait_limit_rejects_bad_values(L):
    from paper_2407_07096_gb300.kde import ExactGaussianKDE
    X, _ = mixture_inputs(1, 100, 1, 4)
    with ExactGaussianKDE(X, 0.1) as kde:
        for bad in (-1, 61 * 10**9):
            with pytest.raises(L.StagKdeError) as e:
                kde.set_wait_limit(bad)
            assert e.value.code == L.EINVAL


@pytest.mark.parametrize("form", ["tc", "simt_f32"])
def test_each_allocation_of_create_fails_cleanly(L, inject, form):
    from paper_2407_07096_gb300.kde import ExactGaussianKDE
    X, Q = mixture_inputs(3, 3000, 200, 16)
    a = 0.2
    failures = 0
    for k in range(1, 60):
        inject(k)
        try:
            kde = ExactGaussianKDE(X, a, form=form)
        except L.StagKdeError as e:
            assert e.code == L.ENOMEM, (k, e)
            failures += 1
            continue
        finally:
            inject(None)
        kde.close()
        break  # k is past the create's last allocation
    else:
        pytest.fail("create kept failing")
    assert failures >= 3
    with ExactGaussianKDE(X, a, form=form) as kde:
        tol = 1e-4 if form == "tc" else 1e-5
        assert oracle.rel_err(kde.query(Q), oracle.kde(X, Q, a)).max() <= tol


def test_query_scratch_allocation_failure(L, inject):
    from paper_2407_07096_gb300.kde import ExactGaussianKDE
    X, Q = mixture_inputs(4, 3000, 300, 16)
    with ExactGaussianKDE(X, 0.2, form="tc") as kde:
        inject(1)  # the first scratch allocation of the query
        with pytest.raises(L.StagKdeError) as e:
            kde.query(Q)
        assert e.value.code == L.ENOMEM
        inject(None)
        assert oracle.rel_err(kde.query(Q), oracle.kde(X, Q, 0.2)).max() <= 1e-4


def test_server_refuses_a_request_whose_admission_allocation_fails(L, inject):
    from paper_2407_07096_gb300.kde import ExactGaussianKDE
    lib = L.load()
    X, Q = mixture_inputs(5, 4000, 300, 16)
    a = 0.2
    ref = oracle.kde(X, Q, a)
    with ExactGaussianKDE(X, a, form="tc") as kde:
        o = L.SrvOpts()
        lib.stag_srv_opts_init(ctypes.byref(o))
        hs = (ctypes.c_void_p * 1)(kde._h.value)
        o.datasets, o.n_datasets, o.slots, o.max_rows = hs, 1, 1, 1024
        srv = ctypes.c_void_p(lib.stag_srv_start(ctypes.byref(o)))
        assert srv.value, L.last_error()
        try:
            def submit():
                out = np.full(len(Q), -1.0)
                t = ctypes.c_uint64()
                L.check(lib.stag_srv_submit(srv, 0, Q.ctypes.data, len(Q), out.ctypes.data, ctypes.byref(t)))
                return out, t.value
            # the slot's first group sets up its view of the dataset: fail that allocation
            inject(1)
            out, t = submit()
            assert lib.stag_srv_wait(srv, t, 30_000_000) == L.ENOMEM
            assert np.all(out == -1.0)
            inject(None)
            for _ in range(2):
                out, t = submit()
                assert lib.stag_srv_wait(srv, t, 30_000_000) == 0
                assert oracle.rel_err(out, ref).max() <= 1e-4
        finally:
            lib.stag_srv_stop(srv)
