"""The batched path (stag_kde_query_batch): instances of uneven n, m, d and a through one
persistent tensor-core launch serving every operand width (a CTA range per width), captured
in a CUDA graph. Every result
must equal a solo query on the same handle within the form's tolerance, and match the
FP64 oracle; replays must be bitwise identical and see new query contents."""

import numpy as np
import pytest

import oracle
from paper_2407_07096_gb300 import datagen as G

pytestmark = pytest.mark.gpu
TOL = 1e-4


def make_instances(count, seed=0, dims=(8, 32, 128)):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        d = dims[i % len(dims)]
        n = int(rng.integers(200, 6000))
        m = int(rng.integers(1, 700))
        a = float(rng.uniform(0.01, 1.0)) / (d / 8)
        mix = G.make_mixture(seed * 1000 + i, 5, d, -4.0, 4.0, 1.0)
        out.append((G.sample(mix, i, n, "data"), G.sample(mix, i, m, "query"), a))
    return out


@pytest.fixture(scope="module")
def lib():
    from paper_2407_07096_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_batch_matches_solo_and_oracle(lib):
    import torch
    from paper_2407_07096_gb300.kde import ExactGaussianKDE, query_batch
    # every operand width (16, 32, 64, 128) in the one launch
    inst = make_instances(13, dims=(8, 32, 128, 64))
    kdes = [ExactGaussianKDE(X, a) for X, _, a in inst]
    # one plain-form instance in the same batch
    X, Q, a = inst[0]
    kdes.append(ExactGaussianKDE(X, a, form="simt_f32"))
    inst.append(inst[0])
    Qs = [torch.from_numpy(Q).cuda() for _, Q, _ in inst]
    outs = query_batch(kdes, Qs)
    torch.cuda.synchronize()
    for k, (X, Q, a), o in zip(kdes, inst, outs):
        got = o.cpu().numpy()
        solo = k.query(Q)
        ref = oracle.kde(X, Q, a)
        assert oracle.rel_err(got, ref).max() <= TOL
        assert oracle.rel_err(got, solo).max() <= TOL
    # replay: bitwise identical
    first = [o.clone() for o in outs]
    outs2 = query_batch(kdes, Qs, outs)
    torch.cuda.synchronize()
    for a1, a2 in zip(first, outs2):
        assert torch.equal(a1, a2)
    # same pointers, new contents: the replayed graph reads the current queries
    X, Q, a = inst[1]
    Qs[1].copy_(torch.from_numpy(Q[::-1].copy()))
    outs3 = query_batch(kdes, Qs, outs)
    torch.cuda.synchronize()
    assert oracle.rel_err(outs3[1].cpu().numpy(), oracle.kde(X, Q[::-1], a)).max() <= TOL
    for k in kdes:
        k.close()


def test_batch_uneven_widths_share_one_launch(lib):
    """The one launch splits its CTAs by each width's share of the work: a width with a
    single tiny instance (one unit) beside a width with a large one still gets its CTA,
    and both match the oracle."""
    import torch
    from paper_2407_07096_gb300.kde import ExactGaussianKDE, query_batch
    mix_big = G.make_mixture(91, 5, 128, -4.0, 4.0, 1.0)
    mix_small = G.make_mixture(92, 5, 8, -4.0, 4.0, 1.0)
    inst = [(G.sample(mix_big, 1, 60000, "data"), G.sample(mix_big, 1, 1500, "query"), 0.02),
            (G.sample(mix_small, 2, 200, "data"), G.sample(mix_small, 2, 1, "query"), 0.5)]
    kdes = [ExactGaussianKDE(X, a) for X, _, a in inst]
    Qs = [torch.from_numpy(Q).cuda() for _, Q, _ in inst]
    outs = query_batch(kdes, Qs)
    torch.cuda.synchronize()
    for (X, Q, a), o in zip(inst, outs):
        idx = np.arange(0, Q.shape[0], max(1, Q.shape[0] // 64))
        got = o.cpu().numpy()[idx]
        assert oracle.rel_err(got, oracle.kde(X, Q[idx], a)).max() <= TOL
    for k in kdes:
        k.close()


def test_batch_argument_checks(lib):
    import torch
    from paper_2407_07096_gb300 import _lib as L
    from paper_2407_07096_gb300.kde import ExactGaussianKDE, query_batch
    X, Q, a = make_instances(1)[0]
    with ExactGaussianKDE(X, a) as k:
        q = torch.from_numpy(Q).cuda()
        with pytest.raises(L.StagKdeError):
            query_batch([k, k], [q, q])
        empty = torch.empty((0, X.shape[1]), dtype=torch.float32, device="cuda")
        out = query_batch([k], [empty])
        assert out[0].numel() == 0
    assert lib.stag_kde_query_batch(None, None, None, None, 0, None) == 0


def test_autotune_keeps_results(lib):
    import torch
    from paper_2407_07096_gb300.kde import ExactGaussianKDE
    X, Q = G.workload_single_d16(0, 20000, 3000)
    with ExactGaussianKDE(X, 0.1) as k:
        before = k.query(Q)
        k.autotune(torch.from_numpy(Q).cuda())
        after = k.query(Q)
    assert oracle.rel_err(after, before).max() <= TOL


@pytest.mark.slow
def test_full_256_instance_workload_every_instance_sampled(lib):
    # the batched workload at its full size (256 instances, n log-U[1e3, 2e5], m
    # log-U[64, 8192], d cycling 8, 32, 128, a U[0.01, 1]) in one graph-replayed call, in
    # the configuration the benchmark times: 16 sampled queries of EVERY instance against
    # the oracle, at the tensor-core form's tolerance for their condition numbers
    import torch
    import bench
    from paper_2407_07096_gb300.kde import ExactGaussianKDE, query_batch
    from tests._common import tol_tc
    inst = bench.build_batched(256)
    kdes = [ExactGaussianKDE(X, a) for X, _, a in inst]
    Qs = [torch.from_numpy(Q).cuda() for _, Q, _ in inst]
    outs = [torch.empty(q.shape[0], dtype=torch.float64, device="cuda") for q in Qs]
    query_batch(kdes, Qs, outs)
    query_batch(kdes, Qs, outs)  # the replay
    torch.cuda.synchronize()
    worst = 0.0
    for i, (X, Q, a) in enumerate(inst):
        idx = np.linspace(0, len(Q) - 1, min(16, len(Q))).astype(int)
        logk, _, kappa = oracle.kde_log(X, Q[idx], a)
        err = oracle.rel_err(outs[i].cpu().numpy()[idx], np.exp(logk))
        assert np.all(err <= tol_tc(kappa, X.shape[1])), (i, X.shape, a, float(err.max()))
        worst = max(worst, float(err.max()))
    assert worst <= 1e-4  # every instance's kappa stays below 400 here
    for k in kdes:
        k.close()


def test_tc_estimate_flags_queries_near_outlying_points_of_a_tile(lib):
    # one instance of the batched workload (index 95: n = 3317, d = 128, a = 0.061) whose
    # k-d tiles mix points of two mixture components: a query's dominant terms then come
    # from points far from their tile's centre, and the error estimate must charge them
    # with the tile's largest radius, not its typical one
    import bench
    from paper_2407_07096_gb300.kde import ExactGaussianKDE
    from tests._common import tol_tc
    X, Q, a = bench.build_batched(96)[95]
    with ExactGaussianKDE(X, a, form="tc") as kde:
        got = kde.query(Q)
    logk, _, kappa = oracle.kde_log(X, Q, a)
    err = oracle.rel_err(got, np.exp(logk))
    assert np.all(err <= tol_tc(kappa, X.shape[1])), float(err.max())
