"""Similarity-graph degrees (Sec. 4.1): the density at every data point, with and without
the j = i term, against the FP64 oracle's self-sum."""
import numpy as np
import pytest

import oracle
from tests._common import mixture_inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("form,d,tol", [("tc", 16, 1e-4), ("simt_f32", 16, 1e-5), ("tc", 64, 1e-4), ("auto", 5, 1e-4)])
def test_degrees(form, d, tol):
    import torch
    from paper_2407_07096_gb300 import build
    build.build()
    from paper_2407_07096_gb300.kde import ExactGaussianKDE
    X, _ = mixture_inputs(d, 3001, 1, d)
    a = 0.5 / d
    want_excl = oracle.kde_self(X, a)
    with ExactGaussianKDE(X, a, form=form) as kde:
        full = kde.degrees().cpu().numpy()
        excl = kde.degrees(exclude_self=True).cpu().numpy()
        torch.cuda.synchronize()
    assert oracle.rel_err(full, want_excl + 1.0).max() <= tol
    # the diagonal term is subtracted after the sum: absolute error as for the full sum
    assert np.max(np.abs(excl - want_excl) / (want_excl + 1.0)) <= tol
