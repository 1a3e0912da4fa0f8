"""Host-side checks of the C-ABI that need no GPU: the library loads, exports every
entry point declared in include/*.h, and rejects bad arguments before touching CUDA."""
import ctypes
import glob
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        for m in re.finditer(r"\b(stag_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_2407_07096_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_the_core_calls():
    names = declared_functions()
    for core in ("stag_kde_create", "stag_kde_query", "stag_kde_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    names = declared_functions()
    assert names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2407_07096_gb300 import _lib
    bound = {s[0] for s in _lib.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_argument_validation_before_any_cuda_call(lib):
    from paper_2407_07096_gb300 import _lib as L
    X = np.ones((4, 3), dtype=np.float32)
    assert not lib.stag_kde_create(None, 4, 3, 1.0)
    assert "NULL" in L.last_error()
    assert not lib.stag_kde_create(X.ctypes.data, 0, 3, 1.0)
    assert not lib.stag_kde_create(X.ctypes.data, 4, 0, 1.0)
    assert not lib.stag_kde_create(X.ctypes.data, 4, 3, -1.0)
    assert "bandwidth" in L.last_error()
    assert not lib.stag_kde_create(X.ctypes.data, 4, 3, float("nan"))
    bad = X.copy()
    bad[2, 1] = np.inf
    assert not lib.stag_kde_create(bad.ctypes.data, 4, 3, 1.0)
    assert "non-finite" in L.last_error()
    big = X.copy()
    big[0, 0] = 1e16
    assert not lib.stag_kde_create(big.ctypes.data, 4, 3, 1.0)
    out = np.empty(4)
    assert lib.stag_kde_query(None, X.ctypes.data, 4, out.ctypes.data) == L.EINVAL
    assert lib.stag_kde_query_dev(None, None, 4, None, None) == L.EINVAL
    assert lib.stag_kde_reserve(None, 4) == L.EINVAL
    lib.stag_kde_destroy(None)  # NULL-safe
    o = L.Opts()
    lib.stag_kde_opts_init(ctypes.byref(o))
    assert (o.form, o.normalise, o.device) == (L.FORM_AUTO, 0, -1)
    assert b"sm_103a" in lib.stag_kde_version()


def test_product_path_does_not_import_the_oracle():
    pkg = os.path.join(ROOT, "paper_2407_07096_gb300")
    for path in glob.glob(os.path.join(pkg, "**", "*.py"), recursive=True) + \
            glob.glob(os.path.join(pkg, "csrc", "*")):
        text = open(path, errors="ignore").read()
        assert not re.search(r"^\s*(import|from)\s+oracle\b", text, flags=re.M), path
        assert "kde_oracle" not in text, path
