"""FP64 CPU oracle for exact Gaussian KDE.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the benchmark's
CPU-baseline leg may use it; the library's product path never imports it, and it
imports nothing from the library. It implements the paper's definition of the
kernel density (Sec. 3) with the Gaussian kernel (Sec. 3) as a plain double loop.
"""
from .kde import (build, kde, kde_weighted, kde_self, kde_log, rel_err,  # noqa: F401
                  avg_rel_err)
