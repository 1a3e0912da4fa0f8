"""GB300-native exact Gaussian kernel density estimation (the exact KDE of the STAG 2.0
report, Sec. 3), behind the C-ABI library libstagkde.so.

Importing the package loads nothing; ``ExactGaussianKDE`` loads the CUDA library on
first use and raises if it has not been built.
"""


def __getattr__(name):
    if name == "ExactGaussianKDE":
        from .kde import ExactGaussianKDE
        return ExactGaussianKDE
    raise AttributeError(name)
