"""Shared helpers for the parity tests: tolerances and small seeded inputs."""
import math

import numpy as np

from paper_2407_07096_gb300 import datagen as G

EPS32 = 2.0 ** -24


def tol_f32(kappa, d, base=1e-5):
    """Per-query tolerance of the plain FP32 form.

    The inputs are exact; each squared distance is summed in FP32 from d exact-to-FP32
    squared differences, so its relative error is about sqrt(d) 2^-24 (random rounding)
    and the term's relative error is that times a d^2 = the condition number kappa of
    the dominant terms. The tolerance is the stated 1e-5, widened to 4 sqrt(d) kappa 2^-24
    only for the ill-conditioned queries where FP32 cannot reach it (kappa sqrt(d) > ~40).
    """
    return np.maximum(base, 4.0 * math.sqrt(d) * np.asarray(kappa) * EPS32)


def mixture_inputs(seed, n, m, d, k=5, spread=3.0, std=1.0, dtype=np.float32):
    mix = G.make_mixture(seed, k, d, -spread, spread, std)
    return G.sample(mix, seed, n, "data", dtype), G.sample(mix, seed, m, "query", dtype)
