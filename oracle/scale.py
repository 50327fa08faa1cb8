"""Spectral scale c of A = c (gamma_5 D_w)^2 by power iteration.

Test infrastructure (see the package docstring): not for the product path.

The workloads scale A by the inverse of a power-iteration estimate of its
largest eigenvalue: v_0 normalised, then K times v <- A v / |A v|, and
lambda_est = |A v_K|, c = 1 / lambda_est.
"""
from __future__ import annotations

import numpy as np


def power_lambda(apply_A_unscaled, v0, iters=100):
    v = v0 / np.linalg.norm(v0)
    for _ in range(iters):
        w = apply_A_unscaled(v)
        v = w / np.linalg.norm(w)
    return float(np.linalg.norm(apply_A_unscaled(v)))


def power_scale(apply_A_unscaled, v0, iters=100):
    return 1.0 / power_lambda(apply_A_unscaled, v0, iters)
