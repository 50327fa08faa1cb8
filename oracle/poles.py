"""Partial fraction expansion of f(A) = A^{-1/2} (Eq. 1).

Test infrastructure (see the package docstring): not for the product path.

Neuberger's expansion (the PFE named in the captions of Figs. 1 and 3):
    omega_s = (1/N_s) / cos^2(theta_s),  sigma_s = tan^2(theta_s),
    theta_s = pi (s - 1/2) / (2 N_s),  s = 1..N_s.
"""
from __future__ import annotations

import numpy as np


def neuberger_poles(ns):
    """(omega, sigma) arrays of length ns."""
    s = np.arange(1, ns + 1, dtype=np.float64)
    theta = np.pi * (s - 0.5) / (2.0 * ns)
    omega = (1.0 / ns) / np.cos(theta) ** 2
    sigma = np.tan(theta) ** 2
    return omega, sigma


def pfe_scalar(z, omega, sigma):
    """sum_s omega_s / (z + sigma_s), Eq. (1) on scalars."""
    z = np.asarray(z, dtype=np.complex128)
    return sum(w / (z + s) for w, s in zip(omega, sigma))
