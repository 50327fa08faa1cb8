"""Partial fraction expansion of f(A) = A^{-1/2} (Eq. 1).

Test infrastructure (see the package docstring): not for the product path.

Neuberger's expansion (the PFE named in the captions of Figs. 1 and 3):
    omega_s = (1/N_s) / cos^2(theta_s),  sigma_s = tan^2(theta_s),
    theta_s = pi (s - 1/2) / (2 N_s),  s = 1..N_s.

Zolotarev's expansion (the alternative the caption of Fig. 3 names for small
mu): the best uniform approximation of sign(x) = x (x^2)^{-1/2} on
[-1, -eps] u [eps, 1] by x R(x^2) with R of type (N_s - 1, N_s), written as
R(z) = sum_s omega_s / (z + sigma_s).  With kappa'^2 = 1 - eps^2, K' the
complete elliptic integral of the first kind at kappa', and
    c_l = eps^2 sn^2(l K' / (2 N_s); kappa') / cn^2(l K' / (2 N_s); kappa'),
    l = 1..2 N_s - 1,
the poles are sigma_s = c_{2s-1} and R(z) = D prod_{i<N_s} (z + c_{2i}) /
prod_s (z + c_{2s-1}); the residues follow by partial fractions and D
centres the error, which equioscillates at the 2 N_s + 1 points
x_j = eps / dn(j K' / (2 N_s); kappa'), j = 0..2 N_s (Zolotarev 1877; as used
for the overlap operator by van den Eshof et al., Comput. Phys. Commun. 146
(2002) 203, and Chiu et al., Phys. Rev. D 66 (2002) 114502).
"""
from __future__ import annotations

import numpy as np
from scipy import special


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


def zolotarev_poles(ns, eps):
    """(omega, sigma, delta): Zolotarev's expansion of z^{-1/2} on [eps^2, 1]
    with ns poles; delta = max |x R(x^2) - 1| over x in [eps, 1]."""
    m = 1.0 - eps * eps                      # parameter kappa'^2 of the elliptic functions
    K = special.ellipk(m)
    sn, cn, _, _ = special.ellipj(np.arange(1, 2 * ns) * K / (2 * ns), m)
    c = eps * eps * sn * sn / (cn * cn)      # c_1 .. c_{2 ns - 1}, increasing
    sigma = c[0::2]                          # c_1, c_3, .., c_{2 ns - 1}
    zeros = c[1::2]                          # c_2, .., c_{2 ns - 2}
    # partial fractions: residue at -sigma_s of prod (z + zeros) / prod (z + sigma),
    # each zero divided by its interlacing neighbour pole (factors in (0, 1))
    res = np.empty(ns)
    for s in range(ns):
        others = np.delete(sigma, s)           # the poles t != s, in order: one per zero
        res[s] = np.prod((zeros - sigma[s]) / (others - sigma[s]))
    # R with D = 1 at the first two alternation points; D centres the error there
    _, _, dn, _ = special.ellipj(np.array([0.0, K / (2 * ns)]), m)
    x = eps / dn
    p = [xi * np.sum(res / (xi * xi + sigma)) for xi in x]
    D = 2.0 / (p[0] + p[1])
    return D * res, sigma, abs(D * p[0] - 1.0)
