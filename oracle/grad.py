"""Adjoint gradient of L = Re <eta, f(A) b> with respect to the links and mu.

Test infrastructure (see the package docstring): not for the product path.

With y = sum_s omega_s x_s, x_s = (A + sigma_s)^{-1} b (Eq. 1) and the
adjoint solutions lambda_s = (A^H + sigma_s)^{-1} eta (sigma_s real):
    dL = -Re sum_s omega_s <lambda_s, dA x_s>,
    dA = c (g5 dD g5 D + g5 D g5 dD)          (A = c (g5 D)^2, c held fixed)
so  <lambda, dA x> = c [ <g5 lambda, dD (g5 D x)> + <g5 D^H g5 lambda, dD x> ].
The link gradient G is defined by dL = Re sum_{x,nu} tr(G_nu(x)^H dU_nu(x));
dL/dmu is the derivative at fixed links.  dL/db = sum_s omega_s lambda_s.
"""
from __future__ import annotations

import numpy as np

from inputs import MU_AXIS
from .dirac import EYE4, GAMMA, Operator, _boundary_weights, gamma5
from .msbicgstab import multishift_single


def _weights(T, nu, mu_chem, t_bc):
    """Per-time-slice weight of the forward hop taken at x and of the backward
    hop taken at x + nu (the two hops that involve the link U_nu(x))."""
    if nu != 3:
        one = np.ones(T)
        return one, one
    fwd, bwd = _boundary_weights(T, mu_chem, t_bc)
    return fwd, np.roll(bwd, -1)


def link_force(U, a, b, mass, mu_chem, t_bc=-1):
    """Derivatives of B = <a, D_w(mu) b> (a^H D b).

    Returns (G, dB_dmu): the variation of B under dU is
    sum_{x,nu,i,j} [dU_ij M_ij + conj(dU_ji) K_ij], so that
    Re dB = Re sum tr(G^H dU) with G = conj(M) + K^T, and dB/dmu (complex).
    M_ij  = -1/2 f+ sum_s conj(a_si(x)) ((1 - g_nu) b(x+nu))_sj   (forward hop at x)
    K_ij  = -1/2 f- sum_s conj(a_si(x+nu)) ((1 + g_nu) b(x))_sj   (backward hop at x+nu)
    """
    T = a.shape[0]
    G = np.zeros(U.shape, dtype=np.complex128)
    dmu = 0.0 + 0j
    for nu in range(4):
        ax = MU_AXIS[nu]
        wf, wb = _weights(T, nu, mu_chem, t_bc)
        wf = wf[:, None, None, None, None, None]
        wb = wb[:, None, None, None, None, None]
        Pb = (EYE4 - GAMMA[nu]) @ np.roll(b, -1, axis=ax)
        Qb = (EYE4 + GAMMA[nu]) @ b
        M = -0.5 * np.einsum("...si,...sj->...ij", np.conj(a), wf * Pb)
        K = -0.5 * np.einsum("...si,...sj->...ij", np.conj(np.roll(a, -1, axis=ax)), wb * Qb)
        G[..., nu, :, :] = np.conj(M) + np.swapaxes(K, -1, -2)
        if nu == 3:
            Unu = U[..., 3, :, :]
            # f+ = e^{mu} (d/dmu: +f+), f- = e^{-mu} (d/dmu: -f-)
            dmu = np.sum(M * Unu) - np.sum(K * np.conj(np.swapaxes(Unu, -1, -2)))
    return G, dmu


def grad_f(U, mass, mu_chem, c, b, eta, omega, sigma, ell, tol, t_bc=-1, max_outer=20000):
    """(L, dL/dU, dL/dmu, dL/db) for L = Re <eta, sum_s omega_s (A + sigma_s)^{-1} b>."""
    op = Operator(U, mass, mu_chem, c, t_bc)
    xs = multishift_single(op.A, b, sigma, ell, tol, max_outer)
    lams = multishift_single(op.A_dagger, eta, sigma, ell, tol, max_outer)
    y = sum(w * x for w, x in zip(omega, xs))
    L = float(np.real(np.vdot(eta, y)))
    G = np.zeros(U.shape, dtype=np.complex128)
    dmu = 0.0
    for w, x, lam in zip(omega, xs, lams):
        a1, b1 = gamma5(lam), gamma5(op.D(x))
        a2, b2 = gamma5(op.D_dagger(gamma5(lam))), x
        G1, d1 = link_force(U, a1, b1, mass, mu_chem, t_bc)
        G2, d2 = link_force(U, a2, b2, mass, mu_chem, t_bc)
        G -= (c * w) * (G1 + G2)
        dmu -= c * w * np.real(d1 + d2)
    db = sum(w * lam for w, lam in zip(omega, lams))
    return L, G, float(dmu), db


def f_value(U, mass, mu_chem, c, b, eta, omega, sigma, ell, tol, t_bc=-1, max_outer=20000):
    """L = Re <eta, f(A) b> alone (for finite differences)."""
    op = Operator(U, mass, mu_chem, c, t_bc)
    xs = multishift_single(op.A, b, sigma, ell, tol, max_outer)
    return float(np.real(np.vdot(eta, sum(w * x for w, x in zip(omega, xs)))))
