"""Wilson-Dirac operator at nonzero chemical potential, in plain numpy FP64.

Test infrastructure (see the package docstring): not for the product path.

Sec. 1 names D_w(mu) without defining it.  This module takes the standard
mass form with the chemical potential on the time links:

    (D psi)(x) = (4 + m) psi(x)
                 - 1/2 sum_nu [ f+_nu(x) (1 - g_nu) U_nu(x)        psi(x + nu)
                              + f-_nu(x) (1 + g_nu) U_nu(x - nu)^H psi(x - nu) ]

with f+_4 = e^{+mu}, f-_4 = e^{-mu}, f_nu = 1 for the spatial directions, and
the time-boundary sign t_bc (-1: antiperiodic) on both hops that cross
t = T-1 <-> 0.  gamma matrices are in the DeGrand-Rossi basis, gamma_5 =
g1 g2 g3 g4 = diag(1, 1, -1, -1).  A = c (gamma_5 D)^2 (Sec. 1, below Eq. 1).
"""
from __future__ import annotations

import numpy as np

from inputs import MU_AXIS

_i = 1j
# DeGrand-Rossi gamma_1..gamma_4
GAMMA = np.array([
    [[0, 0, 0, _i], [0, 0, _i, 0], [0, -_i, 0, 0], [-_i, 0, 0, 0]],
    [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],
    [[0, 0, _i, 0], [0, 0, 0, -_i], [-_i, 0, 0, 0], [0, _i, 0, 0]],
    [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],
], dtype=np.complex128)
GAMMA5 = GAMMA[0] @ GAMMA[1] @ GAMMA[2] @ GAMMA[3]
EYE4 = np.eye(4, dtype=np.complex128)


def _colour(U, psi):
    """(U psi)[s, a] = sum_b U[a, b] psi[s, b] at every site."""
    return psi @ np.swapaxes(U, -1, -2)


def _spin(P, psi):
    """(P psi)[s, a] = sum_t P[s, t] psi[t, a]."""
    return P @ psi


def _dag(U):
    return np.conj(np.swapaxes(U, -1, -2))


def _boundary_weights(T, mu_chem, t_bc):
    """Per-time-slice weights of the forward and backward time hops.

    fwd[t] multiplies the hop x -> x + t_hat taken at time t (crosses the
    boundary at t = T-1); bwd[t] the hop x -> x - t_hat taken at t (crosses it
    at t = 0).
    """
    fwd = np.full(T, np.exp(mu_chem))
    bwd = np.full(T, np.exp(-mu_chem))
    fwd[T - 1] *= t_bc
    bwd[0] *= t_bc
    return fwd, bwd


def dw(U, psi, mass, mu_chem, t_bc=-1):
    """D_w(mu) psi, the definition in the module docstring (Sec. 1)."""
    T = psi.shape[0]
    out = (4.0 + mass) * psi
    fwd_t, bwd_t = _boundary_weights(T, mu_chem, t_bc)
    for nu in range(4):
        ax = MU_AXIS[nu]
        Unu = U[..., nu, :, :]
        hop_f = _colour(Unu, np.roll(psi, -1, axis=ax))              # U(x) psi(x+nu)
        hop_b = _colour(_dag(np.roll(Unu, 1, axis=ax)),               # U(x-nu)^H psi(x-nu)
                        np.roll(psi, 1, axis=ax))
        if nu == 3:
            hop_f = hop_f * fwd_t[:, None, None, None, None, None]
            hop_b = hop_b * bwd_t[:, None, None, None, None, None]
        out = out - 0.5 * (_spin(EYE4 - GAMMA[nu], hop_f) + _spin(EYE4 + GAMMA[nu], hop_b))
    return out


def dw_dagger(U, psi, mass, mu_chem, t_bc=-1):
    """D_w(mu)^H psi, written as the adjoint of each term of `dw`.

    The forward hop F psi(x) = a(x) P U(x) psi(x+nu) has adjoint
    F^H phi(y) = conj(a(y-nu)) P^H U(y-nu)^H phi(y-nu), and the backward hop
    B psi(x) = b(x) Q U(x-nu)^H psi(x-nu) has B^H phi(y) = conj(b(y+nu)) Q^H
    U(y) phi(y+nu).  (Projectors 1 -+ gamma_nu are Hermitian.)
    """
    T = psi.shape[0]
    out = np.conj(4.0 + mass) * psi
    fwd_t, bwd_t = _boundary_weights(T, mu_chem, t_bc)
    for nu in range(4):
        ax = MU_AXIS[nu]
        Unu = U[..., nu, :, :]
        # adjoint of the forward hop: comes from y - nu
        adj_f = _colour(_dag(np.roll(Unu, 1, axis=ax)), np.roll(psi, 1, axis=ax))
        # adjoint of the backward hop: comes from y + nu
        adj_b = _colour(Unu, np.roll(psi, -1, axis=ax))
        if nu == 3:
            adj_f = adj_f * np.conj(np.roll(fwd_t, 1))[:, None, None, None, None, None]
            adj_b = adj_b * np.conj(np.roll(bwd_t, -1))[:, None, None, None, None, None]
        Pf = np.conj(EYE4 - GAMMA[nu]).T
        Pb = np.conj(EYE4 + GAMMA[nu]).T
        out = out - 0.5 * (_spin(Pf, adj_f) + _spin(Pb, adj_b))
    return out


def gamma5(psi):
    return _spin(GAMMA5, psi)


def apply_A(U, psi, mass, mu_chem, c, t_bc=-1):
    """A psi = c gamma_5 D gamma_5 D psi (Sec. 1, A = (gamma_5 D_w)^2, scaled)."""
    return c * gamma5(dw(U, gamma5(dw(U, psi, mass, mu_chem, t_bc)), mass, mu_chem, t_bc))


def apply_A_dagger(U, psi, mass, mu_chem, c, t_bc=-1):
    """A^H psi = conj(c) D^H gamma_5 D^H gamma_5 psi."""
    return np.conj(c) * dw_dagger(U, gamma5(dw_dagger(U, gamma5(psi), mass, mu_chem, t_bc)),
                                  mass, mu_chem, t_bc)


class Operator:
    """Bundles the gauge field and parameters; counts matrix-vector products."""

    def __init__(self, U, mass, mu_chem, c=1.0, t_bc=-1):
        self.U, self.mass, self.mu, self.c, self.t_bc = U, mass, mu_chem, c, t_bc
        self.shape = U.shape[:4] + (4, 3)
        self.n_mv = 0

    def A(self, v):
        self.n_mv += 1
        return apply_A(self.U, v, self.mass, self.mu, self.c, self.t_bc)

    def A_dagger(self, v):
        self.n_mv += 1
        return apply_A_dagger(self.U, v, self.mass, self.mu, self.c, self.t_bc)

    def D(self, v):
        return dw(self.U, v, self.mass, self.mu, self.t_bc)

    def D_dagger(self, v):
        return dw_dagger(self.U, v, self.mass, self.mu, self.t_bc)
