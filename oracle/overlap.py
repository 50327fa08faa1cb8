"""sign(H) b and the overlap operator D_ov(mu) b (Sec. 1), H = gamma_5 D_w(mu).

Test infrastructure (see the package docstring): not for the product path.

Sec. 1 defines D_ov(mu) = 1 + gamma_5 sign(gamma_5 D_w(mu)) and evaluates the
sign function through sign z = z / sqrt(z^2): with A = c H^2 (the scaled
operator of the solver, c > 0), (H^2)^{-1/2} = sqrt(c) A^{-1/2}, so

    sign(H) b = sqrt(c) H f(A) b,     f(A) b = sum_s omega_s (A + sigma_s)^{-1} b

with poles {omega_s, sigma_s} that approximate z^{-1/2} (Eq. 1), and

    D_ov(mu) b = b + gamma_5 sign(H) b = b + sqrt(c) D_w(mu) f(A) b.

`sign_apply` / `overlap_apply` take f(A) b from a caller-supplied solver (the
oracle's multi-shift forms or a direct evaluation); `sign_dense` is the exact
matrix sign function of a small dense H by eigendecomposition (no pole
approximation), the reference the pole form converges to.

`sign_deflated` treats k eigenpairs of H exactly and applies the pole form to
the rest (the deflation of the benchmarks of Sec. 3, Figs. 3 and 4); `smallest_eigenpairs`
supplies them from a dense eigendecomposition on small lattices.

Pinned by tests/test_oracle_pins.py: sign(H)^2 = 1 and the Ginsparg-Wilson
relation (up to the pole approximation), the pole form against the dense
exact sign on tiny lattices, and the deflated form against the exact sign with
an error that falls as eigenpairs are deflated.
"""
from __future__ import annotations

import numpy as np

from . import dirac


def sign_apply(op, y):
    """sign(H) b = sqrt(c) gamma_5 D_w(mu) y, given y = f(A) b (Sec. 1)."""
    return np.sqrt(op.c) * dirac.gamma5(op.D(y))


def overlap_apply(op, b, y):
    """D_ov(mu) b = b + gamma_5 sign(H) b = b + sqrt(c) D_w(mu) y, given y = f(A) b."""
    return b + np.sqrt(op.c) * op.D(y)


def sign_deflated(op, b, lam, R, Lv, f_of_A):
    """sign(H) b with k eigenpairs of H treated exactly (the deflation of the
    benchmarks of Sec. 3, Figs. 3 and 4):
    right eigenvectors R[i], left eigenvectors Lv[i] with Lv[i]^H R[j] = delta_ij,
    eigenvalues lam[i]; a_i = Lv[i]^H b and

        sign(H) b = sum_i sign(Re lam_i) a_i R[i] + sqrt(c) H f(A) (b - sum_i a_i R[i]),

    f_of_A(v) = f(A) v from any solver."""
    a = [np.vdot(Lv[i], b) for i in range(len(lam))]
    rest = b - sum((a[i] * R[i] for i in range(len(lam))), np.zeros_like(b))
    exact = sum((np.sign(np.real(lam[i])) * a[i] * R[i] for i in range(len(lam))), np.zeros_like(b))
    return exact + sign_apply(op, f_of_A(rest))


def overlap_deflated(op, b, lam, R, Lv, f_of_A):
    """D_ov(mu) b = b + gamma_5 sign(H) b with the deflated sign."""
    return b + dirac.gamma5(sign_deflated(op, b, lam, R, Lv, f_of_A))


def smallest_eigenpairs(Hm, k, shape):
    """The k eigenvalues of the dense H smallest in magnitude, with right and
    left eigenvectors (rows of V^{-1}, conjugated) as spinors, Lv_i^H R_j = delta_ij."""
    lam, V = np.linalg.eig(Hm)
    W = np.linalg.inv(V)                     # W V = 1: row i of W is l_i^H
    idx = np.argsort(np.abs(lam))[:k]
    R = [V[:, i].reshape(shape) for i in idx]
    Lv = [np.conj(W[i, :]).reshape(shape) for i in idx]
    return lam[idx], R, Lv


def dense_H(op):
    """The dense matrix of H = gamma_5 D_w(mu) on a small lattice."""
    n = int(np.prod(op.shape))
    Hm = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for k in range(n):
        e[k] = 1.0
        Hm[:, k] = dirac.gamma5(op.D(e.reshape(op.shape))).reshape(-1)
        e[k] = 0.0
    return Hm


def sign_dense(Hm):
    """Exact matrix sign of a diagonalisable H: V diag(sign Re lambda) V^{-1}."""
    lam, V = np.linalg.eig(Hm)
    if np.any(np.abs(lam.real) < 1e-12 * np.abs(lam).max()):
        raise ValueError("H has eigenvalues on the imaginary axis: sign undefined")
    return V @ np.diag(np.sign(lam.real)) @ np.linalg.inv(V)
