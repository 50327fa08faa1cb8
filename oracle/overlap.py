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

Pinned by tests/test_oracle_pins.py: sign(H)^2 = 1 and the Ginsparg-Wilson
relation at mu = 0 (up to the pole approximation), and the pole form against
the dense exact sign on tiny lattices.
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
