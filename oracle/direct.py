"""Direct evaluations of y* = sum_s omega_s (A + sigma_s)^{-1} b (Eq. 1).

Test infrastructure (see the package docstring): not for the product path.

These are the plain definition of what the multi-shift method converges to:
one library solve per shift (SciPy GMRES on a matrix-free operator), or, on
tiny lattices, the dense matrix of A with LU solves or its eigendecomposition.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla


def per_shift_solve(apply_A, b, sigma, rtol=1e-13, restart=200, maxiter=200):
    """x = (A + sigma)^{-1} b by restarted GMRES (library routine)."""
    n = b.size
    shape = b.shape

    def mv(v):
        v = v.reshape(shape)
        return (apply_A(v) + sigma * v).reshape(-1)

    op = spla.LinearOperator((n, n), matvec=mv, dtype=np.complex128)
    x, info = spla.gmres(op, b.reshape(-1), rtol=rtol, atol=0.0, restart=restart,
                         maxiter=maxiter)
    if info != 0:
        raise RuntimeError(f"gmres did not converge (info={info})")
    return x.reshape(shape)


def pfe_per_shift(apply_A, b, omega, sigma, rtol=1e-13):
    """y* by an independent solve per shift."""
    return sum(w * per_shift_solve(apply_A, b, s, rtol) for w, s in zip(omega, sigma))


def dense_matrix(apply, shape):
    """The matrix of a linear map on fields of `shape`, column by column."""
    n = int(np.prod(shape))
    M = np.empty((n, n), dtype=np.complex128)
    e = np.zeros(n, dtype=np.complex128)
    for k in range(n):
        e[k] = 1.0
        M[:, k] = apply(e.reshape(shape)).reshape(-1)
        e[k] = 0.0
    return M


def pfe_dense(Amat, b, omega, sigma):
    """y* by dense LU solves (numpy.linalg.solve) per shift."""
    n = Amat.shape[0]
    bb = b.reshape(-1)
    y = np.zeros(n, dtype=np.complex128)
    for w, s in zip(omega, sigma):
        y += w * np.linalg.solve(Amat + s * np.eye(n), bb)
    return y.reshape(b.shape)


def matfunc_eig(Amat, b, fscalar):
    """V diag(f(lambda)) V^{-1} b for a diagonalisable A."""
    lam, V = np.linalg.eig(Amat)
    coeff = np.linalg.solve(V, b.reshape(-1))
    return (V @ (fscalar(lam) * coeff)).reshape(b.shape)
