"""Pins of the oracle gradient against central finite differences (no GPU)."""
import numpy as np
import pytest

import inputs
from oracle import dirac, grad, poles, scale

DIMS = (2, 2, 2, 4)


def su3_direction(shape, rng):
    """Random Hermitian traceless X per link (a tangent direction i X U)."""
    M = rng.standard_normal(shape + (3, 3)) + 1j * rng.standard_normal(shape + (3, 3))
    X = 0.5 * (M + np.conj(np.swapaxes(M, -1, -2)))
    return X - (np.trace(X, axis1=-2, axis2=-1) / 3.0)[..., None, None] * np.eye(3)


def move(U, X, t):
    return inputs.expi_hermitian(X, t) @ U


def directional(G, X, U):
    """Re sum tr(G^H (i X U)): the derivative along U(t) = exp(i t X) U."""
    dU = 1j * (X @ U)
    return float(np.real(np.sum(np.conj(G) * dU)))


@pytest.mark.parametrize("mu", [0.0, 0.07])
def test_link_force_of_bilinear_against_finite_differences(mu):
    """The force of B = <a, D b> alone, against central differences of B."""
    rng = np.random.default_rng(5)
    dims = (2, 4, 2, 4)
    U = inputs.su3_exp_gauge(dims, 0.5, 6)
    a = inputs.gaussian_spinor(dims, 7)
    b = inputs.gaussian_spinor(dims, 8)
    G, dmu = grad.link_force(U, a, b, -1.8, mu)
    B = lambda UU, m: np.vdot(a, dirac.dw(UU, b, -1.8, m))
    h = 1e-5
    for _ in range(4):
        X = su3_direction(U.shape[:-2], rng)
        fd = np.real(B(move(U, X, h), mu) - B(move(U, X, -h), mu)) / (2 * h)
        assert abs(fd - directional(G, X, U)) < 1e-8 * max(1.0, abs(fd))
        fdi = np.imag(B(move(U, X, h), mu) - B(move(U, X, -h), mu)) / (2 * h)
        # <(-i) a, D b> = i B (conjugate-linear in a), whose real part is -Im B
        Gi, _ = grad.link_force(U, -1j * a, b, -1.8, mu)
        assert abs(-fdi - directional(Gi, X, U)) < 1e-8 * max(1.0, abs(fdi))
    fdm = (B(U, mu + h) - B(U, mu - h)) / (2 * h)
    assert abs(fdm - dmu) < 1e-8 * max(1.0, abs(fdm))


@pytest.fixture(scope="module")
def problem():
    U = inputs.su3_exp_gauge(DIMS, 0.5, 31)
    op = dirac.Operator(U, -1.8, 0.05)
    c = scale.power_scale(op.A, inputs.gaussian_spinor(DIMS, 32), 100)
    b = inputs.gaussian_spinor(DIMS, 33)
    eta = inputs.gaussian_spinor(DIMS, 34)
    om, sg = poles.neuberger_poles(6)
    return U, c, b, eta, om, sg


def test_gradient_of_f_against_finite_differences(problem):
    U, c, b, eta, om, sg = problem
    mu, tol, h = 0.05, 1e-14, 1e-5
    L, G, dmu, db = grad.grad_f(U, -1.8, mu, c, b, eta, om, sg, 2, tol)
    Lf = lambda UU, m, bb: grad.f_value(UU, -1.8, m, c, bb, eta, om, sg, 2, tol)
    assert abs(L - Lf(U, mu, b)) < 1e-12 * abs(L)
    fdm = (Lf(U, mu + h, b) - Lf(U, mu - h, b)) / (2 * h)
    assert abs(fdm - dmu) < 1e-6 * max(1.0, abs(fdm))
    rng = np.random.default_rng(35)
    for _ in range(6):
        X = su3_direction(U.shape[:-2], rng)
        fd = (Lf(move(U, X, h), mu, b) - Lf(move(U, X, -h), mu, b)) / (2 * h)
        assert abs(fd - directional(G, X, U)) < 1e-6 * max(1.0, abs(fd))
    # dL/db: L is real-linear in b, L(b + t v) - L(b) = t Re <db, v>
    v = inputs.gaussian_spinor(DIMS, 36)
    fdb = (Lf(U, mu, b + h * v) - Lf(U, mu, b - h * v)) / (2 * h)
    assert abs(fdb - np.real(np.vdot(db, v))) < 1e-6 * max(1.0, abs(fdb))
