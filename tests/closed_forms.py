"""Closed forms that pin the oracle (and, at full size, the CUDA path).

Free Wilson fermions (U = 1) are diagonal in momentum space.  For a plane wave
psi(x) = e^{i p.x} chi the hops give
    D(p) = (4 + m) - sum_nu cos(pt_nu) + i sum_nu gamma_nu sin(pt_nu),
with pt_4 = p_4 - i mu (the chemical potential shifts the time momentum into
the complex plane) and pt_k = p_k otherwise.  Antiperiodic fields in time have
p_4 = pi (2n + 1) / T.  Then gamma_5 D(p) gamma_5 = a - i gamma.s, so
A(p) = c (gamma_5 D)^2 = c [a(p)^2 + sum_nu s_nu(p)^2] times the unit matrix,
a = 4 + m - sum cos pt, s_nu = sin pt_nu, and f(A) b is the scalar function
applied mode by mode.  Numpy's FFT is the library step.
"""
from __future__ import annotations

import numpy as np

from inputs import lattice_shape

GAMMA_DR = np.array([
    [[0, 0, 0, 1j], [0, 0, 1j, 0], [0, -1j, 0, 0], [-1j, 0, 0, 0]],
    [[0, 0, 0, -1], [0, 0, 1, 0], [0, 1, 0, 0], [-1, 0, 0, 0]],
    [[0, 0, 1j, 0], [0, 0, 0, -1j], [-1j, 0, 0, 0], [0, 1j, 0, 0]],
    [[0, 0, 1, 0], [0, 0, 0, 1], [1, 0, 0, 0], [0, 1, 0, 0]],
], dtype=np.complex128)


def _momenta(dims, mu, t_bc):
    X, Y, Z, T = dims
    shp = lattice_shape(dims)
    kx = 2 * np.pi * np.fft.fftfreq(X)
    ky = 2 * np.pi * np.fft.fftfreq(Y)
    kz = 2 * np.pi * np.fft.fftfreq(Z)
    kt = 2 * np.pi * np.fft.fftfreq(T) + (np.pi / T if t_bc == -1 else 0.0)
    P = np.meshgrid(kt, kz, ky, kx, indexing="ij")   # axes (T, Z, Y, X)
    pt = [P[3], P[2], P[1], P[0] - 1j * mu]            # pt_1..pt_4
    assert P[0].shape == shp
    return pt


def _twist(dims, t_bc):
    T = dims[3]
    t = np.arange(T)
    ph = np.exp(1j * np.pi * t / T) if t_bc == -1 else np.ones(T)
    return ph[:, None, None, None, None, None]


def _to_momentum(psi, dims, t_bc):
    return np.fft.fftn(psi / _twist(dims, t_bc), axes=(0, 1, 2, 3))


def _from_momentum(phi, dims, t_bc):
    return np.fft.ifftn(phi, axes=(0, 1, 2, 3)) * _twist(dims, t_bc)


def free_dw(psi, dims, mass, mu, t_bc=-1):
    """D_w(mu) psi for U = 1, by FFT."""
    pt = _momenta(dims, mu, t_bc)
    a = 4.0 + mass - sum(np.cos(p) for p in pt)
    Dp = a[..., None, None] * np.eye(4)
    for nu in range(4):
        Dp = Dp + 1j * np.sin(pt[nu])[..., None, None] * GAMMA_DR[nu]
    phi = _to_momentum(psi, dims, t_bc)
    return _from_momentum(Dp @ phi, dims, t_bc)


def free_A_eigenvalues(dims, mass, mu, c=1.0, t_bc=-1):
    """The scalar A(p) on every momentum (shape (T, Z, Y, X))."""
    pt = _momenta(dims, mu, t_bc)
    a = 4.0 + mass - sum(np.cos(p) for p in pt)
    return c * (a ** 2 + sum(np.sin(p) ** 2 for p in pt))


def free_matfunc(b, dims, mass, mu, c, fscalar, t_bc=-1):
    """f(A) b for U = 1: fscalar applied to A(p) mode by mode."""
    lam = free_A_eigenvalues(dims, mass, mu, c, t_bc)
    phi = _to_momentum(b, dims, t_bc)
    return _from_momentum(fscalar(lam)[..., None, None] * phi, dims, t_bc)


def neuberger_eps(x, n):
    """Neuberger's rational sign approximation
    eps_N(x) = ((1+x)^{2N} - (1-x)^{2N}) / ((1+x)^{2N} + (1-x)^{2N})."""
    p = (1 + x) ** (2 * n)
    q = (1 - x) ** (2 * n)
    return (p - q) / (p + q)


def gauge_rotate_spinor(g, psi):
    """(G psi)(x) = g(x) psi(x) on the colour index."""
    return psi @ np.swapaxes(g, -1, -2)


def alternation(om, sg, eps, npts=400001):
    """Error of x R(x^2) against sign(x) = 1 on a log grid of [eps, 1]: its
    maximum modulus and the signs at the grid's local extrema that reach it."""
    x = np.geomspace(eps, 1.0, npts)
    err = x * np.sum(om[None, :] / (x[:, None] ** 2 + sg[None, :]), axis=1) - 1.0
    d = np.abs(err).max()
    a = np.abs(err)
    i = np.flatnonzero((a[1:-1] >= a[:-2]) & (a[1:-1] >= a[2:])) + 1
    ends = [0, len(err) - 1]
    pts = sorted(set(j for j in list(i) + ends if a[j] > (1 - 1e-6) * d))
    return d, np.sign(err[pts])
