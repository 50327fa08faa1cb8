"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module holds no arithmetic of the method itself (no Dirac operator, no
partial fractions, no Krylov recurrence): only random fields drawn from seeded
generators, lattice geometry helpers, and the table of workloads.

Canonical layouts (C order, complex128):
    spinor  psi[t, z, y, x, spin(4), colour(3)]
    gauge   U[t, z, y, x, mu(4), a(3), b(3)]     mu = 0,1,2,3 <-> x,y,z,t
so the lexicographic site index is x + X*(y + Y*(z + Z*t)).

The gauge-field recipe U = exp(i*eps*H), H Gaussian traceless Hermitian, is
the synthetic stand-in for the paper's quenched ensembles (beta = 5.32 on
4^3x8, beta = 5.71 on 12^3x24; captions of Figs. 1, 3, 4), which are not
available here.
"""
from __future__ import annotations

import numpy as np

# direction mu -> array axis of the (T, Z, Y, X) site block
MU_AXIS = (3, 2, 1, 0)


def lattice_shape(dims):
    """(X, Y, Z, T) -> array shape (T, Z, Y, X)."""
    X, Y, Z, T = (int(d) for d in dims)
    return (T, Z, Y, X)


def volume(dims):
    X, Y, Z, T = (int(d) for d in dims)
    return X * Y * Z * T


def _complex_gaussian(rng, shape):
    """Entries (N(0,1) + i N(0,1)) / sqrt(2)."""
    g = rng.standard_normal(tuple(shape) + (2,))
    return (g[..., 0] + 1j * g[..., 1]) / np.sqrt(2.0)


def traceless_hermitian(shape, rng):
    """Gaussian traceless Hermitian 3x3 matrices, H = (M + M^H)/2 - tr/3."""
    M = _complex_gaussian(rng, tuple(shape) + (3, 3))
    H = 0.5 * (M + np.conj(np.swapaxes(M, -1, -2)))
    tr = np.trace(H, axis1=-2, axis2=-1).real
    H = H - (tr / 3.0)[..., None, None] * np.eye(3)
    return H


def expi_hermitian(H, eps):
    """exp(i*eps*H) for Hermitian H via its eigendecomposition."""
    w, V = np.linalg.eigh(H)
    ph = np.exp(1j * eps * w)
    return (V * ph[..., None, :]) @ np.conj(np.swapaxes(V, -1, -2))


def su3_exp_gauge(dims, eps, seed):
    """Links U_mu(x) = exp(i eps H), H Gaussian traceless Hermitian (seeded)."""
    rng = np.random.default_rng(seed)
    shp = lattice_shape(dims) + (4,)
    H = traceless_hermitian(shp, rng)
    return np.ascontiguousarray(expi_hermitian(H, eps))


def unit_gauge(dims):
    """Free field U_mu(x) = 1."""
    shp = lattice_shape(dims) + (4,)
    U = np.zeros(shp + (3, 3), dtype=np.complex128)
    U[...] = np.eye(3)
    return U


def random_su3_field(dims, seed, eps=1.0):
    """One SU(3) matrix per site (used as a gauge transformation g(x))."""
    rng = np.random.default_rng(seed)
    H = traceless_hermitian(lattice_shape(dims), rng)
    return np.ascontiguousarray(expi_hermitian(H, eps))


def shift_forward(field, mu):
    """f(x + mu_hat) with periodic wrap (no boundary phase)."""
    return np.roll(field, -1, axis=MU_AXIS[mu])


def gauge_transform(U, g):
    """U^g_mu(x) = g(x) U_mu(x) g(x + mu_hat)^dagger (periodic geometry)."""
    out = np.empty_like(U)
    gd = np.conj(np.swapaxes(g, -1, -2))
    for mu in range(4):
        out[..., mu, :, :] = g @ U[..., mu, :, :] @ shift_forward(gd, mu)
    return out


def pure_gauge(g):
    """U_mu(x) = g(x) g(x + mu_hat)^dagger: the gauge transform of U = 1."""
    gd = np.conj(np.swapaxes(g, -1, -2))
    out = np.empty(g.shape[:4] + (4, 3, 3), dtype=np.complex128)
    for mu in range(4):
        out[..., mu, :, :] = g @ shift_forward(gd, mu)
    return out


def gaussian_spinor(dims, seed):
    """Complex Gaussian spinor, 12 complex components per site."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(_complex_gaussian(rng, lattice_shape(dims) + (4, 3)))


def point_source(dims, spin, colour, site=(0, 0, 0, 0)):
    """Unit vector at lattice site (x, y, z, t), spin and colour index."""
    v = np.zeros(lattice_shape(dims) + (4, 3), dtype=np.complex128)
    x, y, z, t = site
    v[t, z, y, x, spin, colour] = 1.0
    return v


# --------------------------------------------------------------------------
# Workloads.  gauge_seed = 1000 + workload index; the source b uses
# gauge_seed + 1, the adjoint source eta gauge_seed + 2, and the start vector
# of the power iteration for the spectral scale gauge_seed + 3.
# --------------------------------------------------------------------------
WORKLOADS = {
    "wilson_4x4x4x8": dict(
        index=0, dims=(4, 4, 4, 8), eps=0.5, mu=0.05, mass=-1.8, t_bc=-1,
        ell=2, ns=10, tol=1e-10, precision="f64"),
    "wilson_16x16x16x32": dict(
        index=1, dims=(16, 16, 16, 32), eps=0.4, mu=0.1, mass=-1.8, t_bc=-1,
        ell=2, ns=20, tol=1e-10, precision="f32", reliable_every=50),
    "wilson_batched_72": dict(
        index=2, lattices=[(8, 8, 8, 8), (8, 8, 8, 8), (12, 12, 12, 24),
                           (12, 12, 12, 24), (16, 16, 16, 32), (16, 16, 16, 32)],
        eps=0.4, mu_range=(0.0, 0.2), mass=-1.8, t_bc=-1, ell=(2, 4), ns=16,
        tol=1e-10, precision="f32", nrhs=12),
    "wilson_grad_8x8x8x16": dict(
        index=3, dims=(8, 8, 8, 16), eps=0.5, mu=0.05, mass=-1.8, t_bc=-1,
        ell=2, ns=12, tol=1e-13, precision="f64", fd_step=1e-5, n_dirs=32),
    "wilson_32x32x32x64": dict(
        index=4, dims=(32, 32, 32, 64), eps=0.35, mu=0.05, mass=-1.8, t_bc=-1,
        ell=4, ns=32, tol=1e-10, precision="f32", reliable_every=50),
}


def workload_seeds(name):
    gs = 1000 + WORKLOADS[name]["index"]
    return dict(gauge=gs, b=gs + 1, eta=gs + 2, power=gs + 3)


def make_workload(name, dims=None):
    """Gauge field, source and power-iteration start vector of a workload.

    `dims` overrides the lattice size (same generator and seeds), which the
    tests use to run a workload's recipe at a size the oracle finishes fast.
    """
    w = dict(WORKLOADS[name])
    if dims is not None:
        w["dims"] = tuple(dims)
    seeds = workload_seeds(name)
    U = su3_exp_gauge(w["dims"], w["eps"], seeds["gauge"])
    b = gaussian_spinor(w["dims"], seeds["b"])
    v0 = gaussian_spinor(w["dims"], seeds["power"])
    w.update(U=U, b=b, v0=v0, seeds=seeds)
    return w


def make_batched_workload(name="wilson_batched_72"):
    """The batched workload: for lattice k (seeded 100*gauge_seed + k) its gauge
    field, mu_k ~ U[mu_range] (seeded by gauge_seed + 5), the power-iteration
    start vector and its 12 spin-colour point sources at the origin."""
    w = dict(WORKLOADS[name])
    gs = 1000 + w["index"]
    mus = np.random.default_rng(gs + 5).uniform(*w["mu_range"], size=len(w["lattices"]))
    lattices = []
    for k, dims in enumerate(w["lattices"]):
        seed = 100 * gs + k
        lattices.append(dict(
            dims=tuple(dims), mu=float(mus[k]), U=su3_exp_gauge(dims, w["eps"], seed),
            v0=gaussian_spinor(dims, seed + 50),
            sources=[point_source(dims, s, c) for s in range(4) for c in range(3)]))
    w["lattice_systems"] = lattices
    return w
