"""Pins of the FP64 oracle against facts fixed by the mathematics (no GPU).

Each test checks the oracle against something other than itself: closed
forms (free field, Neuberger's rational function), library routines (FFT,
dense LU, eigendecomposition, GMRES), exact invariants, and special cases
that reduce to textbook algorithms.
"""
import numpy as np
import pytest

import inputs
from oracle import dirac, direct, msbicgstab as ms, overlap, poles, scale
from closed_forms import (GAMMA_DR, alternation, free_A_eigenvalues, free_dw, free_matfunc,
                          gauge_rotate_spinor, neuberger_eps)

RNG = np.random.default_rng(12345)


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def vdot(a, b):
    return np.vdot(a, b)


# ---------------------------------------------------------------- poles (Eq. 1)
@pytest.mark.parametrize("n", [1, 4, 10, 20, 32])
def test_neuberger_pfe_closed_form(n):
    """sum_s omega_s/(z + sigma_s) = eps_N(sqrt z)/sqrt z, for complex z."""
    om, sg = poles.neuberger_poles(n)
    z = np.concatenate([np.logspace(-4, 1, 40),
                        (RNG.uniform(0.01, 2, 20) + 1j * RNG.uniform(-0.5, 0.5, 20))])
    x = np.sqrt(z)
    assert np.allclose(poles.pfe_scalar(z, om, sg), neuberger_eps(x, n) / x,
                       rtol=1e-13, atol=0)
    assert np.all(om > 0) and np.all(sg > 0) and np.all(np.diff(sg) > 0)


def test_pfe_approaches_inverse_sqrt():
    """The expansion converges to z^{-1/2} away from 0 (Sec. 1, f(A) = A^{-1/2})."""
    om, sg = poles.neuberger_poles(32)
    z = np.linspace(0.05, 1.0, 50)
    assert np.max(np.abs(poles.pfe_scalar(z, om, sg) * np.sqrt(z) - 1)) < 1e-10


# ---------------------------------------------------------------- gamma algebra
def test_gamma_algebra():
    G = dirac.GAMMA
    for a in range(4):
        assert np.allclose(G[a], G[a].conj().T)
        for b in range(4):
            ac = G[a] @ G[b] + G[b] @ G[a]
            assert np.allclose(ac, 2.0 * (a == b) * np.eye(4))
    assert np.allclose(dirac.GAMMA5, np.diag([1, 1, -1, -1]))
    assert np.allclose(G, GAMMA_DR)


# ---------------------------------------------------------------- operator
DIMS = (4, 4, 4, 8)


@pytest.fixture(scope="module")
def gauge():
    return inputs.su3_exp_gauge(DIMS, 0.5, 77)


def test_links_are_su3(gauge):
    U = gauge
    I = np.eye(3)
    assert np.allclose(U @ np.conj(np.swapaxes(U, -1, -2)), I, atol=1e-13)
    assert np.allclose(np.linalg.det(U), 1.0, atol=1e-13)


@pytest.mark.parametrize("mu,t_bc", [(0.0, -1), (0.05, -1), (0.3, 1), (-0.2, -1)])
def test_free_field_dirac_closed_form(mu, t_bc):
    dims = (4, 6, 2, 8)
    U = inputs.unit_gauge(dims)
    psi = inputs.gaussian_spinor(dims, 5)
    got = dirac.dw(U, psi, -1.8, mu, t_bc)
    assert rel(got, free_dw(psi, dims, -1.8, mu, t_bc)) < 1e-14


@pytest.mark.parametrize("mu", [0.0, 0.1])
def test_gauge_covariance(gauge, mu):
    """D[U^g] (G psi) = G D[U] psi with U^g_nu(x) = g(x) U_nu(x) g(x+nu)^H."""
    g = inputs.random_su3_field(DIMS, 3)
    Ug = inputs.gauge_transform(gauge, g)
    psi = inputs.gaussian_spinor(DIMS, 4)
    lhs = dirac.dw(Ug, gauge_rotate_spinor(g, psi), -1.8, mu)
    rhs = gauge_rotate_spinor(g, dirac.dw(gauge, psi, -1.8, mu))
    assert rel(lhs, rhs) < 1e-14


def test_pure_gauge_reduces_to_free_field():
    g = inputs.random_su3_field(DIMS, 11)
    U = inputs.pure_gauge(g)
    psi = inputs.gaussian_spinor(DIMS, 12)
    got = dirac.dw(U, gauge_rotate_spinor(g, psi), -1.8, 0.07)
    want = gauge_rotate_spinor(g, free_dw(psi, DIMS, -1.8, 0.07))
    assert rel(got, want) < 1e-13


@pytest.mark.parametrize("mu", [0.0, 0.05, 0.4])
def test_dagger_is_adjoint(gauge, mu):
    u = inputs.gaussian_spinor(DIMS, 21)
    v = inputs.gaussian_spinor(DIMS, 22)
    lhs = vdot(u, dirac.dw(gauge, v, -1.8, mu))
    rhs = vdot(dirac.dw_dagger(gauge, u, -1.8, mu), v)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


@pytest.mark.parametrize("mu", [0.05, 0.4])
def test_gamma5_hermiticity_with_mu(gauge, mu):
    """gamma_5 D(mu) gamma_5 = D(-mu)^H; gamma_5 D non-Hermitian for mu != 0 (Sec. 1)."""
    v = inputs.gaussian_spinor(DIMS, 23)
    lhs = dirac.gamma5(dirac.dw(gauge, dirac.gamma5(v), -1.8, mu))
    rhs = dirac.dw_dagger(gauge, v, -1.8, -mu)
    assert rel(lhs, rhs) < 1e-14
    u = inputs.gaussian_spinor(DIMS, 24)
    H = lambda w: dirac.gamma5(dirac.dw(gauge, w, -1.8, mu))
    assert abs(vdot(u, H(v)) - vdot(H(u), v)) > 1e-6 * abs(vdot(u, H(v)))


def test_gamma5_dirac_hermitian_at_mu0(gauge):
    u = inputs.gaussian_spinor(DIMS, 25)
    v = inputs.gaussian_spinor(DIMS, 26)
    H = lambda w: dirac.gamma5(dirac.dw(gauge, w, -1.8, 0.0))
    assert abs(vdot(u, H(v)) - vdot(H(u), v)) < 1e-13 * abs(vdot(u, H(v)))


def test_A_dagger_is_A_at_minus_mu(gauge):
    v = inputs.gaussian_spinor(DIMS, 27)
    u = inputs.gaussian_spinor(DIMS, 28)
    Ad = dirac.apply_A_dagger(gauge, v, -1.8, 0.1, 0.03)
    assert rel(Ad, dirac.apply_A(gauge, v, -1.8, -0.1, 0.03)) < 1e-14
    lhs = vdot(u, dirac.apply_A(gauge, v, -1.8, 0.1, 0.03))
    rhs = vdot(dirac.apply_A_dagger(gauge, u, -1.8, 0.1, 0.03), v)
    assert abs(lhs - rhs) < 1e-13 * abs(lhs)


def test_free_field_A_closed_form():
    dims = (4, 4, 4, 8)
    U = inputs.unit_gauge(dims)
    psi = inputs.gaussian_spinor(dims, 31)
    got = dirac.apply_A(U, psi, -1.8, 0.05, 0.02)
    want = free_matfunc(psi, dims, -1.8, 0.05, 0.02, lambda lam: lam)
    assert rel(got, want) < 1e-14


# ---------------------------------------------------------------- spectral scale
def test_power_iteration_free_field():
    dims = (4, 4, 4, 8)
    op = dirac.Operator(inputs.unit_gauge(dims), -1.8, 0.05)
    lam = scale.power_lambda(op.A, inputs.gaussian_spinor(dims, 41), 100)
    lmax = np.max(np.abs(free_A_eigenvalues(dims, -1.8, 0.05)))
    assert lam <= lmax * (1 + 1e-12)
    assert lam > 0.99 * lmax


def test_power_iteration_dense_tiny():
    dims = (2, 2, 2, 4)
    op = dirac.Operator(inputs.su3_exp_gauge(dims, 0.5, 42), -1.8, 0.05)
    lam = scale.power_lambda(op.A, inputs.gaussian_spinor(dims, 43), 200)
    Am = direct.dense_matrix(op.A, op.shape)
    ev = np.abs(np.linalg.eigvals(Am))
    assert lam <= np.linalg.norm(Am, 2) * (1 + 1e-12)
    assert abs(lam - ev.max()) < 0.02 * ev.max()


# ---------------------------------------------------------------- solvers
TINY = (2, 2, 2, 4)


@pytest.fixture(scope="module")
def tiny_problem():
    U = inputs.su3_exp_gauge(TINY, 0.5, 51)
    op0 = dirac.Operator(U, -1.8, 0.05)
    c = scale.power_scale(op0.A, inputs.gaussian_spinor(TINY, 52), 100)
    op = dirac.Operator(U, -1.8, 0.05, c)
    b = inputs.gaussian_spinor(TINY, 53)
    Am = direct.dense_matrix(op.A, op.shape)
    return op, b, Am


def test_textbook_bicgstab_equals_ell1(tiny_problem):
    """BiCGstab(1) reproduces van der Vorst's BiCGstab iterate by iterate."""
    op, b, _ = tiny_problem
    k = 12
    x = np.zeros_like(b)
    r = b.copy()
    rh = b.copy()
    rho_old = alpha = om = 1.0 + 0j
    v = p = np.zeros_like(b)
    for _ in range(k):
        rho = vdot(rh, r)
        beta = (rho / rho_old) * (alpha / om)
        p = r + beta * (p - om * v)
        v = op.A(p)
        alpha = rho / vdot(rh, v)
        s = r - alpha * v
        t = op.A(s)
        om = vdot(t, s) / vdot(t, t)
        x = x + alpha * p + om * s
        r = s - om * t
        rho_old = rho
    x_ell, _ = ms.seed_recurrence(op.A, b, 1, k)
    assert rel(x_ell, x) < 1e-11


@pytest.mark.parametrize("ell", [1, 2, 3, 4])
def test_seed_solver_converges_to_dense(tiny_problem, ell):
    op, b, Am = tiny_problem
    x, _ = ms.bicgstab_ell(op.A, b, ell, 1e-12)
    want = np.linalg.solve(Am, b.reshape(-1)).reshape(b.shape)
    assert rel(x, want) < 1e-7   # the seed system is the ill-conditioned one


@pytest.mark.parametrize("ell", [1, 2, 3, 4])
def test_shift_collinearity_invariant(tiny_problem, ell):
    """(A + sigma_s) x_s + r_0 / zeta_s = b after every outer iteration."""
    op, b, _ = tiny_problem
    om, sg = poles.neuberger_poles(8)
    worst = [0.0]
    bn = np.linalg.norm(b)

    def obs(m, r0, xs, zeta, active):
        for s in np.flatnonzero(active):
            res = op.A(xs[s]) + sg[s] * xs[s] + r0 / zeta[s] - b
            worst[0] = max(worst[0], np.linalg.norm(res) / bn)

    ms.multishift_single(op.A, b, sg, ell, 1e-11, observer=obs)
    assert worst[0] < 1e-12


@pytest.mark.parametrize("ell", [1, 2, 4])
def test_multishift_matches_dense_lu_and_eig(tiny_problem, ell):
    op, b, Am = tiny_problem
    om, sg = poles.neuberger_poles(10)
    y_lu = direct.pfe_dense(Am, b, om, sg)
    y_eig = direct.matfunc_eig(Am, b, lambda z: neuberger_eps(np.sqrt(z), 10) / np.sqrt(z))
    assert rel(y_eig, y_lu) < 1e-10
    xs = ms.multishift_single(op.A, b, sg, ell, 1e-12)
    for s in range(len(sg)):
        xd = np.linalg.solve(Am + sg[s] * np.eye(Am.shape[0]), b.reshape(-1)).reshape(b.shape)
        assert rel(xs[s], xd) < 1e-9
    y1 = ms.pfe_from_shifts(xs, om)
    y2 = ms.multishift_double(op.A, b, sg, om, ell, 1e-12)
    assert rel(y1, y_lu) < 1e-10
    assert rel(y2, y_lu) < 1e-10


@pytest.mark.parametrize("ell", [1, 2, 4])
def test_single_equals_double_pass(ell):
    """Sec. 2: the double-pass form reproduces the single-pass sum."""
    w = inputs.make_workload("wilson_4x4x4x8")
    op = dirac.Operator(w["U"], w["mass"], w["mu"])
    c = scale.power_scale(op.A, w["v0"], 100)
    op = dirac.Operator(w["U"], w["mass"], w["mu"], c)
    om, sg = poles.neuberger_poles(w["ns"])
    xs = ms.multishift_single(op.A, w["b"], sg, ell, 1e-10)
    y1 = ms.pfe_from_shifts(xs, om)
    y2 = ms.multishift_double(op.A, w["b"], sg, om, ell, 1e-10)
    assert rel(y2, y1) < 1e-13


@pytest.mark.parametrize("ell", [1, 2, 4])
def test_fixed_cost_mode(ell):
    """fixed_outer = M (the fixed-cost runs of Sec. 3, Fig. 2): the shift
    recurrences truncated after M outer iterations.  Pins: a pole at sigma = 0
    reproduces the seed recurrence's own iterate after M outer iterations (the
    shifted system is then the seed system); the double-pass resolution of the
    truncated recurrence equals the single-pass shift vectors; a fixed M past
    the natural stop changes nothing."""
    w = inputs.make_workload("wilson_4x4x4x8")
    op = dirac.Operator(w["U"], w["mass"], w["mu"])
    c = scale.power_scale(op.A, w["v0"], 100)
    op = dirac.Operator(w["U"], w["mass"], w["mu"], c)
    M = 5
    x_seed, _ = ms.seed_recurrence(op.A, w["b"], ell, M)
    st = ms.Stats()
    xs = ms.multishift_single(op.A, w["b"], [0.0, 0.3], ell, 1e-300, fixed_outer=M, stats=st)
    assert st.n_outer == M and list(st.iters_per_shift) == [M, M]
    assert rel(xs[0], x_seed) < 1e-12
    om, sg = poles.neuberger_poles(w["ns"])
    xs = ms.multishift_single(op.A, w["b"], sg, ell, 1e-10, fixed_outer=M)
    y2 = ms.multishift_double(op.A, w["b"], sg, om, ell, 1e-10, fixed_outer=M)
    assert rel(y2, ms.pfe_from_shifts(xs, om)) < 1e-13
    st = ms.Stats()
    y_free = ms.multishift_double(op.A, w["b"], sg, om, ell, 1e-10, stats=st)
    y_long = ms.multishift_double(op.A, w["b"], sg, om, ell, 1e-10, fixed_outer=st.n_outer + 5)
    assert np.array_equal(y_long, y_free)


def test_operation_counts_match_cost_table():
    """Sec. 3 table: #Mv = 2Ml (1-pass), 4Ml (2-pass); #dot = Ml(0.5l+3.5)
    (+1 residual norm per outer iteration for the convergence test)."""
    dims = (2, 2, 2, 4)
    U = inputs.su3_exp_gauge(dims, 0.5, 61)
    op = dirac.Operator(U, -1.8, 0.05, 0.05)
    b = inputs.gaussian_spinor(dims, 62)
    om, sg = poles.neuberger_poles(6)
    for ell in (1, 2, 3, 4):
        st1 = ms.Stats()
        ms.multishift_single(op.A, b, sg, ell, 1e-10, stats=st1)
        M = st1.n_outer
        assert st1.n_mv == 2 * M * ell
        assert st1.n_dot == M * ell * (ell + 7) // 2 + M
        st2 = ms.Stats()
        ms.multishift_double(op.A, b, sg, om, ell, 1e-10, stats=st2)
        assert st2.n_mv == 4 * M * ell
        assert st2.n_dot == M * ell * (ell + 7) // 2 + M


def test_free_field_f_of_A_closed_form():
    """y for U = 1 against the momentum-space PFE (any lattice size)."""
    dims = (4, 4, 4, 8)
    U = inputs.unit_gauge(dims)
    om, sg = poles.neuberger_poles(10)
    op = dirac.Operator(U, -1.8, 0.05, 0.03)
    b = inputs.gaussian_spinor(dims, 71)
    y = ms.multishift_double(op.A, b, sg, om, 2, 1e-11)
    want = free_matfunc(b, dims, -1.8, 0.05, 0.03, lambda lam: poles.pfe_scalar(lam, om, sg))
    assert rel(y, want) < 1e-9


def test_workload_c1_against_per_shift_gmres():
    """The 4^3x8 workload: double-pass y vs one GMRES solve per shift."""
    w = inputs.make_workload("wilson_4x4x4x8")
    op = dirac.Operator(w["U"], w["mass"], w["mu"])
    c = scale.power_scale(op.A, w["v0"], 100)
    op = dirac.Operator(w["U"], w["mass"], w["mu"], c)
    om, sg = poles.neuberger_poles(w["ns"])
    y = ms.multishift_double(op.A, w["b"], sg, om, w["ell"], w["tol"])
    ystar = direct.pfe_per_shift(op.A, w["b"], om, sg, rtol=1e-13)
    assert rel(y, ystar) < 1e-9


def _multishift_cg(A, b, sigma, tol, max_iter=5000):
    """Textbook multi-shift CG for (A + sigma_s) x_s = b with A Hermitian
    positive definite (Jegerlehner, hep-lat/9612014): one CG on A, and for
    every shift the collinear residual r_s = zeta_s r with zeta_s from the
    three-term recurrence of the CG residual polynomials at -sigma_s."""
    sigma = np.asarray(sigma, dtype=np.float64)
    ns = len(sigma)
    x = [np.zeros_like(b) for _ in range(ns)]
    p_s = [b.copy() for _ in range(ns)]
    r, p = b.copy(), b.copy()
    z_prev, z = np.ones(ns), np.ones(ns)
    a_prev, b_prev = 1.0, 0.0
    rr = np.vdot(r, r).real
    bn = np.sqrt(rr)
    live = np.ones(ns, dtype=bool)           # a shift stops once |zeta_s r| <= tol |b|
    for _ in range(max_iter):
        Ap = A(p)
        a = rr / np.vdot(p, Ap).real
        z_new = z.copy()
        for s in np.flatnonzero(live):
            z_new[s] = z[s] * z_prev[s] * a_prev / (a * b_prev * (z_prev[s] - z[s])
                                                     + z_prev[s] * a_prev * (1.0 + sigma[s] * a))
            x[s] = x[s] + (a * z_new[s] / z[s]) * p_s[s]
        r = r - a * Ap
        rr_new = np.vdot(r, r).real
        bt = rr_new / rr
        for s in np.flatnonzero(live):
            p_s[s] = z_new[s] * r + bt * (z_new[s] / z[s]) ** 2 * p_s[s]
        p = r + bt * p
        z_prev, z = np.where(live, z, z_prev), z_new
        a_prev, b_prev, rr = a, bt, rr_new
        live &= np.sqrt(rr) * np.abs(z) > tol * bn
        if not live.any():
            return x
    raise RuntimeError("multi-shift CG did not converge")


@pytest.mark.parametrize("ell", [1, 2, 4])
def test_mu0_multishift_cg_gives_the_same_sum(ell):
    """At mu = 0, A = c (g5 D)^2 is Hermitian positive definite: textbook
    multi-shift CG on it gives the same pole sum and the same x_s as the
    oracle's single- and double-pass multi-shift BiCGstab(l)."""
    U = inputs.su3_exp_gauge(TINY, 0.5, 61)
    op0 = dirac.Operator(U, -1.8, 0.0)
    c = scale.power_scale(op0.A, inputs.gaussian_spinor(TINY, 62), 100)
    op = dirac.Operator(U, -1.8, 0.0, c)
    b = inputs.gaussian_spinor(TINY, 63)
    om, sg = poles.neuberger_poles(10)
    x_cg = _multishift_cg(op.A, b, sg, 1e-13)
    xs = ms.multishift_single(op.A, b, sg, ell, 1e-13)
    for s in range(len(sg)):
        assert rel(xs[s], x_cg[s]) < 1e-10, s
    y_cg = ms.pfe_from_shifts(x_cg, om)
    assert rel(ms.pfe_from_shifts(xs, om), y_cg) < 1e-10
    assert rel(ms.multishift_double(op.A, b, sg, om, ell, 1e-13), y_cg) < 1e-10


def _overlap_problem(mu):
    """Tiny lattice, Wilson mass 1: the spectrum of A = c H^2 stays away from 0,
    so 32 Neuberger poles approximate z^{-1/2} on it to better than 1e-11."""
    U = inputs.su3_exp_gauge(TINY, 0.5, 81)
    op0 = dirac.Operator(U, 1.0, mu)
    c = scale.power_scale(op0.A, inputs.gaussian_spinor(TINY, 82), 200)
    return dirac.Operator(U, 1.0, mu, c), inputs.gaussian_spinor(TINY, 83)


@pytest.mark.parametrize("mu", [0.0, 0.2])
def test_sign_and_overlap_against_dense_exact_sign(mu):
    """Sec. 1: sign(H) b = sqrt(c) H f(A) b (sign z = z / sqrt(z^2)) against the
    exact matrix sign V sign(Re lambda) V^{-1} b of the dense H = g5 D_w(mu);
    D_ov b = b + g5 sign(H) b; sign(H)^2 b = b."""
    op, b = _overlap_problem(mu)
    om, sg = poles.neuberger_poles(32)
    y = ms.multishift_double(op.A, b, sg, om, 2, 1e-13)
    S = overlap.sign_dense(overlap.dense_H(op))
    s_exact = (S @ b.reshape(-1)).reshape(b.shape)
    s = overlap.sign_apply(op, y)
    assert rel(s, s_exact) < 1e-10
    assert rel(overlap.overlap_apply(op, b, y), b + dirac.gamma5(s_exact)) < 1e-10
    y2 = ms.multishift_double(op.A, s, sg, om, 2, 1e-13)
    assert rel(overlap.sign_apply(op, y2), b) < 1e-10


@pytest.mark.parametrize("mu", [0.0, 0.2])
def test_overlap_ginsparg_wilson_relation(mu):
    """D_ov = 1 + g5 sign(H) satisfies g5 D_ov + D_ov g5 = D_ov g5 D_ov, which
    is sign(H)^2 = 1 written out (any mu), here through the pole form."""
    op, b = _overlap_problem(mu)
    om, sg = poles.neuberger_poles(32)

    def D(v):
        return overlap.overlap_apply(op, v, ms.multishift_double(op.A, v, sg, om, 2, 1e-13))

    g5 = dirac.gamma5
    lhs = g5(D(b)) + D(g5(b))
    rhs = D(g5(D(b)))
    assert rel(lhs, rhs) < 1e-10
    # a control: 1 + sign(H) without the gamma_5 does not satisfy it

    def Dx(v):
        return v + overlap.sign_apply(op, ms.multishift_double(op.A, v, sg, om, 2, 1e-13))

    assert rel(g5(Dx(b)) + Dx(g5(b)), Dx(g5(Dx(b)))) > 1e-3


@pytest.mark.parametrize("ns,eps", [(1, 0.5), (2, 0.1), (4, 0.05), (6, 0.01)])
def test_zolotarev_equioscillation(ns, eps):
    """Chebyshev's alternation theorem: the best uniform approximation of
    sign(x) on [eps, 1] by x R(x^2), R of type (ns - 1, ns) (2 ns free
    parameters), has an error that reaches its maximum modulus with alternating
    signs at 2 ns + 1 points.  Found on a dense grid, independently of the
    alternation points the construction uses; the returned delta is that
    maximum."""
    om, sg, delta = poles.zolotarev_poles(ns, eps)
    d, signs = alternation(om, sg, eps)
    assert len(signs) == 2 * ns + 1
    assert np.all(signs[1:] != signs[:-1])
    assert abs(d - delta) <= 1e-6 * delta
    assert np.all(om > 0) and np.all(sg > 0) and np.all(np.diff(sg) > 0)


def test_zolotarev_beats_neuberger_on_its_interval():
    """At equal pole count the optimal expansion is far more accurate on
    [eps^2, 1] than Neuberger's, and its error falls with the pole count."""
    eps = 0.02
    x = np.geomspace(eps, 1.0, 20001)
    prev = 1.0
    for ns in (4, 8, 12):
        om, sg, delta = poles.zolotarev_poles(ns, eps)
        on, snb = poles.neuberger_poles(ns)
        e_n = np.abs(x * poles.pfe_scalar(x * x, on, snb).real - 1).max()
        assert delta < 1e-2 * e_n
        assert delta < 1e-2 * prev
        prev = delta


@pytest.mark.parametrize("mu", [0.0, 0.1])
def test_deflated_sign_converges_to_the_exact_sign(mu):
    """Treating the k eigenpairs of H = g5 D_w smallest in magnitude exactly
    leaves the pole form only the rest of the spectrum, where 20 Neuberger poles
    are accurate: against the dense exact sign the error falls as k grows, and
    deflating every eigenpair gives the exact sign."""
    U = inputs.su3_exp_gauge(TINY, 0.5, 51)
    c = scale.power_scale(dirac.Operator(U, -1.8, mu).A, inputs.gaussian_spinor(TINY, 52), 100)
    op = dirac.Operator(U, -1.8, mu, c)
    b = inputs.gaussian_spinor(TINY, 53)
    Hm = overlap.dense_H(op)
    s_exact = (overlap.sign_dense(Hm) @ b.reshape(-1)).reshape(b.shape)
    Am = direct.dense_matrix(op.A, op.shape)
    om, sg = poles.neuberger_poles(20)

    def f(v):
        return direct.pfe_dense(Am, v, om, sg)

    errs = []
    for k in (0, 4, 16, 64):
        lam, R, Lv = overlap.smallest_eigenpairs(Hm, k, op.shape)
        errs.append(rel(overlap.sign_deflated(op, b, lam, R, Lv, f), s_exact))
    assert all(e1 < 0.7 * e0 for e0, e1 in zip(errs, errs[1:]))
    assert errs[0] > 1e-3 and errs[-1] < 1e-5
    lam, R, Lv = overlap.smallest_eigenpairs(Hm, Hm.shape[0], op.shape)
    assert rel(overlap.sign_deflated(op, b, lam, R, Lv, f), s_exact) < 1e-10
    d_ov = overlap.overlap_deflated(op, b, lam, R, Lv, f)
    assert rel(d_ov, b + dirac.gamma5(s_exact)) < 1e-10


@pytest.mark.parametrize("mu", [0.0, 0.15])
def test_free_field_sign_closed_form(mu):
    """U = 1 on 4^3 x 8: H(p)^2 = a(p)^2 + sum_nu s_nu(p)^2 is a scalar per mode,
    so sign(H) b = H (H^2)^{-1/2} b = sqrt(c) H [A^{-1/2} b] with A^{-1/2} applied
    mode by mode (principal root; FFT).  The oracle's pole form with Zolotarev
    poles for the interval the free spectrum spans (16 poles: uniform error at
    round-off there) and its overlap operator against it."""
    dims = (4, 4, 4, 8)
    U = inputs.unit_gauge(dims)
    lam = free_A_eigenvalues(dims, 1.0, mu, 1.0)
    c = 1.0 / np.abs(lam).max()
    op = dirac.Operator(U, 1.0, mu, c)
    b = inputs.gaussian_spinor(dims, 99)
    isqrt = free_matfunc(b, dims, 1.0, mu, c, lambda z: 1.0 / np.sqrt(z.astype(np.complex128)))
    s_exact = np.sqrt(c) * dirac.gamma5(op.D(isqrt))
    om, sg, delta = poles.zolotarev_poles(16, 0.99 * np.sqrt(np.abs(lam * c).min()))
    assert delta < 1e-13
    y = ms.multishift_double(op.A, b, sg, om, 2, 1e-13)
    assert rel(overlap.sign_apply(op, y), s_exact) < 1e-11
    assert rel(overlap.overlap_apply(op, b, y), b + dirac.gamma5(s_exact)) < 1e-11
