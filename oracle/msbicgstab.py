"""Multi-shift BiCGstab(l): single-pass and double-pass forms, plain FP64.

Test infrastructure (see the package docstring): not for the product path.

Seed system (Sec. 2, BiCGstab(l) of the cited Sleijpen-Fokkema paper), with
<a, b> = a^H b, x = 0, r_0 = b, shadow r~ = b, u_0 = 0, rho_0 = 1, alpha = 0,
omega = 1.  Outer iteration m: rho_0 <- -omega rho_0, then for j = 0..l-1
    rho_1 = <r~, r_j>,  beta = alpha rho_1 / rho_0,  rho_0 = rho_1
    u_i <- r_i - beta u_i                         (i = 0..j)
    u_{j+1} = A u_j,   alpha = rho_0 / <r~, u_{j+1}>
    r_i <- r_i - alpha u_{i+1}                    (i = 0..j)
    r_{j+1} = A r_j,   x <- x + alpha u_0
and the minimal-residual (MR) part: gamma_1..gamma_l minimise
|r_0 - sum_j gamma_j r_j| (normal equations), then
    x <- x + sum_j gamma_j r_{j-1},  r_0 <- r_0 - sum_j gamma_j r_j,
    u_0 <- u_0 - sum_j gamma_j u_j,  omega = gamma_l.
The residual polynomial of one MR step is p(t) = 1 - sum_j gamma_j t^j,
i.e. gamma_0 = -1 in the convention of Sec. 4.

Shifted systems (A + sigma_s) x_s = b share the Krylov space (Sec. 1,
shift invariance).  Each shift keeps x_s, u^s_0..u^s_l (u^s_i = A^i u^s_0)
and scalars zeta_s, zeta'_s with the collinearity r^s = r_0 / zeta_s.
BiCG sub-step j, after the seed's r-update (r_old = r before it):
    zeta_new = (1 + alpha sigma) zeta + (alpha beta / alpha_prev)(zeta' - zeta)
    alpha_s = alpha zeta / zeta_new,     beta_s = beta (zeta' / zeta)^2
    u^s_i <- r_old_i / zeta - beta_s u^s_i                  (i = 0..j)
    u^s_{j+1} <- (r_old_j / zeta - r_j / zeta_new) / alpha_s - sigma u^s_j
    x_s <- x_s + alpha_s u^s_0,   zeta' <- zeta,  zeta <- zeta_new
MR part, with the seed's r_0..r_{l-1} before its MR update:
    p_s = p(-sigma),  c_k = sum_{j=k+1}^{l} gamma_j (-sigma)^{j-1-k}
    x_s <- x_s + (zeta p_s)^{-1} sum_k c_k r_k
    u^s_0 <- (u^s_0 - sum_j gamma_j u^s_j) / p_s,  zeta <- zeta p_s, zeta' <- zeta' p_s
(c_k are the coefficients of (p(-sigma) - p(t)) / (t + sigma).)  A shift is
frozen after the outer iteration at which |r_0| / |zeta_s| <= tol |b|.

Double-pass (Sec. 2, Eqs. 2-3, option 1): every shift vector is a linear
combination of the unshifted iteration vectors v^(i) (Eq. 3).  Pass 1 runs
the seed recurrence with the shift scalars only and resolves the recursion
of each x_s into coefficients gamma_{s,i} over the list of seed-vector
occurrences (r_old_0..r_old_j and r_j in each sub-step, r_0..r_{l-1} in each
MR step); the weighted sums gamma_i = sum_s omega_s gamma_{s,i} are kept.
Pass 2 regenerates the v^(i) with the recorded scalars and forms
sum_i gamma_i v^(i) without any shift-dependent vector.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Record:
    """Scalars of pass 1: alpha, beta per BiCG sub-step, gamma_1..gamma_l per MR."""
    ell: int
    alpha: list = field(default_factory=list)   # [m][j]
    beta: list = field(default_factory=list)    # [m][j]
    gamma: list = field(default_factory=list)   # [m][0..l], gamma[m][0] = -1

    @property
    def n_outer(self):
        return len(self.gamma)


@dataclass
class Stats:
    n_outer: int = 0
    n_mv: int = 0
    n_dot: int = 0
    iters_per_shift: np.ndarray | None = None


def _vdot(a, b):
    return np.vdot(a, b)    # a^H b


def seed_recurrence(A, b, ell, max_outer, substep=None, mr=None, end_outer=None,
                    replay=None, round_vec=None, stats=None):
    """Run the seed BiCGstab(l) recurrence (module docstring), calling hooks.

    substep(m, j, alpha, beta, r_old, r_j)  after the sub-step (r_old: list j+1)
    mr(m, gamma, r_pre)                      before the MR vector update (r_pre: l)
    end_outer(m, r_0) -> bool                after the MR update; False stops.
    With `replay` (a Record), alpha, beta and gamma are taken from it and no
    inner products are formed (pass 2 of the double-pass form).
    Returns (x, record).
    """
    rv = round_vec if round_vec is not None else (lambda v: v)
    st = stats if stats is not None else Stats()
    zero = np.zeros_like(b)
    r = [rv(b.copy())] + [zero] * ell
    u = [zero] * (ell + 1)
    rt = r[0].copy()
    x = zero.copy()
    rho0, alpha, omega = 1.0 + 0j, 0.0 + 0j, 1.0 + 0j
    rec = Record(ell)
    n_outer = replay.n_outer if replay is not None else max_outer
    for m in range(n_outer):
        rho0 = -omega * rho0
        alphas, betas = [], []
        for j in range(ell):
            if replay is None:
                rho1 = _vdot(rt, r[j])
                st.n_dot += 1
                beta = alpha * rho1 / rho0
                rho0 = rho1
            else:
                beta = replay.beta[m][j]
            for i in range(j + 1):
                u[i] = rv(r[i] - beta * u[i])
            u[j + 1] = rv(A(u[j]))
            st.n_mv += 1
            if replay is None:
                den = _vdot(rt, u[j + 1])
                st.n_dot += 1
                if den == 0:
                    raise FloatingPointError("BiCG breakdown: <r~, A u_j> = 0")
                alpha = rho0 / den
            else:
                alpha = replay.alpha[m][j]
            r_old = [r[i] for i in range(j + 1)]
            for i in range(j + 1):
                r[i] = rv(r[i] - alpha * u[i + 1])
            r[j + 1] = rv(A(r[j]))
            st.n_mv += 1
            x = x + alpha * u[0]
            alphas.append(alpha)
            betas.append(beta)
            if substep is not None:
                substep(m, j, alpha, beta, r_old, r[j])
        # MR part: normal equations G gamma = g over r_1..r_l
        if replay is None:
            G = np.empty((ell, ell), dtype=np.complex128)
            g = np.empty(ell, dtype=np.complex128)
            for i in range(1, ell + 1):
                for k in range(1, ell + 1):
                    G[i - 1, k - 1] = _vdot(r[i], r[k])
                g[i - 1] = _vdot(r[i], r[0])
            st.n_dot += ell * (ell + 1) // 2 + ell
            gam = np.concatenate([[-1.0 + 0j], np.linalg.solve(G, g)])
        else:
            gam = np.asarray(replay.gamma[m])
        if mr is not None:
            mr(m, gam, [r[k] for k in range(ell)])
        x = x + sum(gam[j] * r[j - 1] for j in range(1, ell + 1))
        r[0] = rv(r[0] - sum(gam[j] * r[j] for j in range(1, ell + 1)))
        u[0] = rv(u[0] - sum(gam[j] * u[j] for j in range(1, ell + 1)))
        omega = gam[ell]
        rec.alpha.append(alphas)
        rec.beta.append(betas)
        rec.gamma.append(list(gam))
        st.n_outer = m + 1
        if end_outer is not None:
            if replay is None:
                st.n_dot += 1
            if not end_outer(m, r[0]):
                break
    return x, rec


def bicgstab_ell(A, b, ell, tol, max_outer=10000, stats=None):
    """Seed BiCGstab(l) on A x = b alone; stops at |r_0| <= tol |b|."""
    bn = np.linalg.norm(b)
    x, rec = seed_recurrence(A, b, ell, max_outer, stats=stats,
                             end_outer=lambda m, r0: np.linalg.norm(r0) > tol * bn)
    return x, rec


class _ShiftScalars:
    """zeta_s, zeta'_s and the per-step shift coefficients (module docstring)."""

    def __init__(self, sigma, tol, bnorm):
        self.sigma = np.asarray(sigma, dtype=np.float64)
        ns = len(self.sigma)
        self.zeta = np.ones(ns, dtype=np.complex128)
        self.zeta_p = np.ones(ns, dtype=np.complex128)
        self.alpha_prev = 1.0 + 0j
        self.active = np.ones(ns, dtype=bool)
        self.iters = np.zeros(ns, dtype=np.int64)
        self.tol, self.bnorm = tol, bnorm

    def bicg(self, s, alpha, beta):
        sg, z, zp = self.sigma[s], self.zeta[s], self.zeta_p[s]
        zn = (1.0 + alpha * sg) * z + (alpha * beta / self.alpha_prev) * (zp - z)
        return zn, alpha * z / zn, beta * (zp / z) ** 2

    def mr(self, s, gam):
        ell = len(gam) - 1
        ms = -self.sigma[s]
        ps = 1.0 - sum(gam[j] * ms ** j for j in range(1, ell + 1))
        c = [sum(gam[j] * ms ** (j - 1 - k) for j in range(k + 1, ell + 1)) for k in range(ell)]
        return ps, c

    def converge(self, m, r0, last=False):
        """Freeze the shifts whose residual |r_0| / |zeta_s| is below tol |b|; with
        `last` (the final outer iteration of a fixed-cost run) freeze all."""
        rn = np.linalg.norm(r0)
        for s in np.flatnonzero(self.active):
            if last or rn / abs(self.zeta[s]) <= self.tol * self.bnorm:
                self.active[s] = False
                self.iters[s] = m + 1
        return bool(self.active.any())


def _stopper(sh, fixed_outer):
    """end_outer hook: the convergence test, and for a fixed-cost run the
    freezing of every remaining shift after outer iteration fixed_outer."""
    if fixed_outer is None:
        return sh.converge
    return lambda m, r0: sh.converge(m, r0, last=m + 1 >= fixed_outer)


def multishift_single(A, b, sigma, ell, tol, max_outer=10000, round_vec=None, stats=None,
                      observer=None, fixed_outer=None):
    """Single-pass multi-shift BiCGstab(l): returns the list of x_s.

    observer(m, r_0, xs, zeta, active), if given, is called after every outer
    iteration before the convergence test (used to check invariants).
    fixed_outer = M: a fixed-cost run (the setting of Sec. 3, Fig. 2): at most M
    outer iterations; shifts still active after the M-th are frozen there
    instead of raising.
    """
    st = stats if stats is not None else Stats()
    sh = _ShiftScalars(sigma, tol, np.linalg.norm(b))
    ns = len(sh.sigma)
    zero = np.zeros_like(b)
    xs = [zero.copy() for _ in range(ns)]
    us = [[zero.copy() for _ in range(ell + 1)] for _ in range(ns)]

    def substep(m, j, alpha, beta, r_old, r_j):
        for s in np.flatnonzero(sh.active):
            zn, a_s, b_s = sh.bicg(s, alpha, beta)
            z = sh.zeta[s]
            for i in range(j + 1):
                us[s][i] = r_old[i] / z - b_s * us[s][i]
            us[s][j + 1] = (r_old[j] / z - r_j / zn) / a_s - sh.sigma[s] * us[s][j]
            xs[s] = xs[s] + a_s * us[s][0]
            sh.zeta_p[s], sh.zeta[s] = z, zn
        sh.alpha_prev = alpha

    def mr(m, gam, r_pre):
        for s in np.flatnonzero(sh.active):
            ps, c = sh.mr(s, gam)
            xs[s] = xs[s] + sum(c[k] * r_pre[k] for k in range(ell)) / (sh.zeta[s] * ps)
            us[s][0] = (us[s][0] - sum(gam[j] * us[s][j] for j in range(1, ell + 1))) / ps
            sh.zeta[s] *= ps
            sh.zeta_p[s] *= ps

    stop = _stopper(sh, fixed_outer)

    def end_outer(m, r0):
        if observer is not None:
            observer(m, r0, xs, sh.zeta.copy(), sh.active.copy())
        return stop(m, r0)

    n = max_outer if fixed_outer is None else fixed_outer
    seed_recurrence(A, b, ell, n, substep, mr, end_outer, round_vec=round_vec, stats=st)
    st.iters_per_shift = sh.iters.copy()
    if sh.active.any():
        raise RuntimeError("multishift_single: not converged within max_outer")
    return xs


def _occurrences_per_outer(ell):
    return ell * (ell + 1) // 2 + ell + ell


def multishift_double(A, b, sigma, omega, ell, tol, max_outer=10000, round_vec=None,
                      stats=None, return_coefficients=False, fixed_outer=None):
    """Double-pass multi-shift BiCGstab(l): returns y = sum_s omega_s x_s.
    fixed_outer: a fixed-cost run, as in multishift_single."""
    st = stats if stats is not None else Stats()
    sh = _ShiftScalars(sigma, tol, np.linalg.norm(b))
    if fixed_outer is not None:
        max_outer = fixed_outer
    ns = len(sh.sigma)
    cap = max_outer * _occurrences_per_outer(ell)
    CX = np.zeros((ns, cap), dtype=np.complex128)            # x_s  = sum_i CX[s, i] v^(i)
    CU = np.zeros((ns, ell + 1, cap), dtype=np.complex128)   # u^s_k = sum_i CU[s, k, i] v^(i)
    n_occ = [0]

    # ---- pass 1: seed recurrence, shift scalars, resolved recursion (Eq. 3)
    def substep(m, j, alpha, beta, r_old, r_j):
        ids_old = n_occ[0] + np.arange(j + 1)
        id_new = n_occ[0] + j + 1
        n_occ[0] += j + 2
        n = n_occ[0]
        for s in np.flatnonzero(sh.active):
            zn, a_s, b_s = sh.bicg(s, alpha, beta)
            z = sh.zeta[s]
            for i in range(j + 1):
                CU[s, i, :n] *= -b_s
                CU[s, i, ids_old[i]] += 1.0 / z
            CU[s, j + 1, :n] = -sh.sigma[s] * CU[s, j, :n]
            CU[s, j + 1, ids_old[j]] += 1.0 / (a_s * z)
            CU[s, j + 1, id_new] -= 1.0 / (a_s * zn)
            CX[s, :n] += a_s * CU[s, 0, :n]
            sh.zeta_p[s], sh.zeta[s] = z, zn
        sh.alpha_prev = alpha

    def mr(m, gam, r_pre):
        ids = n_occ[0] + np.arange(ell)
        n_occ[0] += ell
        n = n_occ[0]
        for s in np.flatnonzero(sh.active):
            ps, c = sh.mr(s, gam)
            for k in range(ell):
                CX[s, ids[k]] += c[k] / (sh.zeta[s] * ps)
            CU[s, 0, :n] = (CU[s, 0, :n] - sum(gam[j] * CU[s, j, :n]
                                                for j in range(1, ell + 1))) / ps
            sh.zeta[s] *= ps
            sh.zeta_p[s] *= ps

    _, rec = seed_recurrence(A, b, ell, max_outer, substep, mr, _stopper(sh, fixed_outer),
                             round_vec=round_vec, stats=st)
    st.iters_per_shift = sh.iters.copy()
    if sh.active.any():
        raise RuntimeError("multishift_double: not converged within max_outer")
    coef = np.asarray(omega, dtype=np.complex128) @ CX[:, :n_occ[0]]

    # ---- pass 2: regenerate the v^(i) with the recorded scalars, sum gamma_i v^(i)
    y = np.zeros_like(b)
    pos = [0]

    def substep2(m, j, alpha, beta, r_old, r_j):
        nonlocal y
        for i in range(j + 1):
            y = y + coef[pos[0] + i] * r_old[i]
        y = y + coef[pos[0] + j + 1] * r_j
        pos[0] += j + 2

    def mr2(m, gam, r_pre):
        nonlocal y
        for k in range(ell):
            y = y + coef[pos[0] + k] * r_pre[k]
        pos[0] += ell

    seed_recurrence(A, b, ell, max_outer, substep2, mr2, replay=rec,
                    round_vec=round_vec, stats=st)
    assert pos[0] == n_occ[0]
    if return_coefficients:
        return y, coef, rec
    return y


def pfe_from_shifts(xs, omega):
    """sum_s omega_s x_s (Eq. 1 with the per-shift solutions)."""
    return sum(w * x for w, x in zip(omega, xs))
