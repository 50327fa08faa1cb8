"""Plain FP64 CPU oracle for f(A)b = sum_s omega_s (A + sigma_s)^{-1} b.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path imports this package:
only the test-suite, `__graft_entry__.smoke()` and the CPU-baseline leg of
`bench.py` may import or run it.  It shares no code with the CUDA library
(`paper_1010_2592_gb300/csrc`): the two meet only through the seeded input
generators in `inputs/`.

Modules
    dirac      Wilson-Dirac operator D_w(mu), gamma_5, A = c (gamma_5 D_w)^2
    poles      Neuberger and Zolotarev partial-fraction poles {omega_s, sigma_s}, Eq. (1)
    msbicgstab BiCGstab(l) seed recurrence, single-pass multi-shift, and the
               double-pass form of Sec. 2 (Eqs. 2-3)
    direct     y* by per-shift library solves, dense LU and eigendecomposition
    scale      power-iteration estimate of the largest eigenvalue of A
    overlap    sign(gamma_5 D_w) b and the overlap operator D_ov(mu) b of Sec. 1,
               deflated by exactly treated eigenpairs
    grad       gradient of L = Re <eta, f(A) b> with respect to the links and mu

Parity status: every function is pinned by the `-m "not gpu"` tests except
the closed-form double-pass coefficients of Sec. 4 (A_mj, B_m^s, D, E, F, G,
M^m): their symbols are defined only in the cited listing of shifted
BiCGstab(l), which is not available, so they are not implemented here
(parity unpinned; the double-pass weights are instead obtained by resolving
the recursion of Eq. 3 directly).
"""
