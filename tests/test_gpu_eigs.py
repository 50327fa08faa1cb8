"""The deflation eigensolver (fa_eigs_smallest): the k eigenpairs of
H = gamma_5 D_w(mu) smallest in magnitude, right and left eigenvectors, against
the dense eigendecomposition of the oracle's H on a 3^3 x 6 lattice, and fed to
the deflated sign function (Sec. 3, Figs. 3 and 4)."""
import numpy as np
import pytest

import inputs
import paper_1010_2592_gb300 as fa
from fa_cases import make_context, rel, to_dev, to_host
from oracle import dirac, overlap, scale

pytestmark = pytest.mark.gpu


def setup(dims=(3, 3, 3, 6), seed=95, mu=0.1):
    U = inputs.su3_exp_gauge(dims, 0.5, seed)
    c = scale.power_scale(dirac.Operator(U, -1.8, mu).A, inputs.gaussian_spinor(dims, seed + 1), 100)
    op = dirac.Operator(U, -1.8, mu, c)
    om, sg = fa.neuberger_poles(20)
    ctx = make_context(dims, U, -1.8, mu, c, -1, om, sg)
    return op, ctx, om, sg


@pytest.mark.parametrize("mu", [0.0, 0.1])
def test_smallest_eigenpairs_against_dense(mu):
    """Eigenvalues equal to the dense ones (the k smallest in magnitude),
    eigen-residuals |H r - lambda r| and |H^H l - conj(lambda) l| at the solver's
    accuracy, and L^H R = 1 (biorthonormal left and right eigenvectors)."""
    op, ctx, _, _ = setup(mu=mu)
    k = 6
    lam, R, Lv, info = ctx.eigs_smallest(k, m=24, tol=1e-11, ell=2, precision="f64")
    assert info["status"] == 0 and info["converged"] == k and info["solves"] > 0
    Hm = overlap.dense_H(op)
    lam_d = np.linalg.eigvals(Hm)
    want = lam_d[np.argsort(np.abs(lam_d))[:k]]
    for x in lam:
        assert np.min(np.abs(want - x)) < 1e-8 * np.abs(x), (x, want)
    assert np.max(np.abs(lam)) <= np.sort(np.abs(lam_d))[k - 1] * (1 + 1e-8)
    Rh, Lh = to_host(R).reshape(k, -1), to_host(Lv).reshape(k, -1)
    for i in range(k):
        r, l = Rh[i], Lh[i]
        assert np.linalg.norm(Hm @ r - lam[i] * r) < 1e-8 * np.abs(lam[i]) * np.linalg.norm(r)
        assert np.linalg.norm(Hm.conj().T @ l - np.conj(lam[i]) * l) < 1e-8 * np.abs(lam[i]) * np.linalg.norm(l)
    # off the diagonal: eigenvector errors over eigenvalue gaps
    G = Lh.conj() @ Rh.T
    assert np.max(np.abs(G - np.eye(k))) < 1e-7


def test_eigensolver_feeds_the_deflated_sign():
    """sign(H) b with the solver's eigenpairs equals the oracle's deflated sign
    with the dense eigenpairs (the deflated form depends on the pairs only
    through the oblique projector, which both reproduce)."""
    import torch
    from oracle import msbicgstab as ms
    op, ctx, om, sg = setup()
    k = 8
    lam, R, Lv, _ = ctx.eigs_smallest(k, tol=1e-11, ell=2, precision="f64")
    b = inputs.gaussian_spinor((3, 3, 3, 6), 97)
    lam_d, R_d, L_d = overlap.smallest_eigenpairs(overlap.dense_H(op), k, op.shape)

    def f(v):
        return ms.multishift_double(op.A, v, sg, om, 2, 1e-12)

    want = overlap.sign_deflated(op, b, lam_d, R_d, L_d, f)
    r = ctx.apply_sign_deflated(to_dev(b), lam, R, Lv, ell=2, tol=1e-12, precision="f64")
    assert r.stats["status"] == 0
    assert rel(to_host(r.y), want) < 1e-8
    # the context's poles are untouched by the eigensolver
    plain = ctx.apply_sign(to_dev(b), ell=2, tol=1e-12, precision="f64")
    y = ms.multishift_double(op.A, b, sg, om, 2, 1e-12)
    assert rel(to_host(plain.y), overlap.sign_apply(op, y)) < 1e-9
    assert torch.is_tensor(R) and R.shape[0] == k


def test_eigensolver_argument_errors():
    op, ctx, _, _ = setup()
    with pytest.raises(fa.FAError) as e:
        ctx.eigs_smallest(4, m=5)              # m < k + 2
    assert e.value.status == fa.FA_EINVAL
    with pytest.raises(fa.FAError) as e:
        ctx.eigs_smallest(0)
    assert e.value.status == fa.FA_EINVAL
