"""sign(g5 D_w(mu)) b and the overlap operator D_ov(mu) b (Sec. 1) on the GPU
against the FP64 oracle (same pole expansion), and the Ginsparg-Wilson
relation of the GPU's D_ov."""
import numpy as np
import pytest

import inputs
import paper_1010_2592_gb300 as fa
from fa_cases import make_context, oracle_double, rel, to_dev, to_host, workload_case
from oracle import dirac, overlap, scale

pytestmark = pytest.mark.gpu

C1 = "wilson_4x4x4x8"


@pytest.mark.parametrize("mode,precision,tol", [("double", "f64", 1e-9), ("single", "f64", 1e-9),
                                                ("pseudo", "mixed_df", 1e-6), ("double", "f32", 1e-4)])
def test_sign_and_overlap_match_oracle(mode, precision, tol):
    w = workload_case(C1)
    ctx = make_context(w["dims"], w["U"], w["mass"], w["mu"], w["c"], w["t_bc"], w["omega"], w["sigma"])
    op = dirac.Operator(w["U"], w["mass"], w["mu"], w["c"], w["t_bc"])
    y, _ = oracle_double(C1, None, 2, 1e-12)
    b = to_dev(w["b"])
    solver_tol = 1e-12 if precision == "f64" else 1e-10
    kw = dict(ell=2, tol=solver_tol, mode=mode, precision=precision)
    r = ctx.apply_sign(b, **kw)
    assert r.stats["status"] == 0
    assert rel(to_host(r.y), overlap.sign_apply(op, y)) < tol
    r = ctx.apply_overlap(b, **kw)
    assert rel(to_host(r.y), overlap.overlap_apply(op, w["b"], y)) < tol
    # the input is left as it was
    assert np.array_equal(to_host(b), w["b"])


def test_overlap_ginsparg_wilson_relation_on_gpu():
    """g5 D_ov + D_ov g5 = D_ov g5 D_ov (sign(H)^2 = 1) for the GPU's D_ov on
    a lattice where 32 poles resolve the spectrum of A (Wilson mass 1)."""
    dims = (4, 4, 4, 8)
    U = inputs.su3_exp_gauge(dims, 0.5, 91)
    mu = 0.1
    c = scale.power_scale(dirac.Operator(U, 1.0, mu).A, inputs.gaussian_spinor(dims, 92), 100)
    om, sg = fa.neuberger_poles(32)
    ctx = make_context(dims, U, 1.0, mu, c, -1, om, sg)
    g5 = dirac.gamma5
    b = inputs.gaussian_spinor(dims, 93)

    def D(v):
        return to_host(ctx.apply_overlap(to_dev(v), ell=2, tol=1e-12, precision="f64").y)

    Db = D(b)
    lhs = g5(Db) + D(g5(b))
    rhs = D(g5(Db))
    assert rel(lhs, rhs) < 1e-9


def test_sign_argument_errors():
    w = workload_case(C1)
    ctx = make_context(w["dims"], w["U"], w["mass"], w["mu"], w["c"], w["t_bc"], w["omega"], w["sigma"])
    b = to_dev(w["b"])
    with pytest.raises(fa.FAError) as e:
        ctx.apply_sign(b, out=b)
    assert e.value.status == fa.FA_EINVAL
    bare = fa.Context(w["dims"])
    bare.set_gauge(to_dev(w["U"]))
    bare.set_params(w["mass"], w["mu"], w["t_bc"], w["c"])
    with pytest.raises(fa.FAError) as e:
        bare.apply_overlap(b)
    assert e.value.status == fa.FA_ESTATE


@pytest.mark.parametrize("overlap_op", [False, True])
def test_deflated_sign_matches_oracle(overlap_op):
    """k = 8 eigenpairs of H (dense eigendecomposition of the oracle's H on a
    3^3 x 6 lattice) treated exactly, the rest by the pole form: the GPU against
    the oracle's deflated form with the same eigenpairs and poles."""
    import torch
    dims = (3, 3, 3, 6)
    U = inputs.su3_exp_gauge(dims, 0.5, 95)
    mu = 0.1
    c = scale.power_scale(dirac.Operator(U, -1.8, mu).A, inputs.gaussian_spinor(dims, 96), 100)
    op = dirac.Operator(U, -1.8, mu, c)
    om, sg = fa.neuberger_poles(20)
    b = inputs.gaussian_spinor(dims, 97)
    lam, R, Lv = overlap.smallest_eigenpairs(overlap.dense_H(op), 8, op.shape)
    from oracle import msbicgstab as ms

    def f(v):
        return ms.multishift_double(op.A, v, sg, om, 2, 1e-12)

    if overlap_op:
        want = overlap.overlap_deflated(op, b, lam, R, Lv, f)
    else:
        want = overlap.sign_deflated(op, b, lam, R, Lv, f)
    ctx = make_context(dims, U, -1.8, mu, c, -1, om, sg)
    Rd = torch.from_numpy(np.ascontiguousarray(np.stack(R))).cuda()
    Ld = torch.from_numpy(np.ascontiguousarray(np.stack(Lv))).cuda()
    r = ctx.apply_sign_deflated(to_dev(b), lam, Rd, Ld, overlap=overlap_op, ell=2, tol=1e-12, precision="f64")
    assert r.stats["status"] == 0
    assert rel(to_host(r.y), want) < 1e-9
    # k = 0 is the plain sign / overlap
    r0 = ctx.apply_sign_deflated(to_dev(b), np.zeros(0), Rd[:0], Ld[:0], overlap=overlap_op, ell=2, tol=1e-12,
                                 precision="f64")
    plain = (ctx.apply_overlap if overlap_op else ctx.apply_sign)(to_dev(b), ell=2, tol=1e-12, precision="f64")
    assert np.array_equal(to_host(r0.y), to_host(plain.y))
