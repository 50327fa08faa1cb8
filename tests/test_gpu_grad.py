"""GPU adjoint gradient of L = Re <eta, f(A) b> (fa_grad, C-ABI): parity with the
FP64 oracle gradient, central finite differences on the 8^3 x 16 workload
(32 random su(3) link directions and mu, step 1e-5, target 1e-6), and the
torch.autograd.Function."""
import numpy as np
import pytest

import inputs
import paper_1010_2592_gb300 as fa
from fa_cases import make_context, rel, to_dev, to_host, workload_case
from oracle import grad as ograd

pytestmark = pytest.mark.gpu


def su3_direction(shape, rng):
    M = rng.standard_normal(shape + (3, 3)) + 1j * rng.standard_normal(shape + (3, 3))
    X = 0.5 * (M + np.conj(np.swapaxes(M, -1, -2)))
    return X - (np.trace(X, axis1=-2, axis2=-1) / 3.0)[..., None, None] * np.eye(3)


def directional(G, X, U):
    return float(np.real(np.sum(np.conj(G) * (1j * (X @ U)))))


def test_gradient_matches_oracle():
    w = workload_case("wilson_4x4x4x8")
    eta = inputs.gaussian_spinor(w["dims"], w["seeds"]["eta"])
    L_o, G_o, dmu_o, db_o = ograd.grad_f(w["U"], w["mass"], w["mu"], w["c"], w["b"], eta, w["omega"],
                                         w["sigma"], 2, 1e-12)
    ctx = make_context(w["dims"], w["U"], w["mass"], w["mu"], w["c"], w["t_bc"], w["omega"], w["sigma"])
    L, gU, dmu, gb, st = ctx.grad(to_dev(w["b"]), to_dev(eta), ell=2, tol=1e-12)
    assert abs(L - L_o) < 1e-11 * abs(L_o)
    assert rel(to_host(gU), G_o) < 1e-9
    assert abs(dmu - dmu_o) < 1e-9 * abs(dmu_o)
    assert rel(to_host(gb), db_o) < 1e-9
    assert st["n_mv"] > 0


def test_gradient_against_finite_differences_workload():
    name = "wilson_grad_8x8x8x16"
    w = inputs.make_workload(name)
    eta = inputs.gaussian_spinor(w["dims"], w["seeds"]["eta"])
    om, sg = fa.neuberger_poles(w["ns"])
    ctx = fa.Context(w["dims"])
    ctx.set_gauge(to_dev(w["U"]))
    ctx.set_params(w["mass"], w["mu"], w["t_bc"], 1.0)
    c = ctx.estimate_scale(to_dev(w["v0"]), 100)
    ctx.set_params(w["mass"], w["mu"], w["t_bc"], c)
    ctx.set_poles(om, sg)
    b, e = to_dev(w["b"]), to_dev(eta)
    tol, h = w["tol"], w["fd_step"]
    L0, gU, dmu, _, _ = ctx.grad(b, e, ell=w["ell"], tol=tol, want_db=False)
    G = to_host(gU)

    def Lval(U=None, mu=None):
        ctx.set_gauge(to_dev(U if U is not None else w["U"]))
        ctx.set_params(w["mass"], w["mu"] if mu is None else mu, w["t_bc"], c)
        y = to_host(ctx.apply_f(b, ell=w["ell"], tol=tol, mode="single", precision="f64").y)
        return float(np.real(np.vdot(eta, y)))

    fdm = (Lval(mu=w["mu"] + h) - Lval(mu=w["mu"] - h)) / (2 * h)
    assert abs(fdm - dmu) < 1e-6 * max(1.0, abs(fdm)), (fdm, dmu)
    rng = np.random.default_rng(77)
    worst = 0.0
    for _ in range(w["n_dirs"]):
        X = su3_direction(w["U"].shape[:-2], rng)
        Up = inputs.expi_hermitian(X, h) @ w["U"]
        Um = inputs.expi_hermitian(X, -h) @ w["U"]
        fd = (Lval(U=Up) - Lval(U=Um)) / (2 * h)
        worst = max(worst, abs(fd - directional(G, X, w["U"])) / max(1.0, abs(fd)))
    assert worst < 1e-6, worst


def test_autograd_function_matches_fa_grad():
    import torch
    from paper_1010_2592_gb300.autograd import FAFunction
    w = workload_case("wilson_4x4x4x8")
    eta = to_dev(inputs.gaussian_spinor(w["dims"], w["seeds"]["eta"]))
    ctx = make_context(w["dims"], w["U"], w["mass"], w["mu"], w["c"], w["t_bc"], w["omega"], w["sigma"])
    U = to_dev(w["U"]).requires_grad_(True)
    mu = torch.tensor(w["mu"], dtype=torch.float64, device="cuda", requires_grad=True)
    b = to_dev(w["b"]).requires_grad_(True)
    kw = dict(ell=2, tol=1e-12, mode="double", precision="f64")
    y = FAFunction.apply(U, mu, b, ctx, w["mass"], w["t_bc"], w["c"], kw)
    L = torch.real(torch.sum(torch.conj(eta) * y))
    L.backward()
    L2, gU, dmu, gb, _ = ctx.grad(to_dev(w["b"]), eta, ell=2, tol=1e-12)
    assert abs(L.item() - L2) < 1e-10 * abs(L2)
    assert rel(to_host(U.grad), to_host(gU)) < 1e-12
    assert abs(mu.grad.item() - dmu) < 1e-12 * abs(dmu)
    assert rel(to_host(b.grad), to_host(gb)) < 1e-12


@pytest.mark.parametrize("chunk", [1, 3, 4])
def test_chunked_gradient_equals_whole_and_bounds_memory(chunk):
    """shift_chunk = k: the poles are solved k at a time.  Every x_s and lambda_s
    comes from the same seed recurrence and the sums over s run in the same
    order, so L, dL/dU, dL/dmu and dL/db equal the all-poles result bit for bit;
    the lattice-sized device memory no longer grows with N_s (a fresh context
    with twice the poles holds the same field bytes)."""
    w = workload_case("wilson_4x4x4x8")
    eta = to_dev(inputs.gaussian_spinor(w["dims"], w["seeds"]["eta"]))
    b = to_dev(w["b"])
    ctx = make_context(w["dims"], w["U"], w["mass"], w["mu"], w["c"], w["t_bc"], w["omega"], w["sigma"])
    L0, g0, m0, b0, _ = ctx.grad(b, eta, ell=2, tol=1e-11)
    ctx = make_context(w["dims"], w["U"], w["mass"], w["mu"], w["c"], w["t_bc"], w["omega"], w["sigma"])
    L1, g1, m1, b1, st = ctx.grad(b, eta, ell=2, tol=1e-11, shift_chunk=chunk)
    assert L1 == L0 and m1 == m0
    assert np.array_equal(to_host(g1), to_host(g0))
    assert np.array_equal(to_host(b1), to_host(b0))
    assert st["status"] == 0
    fields = []
    for ns in (8, 16):
        om, sg = fa.neuberger_poles(ns)
        c2 = make_context(w["dims"], w["U"], w["mass"], w["mu"], w["c"], w["t_bc"], om, sg)
        c2.grad(b, eta, ell=2, tol=1e-10, shift_chunk=4)
        fields.append(c2.device_bytes()[0])
    assert fields[0] == fields[1]
