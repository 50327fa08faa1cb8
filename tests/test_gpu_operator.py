"""GPU parity of the Wilson-Dirac hop kernels and A = c (g5 D)^2 (C-ABI)
against the FP64 oracle, element by element."""
import numpy as np
import pytest

import inputs
from oracle import dirac, scale
from closed_forms import free_dw
from fa_cases import make_context, rel, to_dev, to_host

pytestmark = pytest.mark.gpu

# lattices spanning one partial block, several blocks with a ragged tail, and
# the multi-block workload shapes
SHAPES = [(3, 3, 3, 6), (6, 4, 6, 10), (4, 4, 4, 8), (8, 8, 8, 16)]
TOL = {"f64": 1e-13, "f32": 5e-6, "df": 1e-11}


@pytest.fixture(scope="module", params=SHAPES, ids=lambda d: "x".join(map(str, d)))
def case(request):
    dims = request.param
    U = inputs.su3_exp_gauge(dims, 0.5, 101)
    psi = inputs.gaussian_spinor(dims, 102)
    return dims, U, psi


@pytest.mark.parametrize("precision", ["f64", "f32", "df"])
@pytest.mark.parametrize("mu,t_bc", [(0.05, -1), (0.0, 1), (0.3, -1)])
def test_dw_matches_oracle(case, precision, mu, t_bc):
    dims, U, psi = case
    ctx = make_context(dims, U, -1.8, mu, 1.0, t_bc)
    got = to_host(ctx.apply_dw(to_dev(psi), precision=precision))
    want = dirac.dw(U, psi, -1.8, mu, t_bc)
    assert rel(got, want) < TOL[precision]
    gotd = to_host(ctx.apply_dw(to_dev(psi), dagger=True, precision=precision))
    wantd = dirac.dw_dagger(U, psi, -1.8, mu, t_bc)
    assert rel(gotd, wantd) < TOL[precision]


@pytest.mark.parametrize("precision", ["f64", "f32", "df"])
def test_A_matches_oracle(case, precision):
    dims, U, psi = case
    ctx = make_context(dims, U, -1.8, 0.1, 0.037)
    got = to_host(ctx.apply_A(to_dev(psi), precision=precision))
    assert rel(got, dirac.apply_A(U, psi, -1.8, 0.1, 0.037)) < TOL[precision]
    gotd = to_host(ctx.apply_A(to_dev(psi), dagger=True, precision=precision))
    assert rel(gotd, dirac.apply_A_dagger(U, psi, -1.8, 0.1, 0.037)) < TOL[precision]


def test_dw_free_field_full_size_closed_form():
    """16^3 x 32 (the bench lattice) with U = 1 against the FFT closed form."""
    dims = (16, 16, 16, 32)
    psi = inputs.gaussian_spinor(dims, 103)
    ctx = make_context(dims, inputs.unit_gauge(dims), -1.8, 0.1, 1.0)
    want = free_dw(psi, dims, -1.8, 0.1)
    assert rel(to_host(ctx.apply_dw(to_dev(psi))), want) < 1e-13
    assert rel(to_host(ctx.apply_dw(to_dev(psi), precision="f32")), want) < TOL["f32"]


def test_dw_full_size_sampled_sites():
    """16^3 x 32 random gauge field: sampled output sites against the oracle."""
    dims = (16, 16, 16, 32)
    U = inputs.su3_exp_gauge(dims, 0.4, 1001)
    psi = inputs.gaussian_spinor(dims, 1002)
    ctx = make_context(dims, U, -1.8, 0.1, 1.0)
    got = to_host(ctx.apply_dw(to_dev(psi)))
    got32 = to_host(ctx.apply_dw(to_dev(psi), precision="f32"))
    want = dirac.dw(U, psi, -1.8, 0.1)
    rng = np.random.default_rng(7)
    idx = tuple(rng.integers(0, n, 256) for n in want.shape[:4])
    assert rel(got[idx], want[idx]) < 1e-13
    assert rel(got32[idx], want[idx]) < TOL["f32"]
    assert rel(got, want) < 1e-13


def test_estimate_scale_matches_oracle():
    dims = (4, 4, 4, 8)
    U = inputs.su3_exp_gauge(dims, 0.5, 1000)
    v0 = inputs.gaussian_spinor(dims, 1003)
    ctx = make_context(dims, U, -1.8, 0.05, 1.0)
    c = ctx.estimate_scale(to_dev(v0), 100)
    op = dirac.Operator(U, -1.8, 0.05, 1.0)
    assert abs(c - scale.power_scale(op.A, v0, 100)) < 1e-10 * c


def test_launches_are_counted():
    dims = (4, 4, 4, 8)
    ctx = make_context(dims, inputs.su3_exp_gauge(dims, 0.5, 1), -1.8, 0.0, 1.0)
    n0 = ctx.launch_count()
    ctx.apply_A(to_dev(inputs.gaussian_spinor(dims, 2)))
    assert ctx.launch_count() >= n0 + 2
