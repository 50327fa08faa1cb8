"""The seeded input generators shared by the oracle tests and the GPU tests:
deterministic, the documented shapes and structure, and different seeds give
different fields."""
import numpy as np
import pytest

import inputs


def test_generators_are_deterministic_and_seed_dependent():
    dims = (2, 3, 2, 4)
    a = inputs.su3_exp_gauge(dims, 0.5, 7)
    assert np.array_equal(a, inputs.su3_exp_gauge(dims, 0.5, 7))
    assert not np.allclose(a, inputs.su3_exp_gauge(dims, 0.5, 8))
    s = inputs.gaussian_spinor(dims, 3)
    assert np.array_equal(s, inputs.gaussian_spinor(dims, 3))
    assert not np.allclose(s, inputs.gaussian_spinor(dims, 4))


def test_shapes_and_link_structure():
    dims = (2, 3, 2, 4)
    U = inputs.su3_exp_gauge(dims, 0.4, 11)
    assert U.shape == (4, 2, 3, 2, 4, 3, 3) and U.dtype == np.complex128
    I = np.eye(3)
    assert np.allclose(U @ np.conj(np.swapaxes(U, -1, -2)), I, atol=1e-13)
    assert np.allclose(np.linalg.det(U), 1.0, atol=1e-13)
    # exp(i eps H) with |H| = O(1): links stay near the unit matrix for small eps
    assert np.abs(inputs.su3_exp_gauge(dims, 1e-3, 11) - I).max() < 1e-2
    assert inputs.gaussian_spinor(dims, 1).shape == (4, 2, 3, 2, 4, 3)
    p = inputs.point_source(dims, 2, 1, site=(1, 2, 0, 3))
    assert p.sum() == 1.0 and p[3, 0, 2, 1, 2, 1] == 1.0


def test_pure_gauge_is_a_gauge_transform_of_the_unit_field():
    dims = (2, 2, 2, 4)
    g = inputs.random_su3_field(dims, 5)
    assert np.allclose(inputs.pure_gauge(g), inputs.gauge_transform(inputs.unit_gauge(dims), g))


@pytest.mark.parametrize("name", ["wilson_4x4x4x8", "wilson_16x16x16x32", "wilson_grad_8x8x8x16",
                                  "wilson_32x32x32x64"])
def test_workload_metadata(name):
    w = inputs.WORKLOADS[name]
    for key in ("dims", "eps", "mu", "mass", "ell", "ns"):
        assert key in w, key
    assert inputs.workload_seeds(name) == inputs.workload_seeds(name)
