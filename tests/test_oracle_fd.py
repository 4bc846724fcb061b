"""Pins of the oracle's finite-difference operators (the derivatives of the
progressive use case, Sec. 5.3) against what the mathematics fixes: exact
derivatives of low-degree polynomials (second-order stencils are exact on
quadratics, the second-difference stencils on cubics), the vorticity of a
rigid rotation, agreement with numpy.gradient (an independent library
implementation of the same first-derivative formulas), and second-order
convergence on a smooth field.  A wrong coefficient, sign, axis or end
formula fails one of them."""
import numpy as np
import pytest

from oracle import derivatives as D


def _grid(shape, h):
    z, y, x = np.meshgrid(*(np.arange(n, dtype=np.float64) * h for n in shape), indexing="ij")
    return x, y, z


@pytest.mark.parametrize("h", [1.0, 0.5, 0.25])
def test_first_derivative_exact_on_quadratics(h):
    x, y, z = _grid((7, 6, 9), h)
    f = 3.0 + 2.0 * x - 5.0 * y + 0.5 * z + 1.5 * x * x - 2.0 * y * y + 0.25 * z * z + x * y - 3.0 * y * z
    assert np.array_equal(D.first_derivative(f, 0, h), 2.0 + 3.0 * x + y)
    assert np.array_equal(D.first_derivative(f, 1, h), -5.0 - 4.0 * y + x - 3.0 * z)
    assert np.array_equal(D.first_derivative(f, 2, h), 0.5 + 0.5 * z - 3.0 * y)


@pytest.mark.parametrize("h", [1.0, 0.5])
def test_second_derivative_exact_on_cubics(h):
    x, y, z = _grid((8, 5, 6), h)
    f = 1.0 + x * x * x - 2.0 * y * y * y + 0.5 * z * z * z + x * x * y + 3.0 * z * z
    assert np.array_equal(D.second_derivative(f, 0, h), 6.0 * x + 2.0 * y)
    assert np.array_equal(D.second_derivative(f, 1, h), -12.0 * y)
    assert np.array_equal(D.second_derivative(f, 2, h), 3.0 * z + 6.0)


def test_vorticity_of_rigid_rotation_and_shear():
    x, y, _ = _grid((4, 5, 6), 1.0)
    # rigid rotation u = -y, v = x: omega_z = 2 everywhere
    assert np.array_equal(D.vorticity_z(-y, x), np.full(x.shape, 2.0))
    # u = y^2, v = x^2: omega_z = 2x - 2y (exact on quadratics, ends included)
    assert np.array_equal(D.vorticity_z(y * y, x * x), 2.0 * x - 2.0 * y)
    # float32 fields are differentiated in float32 (exact here: small integers)
    u32, v32 = (y * y).astype(np.float32), (x * x).astype(np.float32)
    w = D.vorticity_z(u32, v32)
    assert w.dtype == np.float32 and np.array_equal(w, (2.0 * x - 2.0 * y).astype(np.float32))


def test_float32_fields_are_differentiated_in_float32():
    # one float32 rounding per operation: on random data some results differ
    # from the float64 computation rounded once, and all lie within a few
    # float32 ulps of it
    rng = np.random.default_rng(3)
    f = rng.standard_normal((6, 7, 1000)).astype(np.float32)
    for axis, fn in ((0, D.first_derivative), (2, D.second_derivative)):
        d32 = fn(f, axis, 0.1)
        d64 = fn(f.astype(np.float64), axis, 0.1)
        assert d32.dtype == np.float32
        assert (d32 != d64.astype(np.float32)).any()
        assert np.allclose(d32, d64, rtol=1e-4, atol=1e-4 * np.abs(d64).max())


def test_first_derivative_matches_numpy_gradient():
    rng = np.random.default_rng(7)
    f = rng.standard_normal((9, 11, 13))
    for axis in range(3):
        want = np.gradient(f, 0.5, axis=2 - axis, edge_order=2)
        assert np.allclose(D.first_derivative(f, axis, 0.5), want, rtol=0, atol=1e-12)


def test_second_order_convergence_on_a_smooth_field():
    errs1, errs2 = [], []
    for n in (32, 64, 128):
        h = 1.0 / (n - 1)
        t = np.arange(n) * h
        f = np.sin(2.0 * t) * np.ones((3, 3, 1))
        errs1.append(np.abs(D.first_derivative(f, 0, h) - 2.0 * np.cos(2.0 * t)).max())
        errs2.append(np.abs(D.second_derivative(f, 0, h) + 4.0 * np.sin(2.0 * t)).max())
    for e in (errs1, errs2):  # halving h divides the error by about 4
        assert 3.5 < e[0] / e[1] < 4.5 and 3.5 < e[1] / e[2] < 4.5


def test_too_few_points_are_refused():
    with pytest.raises(ValueError):
        D.first_derivative(np.zeros((4, 4, 2)), 0)
    with pytest.raises(ValueError):
        D.second_derivative(np.zeros((3, 4, 4)), 2)
