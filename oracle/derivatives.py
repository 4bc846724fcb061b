"""Finite-difference derivatives of a field on a regular grid: the operators
of the paper's progressive use case (Sec. 5.3).  There the third component
v_x - u_y of the vorticity of a velocity field u = (u, v, w), and the second
derivative w_zz, are computed from progressive reconstructions; a derivative
of order i magnifies the reconstruction error like h^-i, so each needs a
finer tolerance (more components) than the one before.

TEST INFRASTRUCTURE ONLY: imported by tests/ and by bench.py's CPU legs; the
product package never imports it.

The paper names the operators, not their stencils.  The reading used here:
second-order differences at every grid point -- central in the interior, the
second-order one-sided formulas at the two ends of the differentiated axis
(three points for a first derivative, four for a second) -- evaluated in the
field's own precision (as the method's sums are, Sec. 3: "the precision used
for x"), one IEEE rounding per operation in exactly the order written below,
with h first rounded to that type.  Arrays are (nz, ny, nx) in C order (or
(ny, nx), (nx,)); axis 0 is x, the fastest, as in the C ABI.  Parity pinned
by tests/test_oracle_fd.py (exactness on polynomials, the vorticity of rigid
rotation, agreement with numpy.gradient, second-order convergence on smooth
fields).
"""
import numpy as np


def _to_last(g, axis):
    """View with grid axis `axis` (0 = x, the last numpy axis) moved last."""
    return np.moveaxis(g, g.ndim - 1 - axis, -1)


def _from_last(g, axis):
    return np.moveaxis(g, -1, g.ndim - 1 - axis)


def _field(f):
    g = np.asarray(f)
    if g.dtype not in (np.float32, np.float64):
        raise ValueError("fields are float32 or float64")
    return g


def first_derivative(f, axis, h=1.0):
    """df/da in the field's type: (f[i+1] - f[i-1]) / (2h) inside; at the ends
    ((4 f1 - 3 f0) - f2) / (2h) and ((3 f[n-1] - 4 f[n-2]) + f[n-3]) / (2h).
    Needs at least 3 points along the axis."""
    g = _to_last(_field(f), axis)
    T = g.dtype.type
    n = g.shape[-1]
    if n < 3:
        raise ValueError("a first derivative needs 3 points along the axis")
    h2 = T(2) * T(h)
    out = np.empty_like(g)
    out[..., 1:-1] = (g[..., 2:] - g[..., :-2]) / h2
    out[..., 0] = ((T(4) * g[..., 1] - T(3) * g[..., 0]) - g[..., 2]) / h2
    out[..., -1] = ((T(3) * g[..., -1] - T(4) * g[..., -2]) + g[..., -3]) / h2
    return _from_last(out, axis)


def second_derivative(f, axis, h=1.0):
    """d2f/da2 in the field's type: ((f[i+1] - 2 f[i]) + f[i-1]) / h^2 inside;
    at the ends (((2 f0 - 5 f1) + 4 f2) - f3) / h^2 and the mirror image, with
    h^2 = h * h rounded once.  Needs at least 4 points along the axis."""
    g = _to_last(_field(f), axis)
    T = g.dtype.type
    n = g.shape[-1]
    if n < 4:
        raise ValueError("a second derivative needs 4 points along the axis")
    hh = T(h) * T(h)
    out = np.empty_like(g)
    out[..., 1:-1] = ((g[..., 2:] - T(2) * g[..., 1:-1]) + g[..., :-2]) / hh
    out[..., 0] = (((T(2) * g[..., 0] - T(5) * g[..., 1]) + T(4) * g[..., 2]) - g[..., 3]) / hh
    out[..., -1] = (((T(2) * g[..., -1] - T(5) * g[..., -2]) + T(4) * g[..., -3]) - g[..., -4]) / hh
    return _from_last(out, axis)


def vorticity_z(u, v, h=1.0):
    """omega_z = v_x - u_y of a 2D or 3D velocity field, in its type."""
    u, v = _field(u), _field(v)
    if u.dtype != v.dtype or u.shape != v.shape:
        raise ValueError("u and v must have one shape and one type")
    return first_derivative(v, 0, h) - first_derivative(u, 1, h)


def second(w, axis, h=1.0):
    """The second derivative of w along `axis`, in its type."""
    return second_derivative(w, axis, h)
