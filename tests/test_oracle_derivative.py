"""Pins for the oracle's dG first derivative (Sec. 4.2) and its 2D extension.

* block application == dense assembly of Eq. discrete_der / Eq. matrix_xspace (brute force)
* W M_x is skew-symmetric (stated after Eq. matrix_xspace)
* P = 1 reduces to the centred difference (f_{i+1} - f_{i-1}) / 2h (stated in Sec. 3 and 4.2)
* exactness: for a continuous periodic piecewise polynomial of degree <= n-1 the standard
  flux equals the trace, so by Eq. integration-by-parts the dG derivative is the exact
  derivative at the Gauss nodes (closed form)
"""
import numpy as np
import pytest

from oracle.operators import (Operators, dense_ops_2d, derivative_matrix_1d,
                              forward_matrix_1d, from_global, to_global)
from oracle.tables import Grid, Tables


@pytest.mark.parametrize("n", range(1, 6))
def test_block_equals_dense(n):
    g = Grid(3, 4, n, 1.3, 2.1)
    ops = Operators(g, tau=0.3)
    d = dense_ops_2d(g, tau=0.3)
    u = np.random.default_rng(n).standard_normal((4, 3, n, n))
    ug = to_global(u).ravel()
    for name, fn in (("Dx", ops.Dx), ("Dy", ops.Dy), ("A", ops.A)):
        ref = from_global((d[name] @ ug).reshape(4 * n, 3 * n), n)
        assert np.allclose(fn(u), ref, atol=1e-12 * max(1, np.abs(ref).max())), name


@pytest.mark.parametrize("n", range(1, 6))
def test_weighted_derivative_skew(n):
    t = Tables(n)
    N, h = 5, 0.7
    M = derivative_matrix_1d(t, N, h)
    WM = np.diag(np.tile(h * t.w / 2, N)) @ M
    assert np.abs(WM + WM.T).max() < 1e-14 * np.abs(WM).max() * 10


def test_P1_is_centred_difference():
    t = Tables(1)
    N, h = 7, 0.3
    M = derivative_matrix_1d(t, N, h)
    f = np.random.default_rng(0).standard_normal(N)
    fd = (np.roll(f, -1) - np.roll(f, 1)) / (2 * h)
    assert np.allclose(M @ f, fd, atol=1e-14)


def _continuous_piecewise_poly(n, N, L, rng):
    """Periodic C0 function, polynomial of degree n-1 in every cell: face values v_c plus a
    bubble (1 - xi^2) q_c(xi).  Returns (values, derivatives) at the Gauss nodes, (N, n)."""
    t = Tables(n)
    h = L / N
    v = rng.standard_normal(N)
    vals = np.zeros((N, n))
    ders = np.zeros((N, n))
    xi = t.x
    for c in range(N):
        vl, vr = v[c], v[(c + 1) % N]
        q = rng.standard_normal(max(n - 2, 0))          # degree n-3 coefficients
        qv = np.polyval(q, xi) if q.size else np.zeros_like(xi)
        dq = np.polyval(np.polyder(q), xi) if q.size > 1 else np.zeros_like(xi)
        vals[c] = vl * (1 - xi) / 2 + vr * (1 + xi) / 2 + (1 - xi ** 2) * qv
        dxi = (vr - vl) / 2 - 2 * xi * qv + (1 - xi ** 2) * dq
        ders[c] = dxi * 2.0 / h
    return vals, ders


@pytest.mark.parametrize("n", range(2, 6))
def test_exact_on_continuous_piecewise_polynomials(n):
    rng = np.random.default_rng(10 + n)
    N, L = 6, 2.5
    vals, ders = _continuous_piecewise_poly(n, N, L, rng)
    t = Tables(n)
    for M in (derivative_matrix_1d(t, N, L / N), forward_matrix_1d(t, N, L / N)):
        got = (M @ vals.ravel()).reshape(N, n)
        assert np.allclose(got, ders, atol=1e-11 * np.abs(ders).max())
    # 2D: the same function of x only, on a grid with several cell rows
    g = Grid(N, 3, n, L, 1.0)
    ops = Operators(g)
    f = np.broadcast_to(vals[None, :, None, :], (3, N, n, n)).copy()
    df = np.broadcast_to(ders[None, :, None, :], (3, N, n, n))
    assert np.allclose(ops.Dx(f), df, atol=1e-11 * np.abs(ders).max())
    assert np.abs(ops.Dy(f)).max() < 1e-11 * np.abs(vals).max() * n


@pytest.mark.parametrize("n", [1, 3, 5])
def test_summation_by_parts_2d(n):
    """sum W (D f) g = - sum W f (D g) for D = D_x, D_y (discrete integration by parts, Sec. 3)."""
    g = Grid(5, 4, n, 2.0, 3.0)
    ops = Operators(g)
    rng = np.random.default_rng(3)
    f, h = rng.standard_normal((2, 4, 5, n, n))
    for D in (ops.Dx, ops.Dy):
        a, b = ops.inner(D(f), h), -ops.inner(f, D(h))
        assert abs(a - b) < 1e-13 * (1 + abs(a))
