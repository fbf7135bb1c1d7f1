"""Pins for the oracle's Legendre / Gauss-Legendre tables (Sec. 4.1).

Each check compares against something other than the oracle itself: NumPy's Legendre
module (an independent library routine), the closed forms the paper prints, or
identities the paper states (orthogonality, Eq. completeness, Eq. legendre_derivative,
Eq. transformation, Eq. def_norm)."""
import numpy as np
import pytest
from numpy.polynomial import legendre as npleg

from oracle.tables import Tables, gauss_legendre, legendre


@pytest.mark.parametrize("n", range(1, 9))
def test_gauss_legendre_matches_numpy(n):
    x, w = gauss_legendre(n)
    xr, wr = npleg.leggauss(n)
    assert np.allclose(x, xr, rtol=0, atol=1e-15)
    assert np.allclose(w, wr, rtol=0, atol=4e-15)


def test_recursion_matches_numpy():
    xs = np.linspace(-1, 1, 37)
    P = legendre(7, xs)
    for k in range(8):
        c = np.zeros(k + 1)
        c[k] = 1.0
        assert np.allclose(P[k], npleg.legval(xs, c), rtol=0, atol=1e-14)


@pytest.mark.parametrize("n", range(1, 7))
def test_discrete_orthogonality_and_completeness(n):
    t = Tables(n)
    # sum_j w_j p_k(x_j) p_l(x_j) = 2/(2k+1) delta_kl  (exactness to degree 2n-1)
    G = (t.B * t.w[:, None]).T @ t.B
    assert np.allclose(G, np.diag(2.0 / (2 * np.arange(n) + 1)), atol=1e-14)
    # Eq. completeness: sum_k (2k+1)/2 w_j p_k(x_i) p_k(x_j) = delta_ij, i.e. B F = 1, and F B = 1
    assert np.allclose(t.B @ t.F, np.eye(n), atol=1e-14)
    assert np.allclose(t.F @ t.B, np.eye(n), atol=1e-14)


@pytest.mark.parametrize("n", range(1, 7))
def test_D_matrix_closed_form_and_integral(n):
    t = Tables(n)
    # D_ij = int_{-1}^{1} p_i p_j' by NumPy's derivative and a high-order quadrature
    xq, wq = npleg.leggauss(n + 4)
    Dnum = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            ci = np.zeros(i + 1); ci[i] = 1
            cj = np.zeros(j + 1); cj[j] = 1
            dj = npleg.legder(cj) if j > 0 else np.zeros(1)
            Dnum[i, j] = np.sum(wq * npleg.legval(xq, ci) * npleg.legval(xq, dj))
    assert np.allclose(t.D, Dnum, atol=1e-13)
    # Eq. legendre_derivative: (D + L) = (R - D)^T, i.e. D + D^T = R - L
    assert np.array_equal(t.D + t.D.T, t.R - t.L)
    # Eq. legendre_operators: RL_ij = (-1)^j, LR_ij = (-1)^i = RL^T
    j = np.arange(n)
    assert np.array_equal(t.RL, np.tile((-1.0) ** j, (n, 1)))
    assert np.array_equal(t.LR, t.RL.T)


@pytest.mark.parametrize("n", range(1, 6))
@pytest.mark.parametrize("h", [1.0, 0.37])
def test_transformation_and_norm(n, h):
    """F = T B^T W (the index-consistent reading of Eq. transformation) and the two forms
    of the inner product in Eq. def_norm."""
    t = Tables(n)
    assert np.allclose(t.T(h) @ t.B.T @ t.W(h), t.F, atol=1e-14)
    assert np.allclose(t.S(h) @ t.T(h), np.eye(n), atol=1e-15)
    rng = np.random.default_rng(n)
    f, g = rng.standard_normal(n), rng.standard_normal(n)
    x_form = f @ t.W(h) @ g
    l_form = (t.F @ f) @ t.S(h) @ (t.F @ g)
    assert abs(x_form - l_form) < 1e-14 * (1 + abs(x_form))
