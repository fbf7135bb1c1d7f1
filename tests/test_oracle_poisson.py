"""Pins for the oracle's LDG Laplacian and CG Poisson solve (Sec. 6).

* dense brute force on tiny grids: A symmetric, positive semi-definite, kernel = constants
  (for tau = 0 and tau > 0); the block form equals the dense matrix (test_oracle_derivative)
* P = 1, tau = 0 reduces to the 5-point finite-difference Laplacian (textbook)
* PCG reaches the dense direct solution; fixed-iteration mode runs exactly that many steps
* closed form: -Delta psi = (k^2 + l^2) sin kx cos ly converges at order n
* sum W Delta_h u = 0 (vorticity is not created by diffusion)
"""
import numpy as np
import pytest

from oracle.operators import Operators, dense_ops_2d, from_global, to_global
from oracle.solver import pcg, poisson_rhs, solve_poisson, solve_poisson_dense
from oracle.tables import Grid


@pytest.mark.parametrize("n", range(1, 5))
@pytest.mark.parametrize("tau", [0.0, 0.5])
def test_dense_A_symmetric_psd_constant_kernel(n, tau):
    g = Grid(3, 4, n, 1.0, 1.6)
    A = dense_ops_2d(g, tau)["A"]
    assert np.abs(A - A.T).max() < 1e-13 * np.abs(A).max()
    ev, V = np.linalg.eigh(0.5 * (A + A.T))
    scale = np.abs(ev).max()
    assert ev[0] > -1e-12 * scale
    assert ev[1] > 1e-6 * scale                     # exactly one zero eigenvalue
    v0 = V[:, 0] / V[0, 0]
    assert np.allclose(v0, 1.0, atol=1e-8)         # ... and its eigenvector is constant


def test_P1_is_five_point_laplacian():
    g = Grid(7, 5, 1, 2.1, 1.3)
    ops = Operators(g)
    u = np.random.default_rng(0).standard_normal((5, 7, 1, 1))
    U = u[:, :, 0, 0]
    hx, hy = g.hx, g.hy
    fd = ((np.roll(U, -1, 1) - 2 * U + np.roll(U, 1, 1)) / hx ** 2
          + (np.roll(U, -1, 0) - 2 * U + np.roll(U, 1, 0)) / hy ** 2)
    assert np.allclose(ops.laplacian(u)[:, :, 0, 0], fd, atol=1e-12 * np.abs(fd).max())


@pytest.mark.parametrize("n", [1, 2, 3])
def test_pcg_matches_dense_solution(n):
    g = Grid(4, 3, n, 1.5, 1.2)
    ops = Operators(g)
    d = dense_ops_2d(g)
    w = np.random.default_rng(n).standard_normal((3, 4, n, n))
    ref = from_global(solve_poisson_dense(d, to_global(w)), n)
    res = solve_poisson(ops, w, np.zeros_like(w), 1e-13, 10000)
    assert res.converged
    assert np.allclose(res.x, ref, atol=1e-10 * np.abs(ref).max())
    # the solution has W-mean zero and solves -Delta_h psi = omega - mean(omega)
    assert abs(ops.integral(res.x)) < 1e-12 * np.abs(ref).max()
    wm = w - ops.integral(w) / ops.integral(np.ones_like(w))
    assert np.allclose(-ops.laplacian(res.x), wm, atol=1e-9 * np.abs(wm).max())


def test_fixed_iteration_mode():
    g = Grid(6, 6, 3)
    ops = Operators(g)
    w = np.random.default_rng(5).standard_normal((6, 6, 3, 3))
    b = poisson_rhs(ops, w)
    r7 = pcg(ops, b, np.zeros_like(w), 1e-30, 1000, fixed_iters=7)
    assert r7.iters == 7 and r7.relres > 1e-6


@pytest.mark.parametrize("n", [2, 3, 4])
def test_closed_form_poisson_order(n):
    k, l = 1, 2
    errs = []
    for N in (8, 16):
        g = Grid(N, N, n)
        ops = Operators(g)
        X, Y = g.mesh()
        exact = np.sin(k * X) * np.cos(l * Y)
        res = solve_poisson(ops, (k * k + l * l) * exact, np.zeros_like(X), 1e-13, 100000)
        e = res.x - exact
        errs.append(np.sqrt(ops.inner(e, e)))
    order = np.log2(errs[0] / errs[1])
    assert order > n - 0.35, (errs, order)


@pytest.mark.parametrize("n", [1, 3])
def test_diffusion_conserves_vorticity(n):
    g = Grid(5, 6, n)
    ops = Operators(g, tau=0.2)
    u = np.random.default_rng(2).standard_normal((6, 5, n, n))
    assert abs(ops.integral(ops.laplacian(u))) < 1e-12 * np.abs(ops.laplacian(u)).max()
    assert np.abs(ops.laplacian(np.full_like(u, 2.5))).max() < 1e-11


def test_rounding_floor_bounds_the_spectrum_and_the_rounded_solution():
    """The float64 rounding floor of the stopping rule: its eigenvalue bound is not below the
    largest eigenvalue of the scaled operator W^-1/2 A W^-1/2 (dense, tiny grids), and the exact
    solution rounded to float32 -- a stand-in for float64 rounding, 2^29 times larger -- leaves a
    relative residual within the floor scaled by the same factor."""
    from oracle.operators import dense_ops_2d, from_global, to_global
    from oracle.solver import rounding_floor2, solve_poisson_dense
    for Nx, Ny, n, tau in ((4, 3, 2, 0.0), (3, 4, 3, 0.5), (5, 5, 4, 0.0)):
        og = Grid(Nx, Ny, n, 1.3, 0.9)
        ops = Operators(og, tau=tau)
        d = dense_ops_2d(og, tau)
        sw = np.sqrt(d["W"])
        Ahat = d["A"] / sw[:, None] / sw[None, :]
        lam = np.linalg.eigvalsh(Ahat).max()
        bound = np.sqrt(rounding_floor2(ops)) * 2.0 ** 52
        assert bound >= lam * (1 - 1e-12), (bound, lam)
        w = np.random.default_rng(n).standard_normal(og.zeros().shape)
        x = from_global(solve_poisson_dense(d, to_global(w)), n)
        b = poisson_rhs(ops, w)
        x32 = x.astype(np.float32).astype(np.float64)
        r = b - ops.A(x32)
        rel2 = np.sum(r * r / ops.W2) / np.sum(b * b / ops.W2)
        floor2_32 = rounding_floor2(ops) * 2.0 ** 58 * np.sum(ops.W2 * x32 * x32) / np.sum(b * b / ops.W2)
        assert rel2 <= floor2_32, (rel2, floor2_32)
