"""Pins for the oracle's two-level preconditioner (a design choice: Sec. 6 names
none).  It must not change what CG converges to, must be symmetric positive definite, its
coarse solve must invert the Galerkin coarse operator exactly, and the iteration count must
grow far more slowly with the mesh than with W^{-1} (the point of the coarse level; with
cell-sized subdomains and the cell-average coarse space it still grows mildly)."""
import numpy as np
import pytest

from oracle.operators import Operators, dense_ops_2d, from_global, to_global
from oracle.solver import TwoLevel, pcg, poisson_rhs, solve_poisson, solve_poisson_dense
from oracle.tables import Grid
from paper_1311_7477_gb300 import fields


def _dense_of(fn, shape):
    m = int(np.prod(shape))
    M = np.zeros((m, m))
    for k in range(m):
        e = np.zeros(m)
        e[k] = 1.0
        M[:, k] = fn(e.reshape(shape)).ravel()
    return M


@pytest.mark.parametrize("Nx,Ny,n,tau", [(3, 4, 2, 0.0), (4, 3, 3, 0.5), (2, 2, 4, 0.0), (1, 3, 2, 0.0)])
def test_preconditioner_symmetric_positive_definite(Nx, Ny, n, tau):
    g = Grid(Nx, Ny, n, 1.3, 0.9)
    ops = Operators(g, tau)
    M = _dense_of(TwoLevel(ops), (Ny, Nx, n, n))
    assert np.abs(M - M.T).max() < 1e-10 * np.abs(M).max()
    assert np.linalg.eigvalsh(0.5 * (M + M.T)).min() > 0


@pytest.mark.parametrize("Nx,Ny,n", [(5, 4, 2), (3, 6, 3), (1, 4, 2)])
def test_coarse_solve_inverts_galerkin_operator(Nx, Ny, n):
    g = Grid(Nx, Ny, n, 2.0, 1.0)
    ops = Operators(g)
    tl = TwoLevel(ops)
    # A_c = P^T A P assembled column by column
    Ac = np.zeros((Ny * Nx, Ny * Nx))
    for c in range(Ny * Nx):
        e = g.zeros()
        e[c // Nx, c % Nx] = 1.0
        Ac[:, c] = ops.A(e).sum(axis=(2, 3)).ravel()
    rc = np.random.default_rng(1).standard_normal((Ny, Nx))
    rc -= rc.mean()
    uc = tl.coarse_solve(rc)
    assert np.allclose(Ac @ uc.ravel(), rc.ravel(), atol=1e-10 * np.abs(rc).max())
    assert abs(uc.mean()) < 1e-12


@pytest.mark.parametrize("n", [1, 2, 3])
def test_twolevel_pcg_reaches_dense_solution(n):
    g = Grid(5, 4, n, 1.4, 1.0)
    ops = Operators(g)
    w = np.random.default_rng(n).standard_normal((4, 5, n, n))
    ref = from_global(solve_poisson_dense(dense_ops_2d(g), to_global(w)), n)
    res = solve_poisson(ops, w, np.zeros_like(w), 1e-13, 1000, precond=TwoLevel(ops))
    assert res.converged
    assert np.allclose(res.x, ref, atol=1e-10 * np.abs(ref).max())


def test_iterations_grow_slowly_with_the_mesh():
    its = {}
    for pc in ("jacobi", "twolevel"):
        its[pc] = []
        for N in (16, 32, 64):
            g = Grid(N, N, 3)
            ops = Operators(g)
            X, Y = g.mesh()
            w = fields.shear_layer(X, Y, rho=0.2, delta=0.05)
            M = TwoLevel(ops) if pc == "twolevel" else None
            res = pcg(ops, poisson_rhs(ops, w), np.zeros_like(w), 1e-10, 100000, precond=M)
            its[pc].append(res.iters)
    grow_tl = its["twolevel"][2] / its["twolevel"][0]
    grow_j = its["jacobi"][2] / its["jacobi"][0]
    assert grow_tl < 2.0 and grow_j > 4.0 and grow_tl * 2.5 < grow_j, its
    assert its["twolevel"][2] * 1.5 < its["jacobi"][2], its
