"""Pins of the oracle's exact spectral preconditioner (oracle.solver.Spectral): it must be the
pseudo-inverse of the Sec. 6 operator A, checked by brute force against a dense least-squares
solve on tiny grids (odd, even, one-cell and non-square lines, n = 1..5, with and without the
jump penalty), and PCG preconditioned with it must converge in one iteration to the dense
solution."""
import numpy as np
import pytest

from oracle.operators import Operators, dense_ops_2d, to_global
from oracle.solver import Spectral, pcg, poisson_rhs
from oracle.tables import Grid as OGrid

GRIDS = [(4, 3, 2, 2.0, 1.0, 0.0), (5, 4, 3, 1.0, 1.5, 0.0), (3, 2, 4, 1.0, 1.0, 0.0),
         (1, 2, 2, 1.0, 1.0, 0.0), (6, 6, 1, 1.0, 1.0, 0.0), (2, 5, 5, 1.0, 2.0, 0.0),
         (4, 4, 3, 2.0, 2.0, 0.4)]


def _dense_pinv_solve(g, tau, r):
    d = dense_ops_2d(g, tau)
    z = np.linalg.lstsq(d["A"], to_global(r).reshape(-1), rcond=None)[0]
    W = d["W"].reshape(-1)
    return z - np.sum(W * z) / np.sum(W)


@pytest.mark.parametrize("Nx,Ny,n,Lx,Ly,tau", GRIDS)
def test_spectral_is_the_pseudo_inverse(Nx, Ny, n, Lx, Ly, tau):
    g = OGrid(Nx, Ny, n, Lx, Ly)
    o = Operators(g, tau)
    S = Spectral(o)
    r = poisson_rhs(o, np.random.default_rng(Nx * 10 + Ny + n).standard_normal(g.zeros().shape))
    z = S(r)
    ref = _dense_pinv_solve(g, tau, r)
    assert np.abs(to_global(z).reshape(-1) - ref).max() <= 1e-12 * np.abs(ref).max()
    assert np.abs(o.A(z) - r).max() <= 1e-12 * np.abs(r).max()
    assert abs(float(np.sum(o.W2 * z))) <= 1e-12 * float(np.sum(np.abs(o.W2 * z)))


@pytest.mark.parametrize("Nx,Ny,n,Lx,Ly,tau", GRIDS[:4])
def test_pcg_with_spectral_converges_in_one_iteration(Nx, Ny, n, Lx, Ly, tau):
    g = OGrid(Nx, Ny, n, Lx, Ly)
    o = Operators(g, tau)
    r = poisson_rhs(o, np.random.default_rng(3).standard_normal(g.zeros().shape))
    x0 = 0.1 * np.random.default_rng(4).standard_normal(r.shape)
    res = pcg(o, r, x0, 1e-12, 50, precond=Spectral(o))
    assert res.converged and res.iters == 1
    ref = _dense_pinv_solve(g, tau, r)
    assert np.abs(to_global(res.x).reshape(-1) - ref).max() <= 1e-11 * np.abs(ref).max()


def test_spectral_rejects_dirichlet():
    o = Operators(OGrid(4, 4, 2), bc="dirichlet")
    with pytest.raises(ValueError):
        Spectral(o)
