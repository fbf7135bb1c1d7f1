"""GPU parity of the two-level preconditioned CG (DG_PRECOND_TWOLEVEL) against the oracle's
solver.TwoLevel, on power-of-two grids (radix-2 DFT of the cell grid) and other sizes
(direct DFT), in float64 and in the mixed path."""
import numpy as np
import pytest

from oracle.operators import Operators, dense_ops_2d, from_global, to_global
from oracle.solver import TwoLevel, poisson_rhs, solve_poisson, solve_poisson_dense
from oracle.stepper import Simulation
from oracle.tables import Grid as OGrid
from paper_1311_7477_gb300 import fields

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def dg(native):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return native


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


GRIDS = [(16, 8, 3, 2.0, 1.0), (13, 11, 2, 2 * np.pi, 2 * np.pi), (32, 32, 4, 2 * np.pi, 2 * np.pi),
         (12, 20, 5, 1.0, 1.7), (1, 4, 3, 1.0, 1.0), (9, 16, 1, 1.0, 1.0)]


@pytest.mark.parametrize("Nx,Ny,n,Lx,Ly", GRIDS)
def test_fixed_iterations_parity(dg, Nx, Ny, n, Lx, Ly):
    g = dg.Grid(Nx, Ny, n, Lx, Ly)
    g.set_precond("twolevel")
    o = Operators(OGrid(Nx, Ny, n, Lx, Ly))
    rng = np.random.default_rng(Nx + Ny + n)
    w = rng.standard_normal(g.shape)
    x0 = 0.05 * rng.standard_normal(g.shape)
    m = 8
    ref = solve_poisson(o, w, x0, 1e-30, 1000, fixed_iters=m, precond=TwoLevel(o))
    psi = dev(x0)
    rc, it, relres = dg.dg_poisson_solve(g, dev(w), psi, 1e-30, 1000, fixed_iters=m)
    assert it == m
    err = rel(host(psi), ref.x)
    assert err < 1e-12, err
    assert abs(relres - ref.relres) <= 1e-9 * ref.relres


@pytest.mark.parametrize("n", [1, 3])
def test_converged_matches_dense(dg, n):
    g = dg.Grid(6, 4, n, 1.5, 1.0)
    g.set_precond("twolevel")
    og = OGrid(6, 4, n, 1.5, 1.0)
    w = np.random.default_rng(n).standard_normal(g.shape)
    ref = from_global(solve_poisson_dense(dense_ops_2d(og), to_global(w)), n)
    psi = dev(np.zeros(g.shape))
    rc, it, relres = dg.dg_poisson_solve(g, dev(w), psi, 1e-13, 1000)
    assert relres <= 1e-13
    assert rel(host(psi), ref) < 1e-11


@pytest.mark.parametrize("k", [0, 3])
def test_one_step_parity_twolevel(dg, k):
    Nx, Ny, n, D, dt, m = 16, 12, 3, 1e-3, 2e-3, 12
    og = OGrid(Nx, Ny, n)
    o = Operators(og)
    X, Y = og.mesh()
    w0 = fields.random_phase(X, Y, seed=8, kmax=5)
    osim = Simulation(o, w0, D, dt, tol=1e-13, K=3, fixed_iters=m, precond="twolevel")
    osim.step(k)
    g = dg.Grid(Nx, Ny, n)
    g.set_precond("twolevel")
    z = np.zeros(g.shape)
    R1 = osim.R_hist[0] if len(osim.R_hist) > 0 else z
    R2 = osim.R_hist[1] if len(osim.R_hist) > 1 else z
    sim = dg.Sim(g, dev(osim.omega), D=D, dt=dt, cg_tol=1e-13)
    sim.set_state(k, dev(osim.omega), dev(osim.psi), dev(osim.psi_prev), dev(R1), dev(R2))
    sim.set_cg(1e-30, 1000, fixed_iters=m)
    sim.step(1)
    osim.step(1)
    om = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    ps = torch.empty_like(om)
    sim.get(om, ps)
    assert rel(host(om), osim.omega) < 1e-12
    assert rel(host(ps), osim.psi) < 1e-12


def test_full_size_twolevel_fp64_and_mixed(dg):
    """512 x 512 cells, n = 4, shear layer: the preconditioned solves reach the float64
    tolerance (checked by the oracle's residual) with far fewer iterations than W^-1."""
    N, n, D, dt = 512, 4, 1e-4, 5e-4
    og = OGrid(N, N, n)
    o = Operators(og)
    g = dg.Grid(N, N, n)
    xn, yn, _ = g.nodes()
    X, Y = fields.mesh_from_nodes(xn, yn)
    w0 = fields.shear_layer(X, Y)
    b = poisson_rhs(o, w0)
    for prec in (dg.DG_FP64, dg.DG_MIXED):
        g.set_precond("twolevel")
        sim = dg.Sim(g, dev(w0), D=D, dt=dt, precision=prec, cg_tol=1e-10)
        ps = torch.empty(g.shape, dtype=torch.float64, device="cuda")
        sim.get(None, ps)
        p = host(ps)
        r = b - o.A(p)
        relres = np.sqrt(np.sum(r * r / o.W2) / np.sum(b * b / o.W2))
        assert relres < 2e-10, (prec, relres)
        assert abs(o.integral(p)) < 1e-12 * np.abs(p).max() * 4 * np.pi ** 2
        sim.step(3)
        info = sim.status()
        assert info.status == 0
        assert info.cg_iters_last < 600, info.cg_iters_last


def test_mixed_twolevel_one_step_error(dg):
    Nx, n, D, dt = 16, 4, 1e-3, 1e-3
    og = OGrid(Nx, Nx, n)
    o = Operators(og)
    X, Y = og.mesh()
    w0 = fields.random_phase(X, Y, seed=4, kmax=6)
    osim = Simulation(o, w0, D, dt, tol=1e-13, K=3, precond="twolevel")
    osim.step(3)
    g = dg.Grid(Nx, Nx, n)
    g.set_precond("twolevel")
    sim = dg.Sim(g, dev(osim.omega), D=D, dt=dt, precision=dg.DG_MIXED, cg_tol=1e-12)
    sim.set_state(3, dev(osim.omega), dev(osim.psi), dev(osim.psi_prev), dev(osim.R_hist[0]), dev(osim.R_hist[1]))
    sim.step(1)
    osim.step(1)
    om = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    ps = torch.empty_like(om)
    sim.get(om, ps)
    assert rel(host(om), osim.omega) < 1e-9
    assert rel(host(ps), osim.psi) < 1e-9
    assert sim.status().refine_sweeps_last >= 1
