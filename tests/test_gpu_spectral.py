"""GPU parity of the spectral preconditioner (DG_PRECOND_SPECTRAL: the exact pseudo-inverse of
the periodic operator by DFTs over the cells and n x n transforms per wave vector) against the
oracle's solver.Spectral: fixed-iteration PCG iterates on power-of-two grids (radix-2^2 DFTs)
and other sizes (direct DFT), one-cell lines and n = 1..5; the converged solution against a
dense solve; one stepper step in float64, with the float32 preconditioner and in the mixed
modes; the full-size 1024^2, n = 5 solve checked with the oracle's operator."""
import numpy as np
import pytest

from oracle.operators import Operators, dense_ops_2d, from_global, to_global
from oracle.solver import Spectral, poisson_rhs, rounding_floor2, solve_poisson, solve_poisson_dense
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
         (12, 20, 5, 1.0, 1.7), (1, 4, 3, 1.0, 1.0), (9, 16, 1, 1.0, 1.0), (64, 2, 5, 3.0, 1.0),
         (2, 3, 4, 1.0, 1.0)]


def solve_bar(o, Lx, Ly):
    """Two backward-stable solutions of the same system differ by up to about u kappa (u = 2^-52,
    kappa = lambda_max / lambda_min of the scaled operator: the Gershgorin bound over the
    smallest non-zero eigenvalue of -Delta on the periodic box); the exact preconditioner
    makes one PCG iteration such a solve on either side, so the bar is max(1e-12, u kappa)."""
    g = o.g
    lmax = np.sqrt(rounding_floor2(o)) * 2.0 ** 52
    lmin = min((2 * np.pi / Lx) ** 2 if g.Nx > 1 else np.inf, (2 * np.pi / Ly) ** 2 if g.Ny > 1 else np.inf)
    return max(1e-12, 2.0 ** -52 * lmax / lmin)


@pytest.mark.parametrize("Nx,Ny,n,Lx,Ly", GRIDS)
def test_one_iteration_parity(dg, Nx, Ny, n, Lx, Ly):
    """One PCG iteration with the exact preconditioner from the same x0 on both sides (after it
    the residual is rounding noise: further iterations are not comparable)."""
    m = 1
    g = dg.Grid(Nx, Ny, n, Lx, Ly)
    g.set_precond("spectral")
    o = Operators(OGrid(Nx, Ny, n, Lx, Ly))
    rng = np.random.default_rng(Nx + Ny + n)
    w = rng.standard_normal(g.shape)
    x0 = 0.05 * rng.standard_normal(g.shape)
    ref = solve_poisson(o, w, x0, 1e-30, 1000, fixed_iters=m, precond=Spectral(o))
    psi = dev(x0)
    rc, it, relres = dg.dg_poisson_solve(g, dev(w), psi, 1e-30, 1000, fixed_iters=m)
    assert it == ref.iters == 1
    err = rel(host(psi), ref.x)
    assert err < solve_bar(o, Lx, Ly), (err, solve_bar(o, Lx, Ly))


@pytest.mark.parametrize("n", [1, 3, 5])
def test_converged_matches_dense_in_few_iterations(dg, n):
    g = dg.Grid(6, 4, n, 1.5, 1.0)
    g.set_precond("spectral")
    og = OGrid(6, 4, n, 1.5, 1.0)
    w = np.random.default_rng(n).standard_normal(g.shape)
    ref = from_global(solve_poisson_dense(dense_ops_2d(og), to_global(w)), n)
    psi = dev(np.zeros(g.shape))
    rc, it, relres = dg.dg_poisson_solve(g, dev(w), psi, 1e-13, 1000)
    assert relres <= 1e-13 and it <= 2, (it, relres)
    assert rel(host(psi), ref) < 1e-11


def test_dirichlet_rejects_spectral(dg):
    g = dg.Grid(8, 8, 3, bc="dirichlet")
    with pytest.raises(dg.DGError):
        g.set_precond("spectral")


def _step_from_oracle_state(dg, prec, k, m=0):
    Nx, Ny, n, D, dt = 16, 12, 3, 1e-3, 2e-3
    og = OGrid(Nx, Ny, n)
    o = Operators(og)
    X, Y = og.mesh()
    w0 = fields.random_phase(X, Y, seed=8, kmax=5)
    osim = Simulation(o, w0, D, dt, tol=1e-13, K=3, fixed_iters=m, precond="spectral")
    osim.step(k)
    g = dg.Grid(Nx, Ny, n)
    g.set_precond("spectral")
    z = np.zeros(g.shape)
    R1 = osim.R_hist[0] if len(osim.R_hist) > 0 else z
    R2 = osim.R_hist[1] if len(osim.R_hist) > 1 else z
    sim = dg.Sim(g, dev(osim.omega), D=D, dt=dt, precision=prec, cg_tol=1e-12)
    sim.set_state(k, dev(osim.omega), dev(osim.psi), dev(osim.psi_prev), dev(R1), dev(R2))
    if m:
        sim.set_cg(1e-30, 1000, fixed_iters=m)
    sim.step(1)
    osim.step(1)
    om = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    ps = torch.empty_like(om)
    sim.get(om, ps)
    return o, osim, sim, host(om), host(ps)


@pytest.mark.parametrize("k", [0, 3])
def test_one_step_parity_spectral(dg, k):
    """Float64, one fixed PCG iteration per solve on both sides: omega and psi within 1e-12."""
    o, osim, sim, w1, p1 = _step_from_oracle_state(dg, dg.DG_FP64, k, m=1)
    assert rel(w1, osim.omega) < 1e-12
    assert rel(p1, osim.psi) < 1e-12


@pytest.mark.parametrize("mode", ["fp64pc32", "mixed", "mixed64"])
def test_one_step_other_precisions(dg, mode):
    """The float32 preconditioner inside the float64 solve, and the mixed modes (float32 inner
    PCG with the float32 spectral preconditioner): one AB3 step within 1e-10 of the oracle's."""
    prec = {"fp64pc32": dg.DG_FP64_PC32, "mixed": dg.DG_MIXED, "mixed64": dg.DG_MIXED64}[mode]
    o, osim, sim, w1, p1 = _step_from_oracle_state(dg, prec, 3)
    assert rel(w1, osim.omega) < 1e-10
    assert rel(p1, osim.psi) < 1e-10
    b = poisson_rhs(o, w1)
    r = b - o.A(p1)
    relres = np.sqrt(np.sum(r * r / o.W2) / np.sum(b * b / o.W2))
    assert relres < 1.5e-12, relres
    assert sim.status().status == 0


@pytest.mark.parametrize("prec", ["fp64", "fp64pc32", "mixed"])
def test_full_size_spectral(dg, prec):
    """1024 x 1024 cells, n = 5, random-phase field: the initial solve and three steps reach
    the 1e-10 tolerance on the oracle's operator in a handful of iterations."""
    N, n = 1024, 5
    og = OGrid(N, N, n)
    o = Operators(og)
    g = dg.Grid(N, N, n)
    g.set_precond("spectral")
    xn, yn, _ = g.nodes()
    w0 = fields.random_phase_nodes(xn, yn, seed=1)
    p_ = {"fp64": dg.DG_FP64, "fp64pc32": dg.DG_FP64_PC32, "mixed": dg.DG_MIXED}[prec]
    sim = dg.Sim(g, dev(w0), D=0.0, dt=2e-4, precision=p_, cg_tol=1e-10)
    ps = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    sim.get(None, ps)
    p = host(ps)
    b = poisson_rhs(o, w0)
    r = b - o.A(p)
    relres = np.sqrt(np.sum(r * r / o.W2) / np.sum(b * b / o.W2))
    assert relres < 2e-10, relres
    sim.step(3)
    info = sim.status()
    assert info.status == 0
    assert info.cg_iters_last <= 8, info.cg_iters_last


def test_spectral_rejects_long_non_power_of_two_lines(dg):
    """A side that is not a power of two takes the direct DFT, allowed up to 256 cells."""
    g = dg.Grid(300, 64, 2)
    with pytest.raises(dg.DGError):
        g.set_precond("spectral")
    g2 = dg.Grid(200, 64, 2)
    g2.set_precond("spectral")
