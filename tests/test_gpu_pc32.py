"""DG_FP64_PC32: the float64 PCG with the two-level preconditioner applied in float32 (its
cell block solve and coarse DFT solve).  The Krylov vectors, the operator and the stopping
rule stay float64, so the solution meets the float64 tolerance on the true residual; only
the iterates differ from the float64 path, at the level of the tolerance."""
import numpy as np
import pytest

from oracle.operators import Operators
from oracle.solver import poisson_rhs
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


@pytest.mark.parametrize("Nx,Ny,n", [(16, 12, 3), (32, 32, 4), (12, 20, 5)])
def test_steps_match_oracle_to_tolerance(dg, Nx, Ny, n):
    D, dt = 1e-3, 1e-3
    og = OGrid(Nx, Ny, n)
    X, Y = og.mesh()
    w0 = fields.random_phase(X, Y, seed=50 + n, kmax=5)
    osim = Simulation(Operators(og), w0, D, dt, tol=1e-13, precond="twolevel")
    osim.step(4)
    g = dg.Grid(Nx, Ny, n)
    g.set_precond("twolevel")
    sim = dg.Sim(g, dev(w0), D=D, dt=dt, precision=dg.DG_FP64_PC32, cg_tol=1e-13)
    sim.step(4)
    om = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    ps = torch.empty_like(om)
    sim.get(om, ps)
    assert sim.status().status == 0
    assert rel(host(om), osim.omega) < 1e-10
    assert rel(host(ps), osim.psi) < 1e-10


def test_full_size_reaches_float64_tolerance(dg):
    N, n = 512, 4
    og = OGrid(N, N, n)
    o = Operators(og)
    g = dg.Grid(N, N, n)
    g.set_precond("twolevel")
    xn, yn, _ = g.nodes()
    X, Y = fields.mesh_from_nodes(xn, yn)
    w0 = fields.shear_layer(X, Y)
    b = poisson_rhs(o, w0)
    sim = dg.Sim(g, dev(w0), D=1e-4, dt=5e-4, precision=dg.DG_FP64_PC32, cg_tol=1e-10)
    ps = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    sim.get(None, ps)
    p = host(ps)
    r = b - o.A(p)
    relres = np.sqrt(np.sum(r * r / o.W2) / np.sum(b * b / o.W2))
    assert relres < 2e-10, relres
    sim.step(3)
    info = sim.status()
    assert info.status == 0 and info.cg_iters_last < 100, info.cg_iters_last


def test_not_batched(dg):
    g = dg.Grid(8, 8, 2)
    g.set_precond("twolevel")
    sim = dg.Sim(g, dev(np.zeros(g.shape)), D=0.0, dt=1e-3, precision=dg.DG_FP64_PC32)
    b = dg.Batch(2)
    with pytest.raises(RuntimeError):
        b.admit(sim)
    b.close()
