"""The naive bracket J^{++} on the GPU and the Lamb dipole at t = 0.5 (Sec. 6.2, Figures 1-2).

* A simulation stepped with DG_BRACKET_NAIVE matches the oracle's Simulation(bracket="naive").
* Figures 1 (P = 1, N = 100) and 2 (P = 4, N = 50) by norms: with the bracket of Eq. J the
  dipole at t = 0.5 is closer to the exact translated dipole than with J^{++} alone, and
  its enstrophy and energy drift less; both conserve V.
"""
import numpy as np
import pytest

from oracle.operators import Operators
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


def rel(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


@pytest.mark.parametrize("n", [1, 4])
def test_naive_bracket_parity(dg, n):
    Nx, Ny, D, dt, steps = 12, 10, 1e-3, 2e-3, 5
    og = OGrid(Nx, Ny, n)
    X, Y = og.mesh()
    w0 = fields.random_phase(X, Y, seed=40 + n, kmax=4)
    osim = Simulation(Operators(og), w0, D, dt, tol=1e-13, bracket="naive")
    osim.step(steps)
    g = dg.Grid(Nx, Ny, n)
    sim = dg.Sim(g, dev(w0), D=D, dt=dt, cg_tol=1e-13)
    sim.set_bracket("naive")
    sim.step(steps)
    om = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    ps = torch.empty_like(om)
    sim.get(om, ps)
    torch.cuda.synchronize()
    assert rel(om.cpu().numpy(), osim.omega) < 1e-10
    assert rel(ps.cpu().numpy(), osim.psi) < 1e-10


def test_bracket_variant_errors(dg):
    g = dg.Grid(4, 4, 2)
    sim = dg.Sim(g, dev(np.zeros(g.shape)), D=0.0, dt=1e-3)
    with pytest.raises(RuntimeError):
        sim.set_bracket(2)
    sim.set_bracket("naive")
    b = dg.Batch(2)
    with pytest.raises(RuntimeError):
        b.admit(sim)
    b.close()


@pytest.mark.parametrize("N,n", [(100, 1), (50, 4)])
def test_dipole_shape_at_t05(dg, N, n):
    from paper_1311_7477_gb300 import experiments
    a = experiments.dipole_shape(dg, N, n, "arakawa")
    b = experiments.dipole_shape(dg, N, n, "naive")
    assert a["status"] == 0 and b["status"] == 0
    assert a["shape_error"] < b["shape_error"], (a, b)
    assert a["eps_Omega"] < b["eps_Omega"], (a, b)
    for r in (a, b):
        assert abs(r["V"]) < 1e-12
