"""The mixed-precision path (DG_MIXED): bracket and inner CG in float32, float64 refinement
of the Poisson residual, float64 state, update and invariants -- against the FP64 oracle.

Error model of one step from an identical state (stated, then checked with margin): the
float32 right-hand side R carries a relative rounding error of a few eps32 with respect to
the magnitude of the terms that cancel in it, so omega^{k+1} deviates from the float64
update by about  dt * |c| * eps32 * S_R  with S_R the size of those terms; psi^{k+1} is
solved in float64 residuals to the same tolerance as the FP64 path.
"""
import numpy as np
import pytest

from oracle.operators import Operators
from oracle.solver import poisson_rhs
from oracle.stepper import Simulation
from oracle.tables import Grid as OGrid
from paper_1311_7477_gb300 import fields

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

EPS32 = 2.0 ** -24


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


def _state(Nx, n, D, dt, k):
    og = OGrid(Nx, Nx, n)
    o = Operators(og)
    X, Y = og.mesh()
    w0 = fields.random_phase(X, Y, seed=4, kmax=6)
    sim = Simulation(o, w0, D, dt, tol=1e-13, K=3)
    sim.step(k)
    return o, sim


@pytest.mark.parametrize("n", [2, 4])
@pytest.mark.parametrize("k", [0, 3])
def test_mixed_one_step_error(dg, n, k):
    Nx, D, dt = 16, 1e-3, 1e-3
    o, osim = _state(Nx, n, D, dt, k)
    g = dg.Grid(Nx, Nx, n)
    z = np.zeros(g.shape)
    R1 = osim.R_hist[0] if len(osim.R_hist) > 0 else z
    R2 = osim.R_hist[1] if len(osim.R_hist) > 1 else z
    w_k = osim.omega.copy()
    parts = o.bracket_parts(osim.psi, w_k)
    S_R = np.abs(parts[0]) + np.abs(parts[1]) + np.abs(parts[2]) + D * np.abs(o.laplacian(w_k))
    sim = dg.Sim(g, dev(w_k), D=D, dt=dt, precision=dg.DG_MIXED, cg_tol=1e-12)
    sim.set_state(k, dev(w_k), dev(osim.psi), dev(osim.psi_prev), dev(R1), dev(R2))
    sim.step(1)
    osim.tol = 1e-13
    osim.step(1)
    om = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    ps = torch.empty_like(om)
    sim.get(om, ps)
    e_w = np.linalg.norm(host(om) - osim.omega) / np.linalg.norm(osim.omega)
    # R^k enters the update with weight 23/12 (AB3) or, summed over the RK4 stages, ~1
    bound = 32.0 * dt * (23.0 / 12.0) * EPS32 * np.linalg.norm(S_R) / np.linalg.norm(osim.omega)
    assert e_w < bound, (e_w, bound)
    e_p = np.linalg.norm(host(ps) - osim.psi) / np.linalg.norm(osim.psi)
    assert e_p < max(10 * e_w, 1e-11), (e_p, e_w)
    info = sim.status()
    assert info.status == 0


def test_mixed_poisson_meets_float64_tolerance(dg):
    """The float64 residual of the mixed solve reaches the CG tolerance (checked by the oracle)."""
    Nx, n = 48, 3
    og = OGrid(Nx, Nx, n)
    o = Operators(og)
    X, Y = og.mesh()
    w0 = fields.shear_layer(X, Y, rho=0.1, delta=0.05)
    g = dg.Grid(Nx, Nx, n)
    for tol in (1e-8, 1e-10, 1e-12):
        sim = dg.Sim(g, dev(w0), D=0.0, dt=1e-3, precision=dg.DG_MIXED, cg_tol=tol)
        ps = torch.empty(g.shape, dtype=torch.float64, device="cuda")
        sim.get(None, ps)
        b = poisson_rhs(o, w0)
        r = b - o.A(host(ps))
        relres = np.sqrt(np.sum(r * r / o.W2) / np.sum(b * b / o.W2))
        assert relres < 1.5 * tol, (tol, relres)
        info = sim.status()
        assert info.refine_sweeps_last >= 1


def test_mixed_trajectory_tracks_fp64(dg):
    """32 x 32 cells, n = 3, 2 sin x sin y + noise, D = 0, 50 steps: the mixed run stays within
    the accumulated float32 bracket rounding of the FP64 run.  V changes only by the float32
    rounding of sum W R (the update itself is float64): |dV| <= steps dt eps32 |W| |S_R|."""
    Nx, n, dt = 32, 3, 1e-3
    g = dg.Grid(Nx, Nx, n)
    xn, yn, _ = g.nodes()
    X, Y = fields.mesh_from_nodes(xn, yn)
    w0 = fields.sin_sin_noise(X, Y, amp=1e-3, seed=0)
    a = dg.Sim(g, dev(w0), D=0.0, dt=dt, precision=dg.DG_FP64, cg_tol=1e-12)
    b = dg.Sim(g, dev(w0), D=0.0, dt=dt, precision=dg.DG_MIXED, cg_tol=1e-12)
    V0 = b.invariants()[0]
    a.step(50)
    b.step(50)
    wa = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    wb = torch.empty_like(wa)
    a.get(wa, None)
    b.get(wb, None)
    err = np.linalg.norm(host(wa) - host(wb)) / np.linalg.norm(host(wa))
    print("mixed vs fp64 after 50 steps: rel L2 %.3e" % err)
    assert err < 1e-6, err
    dV = abs(b.invariants()[0] - V0)
    print("mixed: |V - V0| after 50 steps %.3e" % dV)
    assert dV < 50 * dt * EPS32 * 4 * np.pi ** 2 * 100
