"""The mixed-precision paths against the FP64 oracle.

DG_MIXED evaluates the bracket and the viscous term in double-float arithmetic on the float32
pipe (dg_bracket_mixed: each value the unevaluated sum of two floats, about 48 significant
bits) and solves the Poisson equation by float64 refinement sweeps around a float32 inner
PCG; DG_MIXED64 keeps the bracket in float64.  State, update and invariants are float64.

Bars: the double-float bracket matches the oracle to 1e-12 in relative L2 (its rounding is
about 2^-46 of the terms that cancel in J, against 2^-52 for float64) and keeps J(f, f) = 0
bitwise; one step of either mode from an identical state is within 1e-10 of the oracle's step
(the target of the mixed-precision pattern), with psi meeting the float64 solver tolerance on
the oracle's own operator.
"""
import numpy as np
import pytest

from oracle.operators import Operators
from oracle.solver import poisson_rhs
from oracle.stepper import Simulation
from oracle.tables import Grid as OGrid
from paper_1311_7477_gb300 import fields
from tests.test_gpu_parity import GRIDS, bracket_scale, rel_l2

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


@pytest.mark.parametrize("Nx,Ny,n,Lx,Ly", GRIDS)
def test_bracket_mixed_parity(dg, Nx, Ny, n, Lx, Ly):
    g = dg.Grid(Nx, Ny, n, Lx, Ly)
    o = Operators(OGrid(Nx, Ny, n, Lx, Ly))
    f, h = np.random.default_rng(Nx * 100 + Ny + n).standard_normal((2, Ny, Nx, n, n))
    J = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    dg.dg_bracket_mixed(g, dev(f), dev(h), J)
    ref = o.bracket(f, h)
    got = host(J)
    assert rel_l2(got, ref, bracket_scale(o, f, h)) < 1e-12
    if Nx > 1 and Ny > 1:  # one cell in a direction: J is a near-total cancellation (see test_gpu_parity)
        assert rel_l2(got, ref) < 1e-12, rel_l2(got, ref)


@pytest.mark.parametrize("n", [1, 3, 5])
def test_bracket_mixed_bitwise_zeros_and_antisymmetry(dg, n):
    g = dg.Grid(10, 7, n, 2.0, 1.0)
    og = OGrid(10, 7, n, 2.0, 1.0)
    f = np.random.default_rng(1).standard_normal(g.shape)
    J = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    dg.dg_bracket_mixed(g, dev(f), dev(f), J)
    assert np.array_equal(host(J), np.zeros(g.shape))
    X, Y = og.mesh()
    psi = fields.sin_sin(X, Y)
    dg.dg_bracket_mixed(g, dev(psi), dev(2.0 * psi), J)
    assert np.array_equal(host(J), np.zeros(g.shape))
    h = np.random.default_rng(2).standard_normal(g.shape)
    J2 = torch.empty_like(J)
    dg.dg_bracket_mixed(g, dev(f), dev(h), J)
    dg.dg_bracket_mixed(g, dev(h), dev(f), J2)
    a, b = host(J), host(J2)
    assert np.array_equal(a, -b)  # antisymmetry holds bitwise: every operation is odd-symmetric


def _state(Nx, n, D, dt, k):
    og = OGrid(Nx, Nx, n)
    o = Operators(og)
    X, Y = og.mesh()
    w0 = fields.random_phase(X, Y, seed=4, kmax=6)
    sim = Simulation(o, w0, D, dt, tol=1e-13, K=3)
    sim.step(k)
    return o, sim


@pytest.mark.parametrize("mode", ["mixed", "mixed64"])
@pytest.mark.parametrize("n", [2, 4])
@pytest.mark.parametrize("k", [0, 3])
def test_mixed_one_step_vs_oracle(dg, mode, n, k):
    """One step (RK4 start-up for k = 0, AB3 for k = 3) from the identical state: omega and the
    increment omega^{k+1} - omega^k within 1e-10 of the oracle's, psi's true residual on the
    oracle's operator within the solver tolerance."""
    Nx, D, dt, tol = 16, 1e-3, 1e-3, 1e-12
    prec = {"mixed": dg.DG_MIXED, "mixed64": dg.DG_MIXED64}[mode]
    o, osim = _state(Nx, n, D, dt, k)
    g = dg.Grid(Nx, Nx, n)
    z = np.zeros(g.shape)
    R1 = osim.R_hist[0] if len(osim.R_hist) > 0 else z
    R2 = osim.R_hist[1] if len(osim.R_hist) > 1 else z
    w_k = osim.omega.copy()
    sim = dg.Sim(g, dev(w_k), D=D, dt=dt, precision=prec, cg_tol=tol)
    sim.set_state(k, dev(w_k), dev(osim.psi), dev(osim.psi_prev), dev(R1), dev(R2))
    sim.step(1)
    osim.step(1)
    om = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    ps = torch.empty_like(om)
    sim.get(om, ps)
    w1, p1 = host(om), host(ps)
    e_w = rel_l2(w1, osim.omega)
    e_inc = rel_l2(w1 - w_k, osim.omega - w_k)
    assert e_w < 1e-10 and e_inc < 1e-10, (e_w, e_inc)
    b = poisson_rhs(o, w1)
    r = b - o.A(p1)
    relres = np.sqrt(np.sum(r * r / o.W2) / np.sum(b * b / o.W2))
    assert relres < 1.5 * tol, relres
    e_p = rel_l2(p1, osim.psi)
    assert e_p < 1e-10, e_p
    assert sim.status().status == 0


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
    """32 x 32 cells, n = 3, 2 sin x sin y + noise, D = 0, 50 steps: the DG_MIXED run stays
    within the solver tolerance's accumulation of the FP64 run (both solve to 1e-12), and V is
    conserved to float64 roundoff (the double-float R converts to float64 exactly and the
    update is float64)."""
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
    assert err < 1e-10, err
    dV = abs(b.invariants()[0] - V0)
    assert dV < 1e-13 * 4 * np.pi ** 2 * np.abs(w0).max(), dV


@pytest.mark.parametrize("mode", [0, 1, 2])
def test_compensated_apply_modes_agree(dg, mode):
    """The inner operator apply of the mixed solves -- float32 (0), double-float (1), adaptive
    (2) -- changes the inner iterates, not the result: on a 256^2, n = 4 shear layer all reach
    the tolerance on the oracle's operator and agree with the float64 solve."""
    N, n = 256, 4
    og = OGrid(N, N, n)
    o = Operators(og)
    g = dg.Grid(N, N, n)
    g.set_precond("twolevel")
    assert g.compensated_apply in (0, 2)
    g.set_compensated_apply(mode)
    assert g.compensated_apply == mode
    X, Y = og.mesh()
    w0 = fields.shear_layer(X, Y)
    s = dg.Sim(g, dev(w0), D=0.0, dt=1e-4, precision=dg.DG_MIXED64, cg_tol=1e-10)
    ps = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    s.get(None, ps)
    p = host(ps)
    b = poisson_rhs(o, w0)
    r = b - o.A(p)
    relres = np.sqrt(np.sum(r * r / o.W2) / np.sum(b * b / o.W2))
    assert relres < 2e-10, relres
    ref = dev(np.zeros(g.shape))
    dg.dg_poisson_solve(g, dev(w0), ref, 1e-10, 100000)
    assert rel_l2(p, host(ref)) < 1e-8
