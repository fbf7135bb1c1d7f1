"""Parity at the full sizes the benchmarks time: 512^2 cells, n = 4 (double shear layer) and
1024^2 cells, n = 5 (random phase), in the launch configurations bench.py uses.

* The bracket J on sampled cells: J at a cell depends only on the 5x5 cells around it, so
  the oracle evaluates it on that patch of the true fields (as a periodic 5x5 grid of the
  same cell size) -- one cell at a time, independent of the full-grid run.
* The Poisson solve (two-level PCG, tolerance 1e-10): the oracle's own operator gives the
  true residual of the returned psi on the whole grid.
* One float64 step and one DG_MIXED64 step from the identical state agree to the solver
  tolerance; V is conserved by the step.
* 1024^2, n = 5: one float64 step against the oracle on the whole grid at 1e-12 (fixed CG
  iteration count on both sides); one DG_MIXED / DG_MIXED64 step against the oracle at 1e-10
  at both sizes; the mixed start-up solve of a 1024^2 shear layer converges.
"""
import numpy as np
import pytest

from oracle.operators import Operators
from oracle.solver import poisson_rhs
from oracle.tables import Grid as OGrid
from paper_1311_7477_gb300 import fields
from tests.test_gpu_parity import bracket_scale as _bracket_scale

pytestmark = [pytest.mark.gpu, pytest.mark.slow]
torch = pytest.importorskip("torch")

CASES = [(512, 4, "shear_layer"), (1024, 5, "random_phase")]


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


def _fields(dg, N, n, kind):
    g = dg.Grid(N, N, n)
    g.set_precond("twolevel")
    xn, yn, _ = g.nodes()
    X, Y = fields.mesh_from_nodes(xn, yn)
    if kind == "shear_layer":
        w = fields.shear_layer(X, Y)
    else:
        w = fields.random_phase(X, Y, seed=1)
    psi = fields.random_phase(X, Y, seed=9, kmax=12)
    return g, w, psi


def _patch(a, cy, cx, r):
    Ny, Nx = a.shape[:2]
    ys = [(cy + d) % Ny for d in range(-r, r + 1)]
    xs = [(cx + d) % Nx for d in range(-r, r + 1)]
    return a[np.ix_(ys, xs)]


@pytest.mark.parametrize("N,n,kind", CASES)
def test_bracket_on_sampled_cells(dg, N, n, kind):
    g, w, psi = _fields(dg, N, n, kind)
    J = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    dg.dg_bracket(g, dev(psi), dev(w), J)
    Jh = host(J)
    h = 2 * np.pi / N
    po = Operators(OGrid(5, 5, n, 5 * h, 5 * h))
    rng = np.random.default_rng(N + n)
    scale = np.abs(Jh).max()
    for cy, cx in zip(rng.integers(0, N, 40), rng.integers(0, N, 40)):
        ref = po.bracket(_patch(psi, cy, cx, 2), _patch(w, cy, cx, 2))[2, 2]
        assert np.abs(Jh[cy, cx] - ref).max() <= 1e-11 * scale, (cy, cx)


@pytest.mark.parametrize("N,n,kind", CASES)
def test_poisson_true_residual(dg, N, n, kind):
    g, w, _ = _fields(dg, N, n, kind)
    o = Operators(OGrid(N, N, n))
    psi = dev(np.zeros(g.shape))
    rc, it, relres = dg.dg_poisson_solve(g, dev(w), psi, 1e-10, 100000)
    assert rc == dg.DG_OK
    p = host(psi)
    b = poisson_rhs(o, w)
    r = b - o.A(p)
    true_rel = np.sqrt(np.sum(r * r / o.W2) / np.sum(b * b / o.W2))
    assert true_rel < 2e-10, true_rel
    assert abs(o.integral(p)) < 1e-11 * np.abs(p).max() * 4 * np.pi ** 2


@pytest.mark.parametrize("N,n,kind", CASES)
def test_step_fp64_vs_mixed64(dg, N, n, kind):
    g, w, _ = _fields(dg, N, n, kind)
    D, dt = (1e-4, 5e-4) if kind == "shear_layer" else (0.0, 2e-4)
    a = dg.Sim(g, dev(w), D=D, dt=dt, precision=dg.DG_FP64, cg_tol=1e-10)
    a.step(3)
    st = [torch.empty(g.shape, dtype=torch.float64, device="cuda") for _ in range(5)]
    k = a.get_state(*st)
    V0 = a.invariants()[0]
    b = dg.Sim(g, st[0], D=D, dt=dt, precision=dg.DG_MIXED64, cg_tol=1e-10)
    b.set_state(k, *st)
    a.step(1)
    b.step(1)
    wa, pa = torch.empty_like(st[0]), torch.empty_like(st[0])
    wb, pb = torch.empty_like(st[0]), torch.empty_like(st[0])
    a.get(wa, pa)
    b.get(wb, pb)
    ew = float(torch.linalg.norm(wa - wb) / torch.linalg.norm(wa))
    ep = float(torch.linalg.norm(pa - pb) / torch.linalg.norm(pa))
    assert ew < 1e-12 and ep < 1e-9, (ew, ep)
    V1 = a.invariants()[0]
    assert abs(V1 - V0) < 1e-12 * float(torch.abs(wa).max()) * 4 * np.pi ** 2


def test_one_step_fp64_whole_field_1024_n5(dg):
    """1024^2 cells, n = 5 (26.2M dof), random phase, D = 0, dt = 2e-4: the benchmark's launch
    configuration.  From the GPU state after three steps (two RK4 start-up steps and one AB3
    step) both sides take one AB3 step with the same number of two-level PCG iterations (the
    per-step parity of Sec. 6 with a fixed iteration count): omega^{k+1} agrees with the
    oracle on the whole grid to 1e-12 in relative L2, the bracket to 1e-12 of its rounding
    scale, psi^{k+1} to the conditioning of the solve."""
    from oracle.solver import TwoLevel, solve_poisson
    N, n, D, dt, m = 1024, 5, 0.0, 2e-4, 16
    g, w, _ = _fields(dg, N, n, "random_phase")
    o = Operators(OGrid(N, N, n))
    sim = dg.Sim(g, dev(w), D=D, dt=dt, cg_tol=1e-10)
    sim.step(3)
    assert sim.status().status == 0
    bufs = [torch.empty(g.shape, dtype=torch.float64, device="cuda") for _ in range(5)]
    sim.get_state(*bufs)
    om, ps, pp, R1, R2 = [host(b) for b in bufs]
    J = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    dg.dg_bracket(g, bufs[1], bufs[0], J)
    Rk = -o.bracket(ps, om)
    # the bracket against the rounding scale of its products (|D| = rho_D / h ~ 3200 here
    # amplifies the rounding of both sides: plain relative L2 about 1e-11); the state after the
    # step is held to the plain 1e-12 below
    Jh = host(J)
    del J
    eJ = np.linalg.norm(Jh + Rk) / max(np.linalg.norm(Rk), _bracket_scale(o, ps, om))
    print("1024^2 n=5 bracket: plain rel L2 %.2e, scaled %.2e"
          % (np.linalg.norm(Jh + Rk) / np.linalg.norm(Rk), eJ))
    assert eJ < 1e-12, eJ
    del Jh
    sim.set_cg(1e-30, 1000, fixed_iters=m)
    sim.step(1)
    om1 = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    ps1 = torch.empty_like(om1)
    sim.get(om1, ps1)
    ref_w = om + dt * (23.0 * Rk - 16.0 * R1 + 5.0 * R2) / 12.0
    e_w = np.linalg.norm(host(om1) - ref_w) / np.linalg.norm(ref_w)
    assert e_w < 1e-12, e_w
    res = solve_poisson(o, ref_w, 2.0 * ps - pp, 1e-30, 1000, fixed_iters=m, precond=TwoLevel(o))
    assert res.iters == m
    # psi after the same 16 Krylov steps: two float64 evaluations of the same iteration differ
    # by their rounding amplified by the operator's condition number (about 5e7 here, the
    # smoothest modes carrying most of psi): observed 1.7e-10.  The bound is that of the
    # conditioning, and the iterate meets the solver tolerance on the oracle's operator.
    e_p = np.linalg.norm(host(ps1) - res.x) / np.linalg.norm(res.x)
    print("1024^2 n=5 psi after %d fixed iterations: rel L2 vs oracle %.2e" % (m, e_p))
    assert e_p < 1e-9, e_p
    # and the fixed-iteration solve is itself converged to the benchmark's tolerance, within the
    # rounding of the oracle's own residual evaluation at this condition number (see
    # test_poisson_true_residual: bound 2 tol)
    assert res.relres < 2e-10, res.relres


@pytest.mark.parametrize("N,n,kind", CASES)
@pytest.mark.parametrize("mode", ["mixed", "mixed64"])
def test_one_step_mixed_vs_oracle(dg, N, n, kind, mode):
    """The mixed-precision step at the benchmark sizes against the oracle: from the FP64 state
    after three steps, one DG_MIXED (double-float bracket) or DG_MIXED64 step; omega^{k+1}
    within 1e-10 of the oracle's AB3 update, psi^{k+1} meeting the 1e-10 tolerance on the
    oracle's own operator (bound 2e-10: the oracle's residual evaluation carries its own
    rounding at this condition number)."""
    g, w, _ = _fields(dg, N, n, kind)
    D, dt = (1e-4, 5e-4) if kind == "shear_layer" else (0.0, 2e-4)
    o = Operators(OGrid(N, N, n))
    a = dg.Sim(g, dev(w), D=D, dt=dt, precision=dg.DG_FP64, cg_tol=1e-10)
    a.step(3)
    st = [torch.empty(g.shape, dtype=torch.float64, device="cuda") for _ in range(5)]
    k = a.get_state(*st)
    a.close()
    om, ps, pp, R1, R2 = [host(b) for b in st]
    prec = {"mixed": dg.DG_MIXED, "mixed64": dg.DG_MIXED64}[mode]
    b = dg.Sim(g, st[0], D=D, dt=dt, precision=prec, cg_tol=1e-10)
    b.set_state(k, *st)
    b.step(1)
    assert b.status().status == 0
    w1 = torch.empty_like(st[0])
    p1 = torch.empty_like(st[0])
    b.get(w1, p1)
    del st
    Rk = -o.bracket(ps, om)
    if D != 0.0:
        Rk = Rk + D * o.laplacian(om)
    ref = om + dt * (23.0 * Rk - 16.0 * R1 + 5.0 * R2) / 12.0
    hw = host(w1)
    e_w = np.linalg.norm(hw - ref) / np.linalg.norm(ref)
    assert e_w < 1e-10, e_w
    bb = poisson_rhs(o, hw)
    r = bb - o.A(host(p1))
    relres = np.sqrt(np.sum(r * r / o.W2) / np.sum(bb * bb / o.W2))
    assert relres < 2e-10, relres


@pytest.mark.parametrize("mode", ["mixed", "mixed64", "fp64"])
@pytest.mark.parametrize("n", [4, 5])
def test_initial_solve_1024_shear_layer(dg, mode, n):
    """The start-up Poisson solve from psi = 0 on 1024^2 cells, n = 4 and 5, of a double shear
    layer, tolerance 1e-10.  There the float64 rounding of psi itself leaves a relative
    residual of about 2e-10 (n = 4) and 4e-10 (n = 5), above the tolerance: every solver
    stops at that floor (the stopping rule accepts a residual that stagnates below the
    rounding bound 2^-52 lambda_max |y|).  The mixed solves switch their inner operator apply to
    double-float when a refinement sweep stalls and reach the floor in a few sweeps; all three
    solutions agree to the attainable accuracy."""
    g, w, _ = _fields(dg, 1024, n, "shear_layer")
    prec = {"mixed": dg.DG_MIXED, "mixed64": dg.DG_MIXED64, "fp64": dg.DG_FP64}[mode]
    s = dg.Sim(g, dev(w), D=1e-4, dt=2e-4, precision=prec, cg_tol=1e-10)
    info = s.status()
    assert info.status == 0 and info.cg_relres_last < 1e-9, (info.status, info.cg_relres_last)
    if mode != "fp64":
        h = s.refinement_history()
        print("1024^2 n=%d shear, %s: %s" % (n, mode, " ".join("%.1e/%d" % x for x in h)))
        assert len(h) <= 12, h
    psi = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    s.get(None, psi)
    ref = dev(np.zeros(g.shape))
    rc, it, rr = dg.dg_poisson_solve(g, dev(w), ref, 1e-10, 100000)
    e = float(torch.linalg.norm(psi - ref) / torch.linalg.norm(ref))
    assert e < 1e-8, e
    s.step(3)
    assert s.status().status == 0
