"""Parity at the full sizes the benchmarks time: 512^2 cells, n = 4 (double shear layer) and
1024^2 cells, n = 5 (random phase), in the launch configurations bench.py uses.

* The bracket J on sampled cells: J at a cell depends only on the 5x5 cells around it, so
  the oracle evaluates it on that patch of the true fields (as a periodic 5x5 grid of the
  same cell size) -- one cell at a time, independent of the full-grid run.
* The Poisson solve (two-level PCG, tolerance 1e-10): the oracle's own operator gives the
  true residual of the returned psi on the whole grid.
* One float64 step and one DG_MIXED64 step from the identical state agree to the solver
  tolerance; V is conserved by the step.
"""
import numpy as np
import pytest

from oracle.operators import Operators
from oracle.solver import poisson_rhs
from oracle.tables import Grid as OGrid
from paper_1311_7477_gb300 import fields

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
