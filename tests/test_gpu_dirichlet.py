"""Homogeneous Dirichlet boundaries on the GPU (dg_grid_create_bc) against the FP64 oracle
with the same reading (tests/test_oracle_dirichlet.py): the bracket (float64 and
double-float), Table 2's Dirichlet row, the LDG operator, the Poisson solve, one time step
(float64 at fixed CG iterations, and the mixed modes), and a batched Dirichlet member."""
import json
import os

import numpy as np
import pytest

from oracle.operators import Operators, dense_ops_2d, from_global, to_global
from oracle.solver import solve_poisson, solve_poisson_dense
from oracle.stepper import Simulation
from oracle.tables import Grid as OGrid
from paper_1311_7477_gb300 import fields
from tests.test_gpu_parity import bracket_scale, rel_l2

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GRIDS = [  # (Nx, Ny, n, Lx, Ly): several tiles, ragged edges, single cells
    (13, 11, 1, 2 * np.pi, 2 * np.pi),
    (19, 9, 2, 2.0, 3.0),
    (21, 18, 3, 2 * np.pi, 2 * np.pi),
    (17, 10, 4, 1.5, 1.0),
    (11, 13, 5, 2 * np.pi, 2 * np.pi),
    (1, 5, 4, 1.0, 2.0),
    (6, 1, 2, 1.0, 1.0),
]


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
@pytest.mark.parametrize("mixed", [False, True])
def test_dirichlet_bracket_parity(dg, Nx, Ny, n, Lx, Ly, mixed):
    g = dg.Grid(Nx, Ny, n, Lx, Ly, bc="dirichlet")
    o = Operators(OGrid(Nx, Ny, n, Lx, Ly), bc="dirichlet")
    f, h = np.random.default_rng(Nx * 10 + n).standard_normal((2, Ny, Nx, n, n))
    J = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    (dg.dg_bracket_mixed if mixed else dg.dg_bracket)(g, dev(f), dev(h), J)
    ref = o.bracket(f, h)
    got = host(J)
    assert rel_l2(got, ref, bracket_scale(o, f, h)) < 1e-12
    if Nx > 1 and Ny > 1:
        assert rel_l2(got, ref) < 1e-12, rel_l2(got, ref)


def test_dirichlet_table2_on_the_gpu(dg):
    from tests.test_oracle_bracket import _printed_match
    gold = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "table2_dirichlet.json")))
    g = dg.Grid(112, 112, 3, np.pi, np.pi, bc="dirichlet")
    xn, yn, W = g.nodes()
    X, Y = fields.mesh_from_nodes(xn, yn)
    f, gg = fields.table2_pair(X, Y)
    J = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    dg.dg_bracket(g, dev(f), dev(gg), J)
    Jh = host(J)
    W4 = np.broadcast_to(W[None, None], f.shape)
    vals = (np.sum(W4 * Jh), np.sum(W4 * f * Jh), np.sum(W4 * gg * Jh))
    for v, p in zip(vals, gold["row"]):
        assert _printed_match(v, p), (v, p)


@pytest.mark.parametrize("Nx,Ny,n,Lx,Ly", GRIDS)
def test_dirichlet_laplace_parity(dg, Nx, Ny, n, Lx, Ly):
    g = dg.Grid(Nx, Ny, n, Lx, Ly, bc="dirichlet")
    o = Operators(OGrid(Nx, Ny, n, Lx, Ly), bc="dirichlet")
    u = np.random.default_rng(5 + n).standard_normal(g.shape)
    y = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    dg.dg_laplace_apply(g, dev(u), y, 0)
    assert rel_l2(host(y), o.A(u)) < 1e-12
    dg.dg_laplace_apply(g, dev(u), y, 1)
    assert rel_l2(host(y), o.laplacian(u)) < 1e-12


def test_dirichlet_poisson(dg):
    # fixed iterations: the same Krylov steps as the oracle's PCG with W^-1
    Nx, Ny, n = 14, 11, 3
    g = dg.Grid(Nx, Ny, n, 2.0, 1.5, bc="dirichlet")
    o = Operators(OGrid(Nx, Ny, n, 2.0, 1.5), bc="dirichlet")
    rng = np.random.default_rng(8)
    w = rng.standard_normal(g.shape)
    x0 = 0.1 * rng.standard_normal(g.shape)
    ref = solve_poisson(o, w, x0, 1e-30, 1000, fixed_iters=20)
    psi = dev(x0)
    rc, it, relres = dg.dg_poisson_solve(g, dev(w), psi, 1e-30, 1000, fixed_iters=20)
    assert it == 20 and rel_l2(host(psi), ref.x) < 1e-12
    # converged: the dense direct solve (A definite, no mean removed)
    og = OGrid(5, 4, 2, 1.3, 1.1)
    g2 = dg.Grid(5, 4, 2, 1.3, 1.1, bc="dirichlet")
    w2 = rng.standard_normal(g2.shape)
    d = from_global(solve_poisson_dense(dense_ops_2d(og, bc="dirichlet"), to_global(w2), bc="dirichlet"), 2)
    p2 = dev(np.zeros(g2.shape))
    dg.dg_poisson_solve(g2, dev(w2), p2, 1e-14, 10000)
    assert rel_l2(host(p2), d) < 1e-12
    with pytest.raises(dg.DGError):
        g.set_precond("twolevel")


@pytest.mark.parametrize("k", [0, 3])
@pytest.mark.parametrize("mode", ["fp64", "mixed", "mixed64"])
def test_dirichlet_one_step(dg, k, mode):
    Nx, Ny, n, D, dt, m = 12, 10, 3, 2e-3, 2e-3, 40
    og = OGrid(Nx, Ny, n)
    o = Operators(og, bc="dirichlet")
    X, Y = og.mesh()
    w0 = 2.0 * np.sin(X) * np.sin(Y) + 0.3 * np.sin(2 * X) * np.sin(3 * Y)
    osim = Simulation(o, w0, D, dt, tol=1e-13, K=3, fixed_iters=m if mode == "fp64" else 0)
    osim.step(k)
    g = dg.Grid(Nx, Ny, n, bc="dirichlet")
    z = np.zeros(g.shape)
    R1 = osim.R_hist[0] if len(osim.R_hist) > 0 else z
    R2 = osim.R_hist[1] if len(osim.R_hist) > 1 else z
    prec = {"fp64": dg.DG_FP64, "mixed": dg.DG_MIXED, "mixed64": dg.DG_MIXED64}[mode]
    sim = dg.Sim(g, dev(osim.omega), D=D, dt=dt, precision=prec, cg_tol=1e-13)
    sim.set_state(k, dev(osim.omega), dev(osim.psi), dev(osim.psi_prev), dev(R1), dev(R2))
    if mode == "fp64":
        sim.set_cg(1e-30, 1000, fixed_iters=m)
    sim.step(1)
    osim.step(1)
    om = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    ps = torch.empty_like(om)
    sim.get(om, ps)
    bar = 1e-12 if mode == "fp64" else 1e-10
    assert rel_l2(host(om), osim.omega) < bar, rel_l2(host(om), osim.omega)
    assert rel_l2(host(ps), osim.psi) < bar, rel_l2(host(ps), osim.psi)
    assert sim.status().status == 0


def test_dirichlet_member_in_a_batch(dg):
    """A Dirichlet grid and a periodic one advanced together match the same steps alone."""
    def make(bc, N, n, seed):
        g = dg.Grid(N, N, n, bc=bc)
        xn, yn, _ = g.nodes()
        X, Y = fields.mesh_from_nodes(xn, yn)
        w = 2.0 * np.sin(X) * np.sin(Y) + 0.1 * fields.random_phase(X, Y, seed=seed, kmax=4)
        if bc == "dirichlet":
            w = w * np.sin(X / 2) * np.sin(Y / 2)          # vanishes on the boundary of [0, 2 pi]^2
        return g, dg.Sim(g, dev(w), D=1e-3, dt=2e-3, precision=dg.DG_FP64, cg_tol=1e-12)
    specs = [("dirichlet", 24, 3, 1), ("periodic", 20, 4, 2), ("dirichlet", 16, 5, 3)]
    members = [make(*s) for s in specs]
    alone = [make(*s) for s in specs]
    b = dg.Batch(4)
    for _, s in members:
        b.admit(s)
    b.step(4)
    for _, s in alone:
        s.step(6)
    for (ga, sa), (gb, sb) in zip(alone, members):
        wa = torch.empty(ga.shape, dtype=torch.float64, device="cuda")
        wb = torch.empty_like(wa)
        sa.get(wa, None)
        sb.get(wb, None)
        assert float(torch.linalg.norm(wa - wb) / torch.linalg.norm(wa)) < 1e-8
    assert b.status()["rc"] == 0
