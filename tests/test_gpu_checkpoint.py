"""Checkpoint and resume (dg_sim_save / dg_sim_load): a run saved at step k and resumed
from the file continues bit-identically to the uninterrupted run, in every precision mode,
for K = 3 and K = 4 and both brackets; the file must match the grid it is loaded on."""
import os

import numpy as np
import pytest

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


def state(dg, sim, g):
    om = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    ps = torch.empty_like(om)
    sim.get(om, ps)
    torch.cuda.synchronize()
    return om.cpu().numpy(), ps.cpu().numpy()


def make(dg, prec, precond="twolevel", N=24, n=3):
    g = dg.Grid(N, N, n)
    g.set_precond(precond)
    xn, yn, _ = g.nodes()
    X, Y = fields.mesh_from_nodes(xn, yn)
    w0 = fields.random_phase(X, Y, seed=5, kmax=6)
    return g, w0


@pytest.mark.parametrize("prec", ["fp64", "mixed", "mixed64"])
@pytest.mark.parametrize("K,bracket", [(3, "arakawa"), (4, "arakawa"), (3, "naive")])
def test_resume_is_bit_identical(dg, tmp_path, prec, K, bracket):
    P = {"fp64": dg.DG_FP64, "mixed": dg.DG_MIXED, "mixed64": dg.DG_MIXED64}[prec]
    g, w0 = make(dg, P)
    a = dg.Sim(g, dev(w0), D=1e-3, dt=2e-3, precision=P, cg_tol=1e-11)
    a.set_multistep(K)
    a.set_bracket(bracket)
    a.set_cg(1e-11, 5000)
    a.step(4)
    path = os.path.join(tmp_path, "sim.dgs")
    a.save(path)
    a.step(5)
    wa, pa = state(dg, a, g)
    b = dg.Sim.load(g, path)
    assert b.status().step == 4
    b.step(5)
    wb, pb = state(dg, b, g)
    assert b.status().step == 9
    assert np.array_equal(wa, wb) and np.array_equal(pa, pb)


def test_load_rejects_other_grid_and_bad_files(dg, tmp_path):
    g, w0 = make(dg, dg.DG_FP64)
    s = dg.Sim(g, dev(w0), D=0.0, dt=1e-3)
    path = os.path.join(tmp_path, "a.dgs")
    s.save(path)
    other = dg.Grid(24, 24, 2)
    with pytest.raises(RuntimeError, match="DG_ERR_ARG"):
        dg.Sim.load(other, path)
    jac = dg.Grid(24, 24, 3)
    with pytest.raises(RuntimeError, match="DG_ERR_ARG"):
        dg.Sim.load(jac, path)            # preconditioner differs (Jacobi vs two-level)
    data = open(path, "rb").read()
    bad = os.path.join(tmp_path, "b.dgs")
    open(bad, "wb").write(b"XX" + data[2:])
    with pytest.raises(RuntimeError, match="DG_ERR_IO"):
        dg.Sim.load(g, bad)
    open(bad, "wb").write(data[:len(data) // 2])
    with pytest.raises(RuntimeError, match="DG_ERR_IO"):
        dg.Sim.load(g, bad)
    with pytest.raises(RuntimeError, match="DG_ERR_IO"):
        dg.Sim.load(g, os.path.join(tmp_path, "missing.dgs"))
    with pytest.raises(RuntimeError, match="DG_ERR_IO"):
        s.save(os.path.join(tmp_path, "no_such_dir", "x.dgs"))
