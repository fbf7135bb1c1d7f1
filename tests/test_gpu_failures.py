"""Failure detection without a GPU fault: a device-side wait that nothing satisfies gives up
after its cap and reports DG_ERR_TIMEOUT, and the context stays usable; solver errors are
reported as status codes."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_wait_cap_reports_timeout_and_context_survives(native):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    dg = native
    rc = dg.lib().dg_selftest_wait_cap(dg._stream(None))
    assert rc == dg.DG_ERR_TIMEOUT, dg.lib().dg_last_error()
    # the context is still usable
    g = dg.Grid(8, 8, 2)
    w = torch.from_numpy(np.random.default_rng(0).standard_normal(g.shape)).cuda()
    psi = torch.zeros_like(w)
    rc, it, relres = dg.dg_poisson_solve(g, w, psi, 1e-12, 1000)
    assert rc == dg.DG_OK and relres <= 1e-12


def test_nonconvergence_is_reported_by_simulations(native):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    dg = native
    g = dg.Grid(16, 16, 3)
    w = torch.from_numpy(np.random.default_rng(1).standard_normal(g.shape)).cuda()
    s = dg.Sim(g, w, D=0.0, dt=1e-3, cg_tol=1e-12)
    s.set_cg(1e-14, 2)            # far too few iterations
    s.step(3)
    info = s.status(check=False)
    assert info.status == dg.DG_ERR_NOCONV
