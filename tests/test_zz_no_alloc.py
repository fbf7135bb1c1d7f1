"""The allocation-free Poisson solve, dg_poisson_solve_static, for callers that cannot
allocate device memory (no dg_grid handle; all scratch in one static device array).

It must give what the allocating entry point dg_poisson_solve gives, on two calls in a row
(the static array keeps the previous call's contents, so the second call checks that nothing
stale leaks into it), within the float64 tolerance of the other parity tests.  This file is
named to be collected last."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def test_static_solve_matches_allocating_solve_twice(native):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    dg = native
    Nx, Ny, n, Lx, Ly, tau = 24, 20, 4, 2.0, 1.7, 0.0     # 7680 values, several tiles, ragged
    g = dg.Grid(Nx, Ny, n, Lx, Ly, tau)
    for call in range(2):
        rng = np.random.default_rng(100 + call)
        w = torch.from_numpy(rng.standard_normal(g.shape)).cuda()
        x0 = torch.from_numpy(0.01 * rng.standard_normal(g.shape)).cuda()
        a, b = x0.clone(), x0.clone()
        rc_a, it_a, rr_a = dg.dg_poisson_solve(g, w, a, tol=1e-12, maxit=20000)
        rc_b, it_b, rr_b = dg.dg_poisson_solve_static(Nx, Ny, n, Lx, Ly, tau, w, b, tol=1e-12, maxit=20000)
        torch.cuda.synchronize()
        assert rc_a == rc_b == dg.DG_OK
        assert it_a == it_b
        err = (torch.linalg.norm(a - b) / torch.linalg.norm(a)).item()
        assert err < 1e-12, (call, err)
        assert abs(rr_a - rr_b) <= 1e-12 * max(rr_a, 1e-300) or rr_a == rr_b
    # a third call with the same n, after the warm-up above: the device's free memory does not
    # change (nothing is allocated, not even by the CUDA runtime on our behalf)
    w = torch.from_numpy(np.random.default_rng(7).standard_normal(g.shape)).cuda()
    b = torch.zeros_like(w)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    rc, _, _ = dg.dg_poisson_solve_static(Nx, Ny, n, Lx, Ly, tau, w, b, tol=1e-12, maxit=20000)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert rc == dg.DG_OK and free1 == free0, (free0, free1)


def test_static_solve_rejects_oversized_grids(native):
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    dg = native
    w = torch.zeros((1,), dtype=torch.float64, device="cuda")
    rc, _, _ = dg.dg_poisson_solve_static(200, 200, 4, 1.0, 1.0, 0.0, w, w.clone(), check=False)
    assert rc == dg.DG_ERR_ARG
    assert b"static scratch" in dg.lib().dg_last_error()
