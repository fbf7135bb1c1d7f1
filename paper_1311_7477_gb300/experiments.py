"""The Lamb dipole runs of Sec. 6.2 through the C ABI.

* table4(): the enstrophy and energy errors of the K-step Adams-Bashforth stepper at
  t = 0.01 (P = 1, N = 200), Table 4.
* dipole_shape(): the dipole at t = 0.5 with the bracket of Eq. J or J^{++} alone, the
  comparison of Figures 1 (P = 1, N = 100) and 2 (P = 4, N = 50).  The figures are not
  available as data, so the comparison is by norms: the relative L2 (Gauss-quadrature)
  distance from the exact dipole translated by U t, and the drifts of E and Omega.

Domain [0, 1]^2, U = 1, R = 0.1, D = 0, the dipole centred at (1/2, 1/2).  With
u = psi_y, v = -psi_x the positive lobe (cos theta > 0, x > 1/2) turns counter-clockwise
and the pair moves in -y; after t = 0.5 on the unit-periodic domain the centre is at
(1/2, 0), the same as (1/2, 1).
"""
import numpy as np

from . import fields, workloads


def _dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def lamb_sim(dg, N, n, dt, K=3, bracket="arakawa", tol=1e-13, precond="twolevel"):
    g = dg.Grid(N, N, n, 1.0, 1.0)
    g.set_precond(precond)
    xn, yn, _ = g.nodes()
    X, Y = fields.mesh_from_nodes(xn, yn)
    sim = dg.Sim(g, _dev(fields.lamb_dipole(X, Y)), D=0.0, dt=dt, cg_tol=tol, cg_maxit=200000)
    sim.set_multistep(K)
    sim.set_bracket(bracket)
    return g, sim, X, Y


def table4(dg, K, steps, t_end=0.01):
    """(eps_Omega, eps_E, V) after `steps` steps to t_end (P = 1, N = 200)."""
    g, sim, _, _ = lamb_sim(dg, 200, 1, t_end / steps, K=K)
    V0, E0, O0 = sim.invariants()
    sim.step(steps)
    V, E, O = sim.invariants()
    sim.close()
    g.close()
    return abs((O - O0) / O0), abs((E - E0) / E0), V


def translated_dipole(X, Y, t, U=1.0):
    """The exact dipole moved by U t in -y, periodically wrapped to the nearest image."""
    yc = (0.5 - U * t) % 1.0
    dy = (Y - yc + 0.5) % 1.0 - 0.5
    return fields.lamb_dipole(X, yc + dy, xc=0.5, yc=yc)


def dipole_shape(dg, N, n, bracket, t_end=0.5, U_bound=4.0, tol=1e-11):
    """Runs the dipole to t_end (CG tolerance tol); returns a dict of the shape error and the
    invariant drifts."""
    import torch
    dt = workloads.stable_dt(dg, N, n, 0.0, L=1.0, U=U_bound, dt_cap=1e-3)
    steps = int(np.ceil(t_end / dt))
    dt = t_end / steps
    g, sim, X, Y = lamb_sim(dg, N, n, dt, K=3, bracket=bracket, tol=tol)
    V0, E0, O0 = sim.invariants()
    sim.step(steps)
    V, E, O = sim.invariants()
    om = torch.empty(g.shape, dtype=torch.float64, device="cuda")
    sim.get(om, None)
    torch.cuda.synchronize()
    w = om.cpu().numpy()
    ex = translated_dipole(X, Y, t_end)
    _, _, wts = g.nodes()
    err = float(np.sqrt(np.sum(wts * (w - ex) ** 2) / np.sum(wts * ex ** 2)))
    st = sim.status()
    sim.close()
    g.close()
    return {"N": N, "n": n, "bracket": bracket, "steps": steps, "dt": dt, "shape_error": err,
            "eps_E": abs((E - E0) / E0), "eps_Omega": abs((O - O0) / O0), "V": V, "status": st.status}
