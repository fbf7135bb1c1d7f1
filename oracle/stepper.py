"""Time stepping of  d omega/dt + {psi, omega} = D Delta omega,  -Delta psi = omega
(Eq. vorticity) -- oracle, test infrastructure only.

Sec. 6: explicit K-step Adams-Bashforth (K = 3 for the Navier-Stokes runs, K = 1..4 in
Table 4), the bracket of Eq. J, the LDG Laplacian for both the viscous term and the
Poisson solve, CG with an initial guess extrapolated from the last two solutions.

Readings where Sec. 6 is silent:
* start-up: the first K-1 steps are classical RK4 steps of the same dt (each RK stage
  solves the Poisson equation with the latest psi as initial guess);
* extrapolation: x0 = 2 psi^k - psi^{k-1} (linear in the last two solutions);
* the right-hand side R(omega) = -J(psi, omega) + D Delta_h omega, J = J(psi, omega).

bracket="naive" replaces J by J^{++} of Eq. J alone: the straightforward discretisation
that Sec. 6.2 (Figures 1-2) compares with the scheme.
"""
import numpy as np

from .solver import solve_poisson

# AB-K weights for R^k, R^{k-1}, ... (standard Adams-Bashforth coefficients).
AB_COEFFS = {
    1: (1.0,),
    2: (3.0 / 2.0, -1.0 / 2.0),
    3: (23.0 / 12.0, -16.0 / 12.0, 5.0 / 12.0),
    4: (55.0 / 24.0, -59.0 / 24.0, 37.0 / 24.0, -9.0 / 24.0),
}


class Simulation:
    """State: omega^k, psi^k, psi^{k-1}, the history R^{k-1}, R^{k-2}, ... and k."""

    def __init__(self, ops, omega0, D, dt, tol=1e-12, maxit=100000, K=3,
                 fixed_iters=0, psi0=None, precond="jacobi", bracket="arakawa"):
        """precond: "jacobi" (W^{-1}), "twolevel" (solver.TwoLevel) or "spectral"
        (solver.Spectral); bracket: "arakawa"
        (Eq. J) or "naive" (J^{++} alone)."""
        if bracket not in ("arakawa", "naive"):
            raise ValueError(bracket)
        self.bracket = bracket
        self.ops, self.D, self.dt = ops, float(D), float(dt)
        from .solver import Spectral, TwoLevel
        self.precond = {"twolevel": TwoLevel, "spectral": Spectral}.get(precond, lambda o: None)(ops)
        self.tol, self.maxit, self.K, self.fixed_iters = float(tol), int(maxit), int(K), int(fixed_iters)
        self.omega = np.array(omega0, dtype=np.float64, copy=True)
        if psi0 is None:
            res = self.solve(self.omega, np.zeros_like(self.omega))
            psi0 = res.x
        self.psi = np.array(psi0, dtype=np.float64, copy=True)
        self.psi_prev = self.psi.copy()
        self.R_hist = []          # R_hist[0] = R^{k-1}, R_hist[1] = R^{k-2}, ...
        self.k = 0
        self.cg_iters = []

    def solve(self, omega, x0):
        res = solve_poisson(self.ops, omega, x0, self.tol, self.maxit, self.fixed_iters, self.precond)
        if not res.converged:
            raise RuntimeError("CG did not converge within maxit")
        self.cg_iters_last = res.iters
        return res

    def rhs(self, psi, omega):
        """R = -J(psi, omega) + D Delta_h omega."""
        if self.bracket == "naive":
            R = -self.ops.bracket_parts(psi, omega)[0]
        else:
            R = -self.ops.bracket(psi, omega)
        if self.D != 0.0:
            R = R + self.D * self.ops.laplacian(omega)
        return R

    def _rk4_step(self):
        dt = self.dt
        w0, p0 = self.omega, self.psi
        k1 = self.rhs(p0, w0)
        wa = w0 + 0.5 * dt * k1
        pa = self.solve(wa, p0).x
        k2 = self.rhs(pa, wa)
        wb = w0 + 0.5 * dt * k2
        pb = self.solve(wb, pa).x
        k3 = self.rhs(pb, wb)
        wc = w0 + dt * k3
        pc = self.solve(wc, pb).x
        k4 = self.rhs(pc, wc)
        w_new = w0 + (dt / 6.0) * (k1 + 2.0 * k2 + 2.0 * k3 + k4)
        res = self.solve(w_new, pc)
        return k1, w_new, res

    def _ab_step(self):
        R = self.rhs(self.psi, self.omega)
        hist = [R] + self.R_hist
        c = AB_COEFFS[self.K]
        incr = sum(ci * Ri for ci, Ri in zip(c, hist[:self.K]))
        w_new = self.omega + self.dt * incr
        x0 = 2.0 * self.psi - self.psi_prev
        res = self.solve(w_new, x0)
        return R, w_new, res

    def step(self, nsteps=1):
        for _ in range(nsteps):
            if self.k < self.K - 1:
                R, w_new, res = self._rk4_step()
            else:
                R, w_new, res = self._ab_step()
            self.R_hist = ([R] + self.R_hist)[:max(self.K - 1, 0)]
            self.psi_prev = self.psi
            self.psi = res.x
            self.omega = w_new
            self.cg_iters.append(res.iters)
            self.k += 1
        return self

    def invariants(self):
        return self.ops.invariants(self.psi, self.omega)
