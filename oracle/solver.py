"""Conjugate-gradient Poisson solve -Delta_h psi = omega (Sec. 6) -- oracle, test only.

The dG Laplacian Delta_h = -W^{-1} A with A symmetric positive semi-definite (kernel =
constants), so -Delta_h psi = omega is the symmetric system  A psi = W omega.  Sec. 6
states only that a conjugate gradient method solves it; the details below are a reading
(parity unpinned for the choice itself, pinned for the result it converges to):

* right-hand side b = W (omega - mean_W(omega)), mean_W(u) = sum W u / sum W, so that
  the system is consistent (b is orthogonal to the constants);
* preconditioner W^{-1} (the inverse of the diagonal X-space mass matrix, Eq. diagonal);
* stopping rule  r . W^{-1} r <= tol^2 * b . W^{-1} b  (relative residual in the
  discrete L2 norm of Eq. def_norm), or a fixed iteration count (parity mode).  The rule is
  on the true residual b - A x: when the recursively updated residual of CG meets it, the
  true residual is computed; if that one does not, CG restarts from it (p = W^{-1} r), at
  most MAX_RESTARTS times.  (Over thousands of iterations the recursive residual drifts away
  from the true one by rounding.)

With x0 of W-mean zero all iterates stay W-mean zero, since every update direction
z = W^{-1} r satisfies sum W z = sum r = 0.
"""
import numpy as np


def poisson_rhs(ops, omega):
    """b = W (omega - mean_W omega).  The mean is evaluated in two passes (the mean of the
    first-pass deviations corrects the first pass), so that b has no rounding-sized component
    along the constants, the kernel of A."""
    W = ops.W2
    sW = float(np.sum(W))
    m1 = float(np.sum(W * omega)) / sW
    m2 = float(np.sum(W * (omega - m1))) / sW
    return W * (omega - (m1 + m2))


MAX_RESTARTS = 20


class CGResult:
    def __init__(self, x, iters, relres, converged):
        self.x, self.iters, self.relres, self.converged = x, iters, relres, converged


def pcg(ops, b, x0, tol, maxit, fixed_iters=0):
    """Preconditioned CG for A x = b with preconditioner W^{-1}.

    Stops when r.W^{-1}r <= tol^2 b.W^{-1}b (fixed_iters == 0) or after exactly
    fixed_iters iterations (fixed_iters > 0); an exactly zero residual also stops.
    Returns a CGResult; converged is False when maxit was reached first."""
    W = ops.W2
    x = np.array(x0, dtype=np.float64, copy=True)
    rho_b = float(np.sum(b * b / W))
    if rho_b == 0.0:
        return CGResult(np.zeros_like(x), 0, 0.0, True)
    r = b - ops.A(x)
    z = r / W
    p = z.copy()
    rho = float(np.sum(r * z))
    it = 0
    restarts = 0
    converged = True
    while True:
        if fixed_iters > 0:
            if it == fixed_iters:
                break
        elif rho <= tol * tol * rho_b:
            r_true = b - ops.A(x)
            rho_true = float(np.sum(r_true * r_true / W))
            if rho_true <= tol * tol * rho_b or restarts == MAX_RESTARTS:
                rho = rho_true
                converged = rho_true <= tol * tol * rho_b
                break
            restarts += 1
            r = r_true
            z = r / W
            p = z.copy()
            rho = float(np.sum(r * z))
            continue
        if rho == 0.0:
            break
        if it == maxit:
            converged = False
            break
        q = ops.A(p)
        alpha = rho / float(np.sum(p * q))
        x = x + alpha * p
        r = r - alpha * q
        z = r / W
        rho_new = float(np.sum(r * z))
        beta = rho_new / rho
        p = z + beta * p
        rho = rho_new
        it += 1
    return CGResult(x, it, float(np.sqrt(max(rho, 0.0) / rho_b)), converged)


def solve_poisson(ops, omega, x0, tol, maxit, fixed_iters=0):
    """psi with -Delta_h psi = omega - mean_W(omega), by pcg from x0."""
    return pcg(ops, poisson_rhs(ops, omega), x0, tol, maxit, fixed_iters)


def solve_poisson_dense(dense, omega_global):
    """Tiny-grid direct solve: (A + (W1)(W1)^T) psi = b, whose unique solution is the
    W-mean-zero solution of A psi = b.  dense = operators.dense_ops_2d(...); arrays in the
    global node order."""
    A, W = dense["A"], dense["W"]
    w = omega_global.ravel()
    b = W * (w - np.sum(W * w) / np.sum(W))
    M = A + np.outer(W, W)
    return np.linalg.solve(M, b).reshape(omega_global.shape)
