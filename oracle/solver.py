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
* the tolerance cannot ask for less than float64 can hold: rounding the exact solution to
  float64 and evaluating b - A x in float64 leave a residual of up to about
  2 u lambda_max |W^{1/2} x| in the norm above (u = 2^-53, lambda_max the largest
  eigenvalue of W^{-1/2} A W^{-1/2}); so the true residual is also accepted once it is below
  that floor and no longer falls (less than a factor 4 below the previous check), with
  lambda_max bounded by the operator's row sums (rounding_floor2).  On fine grids with
  smooth solutions (1024^2 cells, n = 5, a double shear layer) the attainable residual is
  about 3e-10, above a tolerance of 1e-10.

With x0 of W-mean zero all iterates stay W-mean zero, since every update direction
z = W^{-1} r satisfies sum W z = sum r = 0.

Two further preconditioners (design choices; Sec. 6 names none): the additive two-level one
of TwoLevel below (exact solves on every cell plus an exact solve of the Galerkin coarse
problem on cell averages), which makes the iteration count independent of the mesh size, and
Spectral, the exact pseudo-inverse of A on the periodic grid, with which CG converges in one
iteration.  Neither changes the solution CG converges to.
"""
import numpy as np

from .operators import ldg_matrix_1d


def poisson_rhs(ops, omega):
    """b = W (omega - mean_W omega).  The mean is evaluated in two passes (the mean of the
    first-pass deviations corrects the first pass), so that b has no rounding-sized component
    along the constants, the kernel of A.  With homogeneous Dirichlet boundaries A is
    definite and b = W omega."""
    W = ops.W2
    if getattr(ops, "bc", "periodic") == "dirichlet":
        return W * omega
    sW = float(np.sum(W))
    m1 = float(np.sum(W * omega)) / sW
    m2 = float(np.sum(W * (omega - m1))) / sW
    return W * (omega - (m1 + m2))


MAX_RESTARTS = 20


def rounding_floor2(ops):
    """(2^-52 lambda)^2 with lambda the Gershgorin bound (largest absolute row sum) of
    W^{-1/2} A W^{-1/2} = I (x) A1x^ + A1y^ (x) I, A1^ = w^{-1/2} A1 w^{-1/2} per direction: the
    squared float64 rounding floor of the relative residual per unit of W x . x."""
    g = ops.g
    n = g.n
    bound = 0.0
    for h, w in ((g.hx, ops.wx), (g.hy, ops.wy)):
        # the rows of the middle cell of a periodic 3-cell line (a Dirichlet boundary cell's
        # rows are smaller: this bounds both)
        A1 = ldg_matrix_1d(g.t, 3, h, ops.tau)[n:2 * n, :]
        sw = np.sqrt(np.tile(w, 3))
        bound += float(np.max(np.sum(np.abs(A1 / np.sqrt(w)[:, None] / sw[None, :]), axis=1)))
    return (2.0 ** -52 * bound) ** 2


class TwoLevel:
    """Additive two-level preconditioner  M^{-1} = B + P A_c^+ P^T  for A (Sec. 6 operator):

    * B: on every cell, the inverse of the cell's own diagonal block of A,
      A_cc = W_y (x) A1_cc,x + A1_cc,y (x) W_x  (A1_cc = the own-cell block of the 1D LDG
      stiffness); identical for all cells of the uniform grid;
    * P: prolongation of one value per cell to all nodes of the cell (piecewise constants);
    * A_c = P^T A P: the Galerkin coarse operator on the cells -- periodic and translation
      invariant, hence diagonalised by the 2D DFT; its eigenvalues are the DFT of its stencil
      (A applied to the indicator of one cell, summed per cell).  A_c^+ is the pseudo-inverse
      that drops the constant mode (A_c's kernel, the constants).
    B and A_c^+ are symmetric and B is positive definite, so M^{-1} is symmetric positive
    definite and PCG applies."""

    def __init__(self, ops):
        g = ops.g
        n = g.n
        t = g.t
        if getattr(ops, "bc", "periodic") != "periodic":
            raise ValueError("the two-level preconditioner is built for periodic grids")
        A1x = ldg_matrix_1d(t, 3, g.hx, ops.tau)[n:2 * n, n:2 * n]
        A1y = ldg_matrix_1d(t, 3, g.hy, ops.tau)[n:2 * n, n:2 * n]
        Acc = np.kron(np.diag(ops.wy), A1x) + np.kron(A1y, np.diag(ops.wx))   # node index a*n + b
        self.Binv = np.linalg.inv(Acc)
        e = g.zeros()
        e[0, 0] = 1.0
        stencil = ops.A(e).sum(axis=(2, 3))                 # first column of A_c (circulant)
        lam = np.fft.fft2(stencil).real
        inv = np.zeros_like(lam)
        nz = np.ones_like(lam, dtype=bool)
        nz[0, 0] = False                                     # the constant mode
        inv[nz] = 1.0 / lam[nz]
        self.lam, self.lam_inv = lam, inv
        self.n = n

    def coarse_solve(self, rc):
        """A_c^+ rc by the 2D DFT (rc of shape (Ny, Nx))."""
        return np.fft.ifft2(np.fft.fft2(rc) * self.lam_inv).real

    def __call__(self, r):
        Ny, Nx, n, _ = r.shape
        zb = np.einsum("ij,yxj->yxi", self.Binv, r.reshape(Ny, Nx, n * n)).reshape(r.shape)
        uc = self.coarse_solve(r.sum(axis=(2, 3)))
        return zb + uc[:, :, None, None]


class Spectral:
    """Exact preconditioner  M^{-1} = A^+  (the pseudo-inverse of the Sec. 6 operator, a design
    choice; Sec. 6 names no preconditioner): on the uniform periodic grid A is block-circulant
    in cx and in cy, so the 2D DFT over cells splits it into one n^2 x n^2 block per wave
    vector (kx, ky),
        A(kx, ky) = W_y (x) A1_x(kx) + A1_y(ky) (x) W_x,   A1(k) = sum_d B_d exp(2 pi i k d / N),
    B_d the block of the 1D LDG stiffness that couples a cell to its neighbour d cells on
    (d = -1, 0, 1).  Each block is solved exactly; the block of (0, 0) is singular (its
    kernel: the constants) and takes its pseudo-inverse.  The result is returned with W-mean
    zero.  PCG with M^{-1} = A^+ converges in one iteration in exact arithmetic."""

    def __init__(self, ops):
        g = ops.g
        n = g.n
        if getattr(ops, "bc", "periodic") != "periodic":
            raise ValueError("the spectral preconditioner is built for periodic grids")
        def symbol(Nc, h):
            A3 = ldg_matrix_1d(g.t, 3, h, ops.tau)[n:2 * n, :]        # middle cell of a 3-cell line
            Bm, B0, Bp = A3[:, :n], A3[:, n:2 * n], A3[:, 2 * n:]
            th = 2.0 * np.pi * np.arange(Nc) / Nc
            return (B0[None] + np.exp(1j * th)[:, None, None] * Bp[None]
                    + np.exp(-1j * th)[:, None, None] * Bm[None])          # (Nc, n, n)
        Ax = symbol(g.Nx, g.hx)
        Ay = symbol(g.Ny, g.hy)
        Wx, Wy = np.diag(ops.wx), np.diag(ops.wy)
        blocks = (np.einsum("ab,xij->xaibj", Wy, Ax)[None]               # W_y (x) A1_x(kx)
                  + np.einsum("yab,ij->yaibj", Ay, Wx)[:, None])          # A1_y(ky) (x) W_x
        blocks = blocks.reshape(g.Ny, g.Nx, n * n, n * n)
        self.inv = np.empty_like(blocks)
        for ky in range(g.Ny):
            for kx in range(g.Nx):
                if kx == 0 and ky == 0:
                    self.inv[ky, kx] = np.linalg.pinv(blocks[ky, kx], rcond=1e-12, hermitian=True)
                else:
                    self.inv[ky, kx] = np.linalg.inv(blocks[ky, kx])
        self.W = ops.W2
        self.n = n

    def __call__(self, r):
        Ny, Nx, n, _ = r.shape
        rh = np.fft.fft2(r.reshape(Ny, Nx, n * n), axes=(0, 1))
        zh = np.einsum("yxij,yxj->yxi", self.inv, rh)
        z = np.fft.ifft2(zh, axes=(0, 1)).real.reshape(r.shape)
        return z - float(np.sum(self.W * z)) / float(np.sum(self.W))


class CGResult:
    def __init__(self, x, iters, relres, converged):
        self.x, self.iters, self.relres, self.converged = x, iters, relres, converged


def pcg(ops, b, x0, tol, maxit, fixed_iters=0, precond=None):
    """Preconditioned CG for A x = b; preconditioner W^{-1} (precond=None) or a callable
    z = M^{-1} r (e.g. TwoLevel(ops)).

    Stops when r.W^{-1}r <= tol^2 b.W^{-1}b on the true residual (fixed_iters == 0) or after
    exactly fixed_iters iterations (fixed_iters > 0); an exactly zero residual also stops.
    Returns a CGResult; converged is False when maxit was reached first."""
    W = ops.W2
    M = precond if precond is not None else (lambda r: r / W)
    x = np.array(x0, dtype=np.float64, copy=True)
    rho_b = float(np.sum(b * b / W))
    if rho_b == 0.0:
        return CGResult(np.zeros_like(x), 0, 0.0, True)
    r = b - ops.A(x)
    z = M(r)
    p = z.copy()
    rz = float(np.sum(r * z))
    rr = float(np.sum(r * r / W))
    floor2 = rounding_floor2(ops)
    rr_prev = None      # true residual at the previous check
    it = 0
    restarts = 0
    converged = True
    while True:
        if fixed_iters > 0:
            if it == fixed_iters:
                break
        elif rr <= tol * tol * rho_b:
            r_true = b - ops.A(x)
            rr_true = float(np.sum(r_true * r_true / W))
            stagnated = (rr_true <= floor2 * float(np.sum(W * x * x)) and rr_prev is not None
                         and rr_true > 0.25 * rr_prev)
            if rr_true <= tol * tol * rho_b or stagnated or restarts == MAX_RESTARTS:
                rr = rr_true
                converged = rr_true <= tol * tol * rho_b or stagnated
                break
            rr_prev = rr_true
            restarts += 1
            r = r_true
            z = M(r)
            p = z.copy()
            rz = float(np.sum(r * z))
            rr = rr_true
            continue
        if rr == 0.0:
            break
        if it == maxit:
            converged = False
            break
        q = ops.A(p)
        pq = float(np.sum(p * q))
        if pq <= 0.0 and fixed_iters > 0:
            break          # exact convergence reached before the fixed count (tiny systems)
        alpha = rz / pq
        x = x + alpha * p
        r = r - alpha * q
        z = M(r)
        rz_new = float(np.sum(r * z))
        rr = float(np.sum(r * r / W))
        beta = rz_new / rz
        p = z + beta * p
        rz = rz_new
        it += 1
    if precond is not None:
        # A preconditioner other than W^{-1} may move x along the constants (the kernel of
        # A, invisible to the residual); the solution is the W-mean-zero one (G7 reading).
        x = x - float(np.sum(W * x)) / float(np.sum(W))
    return CGResult(x, it, float(np.sqrt(max(rr, 0.0) / rho_b)), converged)


def solve_poisson(ops, omega, x0, tol, maxit, fixed_iters=0, precond=None):
    """psi with -Delta_h psi = omega - mean_W(omega), by pcg from x0."""
    return pcg(ops, poisson_rhs(ops, omega), x0, tol, maxit, fixed_iters, precond)


def solve_poisson_dense(dense, omega_global, bc="periodic"):
    """Tiny-grid direct solve: (A + (W1)(W1)^T) psi = b, whose unique solution is the
    W-mean-zero solution of A psi = b (periodic); A psi = W omega (Dirichlet, A definite).
    dense = operators.dense_ops_2d(...); arrays in the global node order."""
    A, W = dense["A"], dense["W"]
    w = omega_global.ravel()
    if bc == "dirichlet":
        return np.linalg.solve(A, W * w).reshape(omega_global.shape)
    b = W * (w - np.sum(W * w) / np.sum(W))
    M = A + np.outer(W, W)
    return np.linalg.solve(M, b).reshape(omega_global.shape)
