"""dG operators of Secs. 3, 4.2 and 6 (oracle; test infrastructure only).

Two equivalent forms are kept, so that each can be checked against the other:

* dense matrices for tiny grids, assembled exactly as printed: the L-space block
  matrix  Mbar = 1/2 (1^+ (x) RL + 1 (x) (D - D^T) - 1^- (x) LR)  with its periodic
  corner blocks (Eq. discrete_der), mapped to X-space by (1 (x) B T) Mbar (1 (x) F)
  (Eq. matrix_xspace with F = T B^T W), and extended to 2D by Kronecker products
  (Sec. 4.2, last paragraph) in the global node order [Y][X];
* block application on the cell-blocked array f[cy, cx, a, b]: per cell, the same
  three X-space blocks (own cell, right neighbour, left neighbour) applied with
  np.einsum, the neighbours taken with np.roll (periodic wrap).

Derivatives act on the x-node index b (D_x) or the y-node index a (D_y); products of
fields are pointwise in X-space, (fg)_{ni} = f_{ni} g_{ni} (Sec. 4.2).

Boundary conditions: periodic (the default) or homogeneous Dirichlet (bc="dirichlet").
Dirichlet derivative: the numerical flux on a boundary face is the boundary value f^ = 0
(Sec. 3 with the field zero outside); the boundary cells' own L-space blocks become
1/2 R - D^T (first cell) and -1/2 L - D^T (last cell), i.e. 1/2 (D - D^T) + 1/2 L and
1/2 (D - D^T) - 1/2 R, and the periodic corner blocks drop out.  (The corner diagonal blocks
printed in Mbar^dir of Sec. 4.2, 1/2 (D - D^T), do not reproduce the Dirichlet row of
Table 2; these reproduce it to every printed digit.)  For the LDG Laplacian the paper names
no boundary treatment; the reading used here takes u^ = 0 in the forward derivative's flux
on both boundary faces (in the first cell the left-face term -L of the own block drops out)
and penalises the trace on the left boundary face, where q^ is taken from inside:
A1 = D+^T W D+ + (tau_b / h) l_L l_L^T on the first cell (DIRICHLET_PENALTY = tau_b).
"""
import numpy as np

from .tables import Grid


# ----------------------------------------------------------------------------------
# 1D blocks in X-space
# ----------------------------------------------------------------------------------

def central_blocks(t, h):
    """X-space blocks (own, right neighbour c+1, left neighbour c-1) of the 1D derivative
    with the standard flux f^ = (f^+ + f^-)/2 (Eq. standard-flux, Eq. discrete_der):
    L-space blocks 1/2 (D - D^T), 1/2 RL, -1/2 LR, each mapped as B T (.) F."""
    BT = t.B @ t.T(h)
    return (BT @ (0.5 * (t.D - t.D.T)) @ t.F,
            BT @ (0.5 * t.RL) @ t.F,
            BT @ (-0.5 * t.LR) @ t.F)


def forward_blocks(t, h):
    """X-space blocks (own, right neighbour) of the 1D derivative whose flux is taken from
    the right cell, f^_{n+1/2} = f^{n+1}(-1) (the LDG flux choice; Sec. 6, reading of the
    Cockburn-Shu method).  Inserting that flux into Eq. discrete_derivative gives the
    L-space blocks (-L - D^T) on the own cell and RL on the right neighbour."""
    BT = t.B @ t.T(h)
    return BT @ (-t.L - t.D.T) @ t.F, BT @ t.RL @ t.F


def trace_vectors(t):
    """X-space face interpolants: u(-1) = lL . u and u(+1) = lR . u with lL = F^T p(-1),
    lR = F^T p(+1) (f(x) = sum_k fbar^k p_k(x), fbar = F f)."""
    return t.F.T @ t.pL, t.F.T @ t.pR


# ----------------------------------------------------------------------------------
# Dense assembly (tiny grids)
# ----------------------------------------------------------------------------------

def mbar_dirichlet(t, N):
    """L-space block matrix Mbar_x^dir (N cells, homogeneous Dirichlet, f^ = 0 on the boundary
    faces): Mbar^per without its corner blocks, the first and last diagonal blocks corrected
    by +1/2 L and -1/2 R."""
    n = t.n
    M = np.zeros((N * n, N * n))
    for c in range(N):
        r = slice(c * n, (c + 1) * n)
        M[r, r] += 0.5 * (t.D - t.D.T)
        if c == 0:
            M[r, r] += 0.5 * t.L
        if c == N - 1:
            M[r, r] -= 0.5 * t.R
        if c + 1 < N:
            M[r, (c + 1) * n:(c + 2) * n] += 0.5 * t.RL
        if c > 0:
            M[r, (c - 1) * n:c * n] += -0.5 * t.LR
    return M


def mbar_periodic(t, N):
    """L-space block matrix Mbar_x^per of Eq. discrete_der (N cells, periodic corners)."""
    n = t.n
    M = np.zeros((N * n, N * n))
    for c in range(N):
        r = slice(c * n, (c + 1) * n)
        M[r, r] += 0.5 * (t.D - t.D.T)
        cp = (c + 1) % N
        cm = (c - 1) % N
        M[r, cp * n:(cp + 1) * n] += 0.5 * t.RL
        M[r, cm * n:(cm + 1) * n] += -0.5 * t.LR
    return M


def derivative_matrix_1d(t, N, h, bc="periodic"):
    """Dense X-space derivative f_x = (1 (x) B T) Mbar (1 (x) F) f (Eq. matrix_xspace)."""
    I = np.eye(N)
    M = mbar_periodic(t, N) if bc == "periodic" else mbar_dirichlet(t, N)
    return np.kron(I, t.B @ t.T(h)) @ M @ np.kron(I, t.F)


def forward_matrix_1d(t, N, h, bc="periodic"):
    """Dense X-space forward derivative (flux from the right cell); with bc="dirichlet" the
    boundary faces take u^ = 0: no right neighbour for the last cell, no left-face term -L in
    the first cell."""
    n = t.n
    M = np.zeros((N * n, N * n))
    for c in range(N):
        r = slice(c * n, (c + 1) * n)
        M[r, r] += -t.D.T if (bc == "dirichlet" and c == 0) else -t.L - t.D.T
        cp = c + 1
        if cp == N:
            if bc == "dirichlet":
                continue
            cp = 0
        M[r, cp * n:(cp + 1) * n] += t.RL
    I = np.eye(N)
    return np.kron(I, t.B @ t.T(h)) @ M @ np.kron(I, t.F)


def weight_vector_1d(t, N, h):
    """Diagonal of 1 (x) W (Eq. diagonal): h w_j / 2 per node."""
    return np.tile(h * t.w / 2.0, N)


def penalty_matrix_1d(t, N, h, tau):
    """(tau/h) sum over faces of j j^T, j = jump of the face traces u_{c+1}(-1) - u_c(+1)."""
    n = t.n
    lL, lR = trace_vectors(t)
    P = np.zeros((N * n, N * n))
    for c in range(N):
        j = np.zeros(N * n)
        cp = (c + 1) % N
        j[cp * n:(cp + 1) * n] += lL
        j[c * n:(c + 1) * n] -= lR
        P += np.outer(j, j)
    return (tau / h) * P


DIRICHLET_PENALTY = 1.0


def ldg_matrix_1d(t, N, h, tau=0.0, bc="periodic"):
    """A1 = D+^T W D+ + (tau/h) sum_f j_f j_f^T: the 1D LDG stiffness matrix, so that the
    1D dG Laplacian is -W^{-1} A1 (Sec. 6; fluxes: u^ from the right, q^ from the left).
    Dirichlet: u^ = 0 on the boundary faces and the penalty (DIRICHLET_PENALTY / h) u(a)^2 on
    the left boundary face (no jump penalty)."""
    if bc == "dirichlet" and tau != 0.0:
        raise ValueError("the Dirichlet reading has no jump penalty")
    Dp = forward_matrix_1d(t, N, h, bc)
    A1 = Dp.T @ np.diag(weight_vector_1d(t, N, h)) @ Dp
    if tau != 0.0:
        A1 = A1 + penalty_matrix_1d(t, N, h, tau)
    if bc == "dirichlet":
        lL = trace_vectors(t)[0]
        A1[:t.n, :t.n] += (DIRICHLET_PENALTY / h) * np.outer(lL, lL)
    return A1


def dense_ops_2d(g, tau=0.0, bc="periodic"):
    """Dense 2D matrices in the global node order [Y][X] (Y = cy*n + a, X = cx*n + b):
    Dx, Dy (central), A = W_y (x) A1_x + A1_y (x) W_x, and the 2D weights W (x) W."""
    t = g.t
    Dx1 = derivative_matrix_1d(t, g.Nx, g.hx, bc)
    Dy1 = derivative_matrix_1d(t, g.Ny, g.hy, bc)
    Iy = np.eye(g.Ny * g.n)
    Ix = np.eye(g.Nx * g.n)
    wx = weight_vector_1d(t, g.Nx, g.hx)
    wy = weight_vector_1d(t, g.Ny, g.hy)
    A1x = ldg_matrix_1d(t, g.Nx, g.hx, tau, bc)
    A1y = ldg_matrix_1d(t, g.Ny, g.hy, tau, bc)
    A = np.kron(np.diag(wy), A1x) + np.kron(A1y, np.diag(wx))
    return {"Dx": np.kron(Iy, Dx1), "Dy": np.kron(Dy1, Ix), "A": A, "W": np.kron(wy, wx)}


def to_global(f):
    """Cell-blocked f[cy, cx, a, b] -> global node array F[Y, X] (Y = cy*n+a, X = cx*n+b)."""
    Ny, Nx, n, _ = f.shape
    return f.transpose(0, 2, 1, 3).reshape(Ny * n, Nx * n)


def from_global(F, n):
    """Inverse of to_global."""
    Yn, Xn = F.shape
    return F.reshape(Yn // n, n, Xn // n, n).transpose(0, 2, 1, 3).copy()


# ----------------------------------------------------------------------------------
# Block application on f[cy, cx, a, b]
# ----------------------------------------------------------------------------------

def _shift(f, d, axis, zero):
    """f at cell index c + d along axis: periodic wrap, or zero outside the domain."""
    out = np.roll(f, -d, axis=axis)
    if zero:
        idx = [slice(None)] * f.ndim
        idx[axis] = slice(-1, None) if d > 0 else slice(0, 1)
        out[tuple(idx)] = 0.0
    return out


def _apply_x(B0, Bp, Bm, f, zero=False):
    out = np.einsum("ij,yxaj->yxai", B0, f)
    if Bp is not None:
        out += np.einsum("ij,yxaj->yxai", Bp, _shift(f, 1, 1, zero))
    if Bm is not None:
        out += np.einsum("ij,yxaj->yxai", Bm, _shift(f, -1, 1, zero))
    return out


def _apply_y(B0, Bp, Bm, f, zero=False):
    out = np.einsum("ij,yxjb->yxib", B0, f)
    if Bp is not None:
        out += np.einsum("ij,yxjb->yxib", Bp, _shift(f, 1, 0, zero))
    if Bm is not None:
        out += np.einsum("ij,yxjb->yxib", Bm, _shift(f, -1, 0, zero))
    return out


class Operators:
    """The 2D operators on one grid, applied blockwise (cell-blocked layout)."""

    def __init__(self, g: Grid, tau=0.0, bc="periodic"):
        if bc not in ("periodic", "dirichlet"):
            raise ValueError(bc)
        if bc == "dirichlet" and tau != 0.0:
            raise ValueError("the Dirichlet reading has no jump penalty")
        self.g = g
        self.tau = float(tau)
        self.bc = bc
        self.zero = bc == "dirichlet"
        t = g.t
        self.cx = central_blocks(t, g.hx)
        self.cy = central_blocks(t, g.hy)
        self.fx = forward_blocks(t, g.hx)
        self.fy = forward_blocks(t, g.hy)
        # Dirichlet: the first cell's own forward block without the left-face term (u^ = 0),
        # and the corrections of the central derivative's first / last cell blocks (X-space)
        self.fx0 = t.B @ t.T(g.hx) @ (-t.D.T) @ t.F
        self.fy0 = t.B @ t.T(g.hy) @ (-t.D.T) @ t.F
        self.bx = (t.B @ t.T(g.hx) @ (0.5 * t.L) @ t.F, t.B @ t.T(g.hx) @ (-0.5 * t.R) @ t.F)
        self.by = (t.B @ t.T(g.hy) @ (0.5 * t.L) @ t.F, t.B @ t.T(g.hy) @ (-0.5 * t.R) @ t.F)
        self.lL, self.lR = trace_vectors(t)
        self.wx = g.hx * t.w / 2.0
        self.wy = g.hy * t.w / 2.0
        self.W2 = g.weights()

    # --- first derivatives with the standard flux (Sec. 4.2) ---
    def Dx(self, f):
        out = _apply_x(*self.cx, f, zero=self.zero)
        if self.zero:       # f^ = 0 on the boundary faces: first / last cell blocks corrected
            out[:, 0] += np.einsum("ij,yaj->yai", self.bx[0], f[:, 0])
            out[:, -1] += np.einsum("ij,yaj->yai", self.bx[1], f[:, -1])
        return out

    def Dy(self, f):
        out = _apply_y(*self.cy, f, zero=self.zero)
        if self.zero:
            out[0] += np.einsum("ij,xjb->xib", self.by[0], f[0])
            out[-1] += np.einsum("ij,xjb->xib", self.by[1], f[-1])
        return out

    # --- Arakawa bracket, Eq. J ---
    def bracket_parts(self, f, g):
        """J^{++}, J^{+x}, J^{x+} of Eq. J for {f, g} = f_x g_y - f_y g_x."""
        Dx, Dy = self.Dx, self.Dy
        Jpp = Dx(f) * Dy(g) - Dy(f) * Dx(g)
        Jpx = Dx(f * Dy(g)) - Dy(f * Dx(g))
        Jxp = Dy(Dx(f) * g) - Dx(Dy(f) * g)
        return Jpp, Jpx, Jxp

    def bracket(self, f, g):
        """J = (J^{++} + J^{+x} + J^{x+}) / 3 (Eq. J, Sec. 3)."""
        Jpp, Jpx, Jxp = self.bracket_parts(f, g)
        return (Jpp + Jpx + Jxp) / 3.0

    # --- LDG Laplacian (Sec. 6) ---
    def _A1_x(self, u):
        G0, Gp = self.fx
        z = self.zero
        Dp = _apply_x(G0, Gp, None, u, zero=z)                             # D+ u
        if z:
            Dp[:, 0] += np.einsum("ij,yaj->yai", self.fx0 - G0, u[:, 0])  # first cell: no -L term
        v = Dp * self.wx[None, None, None, :]                              # W D+ u
        out = _apply_x(G0.T, None, Gp.T, v, zero=z)                        # D+^T (.)
        if z:
            out[:, 0] += np.einsum("ji,yaj->yai", self.fx0 - G0, v[:, 0])
            tr = np.einsum("j,yaj->ya", self.lL, u[:, 0])                  # u(a) on the left face
            out[:, 0] += (DIRICHLET_PENALTY / self.g.hx) * tr[..., None] * self.lL
        if self.tau != 0.0:
            out += self._penalty_x(u)
        return out

    def _A1_y(self, u):
        G0, Gp = self.fy
        z = self.zero
        Dp = _apply_y(G0, Gp, None, u, zero=z)
        if z:
            Dp[0] += np.einsum("ij,xjb->xib", self.fy0 - G0, u[0])
        v = Dp * self.wy[None, None, :, None]
        out = _apply_y(G0.T, None, Gp.T, v, zero=z)
        if z:
            out[0] += np.einsum("ji,xjb->xib", self.fy0 - G0, v[0])
            tr = np.einsum("j,xjb->xb", self.lL, u[0])
            out[0] += (DIRICHLET_PENALTY / self.g.hy) * self.lL[None, :, None] * tr[:, None, :]
        if self.tau != 0.0:
            out += self._penalty_y(u)
        return out

    def _penalty_x(self, u):
        lL, lR = self.lL, self.lR
        jump = np.einsum("j,yxaj->yxa", lL, np.roll(u, -1, axis=1)) - np.einsum("j,yxaj->yxa", lR, u)
        jump_left = np.roll(jump, 1, axis=1)  # face c-1/2
        return (self.tau / self.g.hx) * (jump_left[..., None] * lL - jump[..., None] * lR)

    def _penalty_y(self, u):
        lL, lR = self.lL, self.lR
        jump = np.einsum("j,yxjb->yxb", lL, np.roll(u, -1, axis=0)) - np.einsum("j,yxjb->yxb", lR, u)
        jump_left = np.roll(jump, 1, axis=0)
        return (self.tau / self.g.hy) * (jump_left[:, :, None, :] * lL[None, None, :, None]
                                         - jump[:, :, None, :] * lR[None, None, :, None])

    def A(self, u):
        """A u with A = W_y (x) A1_x + A1_y (x) W_x: symmetric positive semi-definite,
        kernel = constants; the dG Laplacian is Delta_h = -W^{-1} A."""
        return (self.wy[None, None, :, None] * self._A1_x(u)
                + self.wx[None, None, None, :] * self._A1_y(u))

    def laplacian(self, u):
        """Delta_h u = -W^{-1} A u."""
        return -self.A(u) / self.W2

    # --- integrals, Eq. def_norm and Eq. quantities ---
    def integral(self, f):
        return float(np.sum(self.W2 * f))

    def inner(self, f, g):
        return float(np.sum(self.W2 * f * g))

    def invariants(self, psi, omega):
        """(V, E, Omega) = (int omega, 1/2 int psi omega, 1/2 int omega^2), Gauss quadrature."""
        return (self.integral(omega), 0.5 * self.inner(psi, omega), 0.5 * self.inner(omega, omega))
