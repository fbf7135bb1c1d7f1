"""Legendre / Gauss-Legendre tables of Sec. 4.1 (oracle; test infrastructure only).

Everything is float64 NumPy, computed from the three-term recursion (Eq. recursion) and
the definitions that follow it.  Notation: P = n = number of basis polynomials per
dimension (polynomial degree n-1); indices i, j, k run over 0..n-1.
"""
import numpy as np


def legendre(kmax, x):
    """p_0..p_kmax at the points x by the recursion (k+1) p_{k+1} = (2k+1) x p_k - k p_{k-1}
    with p_0 = 1, p_1 = x (Eq. recursion).  Returns an array of shape (kmax+1,) + x.shape."""
    x = np.asarray(x, dtype=np.float64)
    p = np.zeros((kmax + 1,) + x.shape)
    p[0] = 1.0
    if kmax >= 1:
        p[1] = x
    for k in range(1, kmax):
        p[k + 1] = ((2 * k + 1) * x * p[k] - k * p[k - 1]) / (k + 1)
    return p


def _legendre_derivative(n, x):
    """p_n'(x) from (x^2 - 1) p_n' = n (x p_n - p_{n-1}), valid for |x| < 1."""
    p = legendre(n, x)
    return n * (x * p[n] - p[n - 1]) / (x * x - 1.0)


def gauss_legendre(n):
    """Abscissas x_j and weights w_j of n-point Gauss-Legendre quadrature on [-1, 1]
    (Sec. 4.1): the roots of p_n by Newton's method, w_j = 2 / ((1 - x_j^2) p_n'(x_j)^2).
    Returned in increasing order of x."""
    xs = []
    for j in range(n):
        x = np.cos(np.pi * (j + 0.75) / (n + 0.5))  # classical starting guess
        for _ in range(100):
            if n == 1:
                x = 0.0
                break
            dx = legendre(n, x)[n] / _legendre_derivative(n, x)
            x = x - dx
            if abs(dx) < 1e-17:
                break
        xs.append(float(x))
    x = np.array(sorted(xs))
    if n == 1:
        w = np.array([2.0])
    else:
        w = 2.0 / ((1.0 - x * x) * _legendre_derivative(n, x) ** 2)
    return x, w


class Tables:
    """The n x n matrices of Sec. 4.1 for one polynomial order n (dimensionless, i.e.
    on the reference cell [-1, 1]; the cell size enters through T, W, V only).

    x, w : Gauss-Legendre abscissas and weights
    B    : backward transform, B_{kj} = p_j(x_k)                    (X-space <- L-space)
    F    : forward transform,  F^{kj} = (2k+1)/2 w_j p_k(x_j)        (L-space <- X-space)
    D    : D_ij = int_{-1}^{1} p_i p_j' = 1 - (-1)^{i+j} for i <= j-1, else 0
           (Eq. legendre_operators / Eq. legendre_derivative)
    pR, pL : p_k(1) = 1 and p_k(-1) = (-1)^k
    R, L, RL, LR : the face outer products p(+-1) p(+-1)^T of Eq. legendre_operators
    """

    def __init__(self, n):
        if not (1 <= n <= 8):
            raise ValueError("n must be in 1..8")
        self.n = n
        self.x, self.w = gauss_legendre(n)
        P = legendre(n - 1, self.x)            # P[k, j] = p_k(x_j)
        self.B = P.T.copy()                    # B[j, k] = p_k(x_j)  (B_{kj} := p_j(x_k))
        k = np.arange(n)
        self.F = ((2 * k + 1) / 2.0)[:, None] * self.w[None, :] * P
        self.D = np.zeros((n, n))
        for i in range(n):
            for j in range(n):
                if i <= j - 1:
                    self.D[i, j] = 1.0 - (-1.0) ** (i + j)
        self.pR = np.ones(n)
        self.pL = (-1.0) ** k
        self.R = np.outer(self.pR, self.pR)
        self.L = np.outer(self.pL, self.pL)
        self.RL = np.outer(self.pR, self.pL)
        self.LR = np.outer(self.pL, self.pR)

    # Diagonal matrices of Eq. diagonal for a cell of size h.
    def S(self, h):
        return np.diag(h / (2 * np.arange(self.n) + 1.0))

    def T(self, h):
        return np.diag((2 * np.arange(self.n) + 1.0) / h)

    def W(self, h):
        return np.diag(h * self.w / 2.0)

    def V(self, h):
        return np.diag(2.0 / (h * self.w))


class Grid:
    """Equidistant periodic grid on [0, Lx] x [0, Ly] with Nx x Ny cells and n Gauss
    nodes per cell and dimension (Sec. 4.1: x_{nj} = x_n + (h/2) x_j)."""

    def __init__(self, Nx, Ny, n, Lx=2 * np.pi, Ly=2 * np.pi):
        self.Nx, self.Ny, self.n = int(Nx), int(Ny), int(n)
        self.Lx, self.Ly = float(Lx), float(Ly)
        self.hx, self.hy = self.Lx / self.Nx, self.Ly / self.Ny
        self.t = Tables(self.n)

    def nodes_x(self):
        """x-coordinates of the nodes, shape (Nx, n)."""
        c = (np.arange(self.Nx) + 0.5) * self.hx
        return c[:, None] + 0.5 * self.hx * self.t.x[None, :]

    def nodes_y(self):
        """y-coordinates of the nodes, shape (Ny, n)."""
        c = (np.arange(self.Ny) + 0.5) * self.hy
        return c[:, None] + 0.5 * self.hy * self.t.x[None, :]

    def mesh(self):
        """X, Y of shape (Ny, Nx, n, n) in the layout f[cy, cx, a, b]."""
        xn, yn = self.nodes_x(), self.nodes_y()
        X = np.broadcast_to(xn[None, :, None, :], (self.Ny, self.Nx, self.n, self.n))
        Y = np.broadcast_to(yn[:, None, :, None], (self.Ny, self.Nx, self.n, self.n))
        return np.array(X), np.array(Y)

    def weights(self):
        """2D quadrature weights W (x) W of Eq. def_norm in the layout f[cy, cx, a, b]:
        (hy w_a / 2) (hx w_b / 2)."""
        wy = self.hy * self.t.w / 2.0
        wx = self.hx * self.t.w / 2.0
        w2 = np.outer(wy, wx)
        return np.broadcast_to(w2[None, None], (self.Ny, self.Nx, self.n, self.n)).copy()

    def zeros(self):
        return np.zeros((self.Ny, self.Nx, self.n, self.n))
