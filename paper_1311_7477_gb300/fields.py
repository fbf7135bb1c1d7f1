"""Seeded synthetic initial fields (shared by the tests, the oracle checks and the bench).

This module holds no arithmetic of the dG method: every generator takes the node
coordinates as input (X[cy, cx, a, b], Y[cy, cx, a, b] -- whoever computed the Gauss
nodes) and returns the analytic field sampled there, in the cell-blocked layout
f[cy, cx, a, b] (X-space values; the paper initialises by evaluation at the nodes,
Sec. 4.1 / Sec. 6).  Random draws use numpy.random.default_rng(seed).

Workloads (all periodic on [0, 2pi]^2 unless stated):
* sin_sin_noise   2 sin x sin y + U(-amp, amp) per node           (steady Euler state, Sec. 6)
* shear_layer     double shear layer, rho = delta = 0.05           (large single run)
* random_phase    isotropic random-phase field, E(k) ~ k^4 exp(-(k/k0)^2), |k| <= kmax,
                  normalised to unit enstrophy 1/2 int omega^2 = 1 of the continuous field
* lamb_dipole     Lamb dipole on [0, 1]^2 (Sec. 6, Eq. lamb)
* table2_pair     f = sin x cos y, g = exp(0.1 (x + y)) on [0, pi]^2 (Sec. 5.2)
"""
import numpy as np


def mesh_from_nodes(xn, yn):
    """Node coordinate arrays of shape (Nx, n) and (Ny, n) -> X, Y of shape (Ny, Nx, n, n)."""
    xn = np.asarray(xn, dtype=np.float64)
    yn = np.asarray(yn, dtype=np.float64)
    Nx, n = xn.shape
    Ny = yn.shape[0]
    X = np.broadcast_to(xn[None, :, None, :], (Ny, Nx, n, n))
    Y = np.broadcast_to(yn[:, None, :, None], (Ny, Nx, n, n))
    return np.array(X), np.array(Y)


def sin_sin_noise(X, Y, amp=1e-3, seed=0):
    """omega0 = 2 sin x sin y + i.i.d. U(-amp, amp) on every node value."""
    rng = np.random.default_rng(seed)
    return 2.0 * np.sin(X) * np.sin(Y) + rng.uniform(-amp, amp, size=X.shape)


def sin_sin(X, Y):
    """psi = sin x sin y; omega = 2 psi is the steady solution decaying as exp(-2Dt)."""
    return np.sin(X) * np.sin(Y)


def shear_layer(X, Y, rho=0.05, delta=0.05):
    """Vorticity of the double shear layer u = tanh((y - pi/2)/rho) (y <= pi),
    tanh((3pi/2 - y)/rho) (y > pi), v = delta sin x, taken as omega = v_x - u_y:
    delta cos x - sech^2((y - pi/2)/rho)/rho  (y <= pi),
    delta cos x + sech^2((3pi/2 - y)/rho)/rho (y > pi).  Zero mean."""
    lower = delta * np.cos(X) - 1.0 / (rho * np.cosh((Y - np.pi / 2) / rho) ** 2)
    upper = delta * np.cos(X) + 1.0 / (rho * np.cosh((3 * np.pi / 2 - Y) / rho) ** 2)
    return np.where(Y <= np.pi, lower, upper)


def random_phase(X, Y, seed=1, kmax=32, k0=6.0):
    """Sum over integer wave vectors k in a half plane (ky > 0, or ky == 0 and kx > 0),
    0 < |k| <= kmax, of A_k cos(k.x + phi_k), phi_k ~ U[0, 2pi), A_k = sqrt(|k| E(|k|)/pi),
    E(k) = k^4 exp(-(k/k0)^2); rescaled so that the continuous enstrophy
    1/2 int_{[0,2pi]^2} omega^2 = pi^2 sum A_k^2 equals 1.  X, Y: a tensor mesh (see
    random_phase_nodes)."""
    return random_phase_nodes(X[0, :, 0, :], Y[:, 0, :, 0], seed=seed, kmax=kmax, k0=k0)


def random_phase_nodes(xn, yn, seed=1, kmax=32, k0=6.0):
    """random_phase from the node coordinates xn (Nx, n), yn (Ny, n) of a tensor mesh,
    evaluated separably: with C = A e^{i phi} (ky, kx), the field on node rows ys and node
    columns xs is Re(E_y C E_x^T), E_y = e^{i ys ky}, E_x = e^{i xs kx}, formed as
    Re(P) cos(xs kx)^T - Im(P) sin(xs kx)^T with P = E_y C."""
    rng = np.random.default_rng(seed)
    ks = np.arange(-kmax, kmax + 1)
    kx, ky = np.meshgrid(ks, np.arange(0, kmax + 1), indexing="xy")   # shape (kmax+1, 2kmax+1)
    kk = np.hypot(kx, ky)
    keep = (kk > 0) & (kk <= kmax) & ((ky > 0) | ((ky == 0) & (kx > 0)))
    phi = rng.uniform(0.0, 2.0 * np.pi, size=kx.shape)
    E = np.where(keep, kk ** 4 * np.exp(-(kk / k0) ** 2), 0.0)
    A = np.sqrt(np.where(keep, kk * E / np.pi, 0.0))
    A = A / np.sqrt(np.pi ** 2 * np.sum(A ** 2))
    C = A * np.exp(1j * phi)                                           # (ky, kx)
    xn = np.asarray(xn, dtype=np.float64)
    yn = np.asarray(yn, dtype=np.float64)
    Nx, n = xn.shape
    Ny = yn.shape[0]
    xs = xn.reshape(-1)                                                # (Nx*n,)  x of column index cx*n+b
    ys = yn.reshape(-1)                                                # (Ny*n,)
    P = np.exp(1j * np.outer(ys, np.arange(0, kmax + 1))) @ C          # (Ny*n, 2kmax+1)
    ph = np.outer(ks, xs)                                              # (2kmax+1, Nx*n)
    # Re(P E_x^T) = [Re P, -Im P] [cos; sin]: one real product of inner length 2 (2kmax+1)
    G = np.hstack([P.real, -P.imag]) @ np.vstack([np.cos(ph), np.sin(ph)])   # (Ny*n, Nx*n) [Y][X]
    return G.reshape(Ny, n, Nx, n).transpose(0, 2, 1, 3).copy()


def shear_layer_nodes(xn, yn, rho=0.05, delta=0.05):
    """shear_layer from the node coordinates xn (Nx, n), yn (Ny, n) of a tensor mesh: the
    field is delta cos x plus a function of y, evaluated on the node lines and broadcast
    (the same operations per node as shear_layer)."""
    xn = np.asarray(xn, dtype=np.float64)
    yn = np.asarray(yn, dtype=np.float64)
    cx = delta * np.cos(xn)                                            # (Nx, n)
    lower = 1.0 / (rho * np.cosh((yn - np.pi / 2) / rho) ** 2)         # (Ny, n)
    upper = 1.0 / (rho * np.cosh((3 * np.pi / 2 - yn) / rho) ** 2)
    sy = np.where(yn <= np.pi, -lower, upper)       # c - l is c + (-l) exactly
    return cx[None, :, None, :] + sy[:, None, :, None]


def lamb_dipole(X, Y, R=0.1, U=1.0, xc=0.5, yc=0.5):
    """Lamb dipole (Eq. lamb): omega = 2 lam U / J0(lam R) J1(lam r) cos(theta) for r < R,
    0 outside, lam R = 3.83170597020751231561 (first zero of J1), theta from the x axis."""
    from scipy.special import j0, j1
    lam = 3.83170597020751231561 / R
    dx, dy = X - xc, Y - yc
    r = np.hypot(dx, dy)
    cos_t = np.where(r > 0, dx / np.where(r > 0, r, 1.0), 0.0)
    return np.where(r < R, 2.0 * lam * U / j0(lam * R) * j1(lam * r) * cos_t, 0.0)


def table2_pair(X, Y):
    """f = sin x cos y, g = exp(0.1 (x + y))  (Sec. 5.2, conservation test)."""
    return np.sin(X) * np.cos(Y), np.exp(0.1 * (X + Y))


def uniform_noise(shape, seed, lo=-1.0, hi=1.0):
    """i.i.d. U(lo, hi) field for operator-level parity tests."""
    return np.random.default_rng(seed).uniform(lo, hi, size=shape)
