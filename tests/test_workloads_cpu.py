"""CPU checks of the workload builders: the spectral radii behind the AB3 time-step rule
(computed from the library's host tables through the Fourier symbol of the periodic block
operators) against the eigenvalues of the oracle's dense 1D operators, and the seeded specs."""
import numpy as np
import pytest

from oracle.operators import derivative_matrix_1d, ldg_matrix_1d, weight_vector_1d
from oracle.tables import Tables


@pytest.mark.parametrize("n", range(1, 6))
def test_spectral_radii_match_dense_oracle(native, n):
    from paper_1311_7477_gb300 import workloads
    rh, r2 = workloads.spectral_radii(native, n, samples=513)
    t = Tables(n)
    N, h = 64, 1.0
    D = derivative_matrix_1d(t, N, h)
    L = np.diag(1.0 / weight_vector_1d(t, N, h)) @ ldg_matrix_1d(t, N, h)
    assert abs(np.abs(np.linalg.eigvals(D)).max() - rh) < 1e-3 * rh
    assert abs(np.abs(np.linalg.eigvals(L)).max() - r2) < 1e-3 * r2


def test_dt_rule_and_specs(native):
    from paper_1311_7477_gb300 import workloads
    dt = workloads.stable_dt(native, 256, 5, 1e-3)
    assert 0 < dt < 2e-4                        # the viscous limit binds at 256 cells, n = 5, D = 1e-3
    assert workloads.stable_dt(native, 32, 2, 1e-5) == 2e-4
    a = workloads.ensemble_specs()
    b = workloads.ensemble_specs()
    assert a == b and len(a) == 64
    assert {s["N"] for s in a} <= {32, 64, 128, 256} and {s["n"] for s in a} <= {2, 3, 4, 5}
    tr = workloads.request_trace(count=200)
    gaps = np.diff([r["arrival"] for r in tr])
    assert len(tr) == 200 and (gaps > 0).all() and abs(1.0 / gaps.mean() - 20.0) < 4.0


def test_node_field_generators_match_the_mesh_forms():
    """The node-coordinate generators the workloads use equal the mesh forms: the shear layer
    bit for bit, the random-phase field to rounding against its direct sum over wave vectors."""
    import numpy as np
    from oracle.tables import Grid as OGrid
    from paper_1311_7477_gb300 import fields
    og = OGrid(12, 10, 3, 2 * np.pi, 2 * np.pi)
    X, Y = og.mesh()
    xn, yn = X[0, :, 0, :], Y[:, 0, :, 0]
    assert np.array_equal(fields.shear_layer_nodes(xn, yn), fields.shear_layer(X, Y))
    kmax, k0, seed = 6, 3.0, 5
    got = fields.random_phase_nodes(xn, yn, seed=seed, kmax=kmax, k0=k0)
    assert np.array_equal(got, fields.random_phase(X, Y, seed=seed, kmax=kmax, k0=k0))
    rng = np.random.default_rng(seed)
    ks = np.arange(-kmax, kmax + 1)
    kx, ky = np.meshgrid(ks, np.arange(0, kmax + 1), indexing="xy")
    kk = np.hypot(kx, ky)
    keep = (kk > 0) & (kk <= kmax) & ((ky > 0) | ((ky == 0) & (kx > 0)))
    phi = rng.uniform(0.0, 2.0 * np.pi, size=kx.shape)
    A = np.sqrt(np.where(keep, kk * kk ** 4 * np.exp(-(kk / k0) ** 2) / np.pi, 0.0))
    A = A / np.sqrt(np.pi ** 2 * np.sum(A ** 2))
    ref = np.zeros_like(X)
    for i, j in zip(*np.nonzero(keep)):
        ref += A[i, j] * np.cos(kx[i, j] * X + ky[i, j] * Y + phi[i, j])
    assert np.abs(got - ref).max() <= 1e-13 * np.abs(ref).max()
