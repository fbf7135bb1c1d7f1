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
