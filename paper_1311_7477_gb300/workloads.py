"""Workload builders for the benchmarks and the request server: seeded simulation specs and
the explicit-AB3 stability rule for the time step.

dt rule (a reading: the paper only says the CFL condition is respected, Sec. 6): with the
spectral radii rho_h = rho(D_central) h of the central-flux derivative and
rho_2 = rho(-Delta_1D) h^2 of the 1D LDG Laplacian (both per unit h, from the library's own
tables), the 3-step Adams-Bashforth stability limits 0.7236 (imaginary axis) and 6/11
(negative real axis), and a safety factor 1/2:

    dt = min(dt_cap, 0.5 * 0.7236 * h / (rho_h * U),  0.5 * (6/11) * h^2 / (2 D rho_2))

with U a bound of |u|_inf + |v|_inf of the initial field.
"""
import numpy as np

AB3_IMAG = 0.7236
AB3_REAL = 6.0 / 11.0


def spectral_radii(dg, n, samples=257):
    """(rho_h, rho_2) for n nodes: maxima over the Fourier symbol of the periodic 1D block
    operators built from dg_ref_tables (central derivative; W^-1 A1 for the Laplacian)."""
    t = dg.ref_tables(n)
    w = t["w"] / 2.0
    rh, r2 = 0.0, 0.0
    for th in np.linspace(0.0, 2 * np.pi, samples):
        e = np.exp(1j * th)
        D = t["C0"] + np.outer(t["muR"], t["lL"]) * e - np.outer(t["muL"], t["lR"]) * np.conj(e)
        rh = max(rh, np.abs(np.linalg.eigvals(D)).max())
        A = t["A1cc"] + np.outer(t["betaA"], t["lL"]) * e + np.outer(t["lL"], t["betaA"]) * np.conj(e)
        r2 = max(r2, np.abs(np.linalg.eigvals(A / w[:, None])).max())
    return float(rh), float(r2)


def stable_dt(dg, N, n, D, L=2 * np.pi, U=2.0, dt_cap=2e-4, cache={}):
    if n not in cache:
        cache[n] = spectral_radii(dg, n)
    rh, r2 = cache[n]
    h = L / N
    dt = min(dt_cap, 0.5 * AB3_IMAG * h / (rh * U))
    if D > 0:
        dt = min(dt, 0.5 * AB3_REAL * h * h / (2.0 * D * r2))
    return dt


def ensemble_specs(count=64, seed0=100, Ns=(32, 64, 128, 256), ns=(2, 3, 4, 5), Drange=(1e-5, 1e-3)):
    """Seeded members of the batched ensemble: cells per side and n drawn uniformly, D
    log-uniform, random-phase initial field with the member's seed."""
    out = []
    for i in range(count):
        rng = np.random.default_rng(seed0 + i)
        N = int(rng.choice(Ns))
        n = int(rng.choice(ns))
        D = float(np.exp(rng.uniform(np.log(Drange[0]), np.log(Drange[1]))))
        out.append({"N": N, "n": n, "D": D, "seed": seed0 + i, "field": "random_phase"})
    return out


def request_trace(count=200, rate=20.0, seed=7, Ns=(64, 128, 256, 512, 1024), ns=(3, 4, 5),
                  Drange=(1e-5, 1e-3), steps=(100, 2000)):
    """Served workload: Poisson arrivals (exponential gaps), per request cells per side, n, D,
    step count and the initial field (random phase or shear layer with probability 1/2)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        out.append({"id": i, "arrival": t, "N": int(rng.choice(Ns)), "n": int(rng.choice(ns)),
                    "D": float(np.exp(rng.uniform(np.log(Drange[0]), np.log(Drange[1])))),
                    "steps": int(rng.integers(steps[0], steps[1] + 1)),
                    "field": "random_phase" if rng.uniform() < 0.5 else "shear_layer",
                    "seed": int(rng.integers(0, 2 ** 31 - 1))})
    return out


def initial_field(dg, grid, spec):
    xn, yn, _ = grid.nodes()
    return initial_field_from_nodes(xn, yn, spec)


def initial_field_from_nodes(xn, yn, spec):
    from . import fields
    if spec["field"] == "random_phase":
        return fields.random_phase_nodes(xn, yn, seed=spec["seed"])
    return fields.shear_layer_nodes(xn, yn)
