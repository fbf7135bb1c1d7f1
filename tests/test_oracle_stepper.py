"""Pins for the oracle's time stepper (Sec. 6): Tables 3 and 4 and the invariants.

* Table 4, Lamb dipole, K = 1: every printed digit of eps_Omega and eps_E (10 to 80
  steps).  This fixes E = 1/2 <psi, omega>_W, Omega = 1/2 <omega, omega>_W, the bracket
  and the tau = 0 LDG Poisson operator at P = 1.
* Table 4, K = 2 and K = 3 with RK4 start-up steps: within 3 and 10 percent (start-up
  unspecified).  The printed K = 4 rows are not reproduced by RK4 start-up steps (their
  Omega column does not fall at order 4 either); K = 4 is left unpinned against them and
  pinned instead by its observed order (>= 3.85) and the Adams-Bashforth order conditions
  of the weights of every K.
* Table 3, P = 1, D = 0: the error is exactly zero, as printed (Poisson is solved exactly
  and the bracket vanishes); P = 1, D = 0.01 and P = 2, D = 0: the printed orders.
* Vorticity V is conserved to roundoff in every step (linear scheme, Eq. average1).
* With D = 0 the energy and enstrophy drift only through the time stepper: third order.
"""
import json
import os

import numpy as np
import pytest

from oracle.operators import Operators
from oracle.stepper import Simulation
from oracle.tables import Grid
from paper_1311_7477_gb300 import fields

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _lamb_run(K, steps):
    g = Grid(200, 200, 1, 1.0, 1.0)
    ops = Operators(g)
    X, Y = g.mesh()
    w0 = fields.lamb_dipole(X, Y)
    sim = Simulation(ops, w0, 0.0, 0.01 / steps, tol=1e-13, K=K, precond="twolevel")
    V0, E0, O0 = sim.invariants()
    sim.step(steps)
    V, E, O = sim.invariants()
    return abs((O - O0) / O0), abs((E - E0) / E0), V


@pytest.mark.slow
@pytest.mark.parametrize("steps", [10, 20, 40, 80])
def test_table4_K1_printed_digits(steps):
    gold = json.load(open(os.path.join(GOLD, "table4_lamb.json")))["K1"][str(steps)]
    eO, eE, V = _lamb_run(1, steps)
    assert f"{eO:.2E}" == gold["eps_Omega"].replace("E-00", "E-0")
    assert f"{eE:.2E}" == gold["eps_E"].replace("E-00", "E-0")
    assert abs(V) < 1e-14


@pytest.mark.slow
@pytest.mark.parametrize("steps", [10, 20, 40, 80])
def test_table4_K2_rk4_startup(steps):
    gold = json.load(open(os.path.join(GOLD, "table4_lamb.json")))["K2"][str(steps)]
    eO, eE, V = _lamb_run(2, steps)
    assert abs(eO / float(gold["eps_Omega"]) - 1) < 0.03
    assert abs(eE / float(gold["eps_E"]) - 1) < 0.03
    assert abs(V) < 1e-14


@pytest.mark.slow
@pytest.mark.parametrize("steps", [10, 40])
def test_table4_K3_rk4_startup(steps):
    gold = json.load(open(os.path.join(GOLD, "table4_lamb.json")))["K3"][str(steps)]
    eO, eE, V = _lamb_run(3, steps)
    assert abs(eO / float(gold["eps_Omega"]) - 1) < 0.10
    assert abs(eE / float(gold["eps_E"]) - 1) < 0.10
    assert abs(V) < 1e-14


def _table3_error(n, N, D, nsteps=400):
    g = Grid(N, N, n)
    ops = Operators(g)
    X, Y = g.mesh()
    w0 = 2.0 * fields.sin_sin(X, Y)
    sim = Simulation(ops, w0, D, 2.0 / nsteps, tol=1e-12, K=3)
    sim.step(nsteps)
    e = sim.omega - w0 * np.exp(-2.0 * D * 2.0)
    return np.sqrt(ops.inner(e, e))


def test_table3_P1_D0_exactly_zero():
    gold = json.load(open(os.path.join(GOLD, "table3_periodic.json")))["D0"]["P1"]
    for N in (16, 32):
        assert float(gold[str(N)]) == 0.0
        assert _table3_error(1, N, 0.0) == 0.0


def test_table3_P1_D001_order():
    gold = json.load(open(os.path.join(GOLD, "table3_periodic.json")))["D0.01"]["P1"]
    e16, e32 = _table3_error(1, 16, 0.01), _table3_error(1, 32, 0.01)
    assert abs(np.log2(e16 / e32) - float(gold["order_32"])) < 0.05


@pytest.mark.slow
def test_table3_P2_order_and_magnitude():
    gold = json.load(open(os.path.join(GOLD, "table3_periodic.json")))["D0"]["P2"]
    e16, e32 = _table3_error(2, 16, 0.0), _table3_error(2, 32, 0.0)
    assert abs(np.log2(e16 / e32) - float(gold["order_32"])) < 0.15
    assert abs(e16 / float(gold["16"]) - 1) < 0.15
    assert abs(e32 / float(gold["32"]) - 1) < 0.15


def _random_phase_sim(n, N, D, dt, K=3):
    g = Grid(N, N, n)
    ops = Operators(g)
    X, Y = g.mesh()
    w0 = fields.random_phase(X, Y, seed=3, kmax=6)
    return Simulation(ops, w0, D, dt, tol=1e-13, K=K)


@pytest.mark.parametrize("D", [0.0, 1e-3])
def test_vorticity_conserved_each_step(D):
    sim = _random_phase_sim(3, 12, D, 2e-3)
    scale = np.abs(sim.omega).max() * (2 * np.pi) ** 2
    V0 = sim.invariants()[0]
    for _ in range(6):
        sim.step()
        assert abs(sim.invariants()[0] - V0) < 1e-14 * scale


def test_energy_enstrophy_drift_third_order():
    drifts = []
    for dt, steps in ((8e-3, 10), (4e-3, 20)):
        sim = _random_phase_sim(3, 10, 0.0, dt)
        _, E0, O0 = sim.invariants()
        sim.step(steps)
        _, E, O = sim.invariants()
        drifts.append((abs(E - E0) / E0, abs(O - O0) / O0))
    for i in range(2):
        ratio = drifts[0][i] / drifts[1][i]
        assert ratio > 2.0 ** 3 * 0.7, (drifts, ratio)


def test_naive_bracket_stepper_drifts_at_the_space_error():
    """With J^{++} alone (the comparison of Sec. 6.2) V is still conserved each step (Table 2:
    int J^{++} = 0), but E and Omega drift through the space discretisation: the drift no
    longer falls as dt^3 and exceeds the scheme's by orders of magnitude."""
    out = {}
    for bracket in ("arakawa", "naive"):
        for dt, steps in ((8e-3, 10), (4e-3, 20)):
            g = Grid(10, 10, 3)
            ops = Operators(g)
            X, Y = g.mesh()
            sim = Simulation(ops, fields.random_phase(X, Y, seed=3, kmax=6), 0.0, dt, tol=1e-13, bracket=bracket)
            V0, E0, O0 = sim.invariants()
            sim.step(steps)
            V, E, O = sim.invariants()
            assert abs(V - V0) < 1e-13 * np.abs(sim.omega).max()
            out[(bracket, dt)] = (abs(E - E0) / E0, abs(O - O0) / O0)
    for i in range(2):
        assert out[("naive", 8e-3)][i] / out[("naive", 4e-3)][i] < 2.0
        assert out[("naive", 4e-3)][i] > 100.0 * out[("arakawa", 4e-3)][i], out


def test_adams_bashforth_weights_order_conditions():
    """The K-step Adams-Bashforth weights integrate polynomials of degree < K exactly over one
    step: sum_m c_m (-m)^q = 1 / (q + 1) for q = 0 .. K-1 (m = 0 is R^k, m = 1 is R^{k-1}, ...).
    A closed form for the weights of every K used by Sec. 6 and Table 4."""
    from oracle.stepper import AB_COEFFS
    for K, c in AB_COEFFS.items():
        assert len(c) == K
        for q in range(K):
            s = sum(cm * (-m) ** q for m, cm in enumerate(c))
            assert abs(s - 1.0 / (q + 1)) < 1e-15, (K, q, s)


@pytest.mark.slow
def test_table4_K4_observed_order():
    """K = 4 (Table 4's last rows) with RK4 start-up steps: the errors of the conserved
    quantities fall at least at order 4 (less 0.15) between 10 and 40 steps.  The printed K = 4
    rows themselves are not reproduced by RK4 start-up steps, so this order is the CPU pin of
    the K = 4 weights."""
    e10, e40 = _lamb_run(4, 10), _lamb_run(4, 40)
    for i in (0, 1):
        p = np.log(e10[i] / e40[i]) / np.log(4.0)
        assert p > 4 - 0.15, (i, p)
    assert abs(e40[2]) < 1e-14
