"""Pins for the oracle's Arakawa bracket J = (J++ + J+x + Jx+)/3 (Eq. J, Sec. 3).

* Table 2's periodic rows, to the printed digits (golden fixture)
* the integral constraints of Eqs. average1-3 (sum W J = sum W f J = sum W g J = 0) to
  roundoff for random fields -- fails for any non-skew derivative or wrong product form
* antisymmetry, J(f, f) = 0 and J(psi, 2 psi) = 0 bitwise (steady state)
* P = 1 equals Arakawa's (1966) 9-point Jacobian, written out here as explicit stencils
* closed form {sin x, sin y} = cos x cos y under refinement
"""
import json
import os

import numpy as np
import pytest

from oracle.operators import Operators
from oracle.tables import Grid
from paper_1311_7477_gb300 import fields

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _printed_match(value, printed):
    """value agrees with a printed number to the printed digits; entries printed at the
    1e-16 level are roundoff and only need to stay at roundoff."""
    p = float(printed)
    if abs(p) < 1e-10:
        return abs(value) < 1e-13
    mant = printed.lower().split("e")[0].lstrip("-")
    decimals = len(mant.split(".")[1]) if "." in mant else 0
    if "e" in printed.lower():
        exp = int(printed.lower().split("e")[1])
        half_ulp = 0.5 * 10.0 ** (exp - decimals)
    else:
        half_ulp = 0.5 * 10.0 ** (-decimals)
    return abs(value - p) <= half_ulp * 1.0000001


def test_table2_periodic_rows():
    gold = json.load(open(os.path.join(GOLD, "table2_periodic.json")))
    g = Grid(112, 112, 3, np.pi, np.pi)
    ops = Operators(g)
    X, Y = g.mesh()
    f, gg = fields.table2_pair(X, Y)
    Jpp, Jpx, Jxp = ops.bracket_parts(f, gg)
    J = ops.bracket(f, gg)
    got = {"J++": Jpp, "J+x": Jpx, "Jx+": Jxp, "J": J}
    for row, printed in gold["rows"].items():
        vals = (ops.integral(got[row]), ops.inner(f, got[row]), ops.inner(gg, got[row]))
        for v, p in zip(vals, printed):
            assert _printed_match(v, p), (row, v, p)


@pytest.mark.parametrize("n", range(1, 6))
def test_integral_constraints_random(n):
    g = Grid(6, 5, n, 1.7, 2.9)
    ops = Operators(g)
    rng = np.random.default_rng(n)
    f, gg = rng.standard_normal((2, 5, 6, n, n))
    J = ops.bracket(f, gg)
    scale = np.abs(J).max() * np.abs(f).max() * g.Lx * g.Ly
    for w in (np.ones_like(f), f, gg):
        assert abs(ops.inner(w, J)) < 1e-13 * scale
    # each of the three parts alone violates at least one constraint (Table 2's pattern)
    Jpp, Jpx, Jxp = ops.bracket_parts(f, gg)
    assert abs(ops.inner(f, Jpp)) > 1e-6 * scale
    assert abs(ops.inner(gg, Jxp)) > 1e-6 * scale


@pytest.mark.parametrize("n", [2, 4])
def test_antisymmetry_and_bitwise_zeros(n):
    g = Grid(5, 7, n)
    ops = Operators(g)
    rng = np.random.default_rng(7)
    f, gg = rng.standard_normal((2, 7, 5, n, n))
    J1, J2 = ops.bracket(f, gg), ops.bracket(gg, f)
    assert np.abs(J1 + J2).max() < 1e-13 * np.abs(J1).max()
    assert np.array_equal(ops.bracket(f, f), np.zeros_like(f))
    X, Y = g.mesh()
    psi = fields.sin_sin(X, Y)
    assert np.array_equal(ops.bracket(psi, 2.0 * psi), np.zeros_like(psi))
    # invariance under psi -> psi + c (the discrete derivative of a constant vanishes)
    assert np.abs(ops.bracket(f + 3.25, gg) - J1).max() < 1e-12 * np.abs(J1).max()


def test_P1_equals_arakawa_nine_point():
    N = 9
    g = Grid(N, N, 1, 2.0, 2.0)
    d = g.hx
    ops = Operators(g)
    rng = np.random.default_rng(1)
    psi, zeta = rng.standard_normal((2, N, N, 1, 1))
    P, Z = psi[:, :, 0, 0], zeta[:, :, 0, 0]      # [j (y), i (x)]

    def s(A, di, dj):   # value at (i + di, j + dj), periodic
        return np.roll(np.roll(A, -di, axis=1), -dj, axis=0)

    Jpp = ((s(P, 1, 0) - s(P, -1, 0)) * (s(Z, 0, 1) - s(Z, 0, -1))
           - (s(P, 0, 1) - s(P, 0, -1)) * (s(Z, 1, 0) - s(Z, -1, 0))) / (4 * d * d)
    Jpx = (s(P, 1, 0) * (s(Z, 1, 1) - s(Z, 1, -1)) - s(P, -1, 0) * (s(Z, -1, 1) - s(Z, -1, -1))
           - s(P, 0, 1) * (s(Z, 1, 1) - s(Z, -1, 1)) + s(P, 0, -1) * (s(Z, 1, -1) - s(Z, -1, -1))) / (4 * d * d)
    Jxp = (s(Z, 0, 1) * (s(P, 1, 1) - s(P, -1, 1)) - s(Z, 0, -1) * (s(P, 1, -1) - s(P, -1, -1))
           - s(Z, 1, 0) * (s(P, 1, 1) - s(P, 1, -1)) + s(Z, -1, 0) * (s(P, -1, 1) - s(P, -1, -1))) / (4 * d * d)
    ref = (Jpp + Jpx + Jxp) / 3.0
    got = ops.bracket(psi, zeta)[:, :, 0, 0]
    assert np.allclose(got, ref, atol=1e-13 * np.abs(ref).max())


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_closed_form_bracket_converges(n):
    """The paper states no order for the bracket (rate unpinned); with the central flux the
    error must still fall at least linearly (even n lose one order, odd n do not)."""
    errs = []
    for N in (8, 16, 32):
        g = Grid(N, N, n)
        ops = Operators(g)
        X, Y = g.mesh()
        J = ops.bracket(np.sin(X), np.sin(Y))
        e = J - np.cos(X) * np.cos(Y)
        errs.append(np.sqrt(ops.inner(e, e)))
    assert errs[0] < np.pi                      # ||cos x cos y|| = pi
    expected = n if n % 2 else n - 1             # a lower bound on the observed rate
    for a, b in zip(errs, errs[1:]):
        assert a / b > 2.0 ** expected * 0.85, errs
