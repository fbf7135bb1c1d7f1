"""Pins for the oracle's homogeneous Dirichlet boundaries (Sec. 3 standard flux with the
field zero outside; Sec. 4.2; Tables 2 and 3).

Reading (the paper prints Mbar^dir but names no LDG boundary treatment): the derivative's
flux on a boundary face is the boundary value, f^ = 0, so the first and last cells' own
L-space blocks are 1/2 (D - D^T) + 1/2 L and 1/2 (D - D^T) - 1/2 R; the LDG forward
derivative takes u^ = 0 on the boundary faces, A1 = D+^T W D+ plus a penalty (1/h) u(a)^2 on
the left boundary face.

* Table 2, Dirichlet row: every printed digit of int J, int f J, int g J (the corner blocks
  printed in Mbar^dir, 1/2 (D - D^T), give 0.185, 3e-16, 4e-15 instead);
* P = 1: the derivative is the centred difference with odd-reflected ghost values;
* dense assembly = blockwise application; A symmetric positive definite;
* the closed-form Poisson solution sin x sin y converges at order n (n >= 2);
* Table 3, Dirichlet, D = 0: the printed orders for P = 2 and 4 and the magnitudes within 15%.
"""
import json
import os

import numpy as np
import pytest

from oracle.operators import Operators, dense_ops_2d, to_global
from oracle.solver import solve_poisson, solve_poisson_dense
from oracle.stepper import Simulation
from oracle.tables import Grid
from paper_1311_7477_gb300 import fields
from tests.test_oracle_bracket import _printed_match

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_table2_dirichlet_row_printed_digits():
    gold = json.load(open(os.path.join(GOLD, "table2_dirichlet.json")))
    g = Grid(112, 112, 3, np.pi, np.pi)
    o = Operators(g, bc="dirichlet")
    X, Y = g.mesh()
    f, gg = fields.table2_pair(X, Y)
    J = o.bracket(f, gg)
    vals = (o.integral(J), o.inner(f, J), o.inner(gg, J))
    for v, p in zip(vals, gold["row"]):
        assert _printed_match(v, p), (v, p)


def test_p1_dirichlet_derivative_is_centred_difference_with_odd_ghosts():
    N, h = 9, 0.3
    g = Grid(N, 4, 1, N * h, 1.2)
    o = Operators(g, bc="dirichlet")
    f = np.random.default_rng(3).standard_normal((4, N, 1, 1))
    fe = np.concatenate([-f[:, :1], f, -f[:, -1:]], axis=1)      # odd reflections outside
    ref = (fe[:, 2:] - fe[:, :-2]) / (2 * h)
    assert np.allclose(o.Dx(f), ref, rtol=0, atol=1e-14)


@pytest.mark.parametrize("Nx,Ny,n", [(4, 3, 2), (3, 5, 3), (5, 4, 4), (4, 4, 1), (2, 3, 5)])
def test_dirichlet_dense_equals_blockwise_and_A_is_spd(Nx, Ny, n):
    g = Grid(Nx, Ny, n, 1.3, 0.9)
    o = Operators(g, bc="dirichlet")
    d = dense_ops_2d(g, bc="dirichlet")
    f = np.random.default_rng(n).standard_normal((Ny, Nx, n, n))
    for name, op in (("Dx", o.Dx), ("Dy", o.Dy), ("A", o.A)):
        got = to_global(op(f)).ravel()
        assert np.abs(got - d[name] @ to_global(f).ravel()).max() < 1e-12 * np.abs(got).max(), name
    A = d["A"]
    assert np.abs(A - A.T).max() < 1e-13 * np.abs(A).max()
    assert np.linalg.eigvalsh(A).min() > 1e-6
    # the derivative is not skew in the W inner product at the boundary (why Table 2's
    # Dirichlet row does not vanish): W Dx + (W Dx)^T is non-zero on the boundary cells only
    S = d["W"][:, None] * d["Dx"]
    assert np.abs(S + S.T).max() > 1e-3


def test_dirichlet_poisson_closed_form_order():
    for n in (2, 3):
        errs = []
        for N in (8, 16):
            g = Grid(N, N, n)
            o = Operators(g, bc="dirichlet")
            X, Y = g.mesh()
            r = solve_poisson(o, 2 * np.sin(X) * np.sin(Y), np.zeros(X.shape), 1e-13, 100000)
            e = r.x - np.sin(X) * np.sin(Y)
            errs.append(np.sqrt(o.inner(e, e)))
        assert np.log2(errs[0] / errs[1]) > n - 0.3, (n, errs)
    # and the dense direct solve agrees with CG
    g = Grid(5, 4, 3, 1.1, 0.8)
    o = Operators(g, bc="dirichlet")
    w = np.random.default_rng(1).standard_normal((4, 5, 3, 3))
    x = solve_poisson(o, w, np.zeros_like(w), 1e-14, 10000).x
    from oracle.operators import from_global
    xd = from_global(solve_poisson_dense(dense_ops_2d(g, bc="dirichlet"), to_global(w), bc="dirichlet"), 3)
    assert np.abs(x - xd).max() < 1e-11 * np.abs(xd).max()


@pytest.mark.slow
@pytest.mark.parametrize("P", [2, 4])
def test_table3_dirichlet_order_and_magnitude(P):
    gold = json.load(open(os.path.join(GOLD, "table3_dirichlet.json")))["D0"]["P%d" % P]
    errs = []
    for N in (16, 32):
        g = Grid(N, N, P)
        o = Operators(g, bc="dirichlet")
        X, Y = g.mesh()
        w0 = 2.0 * np.sin(X) * np.sin(Y)
        sim = Simulation(o, w0, 0.0, 2.0 / 400, tol=1e-12, K=3)
        sim.step(400)
        e = sim.omega - w0
        errs.append(np.sqrt(o.inner(e, e)))
    assert abs(np.log2(errs[0] / errs[1]) - float(gold["order_32"])) < 0.15
    assert abs(errs[0] / float(gold["16"]) - 1) < 0.15
    assert abs(errs[1] / float(gold["32"]) - 1) < 0.15
