"""CPU-side checks of the native library: it loads, exports every entry point declared in
include/dg.h, and its host-side setup tables (Sec. 4.1 / 4.2 / Sec. 6) agree with the
independently written oracle.  No GPU compute is called here."""
import ctypes
import os
import re

import numpy as np
import pytest

from oracle.operators import central_blocks, ldg_matrix_1d, trace_vectors
from oracle.tables import Tables

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_symbols():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(dg_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_every_declared_symbol_is_exported(native):
    lib = ctypes.CDLL(native.LIB_PATH)
    syms = _declared_symbols()
    assert len(syms) >= 15
    missing = [s for s in syms if not hasattr(lib, s)]
    assert not missing, missing


@pytest.mark.parametrize("n", range(1, 6))
@pytest.mark.parametrize("tau", [0.0, 0.7])
def test_ref_tables_match_oracle(native, n, tau):
    t = native.ref_tables(n, tau)
    o = Tables(n)
    assert np.allclose(t["x"], o.x, atol=1e-15) and np.allclose(t["w"], o.w, atol=4e-15)
    # central flux: own block and the rank-one neighbour blocks, per unit h
    C0, Cp, Cm = central_blocks(o, 1.0)
    lL, lR = trace_vectors(o)
    assert np.allclose(t["C0"], C0, atol=1e-13)
    assert np.allclose(np.outer(t["muR"], t["lL"]), Cp, atol=1e-13)
    assert np.allclose(-np.outer(t["muL"], t["lR"]), Cm, atol=1e-13)
    assert np.allclose(t["lL"], lL, atol=1e-14) and np.allclose(t["lR"], lR, atol=1e-14)
    # LDG stiffness: blocks of the dense 1D matrix on three unit cells
    A1 = ldg_matrix_1d(o, 3, 1.0, tau)
    blk = lambda i, j: A1[i * n:(i + 1) * n, j * n:(j + 1) * n]
    assert np.allclose(t["A1cc"], blk(1, 1), atol=1e-12 * max(1, np.abs(A1).max()))
    assert np.allclose(np.outer(t["betaA"], t["lL"]), blk(1, 2), atol=1e-12 * max(1, np.abs(A1).max()))
    assert np.allclose(np.outer(t["lL"], t["betaA"]), blk(1, 0), atol=1e-12 * max(1, np.abs(A1).max()))


def test_argument_errors(native):
    lib = native.lib()
    out = (ctypes.c_double * 100)()
    assert lib.dg_ref_tables(0, 0.0, out, 100) == native.DG_ERR_ARG
    assert lib.dg_ref_tables(6, 0.0, out, 100) == native.DG_ERR_ARG
    assert lib.dg_ref_tables(3, -1.0, out, 100) == native.DG_ERR_ARG
    assert lib.dg_ref_tables(3, 0.0, out, 5) == native.DG_ERR_ARG
    assert b"small" in lib.dg_last_error()
    h = ctypes.c_void_p()
    assert lib.dg_grid_create(ctypes.byref(h), 0, 4, 3, 1.0, 1.0, 0.0) == native.DG_ERR_ARG
    assert lib.dg_grid_create(ctypes.byref(h), 4, 4, 6, 1.0, 1.0, 0.0) == native.DG_ERR_ARG
    assert lib.dg_grid_create(ctypes.byref(h), 4, 4, 3, -1.0, 1.0, 0.0) == native.DG_ERR_ARG
    assert lib.dg_grid_dof(None) == 0


def test_no_device_fails_loudly(native):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    rc = native.lib().dg_grid_create(ctypes.byref(h), 4, 4, 3, 1.0, 1.0, 0.0)
    assert rc == native.DG_ERR_CUDA
    with pytest.raises(native.DGError):
        native.Grid(4, 4, 3)


@pytest.mark.parametrize("n", range(1, 6))
@pytest.mark.parametrize("N,k,tau", [(8, 0, 0.0), (8, 3, 0.0), (7, 2, 0.0), (1, 0, 0.0), (2, 1, 0.0),
                                     (16, 8, 0.4), (1024, 1, 0.0), (1024, 512, 0.0)])
def test_spectral_symbol_matches_oracle(native, n, N, k, tau):
    """dg_spectral_symbol (the tables of the spectral preconditioner) against the oracle's LDG
    stiffness: the symbol of the line scaled by w^-1/2 on both sides, built from the blocks of
    the dense 1D matrix on three cells; eigenvalues, V diag(lam) V^* = K and V unitary."""
    L = 2.0
    lam, V = native.spectral_symbol(N, n, L, k, tau)
    o = Tables(n)
    h = L / N
    A3 = ldg_matrix_1d(o, 3, h, tau)[n:2 * n, :]
    w = h * o.w / 2.0
    th = 2.0 * np.pi * k / N
    K = (A3[:, n:2 * n] + np.exp(1j * th) * A3[:, 2 * n:] + np.exp(-1j * th) * A3[:, :n]) / np.sqrt(np.outer(w, w))
    ev = np.linalg.eigvalsh(K)
    if k == 0:
        assert abs(ev[0]) <= 1e-9 * max(abs(ev[-1]), 1e-300)
        ev[0] = 0.0
        assert lam[0] == 0.0
    # the symbol is a cancelling sum of the blocks: rounding is relative to their size
    sc = max(np.abs(A3).max() / w.min(), 1e-300)
    assert np.all(np.diff(lam) >= 0.0)
    assert np.abs(lam - ev).max() <= 1e-13 * sc
    assert np.abs(V @ np.diag(lam) @ V.conj().T - K).max() <= 1e-13 * sc
    assert np.abs(V.conj().T @ V - np.eye(n)).max() <= 1e-13
