"""FP64 CPU oracle for the conservative dG-Arakawa scheme (Einkemmer & Wiesenberger,
"A conservative discontinuous Galerkin scheme for the 2D incompressible Navier-Stokes
equations").

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import, call or link this
package: only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code, tables or
constants with the CUDA library; it is a plain, slow, obviously-checkable restatement
of the paper in NumPy float64, written in the paper's order and notation:

* ``tables``     -- Legendre recursion, Gauss-Legendre quadrature, the transforms F, B
                    and the matrices S, T, W, V, D, R, L, RL, LR (Sec. 4.1).
* ``operators``  -- the 1D dG derivative with the standard (central) flux, its dense
                    block-circulant matrix (Sec. 4.2, Eq. discrete_der, Eq. matrix_xspace),
                    the 2D extension, the Arakawa bracket J (Eq. J, Sec. 3), the LDG
                    Laplacian (Sec. 6, after Cockburn & Shu) and the invariants
                    (Eq. quantities, Eq. def_norm).
* ``solver``     -- the conjugate-gradient Poisson solve of -Delta psi = omega (Sec. 6).
* ``stepper``    -- the K-step Adams-Bashforth vorticity update with RK4 start-up (Sec. 6).

Data layout: a 2D field is a float64 array ``f[cy, cx, a, b]`` (cell row, cell column,
y-node, x-node) holding X-space values, i.e. the field at the Gauss-Legendre nodes of
each cell (Sec. 4.1).  Flattened in C order this is the cell-blocked order
``((cy*Nx + cx)*n + a)*n + b``.

Parity status: every function here is pinned by a ``-m "not gpu"`` test against the
paper's printed tables, closed forms, textbook special cases or dense brute force, with
two exceptions stated in the module docstrings: the LDG penalty for tau > 0 and the CG
preconditioner / stopping rule (the paper does not specify them; parity unpinned).
"""
