"""GB300-native conservative dG-Arakawa solver for 2D incompressible Navier-Stokes
(Einkemmer & Wiesenberger's scheme): CUDA kernels for sm_103a behind the C-ABI library
``libdgk.so`` (declared in ``include/dg.h``), with a thin ctypes binding in ``dg``.

Importing the package loads nothing; ``paper_1311_7477_gb300.dg`` loads the native
library on first use and raises if it is missing -- there is no CPU fallback.
"""
__all__ = ["dg", "fields"]
