"""ctypes binding of libdgk (include/dg.h): the same entry points, argument marshalling only.

Device arrays are torch tensors (float64, contiguous, on the current CUDA device) used as
plain memory; every step of the method runs in the library's CUDA kernels.  There is no
CPU fallback: if the library is missing or fails to load, importing this module raises.
"""
import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libdgk.so")

DG_OK, DG_ERR_ARG, DG_ERR_CUDA, DG_ERR_NOMEM, DG_ERR_NOCONV, DG_ERR_NONFINITE, DG_ERR_TIMEOUT, DG_ERR_IO = range(8)
DG_FP64, DG_MIXED, DG_MIXED64, DG_FP64_PC32 = 0, 1, 2, 3
DG_BC_PERIODIC, DG_BC_DIRICHLET = 0, 1
DG_PRECOND_JACOBI, DG_PRECOND_TWOLEVEL, DG_PRECOND_SPECTRAL = 0, 1, 2
DG_BRACKET_ARAKAWA, DG_BRACKET_NAIVE = 0, 1

ERROR_NAMES = {DG_ERR_ARG: "DG_ERR_ARG", DG_ERR_CUDA: "DG_ERR_CUDA", DG_ERR_NOMEM: "DG_ERR_NOMEM",
               DG_ERR_NOCONV: "DG_ERR_NOCONV", DG_ERR_NONFINITE: "DG_ERR_NONFINITE",
               DG_ERR_TIMEOUT: "DG_ERR_TIMEOUT", DG_ERR_IO: "DG_ERR_IO"}


class DGError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s: %s" % (ERROR_NAMES.get(code, str(code)), msg))
        self.code = code


class SimCounters(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_longlong), ("rhs_launches", ctypes.c_longlong),
                ("cg_launches", ctypes.c_longlong), ("rhs_ms", ctypes.c_double), ("cg_ms", ctypes.c_double)]


class SimInfo(ctypes.Structure):
    _fields_ = [("step", ctypes.c_longlong), ("cg_iters_total", ctypes.c_longlong),
                ("cg_iters_last", ctypes.c_int), ("cg_iters_max", ctypes.c_int),
                ("cg_relres_last", ctypes.c_double), ("refine_sweeps_last", ctypes.c_int),
                ("status", ctypes.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libdgk.so not built (%s); run `python -m paper_1311_7477_gb300.build`" % LIB_PATH)
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, LL = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_longlong
    PP = ctypes.POINTER(ctypes.c_void_p)
    PD = ctypes.POINTER(ctypes.c_double)
    PI = ctypes.POINTER(ctypes.c_int)
    sig = {
        "dg_last_error": (ctypes.c_char_p, []),
        "dg_version": (I, []),
        "dg_selftest_wait_cap": (I, [P]),
        "dg_ref_tables_len": (I, [I]),
        "dg_ref_tables": (I, [I, D, PD, I]),
        "dg_spectral_symbol": (I, [I, I, D, D, I, PD, PD, PD]),
        "dg_grid_create": (I, [PP, I, I, I, D, D, D]),
        "dg_grid_create_bc": (I, [PP, I, I, I, D, D, D, I]),
        "dg_grid_destroy": (I, [P]),
        "dg_grid_dof": (LL, [P]),
        "dg_grid_nodes": (I, [P, PD, PD, PD]),
        "dg_grid_set_tiles": (I, [P, I, I]),
        "dg_grid_set_precond": (I, [P, I]),
        "dg_grid_set_compensated_apply": (I, [P, I]),
        "dg_grid_get_compensated_apply": (I, [P]),
        "dg_bracket": (I, [P, P, P, P, P]),
        "dg_bracket_mixed": (I, [P, P, P, P, P]),
        "dg_bracket_parts": (I, [P, P, P, P, I, P]),
        "dg_laplace_apply": (I, [P, P, P, I, P]),
        "dg_poisson_solve": (I, [P, P, P, D, I, I, PI, PD, P]),
        "dg_invariants": (I, [P, P, P, PD, P]),
        "dg_poisson_solve_static": (I, [I, I, I, D, D, D, P, P, D, I, I, PI, PD, P]),
        "dg_sim_create": (I, [PP, P, D, D, I, D, I, P, P]),
        "dg_sim_destroy": (I, [P]),
        "dg_step": (I, [P, I, P]),
        "dg_sim_status": (I, [P, ctypes.POINTER(SimInfo), P]),
        "dg_sim_refinement_history": (I, [P, ctypes.POINTER(ctypes.c_double), PI, I, PI, P]),
        "dg_sim_get": (I, [P, P, P, P]),
        "dg_sim_get_state": (I, [P, ctypes.POINTER(LL), P, P, P, P, P, P]),
        "dg_sim_set_state": (I, [P, LL, P, P, P, P, P, P]),
        "dg_sim_get_history": (I, [P, I, P, P]),
        "dg_sim_set_history": (I, [P, I, P, P]),
        "dg_sim_set_multistep": (I, [P, I]),
        "dg_batch_set_limit": (I, [P, P, LL]),
        "dg_sim_set_bracket": (I, [P, I]),
        "dg_sim_save": (I, [P, ctypes.c_char_p, P]),
        "dg_sim_load": (I, [PP, P, ctypes.c_char_p, P]),
        "dg_sim_invariants": (I, [P, PD, P]),
        "dg_sim_set_cg": (I, [P, D, I, I]),
        "dg_sim_set_refinement": (I, [P, D, I]),
        "dg_batch_create": (I, [PP, I]),
        "dg_batch_destroy": (I, [P]),
        "dg_batch_admit": (I, [P, P, P]),
        "dg_batch_retire": (I, [P, P]),
        "dg_batch_size": (I, [P]),
        "dg_batch_set_groups": (I, [P, I]),
        "dg_batch_set_tiles": (I, [P, I, I, I, I, I]),
        "dg_batch_set_blocks_per_sm": (I, [P, I]),
        "dg_batch_autotune": (I, [P, I, P]),
        "dg_batch_get_config": (I, [P, ctypes.c_char_p, I]),
        "dg_batch_step": (I, [P, I, P]),
        "dg_batch_status": (I, [P, PI, PI, ctypes.POINTER(LL), P]),
        "dg_sim_upload": (I, [P, LL, P, P, P, P, P, P]),
        "dg_sim_download": (I, [P, P, P, P]),
        "dg_sim_set_timing": (I, [P, I]),
        "dg_sim_get_counters": (I, [P, ctypes.POINTER(SimCounters), P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    return lib


_lib = _load()


def lib():
    return _lib


def _check(rc):
    if rc != DG_OK:
        raise DGError(rc, _lib.dg_last_error().decode())
    return rc


def _ptr(t):
    """Device pointer of a contiguous float64 CUDA tensor (or None)."""
    if t is None:
        return None
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError("expected a contiguous float64 CUDA tensor")
    return ctypes.c_void_p(t.data_ptr())


def _hptr(a):
    """Host pointer of a contiguous float64 CPU tensor or numpy array (or None)."""
    if a is None:
        return None
    import numpy as np
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise TypeError("expected a contiguous float64 array")
        return ctypes.c_void_p(a.ctypes.data)
    if a.is_cuda or a.dtype.itemsize != 8 or not a.is_contiguous():
        raise TypeError("expected a contiguous float64 CPU tensor")
    return ctypes.c_void_p(a.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def ref_tables(n, tau=0.0):
    """Host-only tables (dict of numpy arrays) of dg_ref_tables."""
    import numpy as np
    L = _lib.dg_ref_tables_len(n)
    if L <= 0:
        raise DGError(DG_ERR_ARG, "n outside 1..5")
    out = (ctypes.c_double * L)()
    _check(_lib.dg_ref_tables(n, float(tau), out, L))
    a = np.frombuffer(out, dtype=np.float64).copy()
    o = 0
    res = {}
    for name, size in (("x", n), ("w", n), ("C0", n * n), ("muR", n), ("muL", n), ("lL", n), ("lR", n),
                       ("A1cc", n * n), ("betaA", n)):
        v = a[o:o + size]
        res[name] = v.reshape(n, n) if name in ("C0", "A1cc") else v
        o += size
    return res


def spectral_symbol(N, n, L, k, tau=0.0):
    """Host-only (dg_spectral_symbol): eigenvalues lam (ascending) and unitary eigenvectors V
    (columns) of the scaled 1D CG operator's symbol at wave number k of a periodic line of N
    cells of length L."""
    import numpy as np
    lam = (ctypes.c_double * n)()
    vre = (ctypes.c_double * (n * n))()
    vim = (ctypes.c_double * (n * n))()
    _check(_lib.dg_spectral_symbol(int(N), int(n), float(L), float(tau), int(k), lam, vre, vim))
    V = (np.frombuffer(vre, dtype=np.float64) + 1j * np.frombuffer(vim, dtype=np.float64)).reshape(n, n)
    return np.frombuffer(lam, dtype=np.float64).copy(), V


class Grid:
    """dg_grid: [0, Lx] x [0, Ly], Nx x Ny cells, n nodes per cell and dimension; periodic
    (bc="periodic") or homogeneous Dirichlet (bc="dirichlet") boundaries."""

    def __init__(self, Nx, Ny, n, Lx=6.283185307179586, Ly=6.283185307179586, tau=0.0, bc="periodic"):
        h = ctypes.c_void_p()
        code = {"periodic": DG_BC_PERIODIC, "dirichlet": DG_BC_DIRICHLET}[bc]
        _check(_lib.dg_grid_create_bc(ctypes.byref(h), int(Nx), int(Ny), int(n), float(Lx), float(Ly), float(tau),
                                      code))
        self.h = h
        self.bc = bc
        self.Nx, self.Ny, self.n, self.Lx, self.Ly, self.tau = int(Nx), int(Ny), int(n), float(Lx), float(Ly), float(tau)

    @property
    def shape(self):
        return (self.Ny, self.Nx, self.n, self.n)

    @property
    def dof(self):
        return int(_lib.dg_grid_dof(self.h))

    def nodes(self):
        """(x_nodes (Nx, n), y_nodes (Ny, n), W per node (n, n)) as numpy arrays."""
        import numpy as np
        xn = np.zeros(self.Nx * self.n)
        yn = np.zeros(self.Ny * self.n)
        w = np.zeros(self.n * self.n)
        P = ctypes.POINTER(ctypes.c_double)
        _check(_lib.dg_grid_nodes(self.h, xn.ctypes.data_as(P), yn.ctypes.data_as(P), w.ctypes.data_as(P)))
        return xn.reshape(self.Nx, self.n), yn.reshape(self.Ny, self.n), w.reshape(self.n, self.n)

    def set_tiles(self, TY, TX):
        _check(_lib.dg_grid_set_tiles(self.h, int(TY), int(TX)))

    def set_precond(self, kind):
        """DG_PRECOND_JACOBI (W^-1), DG_PRECOND_TWOLEVEL or DG_PRECOND_SPECTRAL; also accepts
        "jacobi" / "twolevel" / "spectral"."""
        if isinstance(kind, str):
            kind = {"jacobi": DG_PRECOND_JACOBI, "twolevel": DG_PRECOND_TWOLEVEL, "spectral": DG_PRECOND_SPECTRAL}[kind]
        _check(_lib.dg_grid_set_precond(self.h, int(kind)))

    def set_compensated_apply(self, mode):
        """-1 (automatic), 0 (float32), 1 (double-float) or 2 (adaptive): the operator apply of
        the float32 inner solves of the mixed modes on this grid."""
        _check(_lib.dg_grid_set_compensated_apply(self.h, int(mode)))

    @property
    def compensated_apply(self):
        return int(_lib.dg_grid_get_compensated_apply(self.h))

    def close(self):
        if getattr(self, "h", None):
            _lib.dg_grid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dg_bracket(grid, psi, omega, J, stream=None):
    _check(_lib.dg_bracket(grid.h, _ptr(psi), _ptr(omega), _ptr(J), _stream(stream)))


def dg_bracket_mixed(grid, psi, omega, J, stream=None):
    """The bracket as DG_MIXED evaluates it: double-float arithmetic on the float32 pipe."""
    _check(_lib.dg_bracket_mixed(grid.h, _ptr(psi), _ptr(omega), _ptr(J), _stream(stream)))


def dg_bracket_parts(grid, psi, omega, J, parts, stream=None):
    """parts: bit set of 1 (J++), 2 (J+x), 4 (Jx+); 7 = the conservative J."""
    _check(_lib.dg_bracket_parts(grid.h, _ptr(psi), _ptr(omega), _ptr(J), int(parts), _stream(stream)))


def dg_laplace_apply(grid, x, y, mode=0, stream=None):
    _check(_lib.dg_laplace_apply(grid.h, _ptr(x), _ptr(y), int(mode), _stream(stream)))


def dg_poisson_solve(grid, omega, psi, tol=1e-12, maxit=100000, fixed_iters=0, stream=None, check=True):
    """Solves in place (psi holds the initial guess); returns (rc, iterations, relres)."""
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    rc = _lib.dg_poisson_solve(grid.h, _ptr(omega), _ptr(psi), float(tol), int(maxit), int(fixed_iters),
                               ctypes.byref(it), ctypes.byref(rr), _stream(stream))
    if check:
        _check(rc)
    return rc, it.value, rr.value


def dg_poisson_solve_static(Nx, Ny, n, Lx, Ly, tau, omega, psi, tol=1e-12, maxit=100000, fixed_iters=0,
                            stream=None, check=True):
    """The allocation-free Poisson solve (no grid handle); returns (rc, iterations, relres)."""
    it = ctypes.c_int(0)
    rr = ctypes.c_double(0.0)
    rc = _lib.dg_poisson_solve_static(int(Nx), int(Ny), int(n), float(Lx), float(Ly), float(tau), _ptr(omega),
                                      _ptr(psi), float(tol), int(maxit), int(fixed_iters), ctypes.byref(it),
                                      ctypes.byref(rr), _stream(stream))
    if check:
        _check(rc)
    return rc, it.value, rr.value


def dg_invariants(grid, psi, omega, stream=None):
    out = (ctypes.c_double * 3)()
    _check(_lib.dg_invariants(grid.h, _ptr(psi), _ptr(omega), out, _stream(stream)))
    return tuple(out)


class Sim:
    """dg_sim: the K-step Adams-Bashforth time stepper (RK4 start-up, K = 3 by default) on a grid."""

    def __init__(self, grid, omega0, D=0.0, dt=1e-3, precision=DG_FP64, cg_tol=1e-12, cg_maxit=100000, stream=None,
                 _handle=None):
        if _handle is None:
            _handle = ctypes.c_void_p()
            _check(_lib.dg_sim_create(ctypes.byref(_handle), grid.h, float(D), float(dt), int(precision),
                                      float(cg_tol), int(cg_maxit), _ptr(omega0), _stream(stream)))
        self.h = _handle
        self.grid = grid

    @classmethod
    def load(cls, grid, path, stream=None):
        """dg_sim_load: a simulation resumed from a dg_sim_save file on grid."""
        h = ctypes.c_void_p()
        _check(_lib.dg_sim_load(ctypes.byref(h), grid.h, os.fsencode(path), _stream(stream)))
        return cls(grid, None, _handle=h)

    def save(self, path, stream=None):
        _check(_lib.dg_sim_save(self.h, os.fsencode(path), _stream(stream)))

    def set_bracket(self, variant):
        """"arakawa" (Eq. J) or "naive" (J++ alone)."""
        v = {"arakawa": DG_BRACKET_ARAKAWA, "naive": DG_BRACKET_NAIVE}.get(variant, variant)
        _check(_lib.dg_sim_set_bracket(self.h, int(v)))

    def step(self, nsteps=1, stream=None):
        _check(_lib.dg_step(self.h, int(nsteps), _stream(stream)))

    def status(self, stream=None, check=True):
        info = SimInfo()
        rc = _lib.dg_sim_status(self.h, ctypes.byref(info), _stream(stream))
        if check:
            _check(rc)
        return info

    def refinement_history(self, stream=None):
        """[(relres before sweep j, inner iterations of sweep j)] of the last mixed solve."""
        rr = (ctypes.c_double * 48)()
        it = (ctypes.c_int * 48)()
        cnt = ctypes.c_int(0)
        _check(_lib.dg_sim_refinement_history(self.h, rr, it, 48, ctypes.byref(cnt), _stream(stream)))
        return [(rr[j], it[j]) for j in range(min(cnt.value, 48))]

    def get(self, omega=None, psi=None, stream=None):
        _check(_lib.dg_sim_get(self.h, _ptr(omega), _ptr(psi), _stream(stream)))

    def get_state(self, omega, psi, psi_prev, R1, R2, stream=None):
        step = ctypes.c_longlong(0)
        _check(_lib.dg_sim_get_state(self.h, ctypes.byref(step), _ptr(omega), _ptr(psi), _ptr(psi_prev), _ptr(R1),
                                     _ptr(R2), _stream(stream)))
        return step.value

    def set_state(self, step, omega, psi, psi_prev, R1, R2, stream=None):
        _check(_lib.dg_sim_set_state(self.h, int(step), _ptr(omega), _ptr(psi), _ptr(psi_prev), _ptr(R1), _ptr(R2),
                                     _stream(stream)))

    def get_history(self, m, R, stream=None):
        _check(_lib.dg_sim_get_history(self.h, int(m), _ptr(R), _stream(stream)))

    def set_history(self, m, R, stream=None):
        _check(_lib.dg_sim_set_history(self.h, int(m), _ptr(R), _stream(stream)))

    def set_multistep(self, K):
        _check(_lib.dg_sim_set_multistep(self.h, int(K)))

    def invariants(self, stream=None):
        out = (ctypes.c_double * 3)()
        _check(_lib.dg_sim_invariants(self.h, out, _stream(stream)))
        return tuple(out)

    def set_cg(self, tol, maxit, fixed_iters=0):
        _check(_lib.dg_sim_set_cg(self.h, float(tol), int(maxit), int(fixed_iters)))

    def set_refinement(self, tol_in, max_sweeps):
        _check(_lib.dg_sim_set_refinement(self.h, float(tol_in), int(max_sweeps)))

    def upload(self, step, omega, psi, psi_prev, R1, R2, stream=None):
        """Host (CPU) tensors or numpy arrays, float64 contiguous."""
        _check(_lib.dg_sim_upload(self.h, int(step), _hptr(omega), _hptr(psi), _hptr(psi_prev), _hptr(R1),
                                  _hptr(R2), _stream(stream)))

    def download(self, omega=None, psi=None, stream=None):
        _check(_lib.dg_sim_download(self.h, _hptr(omega), _hptr(psi), _stream(stream)))

    def set_timing(self, enable=True):
        _check(_lib.dg_sim_set_timing(self.h, 1 if enable else 0))

    def counters(self, stream=None):
        c = SimCounters()
        _check(_lib.dg_sim_get_counters(self.h, ctypes.byref(c), _stream(stream)))
        return c

    def close(self):
        if getattr(self, "h", None):
            _lib.dg_sim_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """dg_batch: simulations advanced together by one persistent, graph-captured kernel."""

    def __init__(self, max_sims):
        h = ctypes.c_void_p()
        _check(_lib.dg_batch_create(ctypes.byref(h), int(max_sims)))
        self.h = h
        self.members = []

    def admit(self, sim, stream=None):
        _check(_lib.dg_batch_admit(self.h, sim.h, _stream(stream)))
        self.members.append(sim)

    def retire(self, sim):
        _check(_lib.dg_batch_retire(self.h, sim.h))
        self.members.remove(sim)

    def set_groups(self, ngroups):
        _check(_lib.dg_batch_set_groups(self.h, int(ngroups)))

    def set_tiles(self, n, rhs=(0, 0), cg=(0, 0)):
        """Cell tiles (TY, TX) of the batched kernel for members with n nodes ((0, 0): built-in)."""
        _check(_lib.dg_batch_set_tiles(self.h, int(n), int(rhs[0]), int(rhs[1]), int(cg[0]), int(cg[1])))

    def set_blocks_per_sm(self, cap):
        _check(_lib.dg_batch_set_blocks_per_sm(self.h, int(cap)))

    def autotune(self, trial_steps=2, stream=None):
        """dg_batch_autotune: time and keep the fastest launch configuration (advances the members)."""
        _check(_lib.dg_batch_autotune(self.h, int(trial_steps), _stream(stream)))
        return self.config()

    def config(self):
        buf = ctypes.create_string_buffer(512)
        _check(_lib.dg_batch_get_config(self.h, buf, 512))
        return buf.value.decode()

    def set_limit(self, sim, last_step):
        """sim takes no batched step beyond step index last_step (0: no limit)."""
        _check(_lib.dg_batch_set_limit(self.h, sim.h, int(last_step)))

    def step(self, nsteps=1, stream=None):
        _check(_lib.dg_batch_step(self.h, int(nsteps), _stream(stream)))

    def status(self, stream=None, check=True):
        g, ng, nl = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_longlong(0)
        rc = _lib.dg_batch_status(self.h, ctypes.byref(g), ctypes.byref(ng), ctypes.byref(nl), _stream(stream))
        if check:
            _check(rc)
        return {"rc": rc, "graph": bool(g.value), "groups": ng.value, "launches": nl.value}

    def __len__(self):
        return int(_lib.dg_batch_size(self.h))

    def close(self):
        if getattr(self, "h", None):
            _lib.dg_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
