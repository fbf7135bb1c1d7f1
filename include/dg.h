/*
 * dg.h -- C ABI of libdgk: the conservative dG-Arakawa discretisation of the 2D
 * incompressible Navier-Stokes equations in vorticity / stream-function form
 *
 *     d omega/dt + {psi, omega} = D Delta omega,     -Delta psi = omega     (Eq. vorticity)
 *
 * on a periodic Cartesian grid of Nx x Ny square-or-rectangular cells with n Gauss-Legendre
 * nodes per cell and dimension (polynomial degree n-1, 1 <= n <= 5; Sec. 4.1), as CUDA
 * kernels for one NVIDIA GB300 (sm_103a).
 *
 * Conventions
 * -----------
 * - Every function returns an int status (DG_OK = 0 or one of DG_ERR_*); none aborts or
 *   prints.  dg_last_error() returns a message for the last failure on the calling thread.
 * - Fields are arrays of Nx*Ny*n*n values of X-space data (the field at the Gauss nodes of
 *   every cell, Sec. 4.1/4.2) in the cell-blocked layout
 *       idx = ((cy * Nx + cx) * n + a) * n + b
 *   cy, cx = cell row / column, a = y-node, b = x-node; node (a, b) of cell (cy, cx) sits at
 *       x = (cx + 1/2) hx + hx/2 * x_b,  y = (cy + 1/2) hy + hy/2 * x_a,  hx = Lx/Nx, hy = Ly/Ny.
 * - Field pointers passed to the compute calls are DEVICE pointers owned by the caller,
 *   8-byte aligned, non-overlapping unless stated.  The library owns only the memory behind
 *   its handles (dg_grid, dg_sim, dg_batch).
 * - stream is a cudaStream_t passed as void* (NULL = the legacy default stream).  Calls are
 *   asynchronous on that stream except those that return host scalars, which synchronise it.
 * - Calls on one handle must not run concurrently with each other (handles own workspace).
 */
#ifndef DGK_DG_H
#define DGK_DG_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------- */
#define DG_OK 0
#define DG_ERR_ARG 1        /* invalid argument: size, pointer, alignment, parameter range  */
#define DG_ERR_CUDA 2       /* a CUDA runtime call failed (no device, launch failure, ...) */
#define DG_ERR_NOMEM 3      /* device or host allocation failed / over budget              */
#define DG_ERR_NOCONV 4     /* CG reached maxit before the tolerance                       */
#define DG_ERR_NONFINITE 5  /* a reduction saw a NaN or Inf                                */
#define DG_ERR_TIMEOUT 6    /* a device-side wait hit its iteration cap                    */
#define DG_ERR_IO 7         /* a file could not be opened, read or written, or is malformed */

/* ---- CG preconditioners (Sec. 6 names none; see dg_grid_set_precond) ---------------- */
#define DG_PRECOND_JACOBI 0    /* W^-1: the inverse diagonal mass matrix (default)          */
#define DG_PRECOND_TWOLEVEL 1  /* cell block solves + DFT coarse solve on cell averages    */
#define DG_PRECOND_SPECTRAL 2  /* the exact pseudo-inverse of the periodic operator by DFTs */

/* ---- boundary conditions (Sec. 3, Sec. 4.2) ---------------------------------------- */
#define DG_BC_PERIODIC 0   /* periodic in x and y (the default)                             */
#define DG_BC_DIRICHLET 1  /* homogeneous Dirichlet on all four sides (see dg_grid_create_bc) */

/* ---- bracket variants of the time stepper (Sec. 6.2, Figures 1-2) ------------------- */
#define DG_BRACKET_ARAKAWA 0  /* J = (J++ + J+x + Jx+) / 3 of Eq. J: conserves V, E, Omega      */
#define DG_BRACKET_NAIVE 1    /* J++ alone: the straightforward discretisation the paper        */
                              /* compares against (conserves V only)                            */

/* ---- precision modes ------------------------------------------------------------- */
#define DG_FP64 0     /* everything in float64                                             */
#define DG_MIXED 1    /* bracket and viscous term in double-float on the float32 pipe (see  */
                      /* dg_bracket_mixed), inner CG in float32, float64 refinement, state  */
#define DG_MIXED64 2  /* bracket in float64, inner CG in float32, float64 refinement, state  */
#define DG_FP64_PC32 3 /* float64 everywhere except the CG preconditioner, applied in float32 */
                       /* (a float32 copy of the cell block solve and the coarse DFT solve)   */

typedef struct dg_grid dg_grid;
typedef struct dg_sim dg_sim;
typedef struct dg_batch dg_batch;

/* Message for the last error on this thread ("" if none).  Never NULL. */
const char* dg_last_error(void);

/* Library ABI version (major * 100 + minor). */
int dg_version(void);

/*
 * dg_selftest_wait_cap -- checks the cap on device-side waits: launches a small cooperative
 * kernel in which one block never reaches the grid barrier, so the other blocks' waits give
 * up after about a second.  Returns DG_ERR_TIMEOUT (the expected outcome; the context stays
 * usable) or DG_ERR_CUDA.  Synchronises the stream.
 */
int dg_selftest_wait_cap(void* stream);

/*
 * dg_ref_tables -- host-only: the dimensionless per-n tables the kernels are built from
 * (Sec. 4.1: Gauss-Legendre x_j, w_j by Newton's method on the Legendre recursion,
 * Eq. recursion; Sec. 4.2: the central-flux derivative blocks; Sec. 6: the LDG blocks).
 * out receives, in this order (doubles):
 *   x[n], w[n], C0[n*n], muR[n], muL[n], lL[n], lR[n], A1cc[n*n], betaA[n]
 * with  h (f_x)_c = C0 f_c + muR (lL . f_{c+1}) - muL (lR . f_{c-1})        (central flux)
 *       h (A1 u)_c = A1cc u_c + betaA (lL . u_{c+1}) + lL (betaA . u_{c-1}) (LDG, 1D)
 * out_len must be at least dg_ref_tables_len(n) = 7n + 2n^2.
 * Errors: DG_ERR_ARG for n outside 1..5, tau < 0, out NULL or out_len too small.
 */
int dg_ref_tables_len(int n);
int dg_ref_tables(int n, double tau, double* out, int out_len);

/*
 * dg_grid_create -- periodic grid [0,Lx] x [0,Ly] with Nx x Ny cells and n nodes per cell
 * and dimension (Sec. 4.1), LDG jump penalty tau >= 0 (Sec. 6; tau = 0 is the plain
 * alternating-flux LDG).  Allocates the grid's device workspace on the current device.
 * Errors: DG_ERR_ARG (n outside 1..5, Nx or Ny < 1, Lx or Ly <= 0, tau < 0, g NULL),
 * DG_ERR_NOMEM, DG_ERR_CUDA.
 */
int dg_grid_create(dg_grid** g, int Nx, int Ny, int n, double Lx, double Ly, double tau);
/*
 * dg_grid_create_bc -- dg_grid_create with the boundary condition bc: DG_BC_PERIODIC, or
 * DG_BC_DIRICHLET (homogeneous Dirichlet, the fields zero outside [0,Lx] x [0,Ly]).  With
 * Dirichlet boundaries the derivative's numerical flux on a boundary face is the boundary
 * value, 0 (Sec. 3; the first and last cells' own blocks 1/2 (D - D^T) + 1/2 L and
 * 1/2 (D - D^T) - 1/2 R -- the reading that reproduces Table 2's Dirichlet row); the LDG
 * Laplacian takes u^ = 0 on the boundary faces and a penalty (1/h) u^2 on the left face of
 * each line (Sec. 6 names no boundary treatment); A is then symmetric positive definite, so
 * the Poisson solve takes b = W omega without removing the mean.  Dirichlet grids need
 * tau = 0 and the W^-1 preconditioner.  Errors as dg_grid_create, and DG_ERR_ARG for an
 * unknown bc or tau != 0 with Dirichlet.
 */
int dg_grid_create_bc(dg_grid** g, int Nx, int Ny, int n, double Lx, double Ly, double tau, int bc);
int dg_grid_destroy(dg_grid* g);

/* Number of values of one field: Nx*Ny*n*n (0 if g is NULL). */
long long dg_grid_dof(const dg_grid* g);

/*
 * dg_grid_nodes -- host arrays: x node coordinates (Nx*n, index cx*n+b), y node coordinates
 * (Ny*n, index cy*n+a) and the 2D quadrature weights of one cell, W_ab = (hy w_a/2)(hx w_b/2)
 * (n*n, Eq. def_norm).  Any pointer may be NULL.
 */
int dg_grid_nodes(const dg_grid* g, double* x_nodes, double* y_nodes, double* weights);

/*
 * dg_grid_set_tiles -- override the kernels' cell tile (TY x TX cells per thread block);
 * 0 restores the built-in choice for this n (tiles halved on small grids until there is
 * about one per SM).  Batched simulations use the built-in tiles.  Used by the autotuner.
 * Errors: DG_ERR_ARG.
 */
int dg_grid_set_tiles(dg_grid* g, int TY, int TX);

/*
 * dg_grid_set_precond -- the CG preconditioner of every later Poisson solve on this grid
 * (dg_poisson_solve and the simulations on g).  Sec. 6 only says that the symmetric dG
 * Poisson system is solved by conjugate gradients; the choice changes the iterates and their
 * number, and the solutions agree to the solver tolerance (both converge to the W-mean-zero
 * solution of the same system).  DG_PRECOND_JACOBI: W^-1.  DG_PRECOND_TWOLEVEL: the additive two-level
 * preconditioner B + P A_c^+ P^T -- B the exact inverse of every cell's diagonal block of
 * A, P the prolongation of cell values to the cell's nodes, A_c = P^T A P the Galerkin
 * coarse operator, inverted (constant mode dropped) by a 2D DFT of the cell grid; the
 * solution is returned with zero W-mean.  DG_PRECOND_SPECTRAL: M^-1 = A^+ itself.  On the
 * uniform periodic grid the scaled operator W^-1/2 A W^-1/2 = I (x) Kx + Ky (x) I is
 * block-circulant along both cell indices, so a DFT over the cells reduces each 1D operator
 * to one n x n Hermitian matrix per wave number (eigen-decomposed on the host, see
 * dg_spectral_symbol); z = A^+ r is a real 2D DFT of the n^2 node fields, n x n transforms per
 * wave vector, a division by the eigenvalue sums (the constant mode dropped) and the inverse
 * transforms.  CG then converges in one iteration in exact arithmetic (two or three in
 * floating point); the solution is returned with zero W-mean.  Its DFTs are radix-2 for cell
 * counts that are powers of two and direct sums otherwise (a side that is not a power of two
 * may have at most 256 cells).  Errors: DG_ERR_ARG (also for DG_PRECOND_TWOLEVEL and
 * DG_PRECOND_SPECTRAL on a Dirichlet grid: both use periodic DFTs; and for DG_PRECOND_SPECTRAL
 * with a side that is not a power of two above 256 cells).
 */
int dg_grid_set_precond(dg_grid* g, int kind);

/*
 * dg_spectral_symbol -- host-only: the symbol of the scaled 1D CG operator (the operator of
 * Sec. 6 scaled by w^-1/2 on both sides) of a periodic line of N cells of total length L, at
 * wave number k (0 <= k < N): K(k) = M + e^{i th} a r^T + e^{-i th} d s^T, th = 2 pi k / N, for
 * (Op u)_c = M u_c + a (r . u_{c+1}) + d (s . u_{c-1}); returns its eigen-decomposition
 * K = V diag(lam) V^*: lam[n] ascending, V row-major by real (Vre[n*n]) and imaginary (Vim[n*n])
 * parts, column j the eigenvector of lam[j].  At k = 0 the constant mode's eigenvalue is
 * returned as exactly 0.  These are the tables of DG_PRECOND_SPECTRAL.
 * Errors: DG_ERR_ARG.
 */
int dg_spectral_symbol(int N, int n, double L, double tau, int k, double* lam, double* Vre, double* Vim);

/*
 * dg_grid_set_compensated_apply -- how the float32 inner solves of DG_MIXED / DG_MIXED64
 * apply the CG operator on this grid: mode 1 in double-float arithmetic on the float32
 * vectors (an error of about eps32^2 |A| |u| instead of eps32 |A| |u|), 0 in plain float32,
 * 2 adaptively (float32 until a refinement sweep after the second gains less than a factor
 * 100, double-float for the rest of that solve), -1 (default) chosen from the grid: 2 when
 * eps32 times the row-sum bound of the scaled operator exceeds 5% of the smallest non-zero
 * eigenvalue of -Delta on the box (there a float32 apply is wrong by O(1) on the smoothest
 * modes and the sweeps of a solve from a poor guess contract slowly), else 0.  The choice
 * changes the inner iterates only, not what the solve converges to.
 * dg_grid_get_compensated_apply returns the mode in use.  Errors: DG_ERR_ARG.
 */
int dg_grid_set_compensated_apply(dg_grid* g, int mode);
int dg_grid_get_compensated_apply(const dg_grid* g);

/*
 * dg_bracket -- J = {psi, omega} by the conservative dG Arakawa bracket
 *     J = (J++ + J+x + Jx+) / 3                                   (Eq. J, Sec. 3)
 * with the central-flux dG derivatives of Eq. discrete_der / Eq. matrix_xspace and
 * pointwise X-space products (Sec. 4.2).  float64.  J must not alias psi or omega.
 */
int dg_bracket(dg_grid* g, const double* psi, const double* omega, double* J, void* stream);

/*
 * dg_bracket_parts -- the individual discretisations of Eq. J: parts is a bit set of
 * 1 = J++ = D_x f D_y g - D_y f D_x g, 2 = J+x = D_x(f D_y g) - D_y(f D_x g),
 * 4 = Jx+ = D_y(D_x f g) - D_x(D_y f g).  With all three (7) it is dg_bracket (the sum / 3);
 * otherwise the plain sum of the selected parts.  Only 7 conserves the integral
 * constraints (Table 2); 1 is the naive bracket the paper compares against (Figs. 1-2).
 * Errors: DG_ERR_ARG.
 */
int dg_bracket_parts(dg_grid* g, const double* psi, const double* omega, double* J, int parts, void* stream);

/*
 * dg_bracket_mixed -- the bracket of dg_bracket (Eq. J) as the DG_MIXED time stepper evaluates
 * it: the same operations in double-float arithmetic on the float32 pipe (each value the
 * unevaluated sum of two floats, about 48 significant bits; Dekker's TwoProduct and Knuth's
 * TwoSum), read from and written to float64 arrays.  Products are rounded one by one, so
 * J(f, f) = 0 holds bitwise as in float64.  Arguments and errors as dg_bracket.
 */
int dg_bracket_mixed(dg_grid* g, const double* psi, const double* omega, double* J, void* stream);

/*
 * dg_laplace_apply -- the matrix-free LDG operator of Sec. 6 (alternating fluxes, penalty
 * tau): mode 0 writes y = A x with A = W (x) A1 + A1 (x) W symmetric positive semi-definite
 * (kernel = constants); mode 1 writes y = Delta_h x = -W^{-1} A x.  float64.  y must not
 * alias x.  Errors: DG_ERR_ARG for another mode.
 */
int dg_laplace_apply(dg_grid* g, const double* x, double* y, int mode, void* stream);

/*
 * dg_poisson_solve -- -Delta_h psi = omega - mean_W(omega) by conjugate gradients (Sec. 6)
 * on A psi = W (omega - mean), run as CG on the symmetric scaling W^{-1/2} A W^{-1/2} with the
 * grid's preconditioner (dg_grid_set_precond: W^{-1}, i.e. plain CG on the scaled system, by
 * default, or the two-level one), from the initial guess in psi.  Stops when
 * r.W^{-1}r <= tol^2 b.W^{-1}b, or after exactly fixed_iters iterations if fixed_iters > 0
 * (parity mode; tol is then ignored).  The whole loop runs in one persistent cooperative
 * kernel; every device-side wait is capped.  float64.  Synchronises the stream.
 * iters / relres (may be NULL) receive the iteration count and sqrt(r.W^{-1}r / b.W^{-1}b).
 * Errors: DG_ERR_ARG (tol <= 0 with fixed_iters == 0, maxit < 0), DG_ERR_NOCONV (psi then
 * holds the last iterate), DG_ERR_TIMEOUT, DG_ERR_CUDA.
 */
int dg_poisson_solve(dg_grid* g, const double* omega, double* psi, double tol, int maxit,
                     int fixed_iters, int* iters, double* relres, void* stream);

/*
 * dg_poisson_solve_static -- the Poisson solve of dg_poisson_solve for callers that must not
 * allocate device memory: code that runs where cudaMalloc is not allowed or not safe (for
 * example while another framework owns the device allocator, or around a stream capture
 * that must not change the memory pool), and callers that cannot hold a dg_grid handle,
 * since creating one allocates.  The paper has no counterpart; this is an interface choice.
 * It takes the grid as plain parameters (Nx, Ny, n, Lx, Ly, tau as in dg_grid_create) and
 * keeps all its scratch (CG vectors, partial sums, barrier and status words) in one
 * file-scope device array of about 2.8 MB that every GPU loading the library holds until
 * the process exits.  Grids are limited to Nx*Ny*n*n <= 65536 values; larger ones are
 * rejected with DG_ERR_ARG.  It calls no cudaMalloc, cudaFree or other allocating routine.
 * Every call looks up the array's device address on the current device
 * (cudaGetSymbolAddress, which allocates nothing).  The first call for each n on a device
 * also loads that n's solver kernel and sets its shared-memory attribute: make one such
 * warm-up call per n before any stream capture.  All calls share the one array, which keeps
 * the last call's contents: calls that overlap on the GPU (other streams, other host threads)
 * race.  The call synchronises the stream (it returns the iteration count and residual).
 * Arguments, results and errors otherwise as in dg_poisson_solve.
 */
int dg_poisson_solve_static(int Nx, int Ny, int n, double Lx, double Ly, double tau, const double* omega,
                            double* psi, double tol, int maxit, int fixed_iters, int* iters, double* relres,
                            void* stream);

/*
 * dg_invariants -- out[0..2] = (V, E, Omega) = (int omega, 1/2 int psi omega,
 * 1/2 int omega^2) by Gauss-Legendre quadrature (Eq. quantities, Eq. def_norm), summed in
 * float64 in a fixed order.  Synchronises the stream.  Errors: DG_ERR_NONFINITE if a sum is
 * not finite (out is still written).
 */
int dg_invariants(dg_grid* g, const double* psi, const double* omega, double out[3], void* stream);

/* ---- simulations: the time stepper of Sec. 6 ---------------------------------------- */

typedef struct {
  long long step;            /* completed time steps                                        */
  long long cg_iters_total;  /* CG iterations over all solves since creation                */
  int cg_iters_last;         /* iterations of the last Poisson solve                        */
  int cg_iters_max;          /* largest iteration count of any solve                        */
  double cg_relres_last;     /* sqrt(r.W^-1 r / b.W^-1 b) at the end of the last solve      */
  int refine_sweeps_last;    /* float64 refinement sweeps of the last solve (DG_MIXED)      */
  int status;                /* first error seen by a device-side solve (DG_OK if none)    */
} dg_sim_info;

/*
 * dg_sim_create -- a simulation on grid g (which must outlive it) with viscosity D >= 0,
 * time step dt > 0, precision DG_FP64, DG_MIXED, DG_MIXED64 or DG_FP64_PC32, CG tolerance
 * cg_tol > 0 and iteration cap cg_maxit, from the device field omega0.  Solves for psi0 at
 * creation.  The scheme is the explicit K-step Adams-Bashforth method (Sec. 6; K = 3 unless
 * dg_sim_set_multistep changes it) for
 *     R(omega) = -J(psi, omega) + D Delta_h omega,
 * the first K-1 steps being classical RK4 steps of the same dt; each Poisson solve starts
 * from the extrapolation 2 psi^k - psi^{k-1} of the last two solutions (Sec. 6).
 * Synchronises the stream.  Errors: DG_ERR_ARG, DG_ERR_NOMEM, DG_ERR_NOCONV, DG_ERR_CUDA.
 */
int dg_sim_create(dg_sim** s, dg_grid* g, double D, double dt, int precision, double cg_tol,
                  int cg_maxit, const double* omega0, void* stream);
int dg_sim_destroy(dg_sim* s);

/* dg_step -- advance nsteps >= 0 time steps (asynchronous; solver errors are recorded in
 * the simulation and reported by dg_sim_status). */
int dg_step(dg_sim* s, int nsteps, void* stream);

/* dg_sim_status -- synchronises the stream and fills info; returns info->status. */
int dg_sim_status(dg_sim* s, dg_sim_info* info, void* stream);

/*
 * dg_sim_refinement_history -- convergence of the last mixed-precision Poisson solve
 * (DG_MIXED, DG_MIXED64): relres[j] = sqrt(r.W^-1 r / b.W^-1 b) of the float64 residual
 * before refinement sweep j (j = 0: the initial guess's; the last entry is the final residual)
 * and inner_iters[j] = the float32 PCG iterations of sweep j (0 for the last entry).  At most
 * 48 entries are kept; *count receives the number recorded, of which min(count, max) are
 * written.  Synchronises the stream.  Errors: DG_ERR_ARG.
 */
int dg_sim_refinement_history(dg_sim* s, double* relres, int* inner_iters, int max, int* count, void* stream);

/* dg_sim_get -- copies the current omega and psi (device pointers, either may be NULL). */
int dg_sim_get(dg_sim* s, double* omega, double* psi, void* stream);

/*
 * dg_sim_get_state / dg_sim_set_state -- the full stepper state (device pointers, all
 * required): omega^k, psi^k, psi^{k-1}, R^{k-1}, R^{k-2} and the step index k.  Setting the
 * state lets a caller (e.g. a checkpoint or a parity test) resume bit-exactly.  For
 * DG_MIXED the R history is stored in float32 and is converted on get/set.
 */
int dg_sim_get_state(dg_sim* s, long long* step, double* omega, double* psi, double* psi_prev,
                     double* R1, double* R2, void* stream);
int dg_sim_set_state(dg_sim* s, long long step, const double* omega, const double* psi,
                     const double* psi_prev, const double* R1, const double* R2, void* stream);

/*
 * dg_sim_get_history / dg_sim_set_history -- one entry R^{k-m} (m = 1, 2, 3) of the
 * right-hand-side history (device pointer, float64 values); m = 3 is used by K = 4 only.
 * dg_sim_set_state followed by dg_sim_set_history(s, 3, ...) restores a K = 4 state.
 */
int dg_sim_get_history(dg_sim* s, int m, double* R, void* stream);
int dg_sim_set_history(dg_sim* s, int m, const double* R, void* stream);

/*
 * dg_sim_set_bracket -- the bracket used by later steps: DG_BRACKET_ARAKAWA (default, Eq. J)
 * or DG_BRACKET_NAIVE (J++ of Eq. J alone, the comparison of Sec. 6.2).  Batched
 * simulations must use DG_BRACKET_ARAKAWA.  Errors: DG_ERR_ARG.
 */
int dg_sim_set_bracket(dg_sim* s, int variant);

/*
 * dg_sim_save / dg_sim_load -- checkpoint and resume.  save writes the complete stepper
 * state to the file path (host code; synchronises the stream): the grid's Nx, Ny, n, Lx,
 * Ly, tau and preconditioner, D, dt, precision, K, bracket, the CG controls, the step index
 * and six float64 arrays (omega^k, sqrt(W) psi^k, sqrt(W) psi^{k-1} -- the solver's own
 * variables -- and R^{k-1}, R^{k-2}, R^{k-3}).  load creates a new simulation on the
 * caller's grid g from such a file, without any solve; later steps are then bit-identical
 * to those of the saved simulation.  The file is little-endian and not portable to
 * big-endian hosts.  Errors: DG_ERR_ARG (NULL, or g differs from the saved grid),
 * DG_ERR_IO (cannot open/read/write, wrong magic or version, truncated or corrupt file),
 * DG_ERR_NOMEM, DG_ERR_CUDA.
 */
int dg_sim_save(dg_sim* s, const char* path, void* stream);
int dg_sim_load(dg_sim** s, dg_grid* g, const char* path, void* stream);

/*
 * dg_sim_set_multistep -- the number of steps K (1..4) of the Adams-Bashforth method used by
 * later steps (Sec. 6; Table 4 compares K = 1..4).  Default K = 3.  The first K-1 steps of a
 * simulation (step index < K-1) are classical RK4 start-up steps.  Batched simulations
 * (dg_batch_admit) must use K = 3; DG_ERR_ARG for K outside 1..4.
 */
int dg_sim_set_multistep(dg_sim* s, int K);

/* dg_sim_invariants -- (V, E, Omega) of the current state; synchronises the stream. */
int dg_sim_invariants(dg_sim* s, double out[3], void* stream);

/*
 * dg_sim_set_cg -- change the Poisson solver controls of later steps: tolerance tol > 0,
 * iteration cap maxit >= 1 and, if fixed_iters > 0, exactly that many CG iterations per
 * solve (parity mode: two implementations then take the same Krylov steps, Sec. 6).
 */
int dg_sim_set_cg(dg_sim* s, double tol, int maxit, int fixed_iters);

/*
 * dg_sim_set_refinement -- DG_MIXED / DG_MIXED64: each float32 inner CG sweep stops when its
 * residual has fallen by tol_in (0 < tol_in < 1), or by half the factor still missing to the
 * CG tolerance if that is looser; at most max_sweeps >= 1 float64 refinement sweeps per solve
 * (the float64 residual must reach the CG tolerance of dg_sim_create / dg_sim_set_cg).
 * Defaults: tol_in = 1e-4, max_sweeps = 40.
 */
int dg_sim_set_refinement(dg_sim* s, double tol_in, int max_sweeps);

/*
 * dg_sim_upload / dg_sim_download -- the same state transfers with HOST pointers (pinned or
 * pageable), copied by the library on the stream.  upload takes the full stepper state of
 * dg_sim_set_state; download returns omega and psi (either may be NULL) and synchronises.
 */
int dg_sim_upload(dg_sim* s, long long step, const double* omega, const double* psi, const double* psi_prev,
                  const double* R1, const double* R2, void* stream);
int dg_sim_download(dg_sim* s, double* omega, double* psi, void* stream);

/* ---- launch accounting and device timing of the hot kernels ------------------------ */
typedef struct {
  long long launches;      /* kernels this simulation launched since the last reset        */
  long long rhs_launches;  /* right-hand-side kernels (bracket + viscous term + update)     */
  long long cg_launches;   /* persistent Poisson-solve kernels                              */
  double rhs_ms;           /* summed device time of the RHS launches (timing enabled)       */
  double cg_ms;            /* summed device time of the solve launches (timing enabled)     */
} dg_sim_counters;

/* Reset the counters; enable != 0 also brackets every RHS / solve launch with CUDA events on
 * the launching stream (read back by dg_sim_get_counters, which synchronises the stream). */
int dg_sim_set_timing(dg_sim* s, int enable);
int dg_sim_get_counters(dg_sim* s, dg_sim_counters* c, void* stream);

/* ---- batches: many simulations in one persistent kernel ------------------------------ */

/*
 * A batch advances many independent simulations (any grids, n, viscosities, precisions) with
 * ONE cooperative persistent launch per dg_batch_step: the launch's blocks are split into
 * groups; each group runs whole AB3 steps (the fused bracket / viscous term / update of
 * Sec. 6 and the Poisson solve) for the simulations queued on it, one after the other, with
 * its own capped barrier; the groups run concurrently.  Once a plan (members and groups)
 * has served two launches unchanged, the launch is captured in a CUDA graph and replayed.  Simulations keep their state in their own buffers: a simulation
 * can be retired and stepped alone (dg_step) or re-admitted at any time between calls.
 *
 * dg_batch_create  -- room for max_sims >= 1 simulations.  Errors: DG_ERR_ARG, DG_ERR_NOMEM.
 * dg_batch_admit   -- adds s (which must outlive its membership); if s has taken fewer than
 *                     two steps, its RK4 start-up steps run first, alone (synchronously on the
 *                     stream).  Errors: DG_ERR_NOMEM when full, DG_ERR_ARG if already admitted.
 * dg_batch_retire  -- removes s.
 * dg_batch_set_groups -- number of block groups (0: automatic, at most 8); takes effect at the
 *                     next step.
 * dg_batch_step    -- every admitted simulation advances nsteps AB3 steps (asynchronous).
 * dg_batch_status  -- synchronises; reports whether the graph path is used, the group count
 *                     and the launches so far; returns the first error of the batch kernel or
 *                     of any member's solves (DG_ERR_TIMEOUT, DG_ERR_NOCONV, ...).
 */
int dg_batch_create(dg_batch** b, int max_sims);
int dg_batch_destroy(dg_batch* b);
int dg_batch_admit(dg_batch* b, dg_sim* s, void* stream);
int dg_batch_retire(dg_batch* b, dg_sim* s);
int dg_batch_size(const dg_batch* b);
/*
 * dg_batch_set_limit -- s takes no batched step beyond step index last_step (0: no limit):
 * within a dg_batch_step of nsteps, a member that reaches its limit sits the remaining steps
 * out, so members with different step budgets share launches of a fixed length.
 * Errors: DG_ERR_ARG.
 */
int dg_batch_set_limit(dg_batch* b, dg_sim* s, long long last_step);
int dg_batch_set_groups(dg_batch* b, int ngroups);
/*
 * dg_batch_set_tiles -- the cell tiles of the batched kernel for members with n nodes: TY x TX
 * cells per block for the RHS pass and for the solve (0, 0: the built-in tiles).  A tile
 * whose shared memory does not fit makes the next dg_batch_step fail with DG_ERR_ARG.
 * dg_batch_set_blocks_per_sm -- at most cap co-resident blocks per SM (0: as many as fit).
 * Both take effect at the next step.  Errors: DG_ERR_ARG.
 */
int dg_batch_set_tiles(dg_batch* b, int n, int rhs_ty, int rhs_tx, int cg_ty, int cg_tx);
int dg_batch_set_blocks_per_sm(dg_batch* b, int cap);
/*
 * dg_batch_autotune -- picks the batched kernel's launch configuration for the current members
 * by timing it, in two rounds of coordinate descent: the number of block groups, then for
 * each n present (the classes with the most degrees of freedom first) the RHS tile and the
 * solve tile, then a cap on blocks per SM (a tile's shared memory sets how many blocks fit on
 * an SM, so the choices interact); each candidate is timed over trial_steps batched steps
 * (CUDA events on the stream) after one untimed step, and the fastest is kept.  The trial steps are real steps: every member
 * advances (members with a step limit may sit some out, which skews the timings: tune before
 * setting limits).  The result is cached with the members' classes (grid size, n,
 * precision): a later call for the same classes returns at once.  Synchronises the stream.
 * dg_batch_get_config writes a one-line description of the configuration in use.
 * Errors: DG_ERR_ARG, and those of dg_batch_step.
 */
int dg_batch_autotune(dg_batch* b, int trial_steps, void* stream);
int dg_batch_get_config(const dg_batch* b, char* buf, int len);
int dg_batch_step(dg_batch* b, int nsteps, void* stream);
int dg_batch_status(dg_batch* b, int* uses_graph, int* ngroups, long long* launches, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* DGK_DG_H */
