/*
 * topo.h - C ABI of the GB300 MGCG library for variable-thickness-sheet minimum-compliance
 * topology optimisation (Kocvara & Mohammed, "Primal-dual interior-point multigrid method for
 * topology optimization", arXiv 1606.06201).
 *
 * Problem (Eq. (to)):  min 1/2 f^T u  s.t.  K(x) u = f,  sum_i x_i = V,  0 <= x_i <= xbar,
 * with K(x) = sum_i x_i K_i and K_i the element stiffness K0 scattered to element i's DOFs.
 *
 * Conventions (every array argument):
 *   2D grid nx x ny square unit elements, nodes (nx+1)(ny+1), node (i,j) -> i + (nx+1) j.
 *   3D grid nx x ny x nz unit cubes, node (i,j,k) -> i + (nx+1)(j + (ny+1) k).
 *   DOFs interleaved per node: DOF = dim * node + component.  n = dim * nodes.
 *   Elements x-fastest: e = ex + nx (ey + ny ez).  Local element nodes: counter-clockwise from
 *   (ex, ey) in 2D; in 3D the bottom face (z = ez) counter-clockwise, then the top face.
 *   Fixed (Dirichlet) DOFs are given as a byte mask (1 = fixed) on the finest grid.  The library
 *   works on all DOFs and masks: vectors it returns are zero on fixed DOFs, and operators act as
 *   M A M + (I - M) restricted to vectors that vanish on fixed DOFs, which equals the eliminated
 *   system on the free DOFs.
 *   Arrays marked [device] are CUDA device pointers owned by the caller (contiguous, FP64 unless
 *   stated).  Arrays marked [host] are host pointers read during the call only.
 *   All device work is enqueued on the solver's stream (topo_set_stream; default: the legacy
 *   default stream); calls that return iteration counts or norms synchronise that stream.
 *
 * Errors: every call returns a topo_status and never exits or traps.  topo_last_error() returns
 * a thread-local message for the last failing call.  A device-side error flag (breakdown, bounded
 * wait expired) is read back at the synchronisation points and turned into a status.
 */
#ifndef TOPO_H
#define TOPO_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  TOPO_OK = 0,
  TOPO_E_INVALID_ARG = 1,   /* bad size, NaN/Inf, x outside its bounds, V infeasible, ... */
  TOPO_E_NOT_CONVERGED = 2, /* CG reached max_iter; the best iterate is still returned      */
  TOPO_E_BREAKDOWN = 3,     /* p^T A p <= 0 or a non-finite scalar in the CG recurrences     */
  TOPO_E_INFEASIBLE = 4,    /* V outside (0, m xbar)                                         */
  TOPO_E_TIMEOUT = 5,       /* a bounded device-side wait expired                            */
  TOPO_E_OOM = 6,           /* device allocation failed                                      */
  TOPO_E_CUDA = 7           /* any other CUDA runtime error                                  */
} topo_status;

typedef enum { TOPO_FP64 = 0, TOPO_MIXED = 1 } topo_precision;

/* Solver description.  levels >= 1 (1 = coarsest level only: exact dense solve); every
 * coarsening halves nx, ny (, nz), which must stay integers.  The smoother is damped Jacobi
 * (Algorithm MG's opt(), Sec. 5.1: the paper names Gauss-Seidel only as an example) with nu1
 * pre- and nu2 post-sweeps and damping omega; the coarsest level is solved exactly (dense FP64
 * Cholesky).  precision TOPO_MIXED runs the V-cycle (smoother, transfers, coarse operators) in
 * FP32 and keeps the CG recurrences, dot products, the outer operator and the coarsest solve
 * in FP64.  nrhs > 1 batches right-hand sides (vectors [nrhs][n], one CG per right-hand side). */
typedef struct {
  int dim;              /* 2 or 3 */
  int nx, ny, nz;       /* elements per direction (nz ignored in 2D) */
  double E, nu;         /* isotropic material (Sec. 7: E = 1, nu = 0.3) */
  const uint8_t* fixed; /* [host] n bytes, 1 = fixed DOF */
  int levels;
  int precision;        /* topo_precision */
  int nu1, nu2;         /* pre/post smoothing sweeps (>= 0) */
  double omega;         /* Jacobi damping, (0, 1] */
  int max_iter;         /* CG iteration cap (the paper uses 1000, Sec. 9.1) */
  int nrhs;             /* right-hand sides solved together (>= 1) */
  int flexible;         /* 1: Polak-Ribiere beta (safeguard for the FP32 V-cycle) */
  int generic_kernels;  /* 1: use the generic element-matrix kernels on the 2D finest level
                           instead of the specialised Q1 butterfly kernels (for testing) */
} topo_solver_desc;

typedef struct {
  int iterations;       /* CG iterations (max over right-hand sides) */
  double rel_residual;  /* ||r|| / ||b|| of the CG recurrence residual at exit (max over rhs) */
  double wall_ms;       /* device time of the solve (CUDA events) */
  int status;           /* topo_status of the solve */
} topo_solve_info;

typedef struct topo_solver topo_solver;

/* Message of the last failing call on this thread ("" if none).  The string is owned by the
 * library and valid until the next failing call on the same thread. */
const char* topo_last_error(void);

/* Element stiffness K0 (Sec. 7): 2D Q1 plane stress on the unit square with unit thickness
 * (8 x 8), or the 3D trilinear hexahedron on the unit cube (24 x 24), by 2-point Gauss
 * quadrature per direction, row-major, DOFs in local node-major order.  K0_out [host]. */
topo_status topo_element_stiffness(int dim, double E, double nu, double* K0_out);

/* Create a solver: uploads K0 and the masks, allocates the hierarchy and workspaces on the
 * current CUDA device.  Returns TOPO_E_INVALID_ARG if the masks are not compatible with
 * geometric coarsening (a fixed fine DOF must interpolate only from fixed coarse DOFs). */
topo_status topo_solver_create(const topo_solver_desc* desc, topo_solver** out);
topo_status topo_solver_destroy(topo_solver* s);
topo_status topo_set_stream(topo_solver* s, void* cuda_stream);
/* Device bytes held by the solver. */
size_t topo_solver_device_bytes(const topo_solver* s);
/* Number of CUDA kernels this solver has launched since its creation (graph kernel nodes
 * included); instrumentation, no counterpart in the paper. */
unsigned long long topo_solver_launch_count(const topo_solver* s);
/* Live timing of the outer FP64 operator q = K(x) p inside the CG iterations: when on, every
 * captured iteration records CUDA events around that kernel (on the stream it runs on), and
 * topo_get_profile returns the summed duration in ms and the number of timed launches since the
 * last topo_set_profiling call.  Instrumentation, no counterpart in the paper. */
topo_status topo_set_profiling(topo_solver* s, int on);
topo_status topo_get_profile(const topo_solver* s, double* operator_ms_total, long long* count);

/* Set the densities x [device, m FP64] (copied) and rebuild the Galerkin hierarchy
 * A_{k-1} = P^T A_k P (Sec. 5.1) with the coarsest factorisation.  x must be finite, > 0. */
topo_status topo_set_density(topo_solver* s, const double* x);

/* Solve K(x) u = b by Algorithm PCG with one V-cycle (Algorithm MG) as preconditioner
 * (Sec. 5.2), sign convention r = K u - b, stop at ||r||_2 / ||b||_2 <= tol or max_iter.
 * b, u [device, nrhs x n]; if use_x0, u holds the initial guess on entry.  info may be NULL. */
topo_status topo_solve(topo_solver* s, const double* b, double* u, double tol, int use_x0,
                       topo_solve_info* info);

/* y = K(x) v on the finest level in FP64 (masked), v, y [device, nrhs x n]. */
topo_status topo_apply_K(topo_solver* s, const double* v, double* y);

/* y = M^{-1} r: one V-cycle from the zero guess, r, y [device, nrhs x n] (FP64 in and out; in
 * mixed precision the cycle runs in FP32 inside). */
topo_status topo_apply_vcycle(topo_solver* s, const double* r, double* y);

/* Coarse-level data, for inspection: level 0 is the finest.  For 1 <= level < levels the
 * Galerkin element matrices [host out, m_level x ne x ne FP64 with ne = 8 (2D) or 24 (3D)]. */
topo_status topo_get_level_matrices(topo_solver* s, int level, double* out_host);
/* Number of elements of a level (0 = finest). */
int topo_level_elems(const topo_solver* s, int level);

/* c = f^T u per right-hand side: f, u [device, nrhs x n], c [host, nrhs]. */
topo_status topo_compliance(topo_solver* s, const double* f, const double* u, double* c);

/* Element energies E_e = u_e^T K0 u_e (no factor 1/2): u [device, n], E [device, m]. */
topo_status topo_element_energy(topo_solver* s, const double* u, double* E);

/* Adjoint gradient of L = w^T u(x) with K(x) lam = w: g_e = -lam_e^T K0 u_e.
 * lam, u [device, n], g [device, m]. */
topo_status topo_grad_x(topo_solver* s, const double* lam, const double* u, double* g);

#ifdef __cplusplus
}
#endif
#endif /* TOPO_H */
