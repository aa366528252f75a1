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
  TOPO_E_CUDA = 7,          /* any other CUDA runtime error                                  */
  TOPO_E_BOUNDS = 8         /* debug build (TOPO_BOUNDS_CHECK): an index outside its buffer  */
} topo_status;

typedef enum { TOPO_FP64 = 0, TOPO_MIXED = 1 } topo_precision;

/* Solver description.  levels >= 1 (1 = coarsest level only: exact dense solve); every
 * coarsening halves nx, ny (, nz), which must stay integers.  The smoother is damped Jacobi
 * (Algorithm MG's opt(), Sec. 5.1: the paper names Gauss-Seidel only as an example) with nu1
 * pre- and nu2 post-sweeps and damping omega; the coarsest level is solved exactly (an explicit
 * FP64 inverse of the dense coarsest matrix, formed at every hierarchy build).  precision
 * TOPO_MIXED runs the V-cycle (smoother, transfers, coarse operators) in FP32 and keeps the CG
 * recurrences, dot products and the coarsest solve in FP64; the outer operator runs in float
 * pairs (topo_set_outer_precision).  nrhs > 1 batches right-hand sides (vectors [nrhs][n], one
 * CG per right-hand side). */
typedef struct {
  int dim;              /* 2 or 3 */
  int nx, ny, nz;       /* elements per direction (nz ignored in 2D) */
  double E, nu;         /* isotropic material (Sec. 7: E = 1, nu = 0.3) */
  const uint8_t* fixed; /* [host] n bytes, 1 = fixed DOF */
  int levels;
  int precision;        /* topo_precision */
  int nu1, nu2;         /* pre/post smoothing sweeps (>= 0) */
  double omega;         /* Jacobi damping, (0, 1] */
  int max_iter;         /* CG iteration cap (the paper uses 1000, Sec. 8.1) */
  int nrhs;             /* right-hand sides solved together (>= 1) */
  int flexible;         /* 1: Polak-Ribiere beta (safeguard for the FP32 V-cycle) */
  int generic_kernels;  /* 1: use the generic element-matrix kernels on the 2D finest level
                           instead of the specialised Q1 butterfly kernels (for testing) */
  int smoother;         /* 0: damped Jacobi (default); 1: Chebyshev polynomial of degree nu1
                           (pre) / nu2 (post) on D^{-1} A_k over [lambda_k / 4, 1.05 lambda_k],
                           lambda_k from the power iteration (K systems only) */
  int omega_auto;       /* 1: per-level damping omega_k = min(omega, 4 / (3 lambda_k)) with
                           lambda_k ~ lambda_max(D^{-1} A_k) from a power iteration at every
                           hierarchy build: 15 steps from a fixed vector on the first build, 5
                           steps from the previous build's vector afterwards (all levels of IP
                           systems; levels >= 1 otherwise).
                           IP drivers always use it: the element rank-one terms of Z push
                           lambda_max(D^{-1} Z) well above the value for K(x). */
  const double* K0;     /* [host] the element stiffness K_i of Eq. (to) for a unit element, ne x ne
                           row-major (ne = 8 in 2D, 24 in 3D; local node-major DOF order), read
                           during topo_solver_create only; NULL: the analytic K0 of
                           topo_element_stiffness(dim, E, nu), and E, nu are used for nothing
                           else.  It must be finite and symmetric (|K0_ij - K0_ji| <= 1e-12
                           max|K0|), else TOPO_E_INVALID_ARG.  The specialised finest-level
                           kernels (2D butterfly, 3D Walsh-Hadamard basis) are used when K0 has
                           their structure (checked to 1e-14), the generic element-matrix
                           kernels otherwise. */
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
/* Device bytes that topo_solver_create(desc) would allocate (the hierarchy, the coarsest dense
 * matrices, the CG vectors and scratch), computed on the host without a device or an allocation;
 * the same value topo_solver_device_bytes reports after the create.  Descriptor errors as
 * topo_solver_create.  bytes [host]. */
topo_status topo_solver_workspace_bytes(const topo_solver_desc* desc, size_t* bytes);
topo_status topo_solver_destroy(topo_solver* s);
topo_status topo_set_stream(topo_solver* s, void* cuda_stream);
/* Per-solve records: with path [host] non-NULL every solve of this solver (topo_solve, and the
 * linear solves inside the IP and OC drivers that own it) appends one JSON line to the file:
 * the system ("K" or "Z"), grid, levels, precision, smoother, nrhs, free DOFs, tolerance,
 * iterations, final relative residual, wall time, DOF-iterations per second and status.  NULL
 * stops recording.  A file that cannot be opened is skipped silently (recording never fails a
 * solve). */
topo_status topo_set_record_file(topo_solver* s, const char* path);
/* How topo_solve drives the CG iterations of Algorithm PCG (Sec. 5.2); both give the same bits.
 * mode 0 (default): a captured graph of 4 iterations that the host replays, reading the scalars
 * back after each replay.  mode 1: one graph launch per solve, whose conditional while node
 * repeats one captured iteration until every right-hand side has stopped or reached max_iter
 * (falls back to mode 0 where conditional graph nodes are unavailable, and while profiling).
 * Other modes -> E_INVALID_ARG. */
topo_status topo_set_graph_mode(topo_solver* s, int mode);
/* Strip height of the 2D finest-level FP32 warp sweeps (Algorithm MG's smoother, residual and
 * transfers on the finest level of mixed solvers): each warp walks rows node rows of its column
 * tile, recomputing one element row at the strip's lower edge.  0 (default) picks the height that
 * fills about one wave of warps; 2..32 fixes it (a tuning parameter: the outputs do not depend on
 * it, except for the summation order of the fused r~^T y~).  Other values -> E_INVALID_ARG. */
topo_status topo_set_sweep_rows(topo_solver* s, int rows);
/* Bound of the device-side waits on asynchronous copies (the deep V-cycle levels' bulk copies):
 * a wait that has not seen its copies land after ns nanoseconds of the global timer gives up,
 * lets the copies finish under a second wait of the default bound, and stops the CG with
 * TOPO_E_TIMEOUT; the solver stays usable.  Default 1e9 (1 s).  0 makes the first wait give up at
 * once without polling: a way for tests to run the timeout path without a device fault. */
topo_status topo_set_wait_limit_ns(topo_solver* s, unsigned long long ns);
/* Fused kernels in Algorithm MG for 2D K systems with Jacobi smoothing (default on; off: one
 * launch per sweep, residual and transfer).  On the finest level the first two sweeps from zero
 * are one kernel, and so are the residual with the restriction, and the prolongation with the
 * first post-smoothing sweep; the levels
 * from the first one of at most 1024 nodes down to the coarsest run in one launch of a
 * thread-block cluster per right-hand side (where the device can run it).  2D IP systems: the
 * first two sweeps of every coarse level in one kernel.  Both settings give the same bits.  3D
 * and Chebyshev systems ignore the setting. */
topo_status topo_set_vcycle_fusion(topo_solver* s, int on);
/* Arithmetic of the outer operator q = K(x) p of Algorithm PCG on the finest level of K systems
 * (2D Q1 and 3D hex): 0 = FP64; 1 = pairs of FP32 values (hi + lo, about 48 significant bits,
 * FP64 in and out, p^T q accumulated in pairs), which GB300 runs several times faster than FP64.
 * Default: 1 for mixed-precision solvers, 0 for FP64 solvers.  The augmented systems of a
 * mixed-precision IP (topo_ip_*) run the node pass of their outer Z operator in pairs as well, and
 * FP64 IPs keep FP64.  Inputs of
 * magnitude below 2^-100 lose their low part and values beyond float range give a breakdown.
 * Other modes -> E_INVALID_ARG. */
topo_status topo_set_outer_precision(topo_solver* s, int mode);
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
/* Profile a set of kinds (bit k = kind k of topo_get_profile_kernel; 0 = off); topo_set_profiling
 * (s, on) is the mask 1.  Every event pair is a graph node of its own, so each profiled kind adds
 * some time to the iteration.  mask >= 2^8 -> E_INVALID_ARG. */
topo_status topo_set_profiling_mask(topo_solver* s, unsigned mask);
topo_status topo_get_profile(const topo_solver* s, double* operator_ms_total, long long* count);
/* The same for other parts of the iteration (kind 0 = the outer operator, as topo_get_profile).
 * Finest level of the V-cycle, in the V-cycle precision: 1 = the first smoothing kernel with a
 * matrix product (the fused first two sweeps, or the first sweep from z != 0), 2 = the residual
 * b - A z before restriction (with the restriction, where the V-cycle fuses the two), 3 = the
 * restriction P^T r (count 0 where fused into kind 2), 4 = the prolongation and correction
 * z += P z_c (fused with the first post-smoothing sweep where the V-cycle fuses).  Spans of several
 * kernels: 5 = the whole V-cycle (preconditioner), 6 + j = its part on levels >= j + 1 for
 * j = 0..5 (coarsest solve included; a fused deep part counts from its first level).  A kind
 * that the solver's V-cycle does not run has count 0.  kind outside 0..11 -> E_INVALID_ARG. */
topo_status topo_get_profile_kernel(const topo_solver* s, int kind, double* ms_total,
                                    long long* count);

/* Set the densities x [device, m FP64] (copied) and rebuild the Galerkin hierarchy
 * A_{k-1} = P^T A_k P (Sec. 5.1) with the coarsest factorisation.  x must be finite, > 0. */
topo_status topo_set_density(topo_solver* s, const double* x);

/* Solve K(x) u = b by Algorithm PCG with one V-cycle (Algorithm MG) as preconditioner
 * (Sec. 5.2), sign convention r = K u - b, stop at ||r||_2 / ||b||_2 <= tol or max_iter.
 * b, u [device, nrhs x n]; if use_x0, u holds the initial guess on entry.  Entries of b and of
 * the initial guess on fixed DOFs are ignored; u is zero there on return.  info may be NULL. */
topo_status topo_solve(topo_solver* s, const double* b, double* u, double tol, int use_x0,
                       topo_solve_info* info);

/* topo_set_density and topo_solve (from the zero guess) from host memory: x [host, m], b [host,
 * nrhs x n], u [host, nrhs x n, out].  x is copied and the hierarchy built while b is copied on a
 * second stream; u is copied back before the call returns.  Page-locked host buffers let the
 * copies run asynchronously (pageable ones work, with staged copies).  K systems only. */
topo_status topo_solve_host(topo_solver* s, const double* x, const double* b, double* u,
                            double tol, topo_solve_info* info);

/* y = K(x) v on the finest level in FP64 (masked), v, y [device, nrhs x n]. */
topo_status topo_apply_K(topo_solver* s, const double* v, double* y);

/* y = M^{-1} r: one V-cycle from the zero guess, r, y [device, nrhs x n] (FP64 in and out; in
 * mixed precision the cycle runs in FP32 inside). */
topo_status topo_apply_vcycle(topo_solver* s, const double* r, double* y);

/* Coarse-level data, for inspection: level 0 is the finest.  For 1 <= level < levels the
 * Galerkin element matrices [host out, m_level x ne x ne FP64 with ne = 8 (2D) or 24 (3D)].
 * Mixed-precision solvers with fixed damping (Jacobi, omega_auto = 0) compute and keep the
 * matrices below the coarsest level in FP32 only; those are returned widened.  The 2D mixed
 * first coarse level is applied matrix-free and has none (E_INVALID_ARG). */
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

/* ---- Allocation-free compliance (no counterpart in the paper) -------------------------------
 * c[k] = f_k^T u_k for k < nrhs: the reduction of topo_compliance, without a solver object and
 * without allocating anything (no cudaMalloc, cudaFree or pinned host memory).  It is meant for
 * callers that cannot allocate at that point: code that holds no solver (creating one allocates
 * the whole multigrid hierarchy) and code whose device memory a caching allocator has already
 * reserved, where a fresh cudaMalloc can fail and cudaFree synchronizes the device.
 * f, u [device, nrhs x n, right-hand side k at offset k*n]; c [device, nrhs], written by a
 * kernel enqueued on cuda_stream (a cudaStream_t; NULL = the legacy default stream); the call
 * returns without waiting for it.  n = 0 gives c = 0.
 * Scratch: a fixed device array inside the library, 311,552 bytes per device, holding the
 * partial sums of at most 64 right-hand sides; nrhs outside 1..64 or n < 0 -> E_INVALID_ARG with
 * the reason in topo_last_error().  Its ticket counters must be zero when a call starts: they
 * are zero when the library loads and every call leaves them at zero.
 * The first call on a device looks the array up (cudaGetSymbolAddress) with that device
 * current; make it before any stream capture.  Calls that overlap on one device (other
 * streams or host threads) share the array and race: the caller orders them.  The address is kept
 * for the life of the process: after a device reset (cudaDeviceReset) the module may load at
 * another address, so the entry point must not be called on that device again. */
topo_status topo_compliance_noalloc(const double* f, const double* u, long long n, int nrhs,
                                    double* c, void* cuda_stream);

/* ---- Primal-dual interior-point method (Sec. 2-3) ----------------------------------------
 * Newton steps on the KKT conditions KKT1-3 with the perturbed complementarity KKT4p/5p,
 * reduced to the SPD augmented system Z [d_u; d_lambda] = Res^Z of Eq. (nwtr2)-(nwtr2rhs), which
 * is solved by MGCG with the lambda unknown carried to every level by the identity (Sec. 7).
 * Readings: row 3 of Eq. (nwt) uses the right-hand side -1/2 u^T K_i u - lambda - phi_i + psi_i;
 * d_psi = (xbar - x)^{-1} (Res5 + Psi d_x); d_x = D^{-1} (B^T d_u + e d_lambda - tilde Res3);
 * Euclidean norms in the Newton test, evaluated at the new iterate. */
typedef struct topo_ip topo_ip;

typedef struct {
  double sigma;        /* barrier reduction (Sec. 3.2: 0.2) */
  double tau_nwt;      /* Newton stopping tolerance (Sec. 3.4: 0.1) */
  double tau_ip;       /* IP stopping tolerance on max(s, r) (Sec. 3.4: 1e-8) */
  double frac;         /* fraction to the boundary (Sec. 3.3: 0.9) */
  int step_x_only;     /* 1: the step rule bounds x only (the literal Sec. 3.3); 0: also phi, psi */
  int max_newton;      /* Newton step budget */
  double cg_tol;       /* relative residual for the Z systems (Sec. 6.1 uses 1e-2) */
  double cg_tol_init;  /* relative residual of the initial K(x) u = f solve (<= 0: cg_tol) */
  double cg_tol_factor; /* the Z systems of major iteration k (k barrier reductions so far) are
                           solved to cg_tol * cg_tol_factor^k: 1 keeps cg_tol fixed, 0.5 is the
                           "CG tol decreasing" variant of Sec. 8.1 (tab:IP); in (0, 1] */
  int stop_rule;       /* 0: stop once max(s, r) <= tau_ip (Eq. (crit:ip)); 1: stop once the scaled
                          KKT residual of the Remark in Sec. 3.4 is <= tau_kkt after a Newton step:
                          ||Res1||/||f|| + ||tilde Res3||/(||phi|| + ||psi||)
                          + phi^T x/(||phi|| ||x||) + psi^T (xbar - x)/(||psi|| ||xbar - x||) */
  double tau_kkt;      /* tolerance of stop_rule 1 (> 0) */
} topo_ip_opts;

typedef struct {
  int newton;          /* Newton steps so far */
  int ip_iters;        /* barrier reductions so far */
  int feval;           /* linear systems solved (initial solve included) */
  int cg_iters;        /* CG iterations over all systems */
  double s, r, lam, alpha, crit; /* barrier parameters, multiplier, last step, Newton test value */
  int done;            /* 1 once the stop rule holds */
  int status;
  double wall_ms;      /* topo_ip_run: elapsed time of the run */
  double kkt;          /* scaled KKT residual after the last Newton step (stop_rule 1's value) */
} topo_ip_info;

/* f [device, n], copied.  Returns TOPO_E_INFEASIBLE unless 0 < V < m xbar. */
topo_status topo_ip_create(const topo_solver_desc* desc, const double* f, double V, double xbar,
                           topo_ip** out);
topo_status topo_ip_destroy(topo_ip* ip);
topo_status topo_ip_set_stream(topo_ip* ip, void* cuda_stream);
/* topo_set_vcycle_fusion on both solvers of the IP (the same bits either way). */
topo_status topo_ip_set_vcycle_fusion(topo_ip* ip, int on);
/* Switches the problem to the SIMP model with the density filter (Sec. 9).  The equilibrium is
   hat K(x~) u = f with hat K(x~) = sum_i x~_i^p K_i and x~ = W x.  hat W_ij = max(0, rmin - dist(i, j)),
   with dist the Manhattan distance of the element centres in element widths.  Each column of W is
   hat W's column divided by its sum, as Sec. 9 prints it, so sum x~ = sum x.  The volume
   constraint and the bounds act on x.  The Newton systems are Eq. (nwtr)/(nwtr2) with B(u)
   replaced by hat B(u) = B(u) diag(p x~^(p-1)) W; the x-x second derivative of the non-convex
   problem is left out, as in the paper's method.  The outer CG applies that Z exactly (two filter
   passes per product).  The V-cycle's hierarchy is built from its element-local approximation,
   which keeps the row sums of W D^{-1} W^T (= W D^{-1} e) as element weights in place of the matrix:
   exact on the lambda row and column.  Call once, before topo_ip_init.
   p in [1, 8], rmin in [1, 9] (the stencil reaches |o|_1 <= ceil(rmin) - 1); otherwise
   TOPO_E_INVALID_ARG.  p = 1 and rmin = 1 (W = I) is the convex problem. */
topo_status topo_ip_set_simp(topo_ip* ip, double p, double rmin);
/* xt [device, m]: x~ = W x at the current iterate (x itself without topo_ip_set_simp).  Synchronous. */
topo_status topo_ip_filtered_density(topo_ip* ip, double* xt);
/* x = V/m, u = K(x)^{-1} f, lambda = 1, phi = psi = e, s = r = 1 (Sec. 3.1). */
topo_status topo_ip_init(topo_ip* ip, const topo_ip_opts* opts);
/* One Newton step (Sec. 3.1 steps 1-4); info after the step. */
topo_status topo_ip_step(topo_ip* ip, const topo_ip_opts* opts, topo_ip_info* info);
/* init + steps until max(s, r) <= tau_IP or max_newton steps. */
topo_status topo_ip_run(topo_ip* ip, const topo_ip_opts* opts, topo_ip_info* info);
/* Checkpoint / resume: u [device, n], x, phi, psi [device, m], scal [host, 4] = lambda, s, r and
 * the number of barrier reductions so far (as a double). */
topo_status topo_ip_get_state(topo_ip* ip, double* u, double* x, double* phi, double* psi,
                              double* scal);
topo_status topo_ip_set_state(topo_ip* ip, const double* u, const double* x, const double* phi,
                              const double* psi, const double* scal);
/* The rest of the state a bitwise resume needs: the power-iteration vectors of the
 * augmented-system solver.  Its damping omega_k = min(omega, 4/(3 * 1.05 lambda_k)) takes
 * lambda_k ~ lambda_max(D_k^{-1} Z_k) from a power iteration on every level (Sec. 5); the first
 * build runs 15 steps from a fixed start vector, each later build 5 steps from the previous
 * build's vectors.  len [host] receives the number of doubles (0 when no level iterates).
 * get: v [device, len] receives the vectors, ready [host] = 1 if they come from a successful
 * build (else the next build starts from the fixed vector).  set: v [device, len] is copied
 * when ready = 1 (v may be null when ready = 0).  Both synchronize the IP's stream. */
topo_status topo_ip_power_state_size(topo_ip* ip, long long* len);
topo_status topo_ip_get_power_state(topo_ip* ip, double* v, int* ready);
topo_status topo_ip_set_power_state(topo_ip* ip, const double* v, int ready);

/* ---- Optimality Conditions methods (Sec. 4) ----------------------------------------------
 * OC: u = K(x)^{-1} f, E_i = u^T K_i u, bisection on lambda in [0, lam_hi] until the interval is
 * <= tau_lambda, x^NEW = min(max(x E / lambda, xlow), xbar) with x fixed during the bisection and
 * the sum compared with V after a single rounding of an error-free (double-double) reduction.
 * DOC: E replaced by E^q.  AOC: x <- (OC(x) + OC(OC(x))) / 2.  The CG tolerance starts at cg_tol0
 * and, if adaptive_tol, is divided by 10 whenever the compliance increases (Sec. 6.2).
 * The linear systems are warm-started from the previous displacement. */
typedef struct topo_oc topo_oc;
enum { TOPO_OC_PLAIN = 0, TOPO_OC_DOC = 1, TOPO_OC_AOC = 2 };

typedef struct {
  int variant;         /* TOPO_OC_PLAIN, TOPO_OC_DOC or TOPO_OC_AOC */
  double q;            /* DOC damping exponent (Sec. 4.2: 1/2) */
  double xlow;         /* lower bound keeping K(x) nonsingular (Sec. 8.2: 1e-6) */
  double lam_hi;       /* initial upper end of the bisection (Sec. 4.1: 1e4) */
  double tau_lambda;   /* bisection tolerance (Sec. 4.1: 1e-11) */
  double tau_oc;       /* stop when |f^T u_k - f^T u_{k-1}| <= tau_oc (Eq. (OCstop): 1e-5) */
  int max_feval;       /* linear-solve budget */
  double cg_tol0;      /* initial CG tolerance (Sec. 6.2: 1e-4) */
  int adaptive_tol;    /* 1: the Sec. 6.2 heuristic */
} topo_oc_opts;

typedef struct {
  int iters, feval, cg_iters;
  double compliance;       /* f^T u at the iterate of the last step (before its update) */
  double compliance_prev;
  double lam;              /* last bisection midpoint of the step's first OC operator */
  double cg_tol;
  int status;
  double wall_ms;          /* topo_oc_run: elapsed time */
} topo_oc_info;

topo_status topo_oc_create(const topo_solver_desc* desc, const double* f, double V, double xbar,
                           topo_oc** out);
topo_status topo_oc_destroy(topo_oc* oc);
topo_status topo_oc_set_stream(topo_oc* oc, void* cuda_stream);
/* x0 [device, m] or NULL for x = V/m. */
topo_status topo_oc_init(topo_oc* oc, const double* x0);
topo_status topo_oc_step(topo_oc* oc, const topo_oc_opts* opts, topo_oc_info* info);
topo_status topo_oc_run(topo_oc* oc, const topo_oc_opts* opts, topo_oc_info* info);
topo_status topo_oc_get_x(topo_oc* oc, double* x);
topo_status topo_oc_get_u(topo_oc* oc, double* u);
/* Checkpoint / resume of an OC run: x [device, m] (the iterate the next step starts from),
 * u [device, n] (the last displacement, the warm start of the next solve), scal [host, 7] =
 * the CG tolerance in force (Sec. 6.2), the compliance of the previous and of the last iteration
 * (NaN before there is one), whether u holds a solve (1) or not (0), and the counts of linear
 * solves, iterations and CG iterations so far (as doubles).  A run resumed from a snapshot repeats
 * the uninterrupted run bit for bit (with power-iteration damping or Chebyshev smoothing, restore
 * the solver's power-iteration vectors too: topo_oc_get_power_state).  Both synchronize the OC's
 * stream; set returns TOPO_E_INVALID_ARG for a non-finite or negative tolerance or count. */
topo_status topo_oc_get_state(topo_oc* oc, double* x, double* u, double* scal);
/* Per-solve JSONL records of the linear solves inside the OC and IP drivers (as
 * topo_set_record_file; the IP's records name the system "K" for the initial solve and "Z" for the
 * Newton systems). */
topo_status topo_oc_set_record_file(topo_oc* oc, const char* path);
topo_status topo_ip_set_record_file(topo_ip* ip, const char* path);
topo_status topo_oc_set_state(topo_oc* oc, const double* x, const double* u, const double* scal);
/* The power-iteration vectors of the OC's solver (as topo_ip_power_state_size and friends). */
topo_status topo_oc_power_state_size(topo_oc* oc, long long* len);
topo_status topo_oc_get_power_state(topo_oc* oc, double* v, int* ready);
topo_status topo_oc_set_power_state(topo_oc* oc, const double* v, int ready);

/* Self-check of the integer FP64 <-> FP32 conversions that the CG vector kernels use in place of
 * the hardware conversion instructions: converts d[i] (device, n doubles) to float and f[i]
 * (device, n floats) to double both ways and writes to mismatches[0..1] (host) how many results
 * differ (two NaNs count as equal).  Synchronous on the default stream; allocates 16 bytes of
 * device memory for the counts.  TOPO_E_INVALID_ARG for null pointers with n > 0 or n < 0. */
topo_status topo_check_conversions(const double* d, const float* f, long long n,
                                   unsigned long long* mismatches);

/* Index checks (debug build).  A library built with -DTOPO_BOUNDS_CHECK (the package's build with
 * bounds_check=True writes libtopo_gb300_bc.so) checks the indices its operator kernels compute
 * against the sizes of the buffers they address; an index out of range is not used (a load reads
 * entry 0, a store is skipped) and is recorded, and topo_solve, topo_solve_host, topo_apply_K and
 * topo_apply_vcycle then return TOPO_E_BOUNDS.  topo_bounds_check_enabled: 1 in that build, else
 * 0.  topo_bounds_report (host pointers, each may be NULL): the number of indices found out of
 * range since the last reset, the first one of them with the size it was checked against, its
 * source file (NUL-terminated, at most file_len bytes) and line; reset = 1 clears the records.
 * Synchronizes the device.  The release build reports 0.  topo_bounds_selftest (debug build; the
 * release build returns TOPO_E_INVALID_ARG) evaluates one check of index i against size n in a
 * kernel that addresses no buffer, so that a test can see a violation recorded. */
int topo_bounds_check_enabled(void);
topo_status topo_bounds_report(unsigned long long* count, long long* index, long long* size,
                               char* file, int file_len, int* line, int reset);
topo_status topo_bounds_selftest(long long i, long long n);

#ifdef __cplusplus
}
#endif
#endif /* TOPO_H */
