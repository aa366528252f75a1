// Optimisation drivers on top of the MGCG solver: the primal-dual interior-point method (Sec. 2-3)
// and the OC / DOC / AOC methods (Sec. 4).  All state lives on the device; the host loop reads a
// few scalars back once per Newton or OC step.
//
// IP step (Sec. 3.1): residuals and the augmented system (Eq. (nwtr2), (nwtr2Z), (nwtr2rhs)) at
// the current iterate, a Galerkin hierarchy of Z with the lambda unknown carried by the identity
// (Sec. 7), PCG on Z, the direction completed element-wise, the 0.9 step rule (Sec. 3.3), the
// update, and the Newton test (Sec. 3.4) at the new iterate; when it holds, s and r are multiplied
// by sigma (Sec. 3.2) and the method stops once max(s, r) <= tau_IP.  With topo_ip_set_simp the same
// loop runs the SIMP model with the density filter (Sec. 9): the stiffness coefficients are
// (W x)^p and the residuals and the direction take hat B(u).
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "solver.cuh"

struct topo_ip {
  topo_solver* K = nullptr;   // K(x) solves (initial displacement)
  topo_solver* Z = nullptr;   // augmented systems
  Dims d{};
  long long n = 0, m = 0;
  int ne = 8;
  double *u = nullptr, *x = nullptr, *phi = nullptr, *psi = nullptr, *f = nullptr;
  double *g = nullptr, *tR3 = nullptr, *Dinv = nullptr, *t = nullptr;
  double *rhs = nullptr, *du = nullptr, *dx = nullptr, *dphi = nullptr, *dpsi = nullptr;
  IpScalars* ip = nullptr;
  IpScalars* ip_host = nullptr;
  double* partials = nullptr;
  unsigned* counter = nullptr;
  double fnorm = 0.0;
  double kkt = NAN;  // scaled KKT residual after the last Newton step
  bool simp_on = false;  // SIMP model with the density filter (Sec. 9)
  bool started = false;  // topo_ip_init or topo_ip_set_state has run
  SimpArgs sa{};
  int newton = 0, ip_iters = 0, feval = 0, cg_iters = 0;
  bool done = false;
  std::vector<void*> allocs;
  template <typename T>
  topo_status alloc(T** p, size_t count) {
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return cuda_status(e, "cudaMalloc");
    allocs.push_back((void*)*p);
    return TOPO_OK;
  }
};

struct topo_oc {
  topo_solver* K = nullptr;
  long long n = 0, m = 0;
  double *x = nullptr, *x1 = nullptr, *x2 = nullptr, *u = nullptr, *E = nullptr, *f = nullptr;
  double V = 0.0, xbar = 1.0;
  OcScalars* oc = nullptr;
  OcScalars* oc_host = nullptr;
  double* partials = nullptr;
  unsigned* counter = nullptr;
  double c_prev = NAN, c_last = NAN, cg_tol = -1.0;
  int feval = 0, iters = 0, cg_iters = 0;
  bool have_u = false;
  std::vector<void*> allocs;
  template <typename T>
  topo_status alloc(T** p, size_t count) {
    cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(count, 1) * sizeof(T));
    if (e != cudaSuccess) return cuda_status(e, "cudaMalloc");
    allocs.push_back((void*)*p);
    return TOPO_OK;
  }
};

namespace {

__global__ void k_fill(long long n, double* a, double v) {
  pdl_prologue();
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = v;
}

topo_status fill(double* a, long long n, double v, cudaStream_t st) {
  if (n <= 0) return TOPO_OK;
  topo::launch(k_fill, blocks_for(n), kThreads, 0, st, n, a, v);
  TOPO_CHECK_LAUNCH("fill");
  return TOPO_OK;
}

topo_status check_problem(const topo_solver_desc* d, const double* f, double V, double xbar) {
  if (!d || !f) {
    topo::set_error("null argument");
    return TOPO_E_INVALID_ARG;
  }
  const double m = (double)d->nx * d->ny * (d->dim == 3 ? d->nz : 1);
  if (!(xbar > 0.0) || !std::isfinite(xbar)) {
    topo::set_error("xbar must be finite and > 0");
    return TOPO_E_INVALID_ARG;
  }
  if (!(V > 0.0 && V < m * xbar)) {
    topo::set_error("volume V must lie in (0, m xbar)");
    return TOPO_E_INFEASIBLE;
  }
  return TOPO_OK;
}

// Residuals, Z data and right-hand side at the current iterate.
topo_status ip_residuals(topo_ip* a) {
  topo_solver* Z = a->Z;
  TOPO_CUDA(launch_ip_residuals(a->d, Z->K0, a->u, a->x, a->phi, a->psi, a->f, Z->L[0].fixed,
                                a->ip, a->g, a->tR3, a->Dinv, a->t, a->rhs, Z->L[0].w,
                                Z->L[0].invd, a->partials, a->counter, Z->st,
                                a->simp_on ? &a->sa : nullptr));
  return TOPO_OK;
}

// The stiffness coefficients of the current design: x, or rho = (W x)^p for the SIMP model.
topo_status stiffness_coefficients(topo_ip* a, double* dst, cudaStream_t st) {
  const double* src = a->x;
  if (a->simp_on) {
    TOPO_CUDA(launch_simp_density(a->d, a->sa, a->x, st));
    src = a->sa.rho;
  }
  TOPO_CUDA(cudaMemcpyAsync(dst, src, sizeof(double) * a->m, cudaMemcpyDeviceToDevice, st));
  return TOPO_OK;
}

topo_status ip_read(topo_ip* a) {
  TOPO_CUDA(cudaMemcpyAsync(a->ip_host, a->ip, sizeof(IpScalars), cudaMemcpyDeviceToHost, a->Z->st));
  TOPO_CUDA(cudaStreamSynchronize(a->Z->st));
  return TOPO_OK;
}

void fill_ip_info(topo_ip* a, double crit, topo_ip_info* info, int status) {
  if (!info) return;
  const IpScalars& h = *a->ip_host;
  info->newton = a->newton;
  info->ip_iters = a->ip_iters;
  info->feval = a->feval;
  info->cg_iters = a->cg_iters;
  info->s = h.s;
  info->r = h.r;
  info->lam = h.lam;
  info->alpha = h.alpha;
  info->crit = crit;
  info->kkt = a->kkt;
  info->done = a->done ? 1 : 0;
  info->status = status;
}

}  // namespace

extern "C" {

topo_status topo_ip_create(const topo_solver_desc* desc, const double* f, double V, double xbar,
                           topo_ip** out) {
  if (!out) return TOPO_E_INVALID_ARG;
  *out = nullptr;
  TOPO_TRY(check_problem(desc, f, V, xbar));
  if (desc->nrhs != 1) {
    topo::set_error("topo_ip_create: nrhs must be 1");
    return TOPO_E_INVALID_ARG;
  }
  topo_ip* a = new topo_ip();
  auto fail = [&](topo_status st) {
    std::string keep = topo_last_error();
    topo_ip_destroy(a);
    topo::set_error(keep);
    return st;
  };
  topo_status st = topo::solver_create_internal(desc, false, &a->K);
  if (st != TOPO_OK) return fail(st);
  topo_solver_desc dz = *desc;
  dz.omega_auto = 1;  // Z needs the per-level damping (see topo.h)
  st = topo::solver_create_internal(&dz, true, &a->Z);
  if (st != TOPO_OK) return fail(st);
  topo_solver* Z = a->Z;
  a->d = Z->L[0].d;
  a->n = Z->L[0].n;
  a->m = Z->L[0].m;
  a->ne = Z->ne;
  const long long n = a->n, m = a->m;
  topo_status s2 = TOPO_OK;
  s2 = s2 ? s2 : a->alloc(&a->u, n);
  s2 = s2 ? s2 : a->alloc(&a->x, m);
  s2 = s2 ? s2 : a->alloc(&a->phi, m);
  s2 = s2 ? s2 : a->alloc(&a->psi, m);
  s2 = s2 ? s2 : a->alloc(&a->f, n);
  s2 = s2 ? s2 : a->alloc(&a->g, m * a->ne);
  s2 = s2 ? s2 : a->alloc(&a->tR3, m);
  s2 = s2 ? s2 : a->alloc(&a->Dinv, m);
  s2 = s2 ? s2 : a->alloc(&a->t, m);
  s2 = s2 ? s2 : a->alloc(&a->rhs, n + 2);
  s2 = s2 ? s2 : a->alloc(&a->du, n + 2);
  s2 = s2 ? s2 : a->alloc(&a->dx, m);
  s2 = s2 ? s2 : a->alloc(&a->dphi, m);
  s2 = s2 ? s2 : a->alloc(&a->dpsi, m);
  s2 = s2 ? s2 : a->alloc(&a->ip, 1);
  s2 = s2 ? s2 : a->alloc(&a->partials, 12 * (size_t)kRedBlocks + 8 * blocks_for(a->d.nodes()));
  s2 = s2 ? s2 : a->alloc(&a->counter, 1);
  if (s2 != TOPO_OK) return fail(s2);
  if (cudaMallocHost((void**)&a->ip_host, sizeof(IpScalars)) != cudaSuccess)
    return fail(TOPO_E_OOM);
  Z->g = a->g;
  Z->Dinv = a->Dinv;
  Z->zll = &a->ip->zll;
  if (cudaMemset(a->counter, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaMemcpy(a->f, f, sizeof(double) * n, cudaMemcpyDeviceToDevice) != cudaSuccess)
    return fail(TOPO_E_CUDA);
  std::vector<uint8_t>& fx = Z->fixed_host;
  std::vector<double> fh(n);
  if (cudaMemcpy(fh.data(), f, sizeof(double) * n, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(TOPO_E_CUDA);
  double fn = 0.0;
  for (long long i = 0; i < n; ++i) {
    if (!std::isfinite(fh[i])) {
      topo::set_error("topo_ip_create: load vector is not finite");
      return fail(TOPO_E_INVALID_ARG);
    }
    if (!fx[i]) fn += fh[i] * fh[i];
  }
  a->fnorm = std::sqrt(fn);
  if (!(a->fnorm > 0.0)) {
    topo::set_error("topo_ip_create: load vector is zero on the free DOFs");
    return fail(TOPO_E_INVALID_ARG);
  }
  IpScalars h = {};
  h.V = V;
  h.xbar = xbar;
  h.frac = 0.9;
  h.step_all = 1;
  h.lam = 1.0;
  h.s = h.r = 1.0;
  *a->ip_host = h;
  if (cudaMemcpy(a->ip, &h, sizeof(IpScalars), cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(TOPO_E_CUDA);
  *out = a;
  return TOPO_OK;
}

topo_status topo_ip_destroy(topo_ip* a) {
  if (!a) return TOPO_OK;
  if (a->K) topo_solver_destroy(a->K);
  if (a->Z) topo_solver_destroy(a->Z);
  for (void* p : a->allocs) cudaFree(p);
  if (a->ip_host) cudaFreeHost(a->ip_host);
  delete a;
  return TOPO_OK;
}

topo_status topo_ip_set_stream(topo_ip* a, void* stream) {
  if (!a) return TOPO_E_INVALID_ARG;
  topo_set_stream(a->K, stream);
  return topo_set_stream(a->Z, stream);
}

topo_status topo_ip_set_vcycle_fusion(topo_ip* a, int on) {
  if (!a) return TOPO_E_INVALID_ARG;
  TOPO_TRY(topo_set_vcycle_fusion(a->K, on));
  return topo_set_vcycle_fusion(a->Z, on);
}

topo_status topo_ip_set_simp(topo_ip* a, double p, double rmin) {
  if (!a) return TOPO_E_INVALID_ARG;
  if (!(p >= 1.0 && p <= 8.0) || !(rmin >= 1.0 && rmin <= (double)(kSimpMaxR + 1))) {
    topo::set_error("topo_ip_set_simp: p must lie in [1, 8] and rmin in [1, " +
                    std::to_string(kSimpMaxR + 1) + "]");
    return TOPO_E_INVALID_ARG;
  }
  if (a->simp_on || a->started) {
    topo::set_error("topo_ip_set_simp: call once, before topo_ip_init and topo_ip_set_state");
    return TOPO_E_INVALID_ARG;
  }
  StreamGuard gd(a->Z);
  const long long m = a->m;
  SimpArgs& sa = a->sa;
  double* invS = nullptr;
  topo_status s2 = TOPO_OK;
  s2 = s2 ? s2 : a->alloc(&invS, m);
  s2 = s2 ? s2 : a->alloc(&sa.xt, m);
  s2 = s2 ? s2 : a->alloc(&sa.rho, m);
  s2 = s2 ? s2 : a->alloc(&sa.c, m);
  s2 = s2 ? s2 : a->alloc(&sa.E, m);
  s2 = s2 ? s2 : a->alloc(&sa.e3, m);
  s2 = s2 ? s2 : a->alloc(&sa.gh, m * a->ne);
  s2 = s2 ? s2 : a->alloc(&sa.th, m);
  s2 = s2 ? s2 : a->alloc(&sa.Dm, m);
  s2 = s2 ? s2 : a->alloc(&sa.ea, m);
  s2 = s2 ? s2 : a->alloc(&sa.eb, m);
  if (s2 != TOPO_OK) return s2;
  sa.p = p;
  sa.rmin = rmin;
  sa.R = (int)std::ceil(rmin) - 1;
  sa.invS = invS;
  TOPO_CUDA(launch_filter_colsum(a->d, rmin, sa.R, invS, a->Z->st));
  TOPO_CUDA(cudaStreamSynchronize(a->Z->st));
  // the hierarchy of Z takes the element-local columns c_e g_e and the row sums of W D^-1 W^T as
  // weights; the outer CG applies the exact Z
  topo_solver* Z = a->Z;
  Z->g = sa.gh;
  Z->Dinv = sa.Dm;
  Z->simp.on = true;
  Z->simp.rmin = rmin;
  Z->simp.R = sa.R;
  Z->simp.invS = invS;
  Z->simp.Dinv = a->Dinv;
  Z->simp.ea = sa.ea;
  Z->simp.eb = sa.eb;
  a->simp_on = true;
  return TOPO_OK;
}

topo_status topo_ip_filtered_density(topo_ip* a, double* xt) {
  if (!a || !xt) return TOPO_E_INVALID_ARG;
  StreamGuard gd(a->Z);
  cudaStream_t st = a->Z->st;
  if (a->simp_on) {
    TOPO_CUDA(launch_simp_density(a->d, a->sa, a->x, st));
    TOPO_CUDA(cudaMemcpyAsync(xt, a->sa.xt, sizeof(double) * a->m, cudaMemcpyDeviceToDevice, st));
  } else {
    TOPO_CUDA(cudaMemcpyAsync(xt, a->x, sizeof(double) * a->m, cudaMemcpyDeviceToDevice, st));
  }
  TOPO_CUDA(cudaStreamSynchronize(st));
  return TOPO_OK;
}

// The options the IP driver cannot run with.
topo_status check_ip_opts(const topo_ip_opts* o, const char* where) {
  if (!(o->cg_tol > 0.0) || !(o->cg_tol_factor > 0.0 && o->cg_tol_factor <= 1.0) ||
      !(o->sigma > 0.0 && o->sigma < 1.0) || (o->stop_rule != 0 && o->stop_rule != 1) ||
      (o->stop_rule == 1 && !(o->tau_kkt > 0.0))) {
    topo::set_error(std::string(where) +
                    ": cg_tol must be > 0, cg_tol_factor in (0, 1], sigma in (0, 1), stop_rule 0 "
                    "or 1 (with tau_kkt > 0)");
    return TOPO_E_INVALID_ARG;
  }
  return TOPO_OK;
}

topo_status topo_ip_init(topo_ip* a, const topo_ip_opts* o) {
  NvtxRange nvtx("topo: IP init (Sec. 3.1)");
  if (!a || !o) return TOPO_E_INVALID_ARG;
  TOPO_TRY(check_ip_opts(o, "topo_ip_init"));
  StreamGuard gd(a->Z);
  cudaStream_t st = a->Z->st;
  const double V = a->ip_host->V;
  // x = V/m, lambda = 1, phi = psi = e, s = r = 1 (Sec. 3.1); u = K(x)^{-1} f
  TOPO_TRY(fill(a->x, a->m, V / (double)a->m, st));
  TOPO_TRY(fill(a->phi, a->m, 1.0, st));
  TOPO_TRY(fill(a->psi, a->m, 1.0, st));
  IpScalars h = *a->ip_host;
  h.lam = 1.0;
  h.s = h.r = 1.0;
  h.frac = o->frac > 0.0 ? o->frac : 0.9;
  h.step_all = o->step_x_only ? 0 : 1;
  *a->ip_host = h;
  TOPO_CUDA(cudaMemcpyAsync(a->ip, a->ip_host, sizeof(IpScalars), cudaMemcpyHostToDevice, st));
  TOPO_CUDA(cudaStreamSynchronize(st));
  topo_solver* K = a->K;
  {
    StreamGuard gk(K->st, st, K->ev_in, K->ev_out);
    TOPO_TRY(stiffness_coefficients(a, K->x, K->st));
    TOPO_TRY(topo::solver_build(K));
    topo_solve_info si{};
    topo_status s = topo::solver_solve(K, a->f, a->u, o->cg_tol_init > 0 ? o->cg_tol_init : o->cg_tol,
                                       0, &si);
    a->cg_iters += si.iterations;
    if (s != TOPO_OK) return s;
  }
  a->newton = a->ip_iters = 0;
  a->feval = 1;
  a->done = false;
  a->started = true;
  return TOPO_OK;
}

topo_status topo_ip_step(topo_ip* a, const topo_ip_opts* o, topo_ip_info* info) {
  NvtxRange nvtx("topo: IP Newton step (Sec. 3.1)");
  if (!a || !o) return TOPO_E_INVALID_ARG;
  TOPO_TRY(check_ip_opts(o, "topo_ip_step"));
  if (a->done) {
    fill_ip_info(a, 0.0, info, TOPO_OK);
    return TOPO_OK;
  }
  StreamGuard gd(a->Z);
  topo_solver* Z = a->Z;
  cudaStream_t st = Z->st;
  // residuals, Z data and right-hand side at z with the current (s, r)
  TOPO_TRY(ip_residuals(a));
  TOPO_CUDA(cudaMemcpyAsync(Z->x, a->simp_on ? a->sa.rho : a->x, sizeof(double) * a->m,
                            cudaMemcpyDeviceToDevice, st));
  TOPO_TRY(topo::solver_build(Z));
  topo_solve_info si{};
  const double tol = o->cg_tol * std::pow(o->cg_tol_factor, (double)a->ip_iters);
  topo_status ss = topo::solver_solve(Z, a->rhs, a->du, tol, 0, &si);
  a->cg_iters += si.iterations;
  a->feval += 1;
  if (ss != TOPO_OK && ss != TOPO_E_NOT_CONVERGED) {
    fill_ip_info(a, NAN, info, ss);
    return ss;
  }
  TOPO_CUDA(launch_ip_recover_update(a->d, a->g, a->du, a->tR3, a->Dinv, a->u, a->x, a->phi, a->psi,
                                     a->dx, a->dphi, a->dpsi, a->ip, a->partials, a->counter, st,
                                     a->simp_on ? &a->sa : nullptr));
  a->newton += 1;
  // Newton test at the new iterate with the current (s, r)
  TOPO_TRY(ip_residuals(a));
  TOPO_TRY(ip_read(a));
  IpScalars& h = *a->ip_host;
  const double crit = h.nrm_res1 / a->fnorm + h.nrm_tr3 / (h.nrm_phi + h.nrm_psi);
  if (!std::isfinite(crit) || !std::isfinite(h.alpha)) {
    topo::set_error("topo_ip_step: non-finite Newton iterate");
    fill_ip_info(a, crit, info, TOPO_E_BREAKDOWN);
    return TOPO_E_BREAKDOWN;
  }
  // the scaled KKT residual of the Remark in Sec. 3.4, at the new iterate with the current (s, r)
  a->kkt = crit + h.comp_phi / (h.nrm_phi * h.nrm_x) + h.comp_psi / (h.nrm_psi * h.nrm_xu);
  if (o->stop_rule == 1 && a->kkt <= o->tau_kkt) {
    a->done = true;
    fill_ip_info(a, crit, info, ss);
    return TOPO_OK;
  }
  if (crit <= o->tau_nwt) {
    h.s *= o->sigma;
    h.r *= o->sigma;
    a->ip_iters += 1;
    TOPO_CUDA(cudaMemcpyAsync(&a->ip->s, &h.s, sizeof(double), cudaMemcpyHostToDevice, st));
    TOPO_CUDA(cudaMemcpyAsync(&a->ip->r, &h.r, sizeof(double), cudaMemcpyHostToDevice, st));
    TOPO_CUDA(cudaStreamSynchronize(st));
    if (o->stop_rule == 0 && std::max(h.s, h.r) <= o->tau_ip) a->done = true;
  }
  fill_ip_info(a, crit, info, ss);
  return TOPO_OK;
}

topo_status topo_ip_run(topo_ip* a, const topo_ip_opts* o, topo_ip_info* info) {
  if (!a || !o) return TOPO_E_INVALID_ARG;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, a->Z->user);
  topo_status st = topo_ip_init(a, o);
  topo_ip_info last{};
  while (st == TOPO_OK && !a->done && a->newton < o->max_newton)
    st = topo_ip_step(a, o, &last);
  cudaEventRecord(e1, a->Z->user);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (info) {
    *info = last;
    fill_ip_info(a, last.crit, info, st);
    info->wall_ms = ms;
  }
  return st;
}

// State for checkpointing: u [n], x, phi, psi [m] device; scal[0..3] = lambda, s, r and the
// barrier reductions so far (host).
topo_status topo_ip_get_state(topo_ip* a, double* u, double* x, double* phi, double* psi,
                              double* scal) {
  if (!a || !u || !x || !phi || !psi || !scal) return TOPO_E_INVALID_ARG;
  StreamGuard gd(a->Z);
  cudaStream_t st = a->Z->st;
  TOPO_CUDA(cudaMemcpyAsync(u, a->u, sizeof(double) * a->n, cudaMemcpyDeviceToDevice, st));
  TOPO_CUDA(cudaMemcpyAsync(x, a->x, sizeof(double) * a->m, cudaMemcpyDeviceToDevice, st));
  TOPO_CUDA(cudaMemcpyAsync(phi, a->phi, sizeof(double) * a->m, cudaMemcpyDeviceToDevice, st));
  TOPO_CUDA(cudaMemcpyAsync(psi, a->psi, sizeof(double) * a->m, cudaMemcpyDeviceToDevice, st));
  TOPO_TRY(ip_read(a));
  scal[0] = a->ip_host->lam;
  scal[1] = a->ip_host->s;
  scal[2] = a->ip_host->r;
  scal[3] = (double)a->ip_iters;
  return TOPO_OK;
}

topo_status topo_ip_set_state(topo_ip* a, const double* u, const double* x, const double* phi,
                              const double* psi, const double* scal) {
  if (!a || !u || !x || !phi || !psi || !scal) return TOPO_E_INVALID_ARG;
  StreamGuard gd(a->Z);
  cudaStream_t st = a->Z->st;
  TOPO_CUDA(cudaMemcpyAsync(a->u, u, sizeof(double) * a->n, cudaMemcpyDeviceToDevice, st));
  TOPO_CUDA(cudaMemcpyAsync(a->x, x, sizeof(double) * a->m, cudaMemcpyDeviceToDevice, st));
  TOPO_CUDA(cudaMemcpyAsync(a->phi, phi, sizeof(double) * a->m, cudaMemcpyDeviceToDevice, st));
  TOPO_CUDA(cudaMemcpyAsync(a->psi, psi, sizeof(double) * a->m, cudaMemcpyDeviceToDevice, st));
  TOPO_TRY(ip_read(a));
  a->ip_host->lam = scal[0];
  a->ip_host->s = scal[1];
  a->ip_host->r = scal[2];
  a->ip_iters = (int)scal[3];
  TOPO_CUDA(cudaMemcpyAsync(a->ip, a->ip_host, sizeof(IpScalars), cudaMemcpyHostToDevice, st));
  TOPO_CUDA(cudaStreamSynchronize(st));
  a->done = false;
  a->started = true;
  return TOPO_OK;
}

// Power-iteration vectors of the augmented-system solver (start vectors of the next build's
// lambda_max estimates); device copies on the solver's stream.
topo_status topo_ip_power_state_size(topo_ip* a, long long* len) {
  if (!a || !len) return TOPO_E_INVALID_ARG;
  *len = (long long)a->Z->pw_len;
  return TOPO_OK;
}

topo_status topo_ip_get_power_state(topo_ip* a, double* v, int* ready) {
  if (!a || !ready || (a->Z->pw_len && !v)) return TOPO_E_INVALID_ARG;
  StreamGuard gd(a->Z);
  cudaStream_t st = a->Z->st;
  if (a->Z->pw_len)
    TOPO_CUDA(cudaMemcpyAsync(v, a->Z->pw_vec, sizeof(double) * a->Z->pw_len,
                              cudaMemcpyDeviceToDevice, st));
  TOPO_CUDA(cudaStreamSynchronize(st));
  *ready = a->Z->pw_ready ? 1 : 0;
  return TOPO_OK;
}

topo_status topo_ip_set_power_state(topo_ip* a, const double* v, int ready) {
  if (!a || (ready && a->Z->pw_len && !v)) return TOPO_E_INVALID_ARG;
  StreamGuard gd(a->Z);
  cudaStream_t st = a->Z->st;
  if (ready && a->Z->pw_len) {
    TOPO_CUDA(cudaMemcpyAsync(a->Z->pw_vec, v, sizeof(double) * a->Z->pw_len,
                              cudaMemcpyDeviceToDevice, st));
    TOPO_CUDA(cudaStreamSynchronize(st));
  }
  a->Z->pw_ready = ready && a->Z->pw_len;
  return TOPO_OK;
}

// ---- OC -----------------------------------------------------------------------------------

topo_status topo_oc_create(const topo_solver_desc* desc, const double* f, double V, double xbar,
                           topo_oc** out) {
  if (!out) return TOPO_E_INVALID_ARG;
  *out = nullptr;
  TOPO_TRY(check_problem(desc, f, V, xbar));
  if (desc->nrhs != 1) {
    topo::set_error("topo_oc_create: nrhs must be 1");
    return TOPO_E_INVALID_ARG;
  }
  topo_oc* a = new topo_oc();
  auto fail = [&](topo_status st) {
    std::string keep = topo_last_error();
    topo_oc_destroy(a);
    topo::set_error(keep);
    return st;
  };
  topo_status st = topo::solver_create_internal(desc, false, &a->K);
  if (st != TOPO_OK) return fail(st);
  a->n = a->K->L[0].n;
  a->m = a->K->L[0].m;
  a->V = V;
  a->xbar = xbar;
  topo_status s2 = TOPO_OK;
  s2 = s2 ? s2 : a->alloc(&a->x, a->m);
  s2 = s2 ? s2 : a->alloc(&a->x1, a->m);
  s2 = s2 ? s2 : a->alloc(&a->x2, a->m);
  s2 = s2 ? s2 : a->alloc(&a->E, a->m);
  s2 = s2 ? s2 : a->alloc(&a->u, a->n);
  s2 = s2 ? s2 : a->alloc(&a->f, a->n);
  s2 = s2 ? s2 : a->alloc(&a->oc, 1);
  s2 = s2 ? s2 : a->alloc(&a->partials, 2 * (size_t)kRedBlocks);
  s2 = s2 ? s2 : a->alloc(&a->counter, 1);
  if (s2 != TOPO_OK) return fail(s2);
  if (cudaMallocHost((void**)&a->oc_host, sizeof(OcScalars)) != cudaSuccess) return fail(TOPO_E_OOM);
  if (cudaMemset(a->counter, 0, sizeof(unsigned)) != cudaSuccess ||
      cudaMemcpy(a->f, f, sizeof(double) * a->n, cudaMemcpyDeviceToDevice) != cudaSuccess ||
      cudaMemset(a->u, 0, sizeof(double) * a->n) != cudaSuccess)
    return fail(TOPO_E_CUDA);
  *out = a;
  return TOPO_OK;
}

topo_status topo_oc_destroy(topo_oc* a) {
  if (!a) return TOPO_OK;
  if (a->K) topo_solver_destroy(a->K);
  for (void* p : a->allocs) cudaFree(p);
  if (a->oc_host) cudaFreeHost(a->oc_host);
  delete a;
  return TOPO_OK;
}

topo_status topo_oc_set_stream(topo_oc* a, void* stream) {
  if (!a) return TOPO_E_INVALID_ARG;
  return topo_set_stream(a->K, stream);
}

topo_status topo_oc_init(topo_oc* a, const double* x0) {
  if (!a) return TOPO_E_INVALID_ARG;
  StreamGuard gd(a->K);
  cudaStream_t st = a->K->st;
  if (x0)
    TOPO_CUDA(cudaMemcpyAsync(a->x, x0, sizeof(double) * a->m, cudaMemcpyDeviceToDevice, st));
  else
    TOPO_TRY(fill(a->x, a->m, a->V / (double)a->m, st));
  TOPO_CUDA(cudaMemsetAsync(a->u, 0, sizeof(double) * a->n, st));
  TOPO_CUDA(cudaStreamSynchronize(st));
  a->c_prev = a->c_last = NAN;
  a->cg_tol = -1.0;
  a->feval = a->iters = a->cg_iters = 0;
  a->have_u = false;
  return TOPO_OK;
}

namespace {

// One application of the operator OC(.) (Algorithm OC, or DOC with exponent q):
// u = K(xin)^{-1} f (warm start), E_e = u_e^T K0 u_e, bisection on lambda, xout = x^NEW.
topo_status oc_operator(topo_oc* a, const topo_oc_opts* o, const double* xin, double* xout,
                        double* c) {
  topo_solver* K = a->K;
  cudaStream_t st = K->st;
  TOPO_CUDA(cudaMemcpyAsync(K->x, xin, sizeof(double) * a->m, cudaMemcpyDeviceToDevice, st));
  TOPO_TRY(topo::solver_build(K));
  topo_solve_info si{};
  topo_status ss = topo::solver_solve(K, a->f, a->u, a->cg_tol, a->have_u ? 1 : 0, &si);
  a->cg_iters += si.iterations;
  a->feval += 1;
  a->have_u = true;
  if (ss != TOPO_OK && ss != TOPO_E_NOT_CONVERGED) return ss;
  TOPO_CUDA(launch_dot(a->n, 1, a->f, a->u, K->partials, K->counters, K->dots, st));
  TOPO_CUDA(launch_element_energy(K->L[0].d, K->K0, a->u, a->u, a->E, 1.0, st));
  if (o->variant == TOPO_OC_DOC) TOPO_CUDA(launch_pow_inplace(a->m, a->E, o->q, st));
  OcScalars h = {};
  h.lo = 0.0;
  h.hi = o->lam_hi > 0.0 ? o->lam_hi : 1e4;
  h.tau = o->tau_lambda > 0.0 ? o->tau_lambda : 1e-11;
  h.V = a->V;
  h.xlow = o->xlow;
  h.xbar = a->xbar;
  *a->oc_host = h;
  TOPO_CUDA(cudaMemcpyAsync(a->oc, a->oc_host, sizeof(OcScalars), cudaMemcpyHostToDevice, st));
  const int steps = (int)std::ceil(std::log2(std::max(h.hi - h.lo, h.tau) / h.tau)) + 1;
  TOPO_CUDA(launch_oc_bisection(a->m, xin, a->E, a->oc, steps, xout, a->partials, a->counter, st));
  double cdev = 0.0;
  TOPO_CUDA(cudaMemcpyAsync(&cdev, K->dots, sizeof(double), cudaMemcpyDeviceToHost, st));
  TOPO_CUDA(cudaMemcpyAsync(a->oc_host, a->oc, sizeof(OcScalars), cudaMemcpyDeviceToHost, st));
  TOPO_CUDA(cudaStreamSynchronize(st));
  *c = cdev;
  return ss;
}

}  // namespace

topo_status topo_oc_step(topo_oc* a, const topo_oc_opts* o, topo_oc_info* info) {
  NvtxRange nvtx("topo: OC step (Sec. 4)");
  if (!a || !o) return TOPO_E_INVALID_ARG;
  StreamGuard gd(a->K);
  cudaStream_t st = a->K->st;
  if (a->cg_tol < 0.0) a->cg_tol = o->cg_tol0;
  double c = NAN, c2 = NAN;
  double lam_first = NAN;
  topo_status ss;
  if (o->variant == TOPO_OC_AOC) {
    ss = oc_operator(a, o, a->x, a->x1, &c);
    if (ss != TOPO_OK && ss != TOPO_E_NOT_CONVERGED) return ss;
    lam_first = a->oc_host->lam_last;
    ss = oc_operator(a, o, a->x1, a->x2, &c2);
    if (ss != TOPO_OK && ss != TOPO_E_NOT_CONVERGED) return ss;
    TOPO_CUDA(launch_average(a->m, a->x1, a->x2, a->x, st));
  } else {
    ss = oc_operator(a, o, a->x, a->x1, &c);
    if (ss != TOPO_OK && ss != TOPO_E_NOT_CONVERGED) return ss;
    lam_first = a->oc_host->lam_last;
    TOPO_CUDA(cudaMemcpyAsync(a->x, a->x1, sizeof(double) * a->m, cudaMemcpyDeviceToDevice, st));
  }
  TOPO_CUDA(cudaStreamSynchronize(st));
  a->iters += 1;
  a->c_prev = a->c_last;
  a->c_last = c;
  // adaptive CG tolerance (Sec. 6.2): the OC iterates should decrease the compliance
  if (o->adaptive_tol && std::isfinite(a->c_prev) && c > a->c_prev) a->cg_tol *= 0.1;
  if (info) {
    info->iters = a->iters;
    info->feval = a->feval;
    info->cg_iters = a->cg_iters;
    info->compliance = c;
    info->compliance_prev = a->c_prev;
    info->lam = lam_first;
    info->cg_tol = a->cg_tol;
    info->status = ss;
    info->wall_ms = 0.0;
  }
  return TOPO_OK;
}

topo_status topo_oc_run(topo_oc* a, const topo_oc_opts* o, topo_oc_info* info) {
  if (!a || !o) return TOPO_E_INVALID_ARG;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, a->K->user);
  topo_oc_info last{};
  topo_status st = TOPO_OK;
  while (a->feval < o->max_feval) {
    st = topo_oc_step(a, o, &last);
    if (st != TOPO_OK) break;
    if (std::isfinite(a->c_prev) && std::fabs(a->c_last - a->c_prev) <= o->tau_oc) break;
  }
  cudaEventRecord(e1, a->K->user);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (info) {
    *info = last;
    info->wall_ms = ms;
  }
  return st;
}

topo_status topo_oc_get_x(topo_oc* a, double* x) {
  if (!a || !x) return TOPO_E_INVALID_ARG;
  StreamGuard gd(a->K);
  TOPO_CUDA(cudaMemcpyAsync(x, a->x, sizeof(double) * a->m, cudaMemcpyDeviceToDevice, a->K->st));
  return TOPO_OK;
}

topo_status topo_oc_get_u(topo_oc* a, double* u) {
  if (!a || !u) return TOPO_E_INVALID_ARG;
  StreamGuard gd(a->K);
  TOPO_CUDA(cudaMemcpyAsync(u, a->u, sizeof(double) * a->n, cudaMemcpyDeviceToDevice, a->K->st));
  return TOPO_OK;
}

topo_status topo_oc_set_record_file(topo_oc* a, const char* path) {
  if (!a) return TOPO_E_INVALID_ARG;
  return topo_set_record_file(a->K, path);
}

topo_status topo_ip_set_record_file(topo_ip* a, const char* path) {
  if (!a) return TOPO_E_INVALID_ARG;
  if (a->K) TOPO_TRY(topo_set_record_file(a->K, path));
  return topo_set_record_file(a->Z, path);
}

// Checkpoint / resume: the iterate, the warm-start displacement and the host scalars of the run.
topo_status topo_oc_get_state(topo_oc* a, double* x, double* u, double* scal) {
  if (!a || !x || !u || !scal) {
    set_error("topo_oc_get_state: null argument");
    return TOPO_E_INVALID_ARG;
  }
  StreamGuard gd(a->K);
  cudaStream_t st = a->K->st;
  TOPO_CUDA(cudaMemcpyAsync(x, a->x, sizeof(double) * a->m, cudaMemcpyDeviceToDevice, st));
  TOPO_CUDA(cudaMemcpyAsync(u, a->u, sizeof(double) * a->n, cudaMemcpyDeviceToDevice, st));
  TOPO_CUDA(cudaStreamSynchronize(st));
  scal[0] = a->cg_tol;
  scal[1] = a->c_prev;
  scal[2] = a->c_last;
  scal[3] = a->have_u ? 1.0 : 0.0;
  scal[4] = (double)a->feval;
  scal[5] = (double)a->iters;
  scal[6] = (double)a->cg_iters;
  return TOPO_OK;
}

topo_status topo_oc_set_state(topo_oc* a, const double* x, const double* u, const double* scal) {
  if (!a || !x || !u || !scal) {
    set_error("topo_oc_set_state: null argument");
    return TOPO_E_INVALID_ARG;
  }
  // a tolerance not yet set (negative: the next step takes cg_tol0) or a positive finite one
  const bool tol_ok = scal[0] == -1.0 || (std::isfinite(scal[0]) && scal[0] > 0.0);
  bool ok = tol_ok && (scal[3] == 0.0 || scal[3] == 1.0);
  for (int k = 4; k < 7; ++k)
    ok = ok && std::isfinite(scal[k]) && scal[k] >= 0.0 && scal[k] == std::floor(scal[k]) &&
         scal[k] < 2147483647.0;
  if (!ok) {
    set_error("topo_oc_set_state: invalid tolerance, flag or count in scal");
    return TOPO_E_INVALID_ARG;
  }
  StreamGuard gd(a->K);
  cudaStream_t st = a->K->st;
  TOPO_CUDA(cudaMemcpyAsync(a->x, x, sizeof(double) * a->m, cudaMemcpyDeviceToDevice, st));
  TOPO_CUDA(cudaMemcpyAsync(a->u, u, sizeof(double) * a->n, cudaMemcpyDeviceToDevice, st));
  TOPO_CUDA(cudaStreamSynchronize(st));
  a->cg_tol = scal[0];
  a->c_prev = scal[1];
  a->c_last = scal[2];
  a->have_u = scal[3] == 1.0;
  a->feval = (int)scal[4];
  a->iters = (int)scal[5];
  a->cg_iters = (int)scal[6];
  return TOPO_OK;
}

topo_status topo_oc_power_state_size(topo_oc* a, long long* len) {
  if (!a || !len) return TOPO_E_INVALID_ARG;
  *len = (long long)a->K->pw_len;
  return TOPO_OK;
}

topo_status topo_oc_get_power_state(topo_oc* a, double* v, int* ready) {
  if (!a || !ready || (a->K->pw_len && !v)) return TOPO_E_INVALID_ARG;
  StreamGuard gd(a->K);
  cudaStream_t st = a->K->st;
  if (a->K->pw_len)
    TOPO_CUDA(cudaMemcpyAsync(v, a->K->pw_vec, sizeof(double) * a->K->pw_len,
                              cudaMemcpyDeviceToDevice, st));
  TOPO_CUDA(cudaStreamSynchronize(st));
  *ready = a->K->pw_ready ? 1 : 0;
  return TOPO_OK;
}

topo_status topo_oc_set_power_state(topo_oc* a, const double* v, int ready) {
  if (!a || (ready && a->K->pw_len && !v)) return TOPO_E_INVALID_ARG;
  StreamGuard gd(a->K);
  cudaStream_t st = a->K->st;
  if (ready && a->K->pw_len) {
    TOPO_CUDA(cudaMemcpyAsync(a->K->pw_vec, v, sizeof(double) * a->K->pw_len,
                              cudaMemcpyDeviceToDevice, st));
    TOPO_CUDA(cudaStreamSynchronize(st));
  }
  a->K->pw_ready = ready && a->K->pw_len;
  return TOPO_OK;
}

}  // extern "C"
